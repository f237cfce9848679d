// tc.cuh -- fifth-generation tensor-core primitives (sm_100 family: tcgen05, TMEM, bulk async copies,
// mbarriers) in inline PTX, and the exact digit arithmetic the tensor-core path is built on.
//
// Exact products on bf16 tensor cores.  A value x in [-1, 1] is held as the integer X = round(x 2^104) and
// written as 15 balanced base-128 digits, X = sum_i d_i 128^i with d_i in [-64, 63] (the top digit in
// [-64, 64]).  Every digit is an integer of at most 7 bits, so it is exact in bf16, and a product of two
// digits (|.| <= 2^12) is exact in the fp32 accumulator.  The product of two such values keeps the digit
// pairs (i, k) with i + k >= 14: "level" u = 28 - i - k runs over 0..14 and holds u + 1 digit pairs whose
// weight is 128^(28-u).  A level accumulator that has summed P products of each of its pairs satisfies
// |V_u| <= 15 P 2^12; read out every 256 products it stays below 15 2^20 < 2^24, where fp32 holds every
// integer exactly, and a round-to-nearest conversion returns it.  The dropped pairs (i + k <= 13) contribute
// at most 2^-101 of one unit product each, far below the 1e-28 normwise tolerance.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ssh {
namespace tc {

constexpr int kDigits = 15;         // balanced base-128 digits per value
constexpr int kLevels = 15;         // kept levels (digit pairs with i + k >= 14)
constexpr int kFracBits = 104;      // X = round(x 2^104)
constexpr int kTileM = 128;         // accumulator rows (TMEM lanes)
constexpr int kTileN = 32;          // accumulator columns per level
constexpr int kStepK = 16;          // K per MMA instruction (bf16)
constexpr int kChunkSteps = 16;     // K-steps between exact read-outs (256 products per pair)
constexpr int kHeldLevels = 7;      // levels 0..6 (at most 7 pairs) are read out after every second chunk
constexpr int kTmemCols = 512;      // kLevels * kTileN = 480 used
constexpr uint32_t kSliceA = kTileM * kStepK * 2;   // 4096 bytes: one digit slice of one A K-step
constexpr uint32_t kSliceB = kTileN * kStepK * 2;   // 1024 bytes: one digit slice of one B K-step
constexpr uint32_t kStageA = kDigits * kSliceA;      // 61440
constexpr uint32_t kStageB = kDigits * kSliceB;      // 15360
constexpr uint32_t kStageBytes = kStageA + kStageB;  // 76800
constexpr int kStages = 3;
constexpr float kMagic = 12582912.0f;                // 1.5 * 2^23 (small integer -> fp32 by one FADD)
constexpr int32_t kMagicBits = 0x4B400000;

// Byte offset of element (r, k) inside one K-major rows x 16 operand slice, no swizzle: 8x16-byte core
// matrices, K-adjacent core matrices 128 bytes apart (LBO), 8-row groups 256 bytes apart (SBO).
__host__ __device__ __forceinline__ uint32_t slice_off(int r, int k) {
  return (uint32_t)((r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle, version 1.  lbo: byte distance of core matrices adjacent along K;
// sbo: along M (or N).  A core matrix is eight 16-byte rows: for a K-major operand each row holds 8 K-consecutive
// elements of one M row, for an MN-major operand 8 M-consecutive elements of one K row.
__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr, uint32_t lbo = 128, uint32_t sbo = 256) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: D f32, A and B bf16, B K-major, A K-major (a_mn = 0) or MN-major (1), M x N
__host__ __device__ constexpr uint32_t make_idesc(int M, int N, int a_mn = 0) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity to complete.  Gives up (returns false) after `limit`
// clock cycles, or as soon as *abort (when not null) is set by another thread of the CTA.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, long long limit, volatile int* abort) {
  if (mbar_try(b, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try(b, parity)) return true;
    if (abort && *abort) return false;
    if (clock64() - t0 > limit) return false;
  }
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16), completion on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// make a tensor map that the host wrote into global memory visible to the tensor-map proxy of this thread
__device__ __forceinline__ void tmap_acquire(const void* tmap) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
}
// 4-D tiled tensor copy global -> shared (coordinates in elements, innermost first), completion on the mbarrier
__device__ __forceinline__ void tma_load_4d(void* dst, const void* tmap, int c0, int c1, int c2, int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[sdesc] * B[sdesc]^T, issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate));
}
// arrive on the mbarrier when every tcgen05 operation issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
               : "memory");
}

// 16 consecutive accumulator columns of this warp's 32 TMEM lanes, one lane per thread
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// 8 consecutive accumulator columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Exact integer value of an fp32 accumulator word holding an integer x of magnitude below 2^24.  Three forms,
// so that a read-out can spread its conversions over two pipes (the fp32-to-int unit runs at 16 per clock per SM,
// an eighth of the fp32 rate):
//   acc_int       the conversion instruction;
//   acc_int_fma   on the fp32 pipe: q = rint(x / 4096) from the bits of x 2^-12 + 1.5 2^23 (one rounding, to an
//                 integer in [2^23, 2^24), where the spacing is 1), r = x - 4096 q exactly (|r| <= 2048), and r from
//                 the bits of r + 1.5 2^23; x = 4096 q + r, computed modulo 2^32 from the two bit patterns;
//   acc_int_small for |x| < 2^22 only: the bits of x + 1.5 2^23.
__device__ __forceinline__ int32_t acc_int(uint32_t bits) { return __float2int_rn(__uint_as_float(bits)); }
__device__ __forceinline__ int32_t acc_int_fma(uint32_t bits) {
  const float x = __uint_as_float(bits);
  const float h = __fmaf_rn(x, 0x1p-12f, kMagic);
  const float r = __fmaf_rn(__fsub_rn(h, kMagic), -4096.0f, x);
  const float l = __fadd_rn(r, kMagic);
  return (int32_t)(__float_as_uint(h) * 4096u + __float_as_uint(l) - (uint32_t)kMagicBits * 4097u);
}
__device__ __forceinline__ int32_t acc_int_small(uint32_t bits) {
  return (int32_t)(__float_as_uint(__fadd_rn(__uint_as_float(bits), kMagic)) - (uint32_t)kMagicBits);
}

}  // namespace tc
}  // namespace ssh
