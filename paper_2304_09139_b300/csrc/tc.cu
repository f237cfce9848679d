// tc.cu -- the fixed-point hot path for d = 2 on the tensor cores (Eqs. ntilde and force of arXiv:2304.09139).
//
// With a_j(n1) = e^{2 pi i n1 s_j1} and b_j(n2) = e^{2 pi i n2 s_j2}, the collective density factorises per
// axis, n~(n1, n2) = sum_j a_j(n1) b_j(n2): a matrix product over the particles.  Since b_j(-m) = conj(b_j(m)),
// the four real products P_pq(n1, m) = sum_j p_j(n1) q_j(m) (p the cos / sin of axis 1, q of axis 2, m >= 0)
// give both n~(n1, m) = (P_cc - P_ss) + i (P_cs + P_sc) and n~(n1, -m) = (P_cc + P_ss) + i (P_sc - P_cs):
// one real GEMM with rows (n1, p), columns (m, q) and K = particles.
//
// The force F_j = (4 pi / L) sum_k n [C sin th - S cos th] = (4 pi / L) Im sum_k n W_k a_j(n1) b_j(n2), with
// W = C - i S, is grouped per n1: G_j(n1) = sum_n2 W b_j(n2) = sum_{m >= 0} [U(n1, m) cos(2 pi m s_j2) +
// V(n1, m) sin(2 pi m s_j2)], U = W(n1, m) + W(n1, -m), V = i (W(n1, m) - W(n1, -m)) (m = 0: U = W(n1, 0),
// V = 0), and likewise G' with the weight n2.  Rows = particles, K = (m, cos / sin), columns = (n1, Re G,
// Im G, Re G', Im G'); the epilogue forms F_j1 = (4 pi / L) Im sum n1 a_j(n1) G_j(n1) and F_j2 = (4 pi / L)
// Im sum a_j(n1) G'_j(n1).
//
// Both products use the exact digit arithmetic of tc.cuh: operands are 15 bf16 digit slices, the 120 kept
// digit pairs accumulate into 15 TMEM level accumulators, read out exactly every 64 products.
//
// Kernels (one launch each per evaluation, over every tensor-core member of the engine):
//   k_tc_prep         per particle: powers e^{2 pi i m s} of both axes (an exact-phase anchor every 16 powers,
//                     one multiply per power in between), written as digit slices in the tile layouts of the
//                     two GEMMs, and a_j(n1) as Q2.126 for the force epilogue
//   k_tc_gemm         warp-specialised tcgen05 GEMM: one producer thread (bulk async copies, two stages), one
//                     MMA thread (22 MMAs per K-step), eight epilogue warps (level read-out, exact folding)
//   k_tc_dens_finish  fixed-order sum over K ranges, the four real products -> n~(n1, +-m) as Q34.126 partials
//   k_tc_coef         U, V, U', V' from the exact n~ and the power-of-two scale, as digit slices of the force GEMM
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "fx.cuh"
#include "reduce.cuh"
#include "ssh_internal.h"
#include "tc.cuh"

#define SSH_TABLE_QUAL __device__
#include "gen/tables.h"

namespace ssh {

using namespace tc;

namespace {

constexpr int kEpiWarps = 16;                      // four per TMEM lane quadrant
constexpr int kEpiCols = kTileN / (kEpiWarps / 4);  // accumulator columns per epilogue warp (8)
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;  // producer warp, MMA warp, epilogue warps
constexpr long long kWaitLimit = 2000000000LL;     // clock cycles (about one second) for any single wait
constexpr size_t kGemmSmem = (size_t)kStages * kStageBytes;
constexpr int kFinThreads = 64;

__device__ __forceinline__ bool stopped(const CfgDev& c) { return c.run && *c.run; }

__device__ __forceinline__ __int128 q128_to_i128(const q128& a) {
  return (__int128)(((unsigned __int128)a.w[3] << 96) | ((unsigned __int128)a.w[2] << 64) |
                    ((unsigned __int128)a.w[1] << 32) | (unsigned __int128)a.w[0]);
}

// e^{2 pi i t} of an unsigned Q0.128 turn, Q2.126
__device__ __forceinline__ fxc phasor_turn(const q128& t) {
  q128 piq;
#pragma unroll
  for (int i = 0; i < 4; i++) piq.w[i] = SSH_FX_PI_Q3_125[i];
  return fx_sincos_turns(t, SSH_FX_TAB_A, SSH_FX_TAB_B, piq, SSH_FX_INV_FACT);
}

// (t * m) mod 1 for an unsigned Q0.128 turn: exact
__device__ __forceinline__ q128 turn_times(const q128& t, int m) {
  const unsigned __int128 u = (unsigned __int128)q128_to_i128(t);
  return q128_from_i128((__int128)(u * (unsigned __int128)(unsigned)m));
}

// 64 * (128^14 - 1) / 127: the offset that turns balanced digits d_0..d_13 into ordinary base-128 digits
__device__ __forceinline__ __int128 digit_bias() {
  __int128 b = 0;
#pragma unroll
  for (int i = 0; i < 14; i++) b |= (__int128)64 << (7 * i);
  return b;
}

// The 15 balanced digits of X (|X| <= 2^104) as bf16, slice s holding digit 14 - s (top digit first).
__device__ __forceinline__ void put_digits_x(uint8_t* base, uint32_t slice_stride, uint32_t off, __int128 X) {
  const __int128 Y = X + digit_bias();
#pragma unroll
  for (int s = 0; s < kDigits; s++) {
    const int i = kDigits - 1 - s;
    const int d = i == kDigits - 1 ? (int)(Y >> 98) : (int)((Y >> (7 * i)) & 127) - 64;
    *reinterpret_cast<uint16_t*>(base + (size_t)s * slice_stride + off) =
        __bfloat16_as_ushort(__float2bfloat16_rn((float)d));
  }
}

// 192-bit two's-complement accumulator
struct i192 {
  unsigned long long w[3];
};
__device__ __forceinline__ void i192_zero(i192& a) { a.w[0] = a.w[1] = a.w[2] = 0ull; }
// a += v << sh (0 <= sh < 128)
__device__ __forceinline__ void i192_add_shl(i192& a, __int128 v, int sh) {
  const unsigned __int128 lo = (unsigned __int128)v << sh;
  const unsigned long long top =
      sh == 0 ? (v < 0 ? ~0ull : 0ull) : (unsigned long long)(v >> (128 - sh));  // bits 128..191 of v << sh
  const unsigned __int128 a01 = ((unsigned __int128)a.w[1] << 64) | a.w[0];
  const unsigned __int128 s01 = a01 + lo;
  const unsigned long long carry = s01 < a01 ? 1ull : 0ull;
  a.w[0] = (unsigned long long)s01;
  a.w[1] = (unsigned long long)(s01 >> 64);
  a.w[2] = a.w[2] + top + carry;
}
// the low 160 bits of a << sh (0 <= sh < 64) as a Q34.126 accumulator
__device__ __forceinline__ q160 i192_to_q160_shl(const i192& a, int sh) {
  unsigned long long w0 = a.w[0], w1 = a.w[1], w2 = a.w[2];
  if (sh > 0) {
    w2 = (w2 << sh) | (w1 >> (64 - sh));
    w1 = (w1 << sh) | (w0 >> (64 - sh));
    w0 <<= sh;
  }
  q160 r;
  r.w[0] = (uint32_t)w0;
  r.w[1] = (uint32_t)(w0 >> 32);
  r.w[2] = (uint32_t)w1;
  r.w[3] = (uint32_t)(w1 >> 32);
  r.w[4] = (uint32_t)w2;
  return r;
}

// 2^e as a double (normal range)
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// X 2^-S of a 192-bit integer with |X| < 2^150, as a double-double.  X = h 2^106 + m 2^53 + l with l, m in
// [0, 2^53) and h signed are each exact in binary64; the two-sum of the top two pieces is exact, and the last
// piece lies below the unit of the result's low word.
__device__ __forceinline__ dd i192_to_dd(const i192& x, int S) {
  const unsigned long long mask = (1ull << 53) - 1;
  const unsigned long long l = x.w[0] & mask;
  const unsigned long long m = ((x.w[0] >> 53) | (x.w[1] << 11)) & mask;
  const long long h = (long long)((x.w[1] >> 42) | (x.w[2] << 22));
  const dd s = two_sum((double)h * pow2(106 - S), (double)m * pow2(53 - S));
  return fast_two_sum(s.hi, s.lo + (double)l * pow2(-S));
}

// round(a / 2^sh) of a Q34.126 accumulator, for results with |.| <= 2^104; sh may be negative (left shift)
__device__ __forceinline__ __int128 q160_shr_round(const q160& a, int sh) {
  i192 t;  // the 160-bit value sign-extended to 192 bits
  t.w[0] = ((unsigned long long)a.w[1] << 32) | a.w[0];
  t.w[1] = ((unsigned long long)a.w[3] << 32) | a.w[2];
  t.w[2] = (unsigned long long)(long long)(int32_t)a.w[4];
  if (sh <= 0) return (__int128)((((unsigned __int128)t.w[1] << 64) | t.w[0]) << (-sh));
  i192_add_shl(t, (__int128)1, sh - 1);  // round half up
  if (sh >= 64)  // bits sh .. sh + 127, arithmetic
    return (__int128)(((unsigned __int128)t.w[2] << 64) | t.w[1]) >> (sh - 64);
  const unsigned __int128 lo = ((unsigned __int128)t.w[1] << 64) | t.w[0];
  return (__int128)((lo >> sh) | ((unsigned __int128)t.w[2] << (128 - sh)));
}

__device__ __forceinline__ q160 load_q160(const void* p) {
  const uint32_t* u = reinterpret_cast<const uint32_t*>(p);
  q160 r;
#pragma unroll
  for (int i = 0; i < 5; i++) r.w[i] = u[i];
  return r;
}

}  // namespace

// ------------------------------------------------------------------------------------------------ k_tc_prep

namespace {

constexpr int kPrepThreads = 256;
constexpr int kPrepParticles = 16;  // particles per CTA (one K-step of the density GEMM)
constexpr int kPrepM = 80;          // powers per pass (shared-memory staging of their fixed-point values)
constexpr int kPrepLow = 8;         // e^{2 pi i m s} = A[m / 8] T[m % 8]
constexpr int kPrepAnc = kPrepM / kPrepLow;
constexpr int kPrepPitch = 2 * kPrepM + 1;  // staging row pitch (16-byte entries): odd, so rows spread over the banks
constexpr size_t kPrepSmemY = (size_t)kPrepPitch * kPrepParticles * 16;
constexpr size_t kPrepSmem = kPrepSmemY;

// Eight biased values Y = X + B (X = round(x 2^104), B the balanced-digit offset) -> their 15 digits as one
// 16-byte row (8 bf16) per digit slice, slice s holding digit 14 - s.  Digit i < 14 is bits 7i..7i+6 of Y
// minus 64 (one funnel shift from two 32-bit words); the top digit is the signed bits 98..127.
__device__ __forceinline__ void put_digit_rows(uint8_t* base, uint32_t slice_stride, const uint4 (&Y)[8]) {
#pragma unroll
  for (int s = 0; s < kDigits; s++) {
    const int i = kDigits - 1 - s;
    uint32_t f[8];
#pragma unroll
    for (int v = 0; v < 8; v++) {
      const uint32_t w[4] = {Y[v].x, Y[v].y, Y[v].z, Y[v].w};
      int d;
      if (i == kDigits - 1) {
        d = (int32_t)w[3] >> 2;
      } else {
        const int o = 7 * i;
        d = (int)(__funnelshift_r(w[o >> 5], w[(o >> 5) + 1 < 4 ? (o >> 5) + 1 : 3], o & 31) & 127u) - 64;
      }
      // small integer -> fp32 (exact) whose upper half is the bf16 of the same value
      f[v] = __float_as_uint(__int_as_float(kMagicBits + d) - kMagic);
    }
    uint4 row;
    row.x = __byte_perm(f[0], f[1], 0x7632);
    row.y = __byte_perm(f[2], f[3], 0x7632);
    row.z = __byte_perm(f[4], f[5], 0x7632);
    row.w = __byte_perm(f[6], f[7], 0x7632);
    *reinterpret_cast<uint4*>(base + (size_t)s * slice_stride) = row;
  }
}

// first-quadrant phasor -> (re, im) as round(x 2^104) + balanced-digit offset, and as signed Q2.126
__device__ __forceinline__ void qent_out(const qent& z, uint4& yre, uint4& yim, fxc* q126) {
  // unsigned Q1.127 components (value 1 is 2^127: unsigned arithmetic until after the shift)
  const unsigned __int128 c = (unsigned __int128)q128_to_i128(z.c), sn = (unsigned __int128)q128_to_i128(z.s);
  const uint32_t q = z.cs.w[0] & 3u;
  const __int128 xc = (__int128)((c + ((unsigned __int128)1 << 22)) >> 23);
  const __int128 xs = (__int128)((sn + ((unsigned __int128)1 << 22)) >> 23);
  __int128 re, im;
  switch (q) {  // z = i^q (c + i s)
    case 0: re = xc; im = xs; break;
    case 1: re = -xs; im = xc; break;
    case 2: re = -xc; im = -xs; break;
    default: re = xs; im = -xc; break;
  }
  const __int128 b = digit_bias();
  const unsigned __int128 ur = (unsigned __int128)(re + b), ui = (unsigned __int128)(im + b);
  yre = make_uint4((uint32_t)ur, (uint32_t)(ur >> 32), (uint32_t)(ur >> 64), (uint32_t)(ur >> 96));
  yim = make_uint4((uint32_t)ui, (uint32_t)(ui >> 32), (uint32_t)(ui >> 64), (uint32_t)(ui >> 96));
  if (q126) {
    const __int128 hc = (__int128)(c >> 1), hs = (__int128)(sn >> 1);  // Q2.126
    __int128 r2, i2;
    switch (q) {
      case 0: r2 = hc; i2 = hs; break;
      case 1: r2 = -hs; i2 = hc; break;
      case 2: r2 = -hc; i2 = -hs; break;
      default: r2 = hs; i2 = -hc; break;
    }
    fxc o;
    o.re = q128_from_i128(r2);
    o.im = q128_from_i128(i2);
    *q126 = o;
  }
}

}  // namespace

// Thread per (particle, axis): the tables T[k] = e^{2 pi i k s} (k < 8) and A[b] = e^{2 pi i 8 b s}
// (b < ceil((R + 1) / 8)) as first-quadrant phasors, from exact-phase values of e^{2 pi i s} and e^{2 pi i 8 s}
// and chains of multiplies (each product at most 8 units of 2^-126 low; about 17 in the longest chain).
// Grid (particle blocks, tensor-core members); layout tc_tab[(axis N + j) tc_ntab + (k | 8 + b)].
__global__ void __launch_bounds__(128) k_tc_tables(const CfgDev* __restrict__ cfgs, const int* __restrict__ list) {
  grid_dep_wait();
  const CfgDev& c = cfgs[list[blockIdx.y]];
  if (stopped(c)) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * c.N) return;
  const int axis = (int)(idx / c.N);
  const int64_t j = idx - (int64_t)axis * c.N;
  const int R = axis == 0 ? c.tc_R1 : c.tc_R2;
  const int nA = R / kPrepLow + 1;
  const q128 u = turns_from_dd(c.s_hi[axis * c.N + j], c.s_lo[axis * c.N + j]);
  qent* tab = reinterpret_cast<qent*>(c.tc_tab) + idx * c.tc_ntab;
  const qent one = to_quadrant(phasor_turn(q128_zero()));
  const qent e1 = to_quadrant(phasor_turn(u));
  qent t = one;
#pragma unroll 1
  for (int k = 0; k < kPrepLow; k++) {
    tab[k] = t;
    if (k + 1 < kPrepLow) t = qmul(t, e1);
  }
  const qent e8 = to_quadrant(phasor_turn(turn_times(u, kPrepLow)));
  qent a = one;
#pragma unroll 1
  for (int b = 0; b < nA; b++) {
    tab[kPrepLow + b] = a;
    if (b + 1 < nA) a = qmul(a, e8);
  }
}

// CTA per (configuration, axis, 16 particles); items TwItem {cfg, axis, first particle}.  Per pass over at
// most 80 powers m0.. : phase 1 forms every power as one product A[m / 8] T[m % 8] of the particle's tables
// (all threads, independent) into shared memory; phase 2 writes the digit slices as whole 16-byte
// core-matrix rows (8 K-consecutive values of one operand row), which consecutive threads fill contiguously.
// Axis 1 (n1) feeds the density GEMM's A operand and the Q2.126 table a_j(n1) of the force epilogue; axis 2
// feeds the density GEMM's B operand and the force GEMM's A operand.
__global__ void __launch_bounds__(kPrepThreads) k_tc_prep(const CfgDev* __restrict__ cfgs,
                                                          const TwItem* __restrict__ items) {
  grid_dep_wait();
  extern __shared__ __align__(16) uint8_t psm[];
  uint4* Ys = reinterpret_cast<uint4*>(psm);  // [j][2 (m - m0) + p], pitch kPrepPitch
  const TwItem it = items[blockIdx.x];
  const CfgDev& c = cfgs[it.cfg];
  if (stopped(c)) return;
  const int axis = it.pad;
  const int64_t N = c.N;
  const int64_t j0 = it.start;
  const int R = axis == 0 ? c.tc_R1 : c.tc_R2;
  const int tid = threadIdx.x;
  const __int128 bias = digit_bias();
  const uint4 yzero = make_uint4((uint32_t)bias, (uint32_t)(bias >> 32), (uint32_t)(bias >> 64), (uint32_t)(bias >> 96));
  const qent* tab = reinterpret_cast<const qent*>(c.tc_tab);
  for (int m0 = 0; m0 <= R; m0 += kPrepM) {
    const int mcount = min(kPrepM, R + 1 - m0);
    // phase 1: every (particle, power) of the pass, one product each
    for (int task = tid; task < mcount * kPrepParticles; task += kPrepThreads) {
      const int jl = task % kPrepParticles, ml = task / kPrepParticles;
      const int64_t j = j0 + jl;
      const int m = m0 + ml;
      uint4 yr = yzero, yi = yzero;
      if (j < N) {
        const qent* tj = tab + ((int64_t)axis * N + j) * c.tc_ntab;
        const qent z = qmul(tj[kPrepLow + (m >> 3)], tj[m & 7]);
        fxc zq;
        qent_out(z, yr, yi, axis == 0 ? &zq : nullptr);
        if (axis == 0) reinterpret_cast<fxc*>(c.tc_a1)[(int64_t)m * N + j] = zq;
      }
      Ys[jl * kPrepPitch + ml * 2 + 0] = yr;
      Ys[jl * kPrepPitch + ml * 2 + 1] = yi;
    }
    __syncthreads();
    // phase 2a: rows (m, cos / sin) x 8 particles, into the density GEMM operand of this axis
    const int nrow = 2 * mcount;
    for (int task = tid; task < nrow * (kPrepParticles / 8); task += kPrepThreads) {
      const int rl = task % nrow, g8 = task / nrow;
      const int r = 2 * m0 + rl;
      const int64_t jg = j0 + 8 * g8;
      if (jg >= N) continue;  // K-steps past the last particle stay zero
      uint4 Y[8];
#pragma unroll
      for (int v = 0; v < 8; v++) Y[v] = Ys[(8 * g8 + v) * kPrepPitch + rl];
      const int64_t ks = jg >> 4;
      const int k0 = (int)(jg & 15);
      if (axis == 0)
        put_digit_rows(c.tc_dA + ((int64_t)(r >> 7) * c.tc_KS + ks) * kStageA + slice_off(r & 127, k0), kSliceA, Y);
      else
        put_digit_rows(c.tc_dB + ((int64_t)(r >> 5) * c.tc_KS + ks) * kStageB + slice_off(r & 31, k0), kSliceB, Y);
    }
    // phase 2b (axis 2): particles x 8 values of (m, cos / sin), into the force GEMM's A operand
    if (axis == 1) {
      const int groups = (nrow + 7) / 8;  // 2 m0 is a multiple of 8; a partial last group is padded with zeros
      const uint4 yz = yzero;
      for (int task = tid; task < groups * kPrepParticles; task += kPrepThreads) {
        const int jl = task % kPrepParticles, g = task / kPrepParticles;
        const int64_t j = j0 + jl;
        if (j >= N) continue;
        uint4 Y[8];
#pragma unroll
        for (int v = 0; v < 8; v++) {
          const int rl = 8 * g + v;
          Y[v] = rl < nrow ? Ys[jl * kPrepPitch + rl] : yz;
        }
        const int kf0 = 2 * m0 + 8 * g;
        put_digit_rows(c.tc_fA + ((int64_t)(j >> 7) * c.tc_KSf + (kf0 >> 4)) * kStageA + slice_off((int)(j & 127), kf0 & 15),
                       kSliceA, Y);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------------ k_tc_gemm

// Persistent: CTA b takes items b, b + gridDim.x, ...  Density items: A = density row tile it.a, B = column
// tile it.b, K-steps [ks0, ks0 + nks); the epilogue stores the three int64 level groups of every output into
// tc_part slot it.slot.  Force items: A = particle tile it.a, B = column tile it.b (8 values of n1), every
// K-step; the epilogue writes force partials fpart[2 it.b + half][axis][j].  Stage and accumulator barrier
// phases run on across items, so the producer streams the next item's operands while the epilogue finishes
// the previous item (the accumulator is released as soon as its last level has been read).
__global__ void __launch_bounds__(kGemmThreads, 1) k_tc_gemm(const CfgDev* __restrict__ cfgs,
                                                              const TcItem* __restrict__ items, int n_items) {
  grid_dep_wait();
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t bar_full[kStages], bar_empty[kStages], bar_acc_full, bar_acc_empty, bar_drain;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], 1);
    }
    mbar_init(&bar_acc_full, 1);
    mbar_init(&bar_acc_empty, kEpiWarps);
    mbar_init(&bar_drain, 1);
    abort_sh = 0;
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base_sh, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base_sh;
  volatile int* abort_flag = &abort_sh;

  if (warp == 0) {
    // ---- producer: one thread streams every item's K-steps through the stages
    if (lane == 0) {
      long long gs = 0;  // K-steps issued so far (all items)
      bool stop = false;
      for (int item = blockIdx.x; item < n_items && !stop; item += gridDim.x) {
        const TcItem it = items[item];
        const CfgDev& c = cfgs[it.cfg];
        if (stopped(c)) continue;
        const uint8_t* gA;
        const uint8_t* gB;
        if (it.kind == 0) {
          gA = c.tc_dA + ((int64_t)it.a * c.tc_KS + it.ks0) * kStageA;
          gB = c.tc_dB + ((int64_t)it.b * c.tc_KS + it.ks0) * kStageB;
        } else {
          gA = c.tc_fA + ((int64_t)it.a * c.tc_KSf + it.ks0) * kStageA;
          gB = c.tc_fB + ((int64_t)it.b * c.tc_KSf + it.ks0) * kStageB;
        }
        for (int ks = 0; ks < it.nks; ks++, gs++) {
          const int s = (int)(gs % kStages);
          const long long use = gs / kStages;
          if (use > 0 && !mbar_wait(&bar_empty[s], (uint32_t)((use - 1) & 1), kWaitLimit, abort_flag)) {
            *abort_flag = 1;
            atomicOr(c.tc_err, 1);
            stop = true;
            break;
          }
          uint8_t* dst = smem + (size_t)s * kStageBytes;
          mbar_expect_tx(&bar_full[s], kStageBytes);
          bulk_g2s(dst, gA + (size_t)ks * kStageA, kStageA, &bar_full[s]);
          bulk_g2s(dst + kStageA, gB + (size_t)ks * kStageB, kStageB, &bar_full[s]);
        }
      }
      if (*abort_flag) {
        // let the copies in flight land before the CTA can exit
        for (long long k = gs > kStages ? gs - kStages : 0; k < gs; k++)
          mbar_wait(&bar_full[k % kStages], (uint32_t)((k / kStages) & 1), kWaitLimit, nullptr);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer: 22 MMAs per K-step; level u of the accumulator receives digit slice pairs (s, u - s)
    if (lane == 0) {
      long long gs = 0, gc = 0;  // K-steps and chunks consumed so far (all items)
      bool stop = false;
      for (int item = blockIdx.x; item < n_items && !stop; item += gridDim.x) {
        const TcItem it = items[item];
        const CfgDev& c = cfgs[it.cfg];
        if (stopped(c)) continue;
        for (int ks = 0; ks < it.nks; ks++, gs++) {
          const int s = (int)(gs % kStages);
          const long long use = gs / kStages;
          const bool first = ks % kChunkSteps == 0;
          const bool last = ks % kChunkSteps == kChunkSteps - 1 || ks == it.nks - 1;
          if (!mbar_wait(&bar_full[s], (uint32_t)(use & 1), kWaitLimit, abort_flag)) {
            *abort_flag = 1;
            atomicOr(c.tc_err, 2);
            stop = true;
            break;
          }
          if (first && gc > 0 && !mbar_wait(&bar_acc_empty, (uint32_t)((gc - 1) & 1), kWaitLimit, abort_flag)) {
            *abort_flag = 1;
            atomicOr(c.tc_err, 4);
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(smem + (size_t)s * kStageBytes);
          const uint32_t b0 = a0 + kStageA;
#pragma unroll
          for (int sl = 0; sl < kDigits; sl++) {
            const int ntot = (kLevels - sl) * kTileN;
            const int n1 = ntot < 256 ? ntot : 256;
            const uint32_t acc = (first && sl == 0) ? 0u : 1u;
            const uint64_t ad = make_sdesc(a0 + sl * kSliceA);
            mma_bf16(tbase + sl * kTileN, ad, make_sdesc(b0), make_idesc(kTileM, n1), acc);
            if (ntot > 256)
              mma_bf16(tbase + sl * kTileN + 256, ad, make_sdesc(b0 + 256 * 32), make_idesc(kTileM, ntot - 256), acc);
          }
          mma_commit(&bar_empty[s]);
          if (last) {
            mma_commit(&bar_acc_full);
            gc++;
          }
        }
      }
      // every MMA issued by this thread has completed once the drain barrier flips
      mma_commit(&bar_drain);
      if (!mbar_wait(&bar_drain, 0, kWaitLimit, nullptr)) *abort_flag = 1;
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 and accumulator columns 8 hq .. 8 hq + 7
    const int q = warp & 3, hq = (warp - 2) >> 2;
    const int row = 32 * q + lane;
    const uint32_t trow = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(kEpiCols * hq);
    long long gc = 0;  // chunks read (all items of this CTA)
    bool stop = false;
    for (int item = blockIdx.x; item < n_items && !stop; item += gridDim.x) {
      const TcItem it = items[item];
      const CfgDev& c = cfgs[it.cfg];
      if (stopped(c)) continue;
      long long st[3][kEpiCols];
#pragma unroll
      for (int g = 0; g < 3; g++)
#pragma unroll
        for (int i = 0; i < kEpiCols; i++) st[g][i] = 0;
      const int nch = (it.nks + kChunkSteps - 1) / kChunkSteps;
      for (int ch = 0; ch < nch; ch++, gc++) {
        // the warp leaves together (tcgen05.ld is warp-collective)
        const bool got = mbar_wait(&bar_acc_full, (uint32_t)(gc & 1), kWaitLimit, abort_flag);
        if (!__all_sync(0xffffffffu, got)) {
          *abort_flag = 1;
          if (lane == 0) atomicOr(c.tc_err, 16);
          stop = true;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int g = 0; g < 3; g++) {
          long long t[kEpiCols];
#pragma unroll
          for (int i = 0; i < kEpiCols; i++) t[i] = 0;
          uint32_t r[5][kEpiCols];  // the group's five levels, loaded together, one wait
#pragma unroll
          for (int l = 0; l < 5; l++) tmem_ld8(trow + (uint32_t)((5 * g + l) * kTileN), r[l]);
          tmem_ld_wait();
#pragma unroll
          for (int l = 0; l < 5; l++)
#pragma unroll
            for (int i = 0; i < kEpiCols; i++)
              t[i] += (long long)acc_int(r[l][i]) * (1ll << (7 * (4 - l)));
#pragma unroll
          for (int i = 0; i < kEpiCols; i++) st[g][i] += t[i];
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_acc_empty);
      }
      if (stop) break;
      if (it.kind == 0) {
        // level groups of every output, R' = st0 2^70 + st1 2^35 + st2 (value = R' 2^-110), added into the
        // tile's accumulator: integer addition, so the K ranges combine exactly in any order
        unsigned long long* out = reinterpret_cast<unsigned long long*>(c.tc_acc) + (size_t)it.slot * (3 * kTileN * kTileM);
#pragma unroll
        for (int g = 0; g < 3; g++)
#pragma unroll
          for (int i = 0; i < kEpiCols; i++)
            atomicAdd(out + ((size_t)g * kTileN + kEpiCols * hq + i) * kTileM + row, (unsigned long long)st[g][i]);
      } else {
        // two n1 values per warp, columns (Re G, Im G, Re G', Im G') each.  G~ = R' 2^-110 is taken as R' 2^gs
        // (|.| < 2^126); the top halves of a * G are value 2^(108 + gs), shifted to value 2^ts.
        const int64_t j = (int64_t)it.a * kTileM + row;
        const int gsh = c.tc_gs, tsh = 108 + c.tc_gs - c.tc_ts;
        __int128 F1 = 0, F2 = 0;  // value 2^ts
#pragma unroll
        for (int v = 0; v < kEpiCols / 4; v++) {
          const int n1 = it.b * (kTileN / 4) + hq * (kEpiCols / 4) + v;
          if (n1 > c.tc_R1 || j >= c.N) continue;
          q128 gcol[4];
#pragma unroll
          for (int g4 = 0; g4 < 4; g4++) {
            const int i = 4 * v + g4;
            const __int128 R = ((__int128)st[0][i] << 70) + ((__int128)st[1][i] << 35) + (__int128)st[2][i];
            gcol[g4] = q128_from_i128(R << gsh);
          }
          const fxc a = reinterpret_cast<const fxc*>(c.tc_a1)[(int64_t)n1 * c.N + j];
          uint32_t p[5], r2[5];
          // Im(a G) = Re a Im G + Im a Re G
          smul_top(a.re, gcol[1], p);
          smul_top(a.im, gcol[0], r2);
          __int128 T = (q128_to_i128(q128{{p[1], p[2], p[3], p[4]}}) + q128_to_i128(q128{{r2[1], r2[2], r2[3], r2[4]}})) >> tsh;
          F1 += T * (__int128)n1;
          smul_top(a.re, gcol[3], p);
          smul_top(a.im, gcol[2], r2);
          T = (q128_to_i128(q128{{p[1], p[2], p[3], p[4]}}) + q128_to_i128(q128{{r2[1], r2[2], r2[3], r2[4]}})) >> tsh;
          F2 += T;
        }
        if (j < c.N) {
          // F = L2 2^88 + L1 2^44 + L0 (L0, L1 in [0, 2^44)): the limbs of all column blocks add up exactly
          unsigned long long* fa = reinterpret_cast<unsigned long long*>(c.tc_facc);
          const unsigned long long m44 = (1ull << 44) - 1;
#pragma unroll
          for (int a = 0; a < 2; a++) {
            const __int128 F = a == 0 ? F1 : F2;
            atomicAdd(fa + ((size_t)a * 3 + 0) * c.N + j, (unsigned long long)F & m44);
            atomicAdd(fa + ((size_t)a * 3 + 1) * c.N + j, (unsigned long long)(F >> 44) & m44);
            atomicAdd(fa + ((size_t)a * 3 + 2) * c.N + j, (unsigned long long)(long long)(F >> 88));
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, kTmemCols);
  }
}

// ------------------------------------------------------------------------------------------------ finish

// grid (finish blocks, tensor-core members), 64 threads: n~(n1, m), n~(n1, -m) from the four real products of
// the tile accumulator (which it clears for the next evaluation), as exact Q34.126 values (for the force
// coefficients) and as dd (C, S), with the block's Phi / max |n~|^2 / max |C|, |S| partials.
__global__ void __launch_bounds__(kFinThreads) k_tc_dens_finish(const CfgDev* __restrict__ cfgs,
                                                                const int* __restrict__ list) {
  grid_dep_wait();
  const CfgDev& c = cfgs[list[blockIdx.y]];
  if (stopped(c) || (int)blockIdx.x >= c.tc_nblk) return;  // uniform per block
  RedPart v = {0, 0, 0, 0, 0, 0, 0, 0};
  const int W1 = c.tc_R1 + 1;
  const int64_t idx = (int64_t)blockIdx.x * kFinThreads + threadIdx.x;
  if (idx < (int64_t)W1 * (c.tc_R2 + 1)) {
    const int n1 = (int)(idx % W1), m = (int)(idx / W1);  // n1 fastest: neighbours read neighbouring rows
    const int span = 2 * c.tc_R2 + 1;
    const int kp = c.tc_kmap[(int64_t)n1 * span + (c.tc_R2 + m)];
    const int km = m > 0 ? c.tc_kmap[(int64_t)n1 * span + (c.tc_R2 - m)] : -1;
    const int r = 2 * n1, col = 2 * m;
    const int ti = (kp >= 0 || km >= 0) ? c.tc_tilemap[(r >> 7) * c.tc_CTd + (col >> 5)] : -1;
    if (ti >= 0) {
      const int rr = r & 127, cc = col & 31;
      long long* acc = c.tc_acc + (size_t)ti * (3 * kTileN * kTileM);
      long long P[4][3];  // 0 = cos cos, 1 = cos sin, 2 = sin cos, 3 = sin sin
#pragma unroll
      for (int p = 0; p < 2; p++)
#pragma unroll
        for (int qq = 0; qq < 2; qq++)
#pragma unroll
          for (int g = 0; g < 3; g++) {
            long long* e = acc + ((size_t)g * kTileN + cc + qq) * kTileM + rr + p;
            P[2 * p + qq][g] = *e;
            *e = 0;
          }
      FxAcc* part = reinterpret_cast<FxAcc*>(c.part);
      // C = P_cc + ss_sign P_ss, S = cs_sign P_cs + P_sc
      auto emit = [&](int k, int ss_sign, int cs_sign) {
        i192 C, S;
        i192_zero(C);
        i192_zero(S);
#pragma unroll
        for (int g = 0; g < 3; g++) {
          const int sh = 70 - 35 * g;
          i192_add_shl(C, (__int128)P[0][g] + (ss_sign > 0 ? (__int128)P[3][g] : -(__int128)P[3][g]), sh);
          i192_add_shl(S, (cs_sign > 0 ? (__int128)P[1][g] : -(__int128)P[1][g]) + (__int128)P[2][g], sh);
        }
        FxAcc o;
        o.re = i192_to_q160_shl(C, 16);  // value 2^-110 -> Q34.126
        o.im = i192_to_q160_shl(S, 16);
        part[k] = o;
        const dd cd = i192_to_dd(C, 110), sd = i192_to_dd(S, 110);
        c.C_hi[k] = cd.hi;
        c.C_lo[k] = cd.lo;
        c.S_hi[k] = sd.hi;
        c.S_lo[k] = sd.lo;
        RedPart t;
        const dd a2 = dd_add(dd_sqr(cd), dd_sqr(sd));
        t.phi_hi = a2.hi;
        t.phi_lo = a2.lo;
        t.a2max_hi = a2.hi;
        t.a2max_lo = a2.lo;
        t.cmax = fmax(fabs(cd.hi), fabs(sd.hi));
        red_combine(v, t);
      };
      if (kp >= 0) emit(kp, -1, +1);  // n~(n1, m) = (P_cc - P_ss) + i (P_cs + P_sc)
      if (km >= 0) emit(km, +1, -1);  // n~(n1, -m) = (P_cc + P_ss) + i (P_sc - P_cs)
    }
  }
  red_warp(v);
  __shared__ RedPart sh[kFinThreads / 32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    RedPart a = sh[0];
#pragma unroll
    for (int w = 1; w < kFinThreads / 32; w++) red_combine(a, sh[w]);
    reinterpret_cast<RedPart*>(c.blk)[blockIdx.x] = a;
  }
}

// grid (coordinate blocks, tensor-core members), 64 threads: F[a][j] from the force limbs (which it clears),
// times 4 pi / L and the power-of-two scale of the coefficients
__global__ void __launch_bounds__(kFinThreads) k_tc_force_finish(const CfgDev* __restrict__ cfgs,
                                                                 const int* __restrict__ list) {
  grid_dep_wait();
  const CfgDev& c = cfgs[list[blockIdx.y]];
  if (stopped(c)) return;
  const int64_t i = (int64_t)blockIdx.x * kFinThreads + threadIdx.x;  // over [a][j]
  if (i >= 2 * c.N) return;
  const int a = (int)(i / c.N);
  const int64_t j = i - (int64_t)a * c.N;
  long long* fa = c.tc_facc + (size_t)a * 3 * c.N + j;
  const long long L0 = fa[0], L1 = fa[c.N], L2 = fa[2 * c.N];
  fa[0] = 0;
  fa[c.N] = 0;
  fa[2 * c.N] = 0;
  i192 X;
  i192_zero(X);
  i192_add_shl(X, (__int128)L0, 0);
  i192_add_shl(X, (__int128)L1, 44);
  i192_add_shl(X, (__int128)L2, 88);
  // value = X 2^-ts in units of 2^e (axis 2: of 2^(e + bexp))
  const int e = (int)c.scal[kScScaleExp];
  dd f = dd_mul(i192_to_dd(X, c.tc_ts), c.pref);
  const double sc = pow2(e + (a == 1 ? c.tc_bexp : 0));
  c.F_hi[i] = f.hi * sc;
  c.F_lo[i] = f.lo * sc;
}

// grid ((R1 + 1) (R2 + 1) / 128 blocks, tensor-core members): the force GEMM's coefficient digits
__global__ void k_tc_coef(const CfgDev* __restrict__ cfgs, const int* __restrict__ list) {
  grid_dep_wait();
  const CfgDev& c = cfgs[list[blockIdx.y]];
  if (stopped(c)) return;
  const int W2 = c.tc_R2 + 1;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)(c.tc_R1 + 1) * W2) return;
  const int n1 = (int)(idx / W2), m = (int)(idx % W2);
  const int span = 2 * c.tc_R2 + 1;
  const int kp = c.tc_kmap[(int64_t)n1 * span + (c.tc_R2 + m)];
  const int km = m > 0 ? c.tc_kmap[(int64_t)n1 * span + (c.tc_R2 - m)] : -1;
  const FxAcc* part = reinterpret_cast<const FxAcc*>(c.part);
  const q160 z = q160_zero();
  const q160 Cp = kp >= 0 ? load_q160(&part[kp].re) : z, Sp = kp >= 0 ? load_q160(&part[kp].im) : z;
  const q160 Cm = km >= 0 ? load_q160(&part[km].re) : z, Sm = km >= 0 ? load_q160(&part[km].im) : z;
  const int e = (int)c.scal[kScScaleExp];
  // W = C - i S:  Re U = C+ + C-,  Im U = -(S+ + S-),  Re V = S+ - S-,  Im V = C+ - C-
  //               Re U' = m (C+ - C-), Im U' = -m (S+ - S-), Re V' = m (S+ + S-), Im V' = m (C+ + C-)
  q160 cpl = Cp, cmi = Cp, spl = Sp, smi = Sp;
  q160_add160(cpl, Cm);
  cmi = q160_sub160(Cp, Cm);
  q160_add160(spl, Sm);
  smi = q160_sub160(Sp, Sm);
  const int shG = 22 + e, shW = 22 + e + c.tc_bexp;
  __int128 X[4][2];
  X[0][0] = q160_shr_round(cpl, shG);
  X[0][1] = q160_shr_round(smi, shG);
  X[1][0] = -q160_shr_round(spl, shG);
  X[1][1] = q160_shr_round(cmi, shG);
  X[2][0] = q160_shr_round(q160_mul_int(cmi, m), shW);
  X[2][1] = q160_shr_round(q160_mul_int(spl, m), shW);
  X[3][0] = -q160_shr_round(q160_mul_int(smi, m), shW);
  X[3][1] = q160_shr_round(q160_mul_int(cpl, m), shW);
  if (m == 0) {  // sin(0) = 0 and the weight n2 = 0
    X[0][1] = X[1][1] = 0;
    X[2][0] = X[2][1] = X[3][0] = X[3][1] = 0;
  }
#pragma unroll
  for (int g = 0; g < 4; g++) {
    const int col = 4 * n1 + g;
#pragma unroll
    for (int qq = 0; qq < 2; qq++) {
      const int kf = 2 * m + qq;
      uint8_t* base = c.tc_fB + ((int64_t)(col >> 5) * c.tc_KSf + (kf >> 4)) * kStageB;
      put_digits_x(base, kSliceB, slice_off(col & 31, kf & 15), X[g][qq]);
    }
  }
}

// ------------------------------------------------------------------------------------------------ host side

static cudaError_t tc_dev_alloc(DevBuf* b, size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 16;
  b->bytes = bytes;
  cudaError_t e = cudaMalloc(&b->p, bytes);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(b->p, 0, bytes, st);  // padding rows, columns and K stay zero for good
}

bool tc_eligible(const Ctx& c) { return c.d == 2 && c.N >= 1 && c.M >= 1; }

int tc_finish_blocks(const Ctx& c) {
  if (!c.tc.on) return 0;
  return (int)(((int64_t)(c.tc.R1 + 1) * (c.tc.R2 + 1) + kFinThreads - 1) / kFinThreads);
}

// Tile plan and device buffers of one configuration.
cudaError_t tc_setup(Ctx* c) {
  TcPlan& t = c->tc;
  t = TcPlan();
  if (!c->tc_requested || !tc_eligible(*c)) return cudaSuccess;
  const KSet& ks = c->ks;
  t.R1 = std::max(0, ks.nmax[0]);
  t.R2 = std::max(std::abs(ks.nmin[1]), std::abs(ks.nmax[1]));
  t.KS = (c->N + kStepK - 1) / kStepK;
  t.RT = (2 * (t.R1 + 1) + kTileM - 1) / kTileM;
  t.CTd = (2 * (t.R2 + 1) + kTileN - 1) / kTileN;
  t.PT = (int)((c->N + kTileM - 1) / kTileM);
  t.KSf = (2 * (t.R2 + 1) + kStepK - 1) / kStepK;
  t.CTf = (4 * (t.R1 + 1) + kTileN - 1) / kTileN;
  t.bexp = 0;
  while ((1 << t.bexp) <= t.R2) t.bexp++;
  const int span = 2 * t.R2 + 1;
  t.kmap.assign((size_t)(t.R1 + 1) * span, -1);
  t.tilemap.assign((size_t)t.RT * t.CTd, -1);
  for (int64_t k = 0; k < c->M; k++) {
    const int n1 = ks.n_int[2 * k], n2 = ks.n_int[2 * k + 1];
    t.kmap[(size_t)n1 * span + (n2 + t.R2)] = (int32_t)k;
    const int ti = ((2 * n1) >> 7) * t.CTd + ((2 * std::abs(n2)) >> 5);
    t.tilemap[ti] = 1;
  }
  t.tiles.clear();
  for (int i = 0; i < t.RT * t.CTd; i++)
    if (t.tilemap[i] >= 0) {
      t.tilemap[i] = (int32_t)t.tiles.size();
      t.tiles.push_back(i);
    }
  const int nt = (int)t.tiles.size();
  const int64_t max_split = std::max<int64_t>(1, t.KS / kChunkSteps);
  // one CTA per SM: as many K ranges per tile as fit in a single wave
  t.ksplit = (int)std::max<int64_t>(1, std::min<int64_t>(max_split, c->sm_count / std::max(1, nt)));
  // each K range holds at most 1024 read-outs, so the int64 level groups (below 2^52 per read-out) cannot overflow
  t.ksplit = (int)std::max<int64_t>(t.ksplit, (t.KS + 1024 * kChunkSteps - 1) / (1024 * kChunkSteps));
  cudaStream_t st = c->stream;
  cudaError_t e;
  if ((e = tc_dev_alloc(&t.dA, (size_t)t.RT * t.KS * kStageA, st)) != cudaSuccess) return e;
  if ((e = tc_dev_alloc(&t.dB, (size_t)t.CTd * t.KS * kStageB, st)) != cudaSuccess) return e;
  if ((e = tc_dev_alloc(&t.fA, (size_t)t.PT * t.KSf * kStageA, st)) != cudaSuccess) return e;
  if ((e = tc_dev_alloc(&t.fB, (size_t)t.CTf * t.KSf * kStageB, st)) != cudaSuccess) return e;
  if ((e = tc_dev_alloc(&t.a1, (size_t)(t.R1 + 1) * c->N * sizeof(fxc), st)) != cudaSuccess) return e;
  t.ntab = kPrepLow + std::max(t.R1, t.R2) / kPrepLow + 1;
  if ((e = tc_dev_alloc(&t.tab, (size_t)2 * c->N * t.ntab * sizeof(qent), st)) != cudaSuccess) return e;
  if ((e = tc_dev_alloc(&t.acc, (size_t)nt * 3 * kTileN * kTileM * 8, st)) != cudaSuccess) return e;
  if ((e = tc_dev_alloc(&t.facc, (size_t)2 * 3 * c->N * 8, st)) != cudaSuccess) return e;
  if ((e = tc_dev_alloc(&t.kmap_d, t.kmap.size() * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(t.kmap_d.p, t.kmap.data(), t.kmap.size() * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  if ((e = tc_dev_alloc(&t.tilemap_d, t.tilemap.size() * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(t.tilemap_d.p, t.tilemap.data(), t.tilemap.size() * 4, cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return e;
  if ((e = tc_dev_alloc(&t.err, 16, st)) != cudaSuccess) return e;
  // force epilogue scales: G~ (|.| <= 2 (R2 + 1)) held as R' 2^gs below 2^126; partial sums of four n1 terms
  // weighted by n1 <= R1 held at value 2^ts below 2^126
  int lg = 0;
  while ((1ll << lg) < 2ll * (t.R2 + 1)) lg++;
  t.gs = 16 - lg;
  int lf = 0;
  while ((1ll << lf) < 4ll * std::max(1, t.R1) * 2ll * (t.R2 + 1)) lf++;
  t.ts = 126 - lf;
  if (t.gs < 1 || t.ts < 64) return cudaErrorInvalidValue;  // wavevector range beyond the scales used here
  t.on = true;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
    cudaFuncSetAttribute(k_tc_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPrepSmem);
    attr = true;
  }
  return cudaGetLastError();
}

void tc_free(Ctx* c) {
  TcPlan& t = c->tc;
  for (DevBuf* b : {&t.dA, &t.dB, &t.fA, &t.fB, &t.a1, &t.tab, &t.acc, &t.facc, &t.kmap_d, &t.tilemap_d, &t.err}) {
    if (b->p) cudaFree(b->p);
    b->p = nullptr;
    b->bytes = 0;
  }
  t.on = false;
}

size_t tc_footprint(const Ctx& c) {
  const TcPlan& t = c.tc;
  if (!t.on) return 0;
  return t.dA.bytes + t.dB.bytes + t.fA.bytes + t.fB.bytes + t.a1.bytes + t.tab.bytes + t.acc.bytes + t.facc.bytes + t.kmap_d.bytes +
         t.tilemap_d.bytes;
}

void tc_fill_cfgdev(const Ctx* c, CfgDev* g) {
  const TcPlan& t = c->tc;
  g->tc = t.on ? 1 : 0;
  if (!t.on) return;
  g->tc_R1 = t.R1;
  g->tc_R2 = t.R2;
  g->tc_RT = t.RT;
  g->tc_CTd = t.CTd;
  g->tc_PT = t.PT;
  g->tc_KSf = t.KSf;
  g->tc_CTf = t.CTf;
  g->tc_bexp = t.bexp;
  g->tc_ksplit = t.ksplit;
  g->tc_KS = t.KS;
  g->tc_dA = (uint8_t*)t.dA.p;
  g->tc_dB = (uint8_t*)t.dB.p;
  g->tc_fA = (uint8_t*)t.fA.p;
  g->tc_fB = (uint8_t*)t.fB.p;
  g->tc_a1 = t.a1.p;
  g->tc_tab = t.tab.p;
  g->tc_ntab = t.ntab;
  g->tc_acc = (long long*)t.acc.p;
  g->tc_facc = (long long*)t.facc.p;
  g->tc_nblk = tc_finish_blocks(*c);
  g->tc_kmap = (const int32_t*)t.kmap_d.p;
  g->tc_tilemap = (const int32_t*)t.tilemap_d.p;
  g->tc_err = (int*)t.err.p;
  g->tc_gs = t.gs;
  g->tc_ts = t.ts;
  g->psplit[SSH_FX] = 1;
}

// work items of one member (engine member index i)
void tc_items(const Ctx* c, int i, std::vector<TwItem>& prep, std::vector<TcItem>& dens, std::vector<TcItem>& force) {
  const TcPlan& t = c->tc;
  for (int axis = 0; axis < 2; axis++)
    for (int64_t j = 0; j < c->N; j += kPrepParticles) prep.push_back({i, axis, j});  // one K-step each
  for (int ti = 0; ti < (int)t.tiles.size(); ti++) {
    const int rt = t.tiles[ti] / t.CTd, ct = t.tiles[ti] % t.CTd;
    for (int sp = 0; sp < t.ksplit; sp++) {
      const int64_t k0 = t.KS * sp / t.ksplit, k1 = t.KS * (sp + 1) / t.ksplit;
      dens.push_back({i, 0, rt, ct, (int32_t)k0, (int32_t)(k1 - k0), ti, 0});
    }
  }
  // force items: column tile ct holds n1 in [8 ct, 8 ct + 8); its K range (m, cos / sin) stops at the largest m
  // with (n1, +-m) in the set for one of those n1 (the coefficients beyond are zero).  Largest items first, so
  // the round-robin assignment to the persistent CTAs balances.
  const int span = 2 * t.R2 + 1;
  std::vector<int> ks_of(t.CTf, 0);
  for (int ct = 0; ct < t.CTf; ct++) {
    int mmax = -1;
    for (int n1 = 8 * ct; n1 < std::min(8 * ct + 8, t.R1 + 1); n1++)
      for (int m = 0; m <= t.R2; m++)
        if (t.kmap[(size_t)n1 * span + t.R2 + m] >= 0 || t.kmap[(size_t)n1 * span + t.R2 - m] >= 0) mmax = std::max(mmax, m);
    ks_of[ct] = mmax < 0 ? 0 : (2 * (mmax + 1) + kStepK - 1) / kStepK;
  }
  std::vector<TcItem> fi;
  for (int pt = 0; pt < t.PT; pt++)
    for (int ct = 0; ct < t.CTf; ct++)
      if (ks_of[ct] > 0) fi.push_back({i, 1, pt, ct, 0, ks_of[ct], ct, 0});
  std::stable_sort(fi.begin(), fi.end(), [](const TcItem& a, const TcItem& b) { return a.nks > b.nks; });
  force.insert(force.end(), fi.begin(), fi.end());
}

size_t tc_gemm_smem() { return kGemmSmem; }

cudaError_t tc_launch_force_finish(const EngineView& v, cudaStream_t st, Prof* prof) {
  if (v.ntc_list == 0) return cudaSuccess;
  prof_begin(prof, st, kKTcFinish);
  const dim3 g((unsigned)std::max<int64_t>(1, (v.maxND + kFinThreads - 1) / kFinThreads), (unsigned)v.ntc_list);
  cudaError_t le = launch_pdl(k_tc_force_finish, g, dim3(kFinThreads), 0, st, v.cfgs, v.tc_list);
  if (le != cudaSuccess) return le;
  prof_end(prof, st);
  return cudaGetLastError();
}

cudaError_t tc_launch_density(const EngineView& v, cudaStream_t st, Prof* prof) {
  if (v.ntc_list == 0) return cudaSuccess;
  prof_begin(prof, st, kKTcPrep);
  cudaError_t le = launch_pdl(k_tc_tables, dim3((unsigned)std::max<int64_t>(1, (v.maxND + 127) / 128), (unsigned)v.ntc_list),
                              dim3(128), 0, st, v.cfgs, v.tc_list);
  if (le == cudaSuccess)
    le = launch_pdl(k_tc_prep, dim3((unsigned)v.ntc_prep), dim3(kPrepThreads), kPrepSmem, st, v.cfgs, v.tc_prep);
  if (le != cudaSuccess) return le;
  prof_end(prof, st);
  prof_begin(prof, st, kKTcDens);
  le = launch_pdl(k_tc_gemm, dim3((unsigned)std::min(v.ntc_dens, v.sm_count)), dim3(kGemmThreads), kGemmSmem, st, v.cfgs,
                  v.tc_dens, v.ntc_dens);
  if (le != cudaSuccess) return le;
  prof_end(prof, st);
  prof_begin(prof, st, kKTcFinish);
  const dim3 g((unsigned)std::max<int64_t>(1, (v.tc_max_grid + kFinThreads - 1) / kFinThreads), (unsigned)v.ntc_list);
  le = launch_pdl(k_tc_dens_finish, g, dim3(kFinThreads), 0, st, v.cfgs, v.tc_list);
  if (le != cudaSuccess) return le;
  prof_end(prof, st);
  return cudaGetLastError();
}

cudaError_t tc_launch_force(const EngineView& v, cudaStream_t st, Prof* prof) {
  if (v.ntc_list == 0) return cudaSuccess;
  prof_begin(prof, st, kKTcCoef);
  const dim3 g((unsigned)std::max<int64_t>(1, (v.tc_max_grid + 127) / 128), (unsigned)v.ntc_list);
  cudaError_t le = launch_pdl(k_tc_coef, g, dim3(128), 0, st, v.cfgs, v.tc_list);
  if (le != cudaSuccess) return le;
  prof_end(prof, st);
  prof_begin(prof, st, kKTcForce);
  le = launch_pdl(k_tc_gemm, dim3((unsigned)std::min(v.ntc_force, v.sm_count)), dim3(kGemmThreads), kGemmSmem, st, v.cfgs,
                  v.tc_force, v.ntc_force);
  if (le != cudaSuccess) return le;
  prof_end(prof, st);
  return cudaGetLastError();
}

}  // namespace ssh
