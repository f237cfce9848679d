// tc.cu -- the fixed-point hot path for d = 2, 3 and 4 on the tensor cores (Eqs. ntilde and force of
// arXiv:2304.09139; d = 1 runs on two lifted axes).
//
// Write a wavevector as n = (n1, p), p = (n2), (n2, n3) or (n2, n3, n4), and the phasor of particle j per factor:
// a_j(n1) = e^{2 pi i n1 s_j1}, w_j(p) = e^{2 pi i p . (s_j2, .., s_jd)}.  The collective density is then a matrix
// product over the particles, n~(n1, p) = sum_j a_j(n1) w_j(p).  The half set H (first non-zero component > 0)
// has n1 >= 0; p runs over a half of its space, P = {p : the last non-zero component of p is > 0, or p = 0}
// ("canonical" p), since every k in H is (n1, p) or (n1, -p) with p in P.  As a_j(-n1) = conj(a_j(n1)), the four real products
// P_xy(p, n1) = sum_j x_j(p) y_j(n1) (x the cos / sin of w, y of a) give
//   n~(n1, p)  = (P_cc - P_ss) + i (P_sc + P_cs),
//   n~(n1, -p) = conj n~(-n1, p) = (P_cc + P_ss) + i (P_cs - P_sc):
// one real GEMM with rows (p, cos / sin), columns (n1, cos / sin) and K = particles.  For d = 3, w_j(p) is the
// product b_j(n2) c_j(n3) of the axis-2 and axis-3 powers, for d = 4 b_j(n2) c_j(n3) e_j(n4), formed once per
// particle and p.
//
// The force F_j = (4 pi / L) sum_k n [C sin th - S cos th] = (4 pi / L) Im sum_k n W_k e^{i th_jk}, W = C - i S,
// is grouped per n1: G_j(n1) = sum_{p in P} [U(n1, p) cos(2 pi p . s_j) + V(n1, p) sin(2 pi p . s_j)] with
// U = W(n1, p) + W(n1, -p), V = i (W(n1, p) - W(n1, -p)) (W = 0 off the set; p = 0 counted once), and
// G^a_j(n1) with the weight n_a (a >= 2): U^a = n_a (W(n1, p) - W(n1, -p)), V^a = i n_a (W(n1, p) + W(n1, -p)).
// Rows = particles, K = (p, cos / sin), columns = (n1, axis, Re / Im); the epilogue forms
// F_j1 = (4 pi / L) Im sum n1 a_j(n1) G_j(n1) and F_ja = (4 pi / L) Im sum a_j(n1) G^a_j(n1).
//
// Both products use the exact digit arithmetic of tc.cuh: operands are 15 bf16 digit slices, the 120 kept
// digit pairs accumulate into 15 TMEM level accumulators, read out exactly every 256 products.  The digits of
// w are written once, as a 4-D tensor [slice][row group][particle group][8 x 8 core] (a core: 8 rows (p, cos /
// sin) x 8 particles, particles contiguous); the density GEMM reads it through a tensor-map box as its K-major A
// operand (rows (p, cos / sin), K = particles) and the force GEMM through a second box as its MN-major A operand
// (rows = particles, K = (p, cos / sin)).
//
// Kernels (one launch each per evaluation, over every tensor-core member of the engine):
//   k_tc_tables       per (particle, axis): e^{2 pi i k s} (k < 8) and e^{2 pi i 8 b s} as first-quadrant phasors
//   k_tc_prep         per particle block: a_j(n1) as digit slices of the density B operand and as Q2.126 for the
//                     force epilogue; w_j(p) as the digit tensor
//   k_tc_gemm         warp-specialised persistent tcgen05 GEMM: one producer thread (tensor-map and bulk async
//                     copies, three stages), one MMA thread (22 MMAs per K-step), sixteen epilogue warps (level
//                     read-out, exact folding, integer atomics)
//   k_tc_dens_finish  the four real products -> n~(k) as Q34.126 partials and dd (C, S), Phi / S_max partials
//   k_tc_coef         U, V, U^a, V^a from the exact n~ and the power-of-two scale, as digit slices of the force GEMM
//   k_tc_force_finish force limbs -> dd F
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>

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
constexpr size_t kGemmSmem = (size_t)kStages * kStageBytes + 128;  // + alignment slack of the stages
constexpr int kFinThreads = 64;
constexpr int kRing = 8;                           // item indices in flight between the producer and consumers

__device__ __forceinline__ bool stopped(const CfgDev& c) { return c.run && *c.run; }

// Limit of the GEMM's waits on work (stages, items, the accumulator), in clock cycles; ssh_set_wait_limit changes
// it.  The waits that let copies and MMAs in flight land before a CTA exits always use kWaitLimit.
__device__ long long g_tc_wait_limit = kWaitLimit;

// Cycle counters of the GEMM (ssh_gemm_counters): one record of kGcFields words per CTA and launch kind (density,
// force), written by the counting instance of k_tc_gemm only.  The production instance has none of this code.
constexpr int kGcCtas = 256, kGcFields = 16;
__device__ unsigned long long g_tc_counters[2][kGcCtas][kGcFields];
// on for this process between ssh_gemm_counters(.., 1) and (.., 0): GEMM launches use the counting instance (an
// atomic, since a server's worker thread may launch while another thread switches it)
std::atomic<bool> g_counters_on{false};
enum { kGcCycles = 0, kGcProdWaitStage, kGcMmaWaitOperands, kGcMmaWaitAcc, kGcMmaWaitItem, kGcEpiWaitAcc,
       kGcEpiRead, kGcEpiMath, kGcItems, kGcKsteps, kGcMmaCycles, kGcT0, kGcT1 };
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// A wait gave up: record `code` in the error word of every configuration with items in this launch, since the
// items this CTA had claimed or published (and so skips) may belong to any of them.
__device__ __noinline__ void tc_flag_all(const CfgDev* __restrict__ cfgs, const TcItem* __restrict__ items,
                                         int n_items, int code) {
  int last = -1;
  for (int i = 0; i < n_items; i++) {
    const int ci = items[i].cfg;
    if (ci == last) continue;
    last = ci;
    const CfgDev& c = cfgs[ci];
    if (!stopped(c) && c.tc_err) atomicOr(c.tc_err, code);
  }
}

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

// The 15 balanced digits of two values X0, X1 (|X| <= 2^104) as bf16 pairs, one 32-bit word per slice (X0 in the
// low half), slice s holding digit 14 - s (top digit first).  Digit i < 14 is d = u - 64 with u the bits 7i..7i+6
// of X + B (B the balanced-digit offset); the bf16 of 192 + d is 0x4300 | u, so one packed bf16 subtraction of
// 192 gives both digits exactly.  The top digit, the signed bits 98..127 (it may be 64), goes through fp32.
__device__ __forceinline__ void put_digit_pair(uint8_t* base, uint32_t slice_stride, uint32_t off, __int128 X0,
                                               __int128 X1) {
  const unsigned __int128 Y0 = (unsigned __int128)(X0 + digit_bias()), Y1 = (unsigned __int128)(X1 + digit_bias());
  {
    const uint32_t f0 = __float_as_uint(__int_as_float(kMagicBits + (int)((__int128)Y0 >> 98)) - kMagic);
    const uint32_t f1 = __float_as_uint(__int_as_float(kMagicBits + (int)((__int128)Y1 >> 98)) - kMagic);
    *reinterpret_cast<uint32_t*>(base + off) = __byte_perm(f0, f1, 0x7632);
  }
  const __nv_bfloat162 b192 = __halves2bfloat162(__ushort_as_bfloat16((unsigned short)0x4340),
                                                 __ushort_as_bfloat16((unsigned short)0x4340));
#pragma unroll
  for (int s = 1; s < kDigits; s++) {
    const int i = kDigits - 1 - s;
    const uint32_t u0 = (uint32_t)(Y0 >> (7 * i)) & 127u, u1 = (uint32_t)(Y1 >> (7 * i)) & 127u;
    const uint32_t t = u0 | (u1 << 16) | 0x43004300u;
    const __nv_bfloat162 r = __hsub2(*reinterpret_cast<const __nv_bfloat162*>(&t), b192);
    *reinterpret_cast<uint32_t*>(base + (size_t)s * slice_stride + off) = *reinterpret_cast<const uint32_t*>(&r);
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
// a << sh (0 <= sh < 64), two's complement
__device__ __forceinline__ i192 i192_shl(const i192& a, int sh) {
  if (sh == 0) return a;
  i192 r;
  r.w[2] = (a.w[2] << sh) | (a.w[1] >> (64 - sh));
  r.w[1] = (a.w[1] << sh) | (a.w[0] >> (64 - sh));
  r.w[0] = a.w[0] << sh;
  return r;
}
__device__ __forceinline__ i192 i192_add(const i192& a, const i192& b) {
  const unsigned __int128 a01 = ((unsigned __int128)a.w[1] << 64) | a.w[0];
  const unsigned __int128 s01 = a01 + (((unsigned __int128)b.w[1] << 64) | b.w[0]);
  i192 r;
  r.w[0] = (unsigned long long)s01;
  r.w[1] = (unsigned long long)(s01 >> 64);
  r.w[2] = a.w[2] + b.w[2] + (s01 < a01 ? 1ull : 0ull);
  return r;
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

// a += round(x 2^126) for a double with |x| < 2^33 (round half up; terms below 2^-190 are dropped)
__device__ __forceinline__ void i192_add_double_126(i192& a, double x) {
  if (x == 0.0) return;
  int ex;
  const double fr = frexp(x, &ex);                 // x = fr 2^ex, 1/2 <= |fr| < 1
  const long long m = (long long)ldexp(fr, 53);     // exact: x = m 2^(ex - 53)
  const int sh = ex - 53 + 126;
  if (sh >= 0) {
    i192_add_shl(a, (__int128)m, sh);
  } else if (sh > -62) {
    i192_add_shl(a, (__int128)((m + (1ll << (-sh - 1))) >> (-sh)), 0);
  }
}

// 2^e as a double (normal range)
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// 320-bit unsigned integer, five little-endian 64-bit words: exact sums of |n~|^2 in units of 2^-220
struct u320 {
  unsigned long long w[5];
};
__device__ __forceinline__ void u320_zero(u320& a) {
#pragma unroll
  for (int i = 0; i < 5; i++) a.w[i] = 0ull;
}
__device__ __forceinline__ void u320_add(u320& a, const u320& b) {
  unsigned long long cy = 0;
#pragma unroll
  for (int i = 0; i < 5; i++) {
    const unsigned __int128 t = (unsigned __int128)a.w[i] + b.w[i] + cy;
    a.w[i] = (unsigned long long)t;
    cy = (unsigned long long)(t >> 64);
  }
}
// a += v 2^(64 i) (the sum stays below 2^320)
__device__ __forceinline__ void u320_add_at(u320& a, int i, unsigned __int128 v) {
  unsigned long long add[5] = {0ull, 0ull, 0ull, 0ull, 0ull};
  add[i] = (unsigned long long)v;
  if (i + 1 < 5) add[i + 1] = (unsigned long long)(v >> 64);
  u320 b;
#pragma unroll
  for (int k = 0; k < 5; k++) b.w[k] = add[k];
  u320_add(a, b);
}
// x^2 of a 192-bit two's-complement integer with |x| < 2^159
__device__ __forceinline__ u320 u320_sq(const i192& x) {
  unsigned long long a0 = x.w[0], a1 = x.w[1], a2 = x.w[2];
  if ((long long)a2 < 0) {  // |x|
    a0 = ~a0;
    a1 = ~a1;
    a2 = ~a2;
    a0 += 1ull;
    const unsigned long long c0 = a0 == 0ull ? 1ull : 0ull;
    a1 += c0;
    a2 += (c0 && a1 == 0ull) ? 1ull : 0ull;
  }
  // x^2 = a0^2 + 2 a0 a1 2^64 + (a1^2 + 2 a0 a2) 2^128 + 2 a1 a2 2^192 + a2^2 2^256
  u320 r;
  u320_zero(r);
  const unsigned __int128 p01 = (unsigned __int128)a0 * a1, p02 = (unsigned __int128)a0 * a2,
                          p12 = (unsigned __int128)a1 * a2;
  u320_add_at(r, 0, (unsigned __int128)a0 * a0);
  u320_add_at(r, 1, p01);
  u320_add_at(r, 1, p01);
  u320_add_at(r, 2, (unsigned __int128)a1 * a1);
  u320_add_at(r, 2, p02);
  u320_add_at(r, 2, p02);
  u320_add_at(r, 3, p12);
  u320_add_at(r, 3, p12);
  r.w[4] += a2 * a2;
  return r;
}
// word q of a little-endian array of n words (0 outside), by selects: no indexed access to registers
template <int n>
__device__ __forceinline__ unsigned long long word_at(const unsigned long long (&w)[n], int q) {
  unsigned long long v = 0ull;
#pragma unroll
  for (int k = 0; k < n; k++) v = k == q ? w[k] : v;
  return v;
}
// 64 bits of x from bit b up (b may be negative: zeros shifted in below bit 0)
__device__ __forceinline__ unsigned long long u320_bits(const u320& x, int b) {
  if (b <= -64) return 0ull;
  if (b < 0) return x.w[0] << (-b);
  const int q = b >> 6, r = b & 63;
  const unsigned long long lo = word_at(x.w, q), hi = word_at(x.w, q + 1);
  return r ? (lo >> r) | (hi << (64 - r)) : lo;
}
// x 2^-S as a double-double from the top 106 bits of x (the bits below are dropped: relative error < 2^-105);
// S - 320 >= -1022 keeps both words normal
__device__ __forceinline__ dd u320_to_dd(const u320& x, int S) {
  int t = 0;
#pragma unroll
  for (int k = 1; k < 5; k++) t = x.w[k] != 0ull ? k : t;
  const unsigned long long top = word_at(x.w, t);
  if (top == 0ull) return dd_make(0.0);
  const int lead = 64 * t + 63 - __clzll((long long)top);
  const unsigned long long m53 = (1ull << 53) - 1;
  const unsigned long long h = u320_bits(x, lead - 52) & m53, l = u320_bits(x, lead - 105) & m53;
  return fast_two_sum((double)h * pow2(lead - 52 - S), (double)l * pow2(lead - 105 - S));
}
// round(x w) for a weight 0 <= w <= 1024 (round half up; x w < 2^320)
__device__ __forceinline__ u320 u320_mul_weight(const u320& x, double w) {
  u320 r;
  u320_zero(r);
  if (!(w > 0.0)) return r;
  int ex;
  const double fr = frexp(w, &ex);                                  // w = fr 2^ex, 1/2 <= fr < 1
  const unsigned long long m = (unsigned long long)ldexp(fr, 53);  // exact: w = m 2^(ex - 53)
  unsigned long long y[6];
  unsigned long long cy = 0;
#pragma unroll
  for (int i = 0; i < 5; i++) {
    const unsigned __int128 t = (unsigned __int128)x.w[i] * m + cy;
    y[i] = (unsigned long long)t;
    cy = (unsigned long long)(t >> 64);
  }
  y[5] = cy;
  const int sh = 53 - ex;  // >= 42
  if (sh >= 6 * 64) return r;
  {  // + 2^(sh - 1)
    const int q = (sh - 1) >> 6;
    unsigned long long c = 0ull;
#pragma unroll
    for (int i = 0; i < 6; i++) {
      const unsigned long long o = y[i], a = (i == q ? 1ull << ((sh - 1) & 63) : 0ull) + c;
      y[i] = o + a;
      c = y[i] < o ? 1ull : 0ull;
    }
  }
  const int q = sh >> 6, b = sh & 63;
#pragma unroll
  for (int i = 0; i < 5; i++) {
    const unsigned long long lo = word_at(y, i + q), hi = word_at(y, i + q + 1);
    r.w[i] = b ? (lo >> b) | (hi << (64 - b)) : lo;
  }
  return r;
}

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
constexpr int kPrepStaged = 16;     // particles per d >= 3 w item (their axis powers staged in shared memory)
constexpr int kPrepTable = 128;     // at most this many particles per table item (a(n1); w of d = 1, 2)
constexpr int kPrepLow = 8;         // e^{2 pi i m s} = A[m / 8] T[m % 8]
constexpr size_t kPrepSmemMax = 200 * 1024;

// the components of a packed canonical p: (n2 & 0xffff) | n3 << 16 on two or three axes, 10-bit fields
// n2 | n3 << 10 | n4 << 20 on four (each sign-extended)
__device__ __forceinline__ void unpack_p(int32_t pv, int d, int& n2, int& n3, int& n4) {
  if (d == 4) {
    n2 = (int32_t)((uint32_t)pv << 22) >> 22;
    n3 = (int32_t)((uint32_t)pv << 12) >> 22;
    n4 = (int32_t)((uint32_t)pv << 2) >> 22;
  } else {
    n2 = (int)(int16_t)(pv & 0xffff);
    n3 = pv >> 16;
    n4 = 0;
  }
}

// conj of a first-quadrant phasor: conj(i^q (c + i s)) = i^{-q} (c - i s) = i^{3 - q} (s + i c)
__device__ __forceinline__ qent qconj(const qent& z) {
  qent r;
  r.c = z.s;
  r.s = z.c;
  r.cs = z.cs;
  r.cs.w[0] = (z.cs.w[0] & ~3u) | ((3u - (z.cs.w[0] & 3u)) & 3u);
  return r;
}

// Eight biased values Y = X + B (X = round(x 2^104), B the balanced-digit offset) -> their 15 digits as one
// 16-byte row (8 bf16) per digit slice, slice s holding digit 14 - s.  Digit i < 14 is d = u - 64 with u the
// bits 7i..7i+6 of Y; the bf16 of 192 + d = 128 + u is 0x4300 | u (exponent 2^7, mantissa u), so one packed
// bf16 subtraction of 192 gives two digits exactly.  The top digit, the signed bits 98..127 (it may be 64), is
// converted through fp32.  With base2 set, every row is also stored at base2 (slices slice_stride2 apart): the digits
// are formed once.
__device__ __forceinline__ void put_digit_rows(uint8_t* base, size_t slice_stride, const uint4 (&Y)[8],
                                               uint8_t* base2 = nullptr, size_t slice_stride2 = 0) {
  {
    uint32_t f[8];
#pragma unroll
    for (int v = 0; v < 8; v++) {
      const int d = (int32_t)Y[v].w >> 2;
      // small integer -> fp32 (exact) whose upper half is the bf16 of the same value
      f[v] = __float_as_uint(__int_as_float(kMagicBits + d) - kMagic);
    }
    uint4 row;
    row.x = __byte_perm(f[0], f[1], 0x7632);
    row.y = __byte_perm(f[2], f[3], 0x7632);
    row.z = __byte_perm(f[4], f[5], 0x7632);
    row.w = __byte_perm(f[6], f[7], 0x7632);
    *reinterpret_cast<uint4*>(base) = row;
    if (base2) *reinterpret_cast<uint4*>(base2) = row;
  }
  const __nv_bfloat162 b192 = __halves2bfloat162(__ushort_as_bfloat16((unsigned short)0x4340),
                                                 __ushort_as_bfloat16((unsigned short)0x4340));
#pragma unroll
  for (int s = 1; s < kDigits; s++) {
    const int o = 7 * (kDigits - 1 - s);
    const int lo = o >> 5, hi = lo + 1 < 4 ? lo + 1 : 3;
    uint32_t wv[4];
#pragma unroll
    for (int pr = 0; pr < 4; pr++) {
      const uint32_t a0[4] = {Y[2 * pr].x, Y[2 * pr].y, Y[2 * pr].z, Y[2 * pr].w};
      const uint32_t a1[4] = {Y[2 * pr + 1].x, Y[2 * pr + 1].y, Y[2 * pr + 1].z, Y[2 * pr + 1].w};
      const uint32_t u0 = __funnelshift_r(a0[lo], a0[hi], o & 31), u1 = __funnelshift_r(a1[lo], a1[hi], o & 31);
      const uint32_t t = (__byte_perm(u0, u1, 0x5410) & 0x007F007Fu) | 0x43004300u;
      const __nv_bfloat162 r = __hsub2(*reinterpret_cast<const __nv_bfloat162*>(&t), b192);
      wv[pr] = *reinterpret_cast<const uint32_t*>(&r);
    }
    const uint4 row = make_uint4(wv[0], wv[1], wv[2], wv[3]);
    *reinterpret_cast<uint4*>(base + (size_t)s * slice_stride) = row;
    if (base2) *reinterpret_cast<uint4*>(base2 + (size_t)s * slice_stride2) = row;
  }
}

// The product z b of two first-quadrant phasors -> (re, im) as round(x 2^104) + balanced-digit offset, and as
// signed Q2.126.  The three products of qmul give (re, im), im >= 0 (clamped at 0 as there); the product is
// i^(q1 + q2) (re + i im), turned without renormalising to the first quadrant, and each signed component is
// rounded to the nearest multiple of 2^-104 (ties upward; error at most 2^-105).
__device__ __forceinline__ void qmul_out(const qent& z, const qent& b, uint4& yre, uint4& yim, fxc* q126) {
  const q128 p1 = umulhi(z.c, b.c), p2 = umulhi(z.s, b.s), p3 = umulhi(z.cs, b.cs);
  const q128 re = q128_sub(p1, p2);
  q128 im = q128_sub(q128_sub(p3, p1), p2);
  if ((int32_t)im.w[3] < 0) im = q128_zero();
  const uint32_t q = (z.cs.w[0] + b.cs.w[0]) & 3u;
  const __int128 R = q128_to_i128(re), I = q128_to_i128(im);
  __int128 xr, xi;
  switch (q) {  // i^q (R + i I)
    case 0: xr = R; xi = I; break;
    case 1: xr = -I; xi = R; break;
    case 2: xr = -R; xi = -I; break;
    default: xr = I; xi = -R; break;
  }
  // to the nearest multiple of 2^-104 (ties upward): an add and an arithmetic shift
  const auto rnd = [](__int128 x) -> __int128 { return (x + ((__int128)1 << 21)) >> 22; };
  const __int128 bias = digit_bias();
  const unsigned __int128 ur = (unsigned __int128)(rnd(xr) + bias), ui = (unsigned __int128)(rnd(xi) + bias);
  yre = make_uint4((uint32_t)ur, (uint32_t)(ur >> 32), (uint32_t)(ur >> 64), (uint32_t)(ur >> 96));
  yim = make_uint4((uint32_t)ui, (uint32_t)(ui >> 32), (uint32_t)(ui >> 64), (uint32_t)(ui >> 96));
  if (q126) {
    q126->re = q128_from_i128(xr);
    q126->im = q128_from_i128(xi);
  }
}

}  // namespace

// Two threads per (particle, axis), in two halves of the grid so that every warp runs one of the two tables:
// half 0 the tables T[k] = e^{2 pi i k s} (k < 8), half 1 the tables A[b] = e^{2 pi i 8 b s} (b <= Rax / 8), as
// first-quadrant phasors.  Each table starts from an exact-phase evaluation z (e^{2 pi i s}, e^{2 pi i 8 s}) and
// runs as two interleaved chains of step z^2, the even and the odd powers, which halves the dependent multiplies
// of the thread (each product at most 8 units of 2^-126 low, so the error of a power grows linearly in its
// exponent: far below the 2^-104 digits).
// Block map over the tensor-core members' chunks; layout tc_tab[(axis nbuf + j) tc_ntab + (k | 8 + b)], j within
// the chunk.
__global__ void __launch_bounds__(128) k_tc_tables(const CfgDev* __restrict__ cfgs, const BlockMap* __restrict__ bm) {
  grid_dep_wait();
  const BlockMap m = bm[blockIdx.x];
  const CfgDev& c = cfgs[m.cfg];
  if (stopped(c)) return;
  const int64_t nd = (int64_t)c.tc_d * c.tc_n;  // this chunk's particles
  const int64_t idx = (int64_t)m.blk * blockDim.x + threadIdx.x;
  if (idx >= 2 * nd) return;
  const int h = idx >= nd ? 1 : 0;
  const int64_t r = idx - h * nd;
  const int axis = (int)(r / c.tc_n);
  const int64_t j = r - (int64_t)axis * c.tc_n;  // within the chunk; particle tc_j0 + j
  const int cnt = h == 0 ? kPrepLow : c.tc_Rax[axis] / kPrepLow + 1;
  // d = 1 lifted to two axes: axis 0 holds the phase 2^lift s (mod 1, exact), axis 1 the phase s
  const int src = c.tc_lift ? 0 : axis;
  q128 u = turns_from_dd(c.s_hi[src * c.N + c.tc_j0 + j], c.s_lo[src * c.N + c.tc_j0 + j]);
  if (c.tc_lift && axis == 0) u = turn_times(u, 1 << c.tc_lift);
  qent* tab = reinterpret_cast<qent*>(c.tc_tab) + ((int64_t)axis * c.tc_nbuf + j) * c.tc_ntab + (h == 0 ? 0 : kPrepLow);
  // e^0 = 1 exactly (the exact-phase evaluation returns (2^126, 0) at t = 0): c = 1 in Q1.127, s = 0, quadrant 0
  qent xe;
  xe.c = q128_zero();
  xe.c.w[3] = 0x80000000u;
  xe.s = q128_zero();
  xe.cs = xe.c;
  const qent e = to_quadrant(phasor_turn(h == 0 ? u : turn_times(u, kPrepLow)));
  const qent e2 = qmul(e, e);
  qent xo = e;
#pragma unroll 1
  for (int k = 0; k < cnt; k += 2) {  // xe = z^k, xo = z^(k + 1)
    tab[k] = xe;
    if (k + 1 < cnt) tab[k + 1] = xo;
    if (k + 2 < cnt) xe = qmul(xe, e2);
    if (k + 3 < cnt) xo = qmul(xo, e2);
  }
}

// CTA per item.  Items TwItem {cfg, kind | staged << 8 | groups << 9, first particle}: 8 x groups particles (16
// for a staged w item of three or four axes; a table item enough for 128 (entry, group) lane pairs, at most 128).
// Kind 0: a_j(n1), n1 in [0, R1] -> density B digit slices (rows (n1, cos / sin) of
// K-major 32 x 16 tiles) and the Q2.126 table of the force epilogue.  Kind 1: w_j(p) for the nP canonical p ->
// the digit tensor.  A lane pair takes one entry and eight consecutive particles: each lane forms four of the
// products, the pair swaps halves, and lane 0 writes the entry's cos row, lane 1 its sin row, as 16-byte
// core-matrix rows, so that a warp's store covers whole 128-byte core matrices.  Table items (kind 0, and kind
// 1 for d = 2) multiply two entries of each particle's tables; staged w items cover 16 particles whose axis
// powers b_j(n2), c_j(n3) (and e_j(n4) on four axes; every exponent >= 0) are formed first into shared memory,
// and w = b_j(|n2|) (conjugated for n2 < 0) c_j(n3) on three axes, w = b_j(|n2|) c_j(|n3|) e_j(n4) on four (each
// factor of a negative exponent conjugated).
// kFour: the instance for members of four axes (their items are launched apart, after the others'), whose w
// takes a third factor; the other instance is free of that code and of its registers.
template <bool kFour>
__global__ void __launch_bounds__(kPrepThreads) k_tc_prep(const CfgDev* __restrict__ cfgs,
                                                                         const TwItem* __restrict__ items) {
  grid_dep_wait();
  extern __shared__ __align__(16) uint8_t psm[];
  const TwItem it = items[blockIdx.x];
  const CfgDev& c = cfgs[it.cfg];
  if (stopped(c)) return;
  const int kind = it.pad & 0xff, ng = it.pad >> 9;  // particle groups of 8
  const bool staged = (it.pad >> 8) & 1;
  const int64_t N = c.tc_n;                 // this chunk's particles (indices within the chunk)
  const int64_t Npad = (N + 15) & ~(int64_t)15;  // groups up to the K-step boundary are written (zeros past N)
  const int64_t j0 = it.start;
  const int tid = threadIdx.x, lane = tid & 31, h = lane & 1;
  const __int128 bias = digit_bias();
  const uint4 yzero = make_uint4((uint32_t)bias, (uint32_t)(bias >> 32), (uint32_t)(bias >> 64), (uint32_t)(bias >> 96));
  const qent* tab = reinterpret_cast<const qent*>(c.tc_tab);
  // staged powers per particle: axis 2 (W2 of them), axis 3 (W3), axis 4 (W4)
  const int W2 = c.tc_Rax[1] + 1, W3 = c.tc_d >= 3 ? c.tc_Rax[2] + 1 : 0, W4 = kFour ? c.tc_Rax[3] + 1 : 0;
  const int W23 = W2 + W3 + W4;
  const int count = kind == 0 ? c.tc_R1 + 1 : c.tc_nP;
  int32_t* pvs = reinterpret_cast<int32_t*>(psm);  // kind 1: the packed p of every entry
  // staged: [particle][powers of axis 2, then 3, then 4]
  qent* Pw = reinterpret_cast<qent*>(psm + (((size_t)c.tc_nP * 4 + 15) & ~(size_t)15));
  if (kind == 1) {
    for (int e = tid; e < count; e += kPrepThreads) pvs[e] = c.tc_pvec[e];
    if (staged) {
      for (int task = tid; task < kPrepStaged * W23; task += kPrepThreads) {
        const int jl = task % kPrepStaged, e = task / kPrepStaged;
        const int64_t j = min(j0 + jl, N - 1);  // entries of particles past N are never read
        const int axis = e < W2 ? 1 : (e < W2 + W3 ? 2 : 3);
        const int m = e < W2 ? e : (e < W2 + W3 ? e - W2 : e - W2 - W3);
        const qent* tj = tab + ((int64_t)axis * c.tc_nbuf + j) * c.tc_ntab;
        Pw[jl * W23 + e] = qmul(tj[kPrepLow + (m >> 3)], tj[m & 7]);
      }
    }
    __syncthreads();
  }
  const int axis = kind == 0 ? 0 : 1;
  const size_t wstride = (size_t)c.tc_NPg * (size_t)c.tc_NJ * 128;  // bytes between digit slices of the tensor
  const int total = count * ng;  // (entry, group) pairs of lanes
  for (int q0 = (tid >> 5) * 16; q0 < total; q0 += kPrepThreads / 2) {  // warp-uniform: 16 pairs per warp
    const int q = q0 + (lane >> 1);
    const bool valid = q < total;
    const int e = valid ? q % count : 0, g = valid ? q / count : 0;
    const int64_t jg = j0 + 8 * g;
    const bool live = valid && jg < Npad;  // digits of particles past the last one are written as zeros
    int m = e, n2 = 0, n3 = 0, n4 = 0;
    if (kind == 1) {
      unpack_p(pvs[e], kFour ? 4 : 2, n2, n3, n4);
      m = n2;  // d = 2: n2 = m >= 0
    }
    uint4 Yr[4], Yi[4];
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const int jl = 8 * g + 4 * h + v;
      const int64_t j = jg + 4 * h + v;
      Yr[v] = yzero;
      Yi[v] = yzero;
      if (live && j < N) {
        qent za, zb;
        if (staged) {
          const qent* pj = Pw + jl * W23;
          const qent b = pj[n2 < 0 ? -n2 : n2];
          za = n2 < 0 ? qconj(b) : b;
          if (kFour) {  // w = b(n2) c(n3) e(n4), n4 >= 0
            const qent cz = pj[W2 + (n3 < 0 ? -n3 : n3)];
            za = qmul(za, n3 < 0 ? qconj(cz) : cz);
            zb = pj[W2 + W3 + n4];
          } else {
            zb = pj[W2 + n3];
          }
        } else {
          const qent* tj = tab + ((int64_t)axis * c.tc_nbuf + j) * c.tc_ntab;
          za = tj[kPrepLow + (m >> 3)];
          zb = tj[m & 7];
        }
        if (kind == 0) {
          fxc zq;
          qmul_out(za, zb, Yr[v], Yi[v], &zq);
          reinterpret_cast<fxc*>(c.tc_a1)[(int64_t)e * c.tc_nbuf + j] = zq;
        } else {
          qmul_out(za, zb, Yr[v], Yi[v], nullptr);
        }
      }
    }
    // lane 0 of the pair keeps the cos values and receives those of particles 4..7; lane 1 the sin values of
    // particles 0..3
    uint4 Y[8];
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const uint4 send = h == 0 ? Yi[v] : Yr[v];
      uint4 got;
      got.x = __shfl_xor_sync(0xffffffffu, send.x, 1);
      got.y = __shfl_xor_sync(0xffffffffu, send.y, 1);
      got.z = __shfl_xor_sync(0xffffffffu, send.z, 1);
      got.w = __shfl_xor_sync(0xffffffffu, send.w, 1);
      Y[v] = h == 0 ? Yr[v] : got;
      Y[4 + v] = h == 0 ? got : Yi[v];
    }
    if (live) {
      const int r = 2 * e + h;  // row (entry, cos / sin)
      uint8_t* base = kind == 0
          ? c.tc_aB + ((int64_t)(r >> 5) * c.tc_KS + (jg >> 4)) * kStageB + slice_off(r & 31, (int)(jg & 15))
          : c.tc_wT + ((size_t)(r >> 3) * (size_t)c.tc_NJ + (size_t)(jg >> 3)) * 128 + (r & 7) * 16;
      // the transposed remainder tile: a_j(n1) also as digit-tensor rows, w_j(p) of the last row tile also as the
      // columns of its B operand (the last density column tile)
      uint8_t* b2 = nullptr;
      if (c.tc_tr && (kind == 0 ? e < c.tc_trN1 : e >= c.tc_trP0)) {
        if (kind == 0) {
          const int rt = kTileM * (c.tc_RT - 1) + c.tc_trRow0 + r;
          b2 = c.tc_wT + ((size_t)(rt >> 3) * (size_t)c.tc_NJ + (size_t)(jg >> 3)) * 128 + (rt & 7) * 16;
        } else {
          const int col = 2 * (e - c.tc_trP0) + h;
          b2 = c.tc_aB + ((int64_t)(c.tc_CTd - 1) * c.tc_KS + (jg >> 4)) * kStageB + slice_off(col, (int)(jg & 15));
        }
      }
      put_digit_rows(base, kind == 0 ? (size_t)kSliceB : wstride, Y, b2, kind == 0 ? wstride : (size_t)kSliceB);
    }
  }
}

// ------------------------------------------------------------------------------------------------ k_tc_gemm

// Persistent, with a dynamic queue: the producer thread claims items in list order (queue[0], an atomic
// counter) and passes each index to the MMA thread and the epilogue warps through a ring in shared memory, so a
// CTA that finishes early takes the next item (queue[1] counts finished CTAs; the last one resets both).
// Density items: A = rows (p, cos / sin) of row tile it.a
// (tensor-map box, K-major), B = column tile it.b of the a_j(n1) slices, K-steps [ks0, ks0 + nks) of 16
// particles; the epilogue adds the three int64 level groups of every output into tile accumulator it.slot.
// Force items: A = particle tile it.a (tensor-map box, MN-major), B = column tile it.b (16 / d values of n1, all
// axes) of the coefficient slices, K-steps of 16 rows (p, cos / sin); the epilogue adds the tile's force limbs.
// Stage and accumulator barrier phases run on across items, so the producer streams the next item's operands
// while the epilogue finishes the previous item (the accumulator is released as soon as its last level has
// been read).
template <bool kCount>
__global__ void __launch_bounds__(kGemmThreads, 1) k_tc_gemm(const CfgDev* __restrict__ cfgs,
                                                              const TcItem* __restrict__ items, int n_items,
                                                              int* __restrict__ queue) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  // tensor-map destinations must be 128-byte aligned
  uint8_t* smem = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  __shared__ uint64_t bar_full[kStages], bar_empty[kStages], bar_acc_full, bar_acc_empty, bar_drain;
  __shared__ uint64_t bar_item_full[kRing], bar_item_empty[kRing];
  __shared__ int item_ring[kRing];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], 1);
    }
    for (int r = 0; r < kRing; r++) {
      mbar_init(&bar_item_full[r], 1);
      mbar_init(&bar_item_empty[r], 1 + kEpiWarps);  // the MMA thread and every epilogue warp have read it
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
  // the set-up above touches no global memory, so it overlaps the end of the previous kernel; the operands, the
  // queue and the accumulators are used only after that kernel has completed
  grid_dep_wait();
  const uint32_t tbase = tmem_base_sh;
  volatile int* abort_flag = &abort_sh;
  const long long wlim = g_tc_wait_limit;  // waits on work; the drains below always use kWaitLimit
  // counting instance: cycles spent in each wait and phase (kGc* fields), one record per CTA
  const long long T0 = kCount ? clock64() : 0;
  const unsigned long long G0 = kCount ? global_ns() : 0;
  long long c_prod = 0, c_full = 0, c_acc = 0, c_item = 0, c_items = 0, c_ks = 0, c_eacc = 0, c_eread = 0, c_emath = 0;

  if (warp == 0) {
    // ---- producer: one thread streams every item's K-steps through the stages
    if (lane == 0) {
      long long gs = 0;  // K-steps issued so far (all items)
      bool stop = false;
      int pre = -1;      // the next claim, made while the previous item's last K-step is copied (-1: none yet)
      for (long long n = 0; !stop; n++) {
        // claim the next item and publish it to the MMA thread and the epilogue warps
        const int r = (int)(n % kRing);
        const long long use = n / kRing;
        if (use > 0 && !mbar_wait(&bar_item_empty[r], (uint32_t)((use - 1) & 1), wlim, abort_flag)) {
          *abort_flag = 1;
          tc_flag_all(cfgs, items, n_items, 32);
          break;
        }
        const int item = pre >= 0 ? pre : atomicAdd(queue, 1);
        pre = -1;
        item_ring[r] = item < n_items ? item : -1;
        mbar_arrive(&bar_item_full[r]);
        if (item >= n_items) break;
        const TcItem it = items[item];
        const CfgDev& c = cfgs[it.cfg];
        if (stopped(c)) continue;
        const void* tmap = reinterpret_cast<const uint8_t*>(c.tc_tmap) + (it.kind == 0 ? 0 : 128);
        tmap_acquire(tmap);
        const uint8_t* gB = it.kind == 0 ? c.tc_aB + ((int64_t)it.b * c.tc_KS + it.ks0) * kStageB
                                         : c.tc_fB + ((int64_t)it.b * c.tc_KSf + it.ks0) * kStageB;
        for (int ks = 0; ks < it.nks; ks++, gs++) {
          const int s = (int)(gs % kStages);
          const long long use = gs / kStages;
          const long long tw0 = kCount ? clock64() : 0;
          const bool free_stage = use == 0 || mbar_wait(&bar_empty[s], (uint32_t)((use - 1) & 1), wlim, abort_flag);
          if (kCount) c_prod += clock64() - tw0;
          if (!free_stage) {
            *abort_flag = 1;
            tc_flag_all(cfgs, items, n_items, 1);
            stop = true;
            break;
          }
          if (ks == it.nks - 1) pre = atomicAdd(queue, 1);  // its latency overlaps the last copies and MMAs
          uint8_t* dst = smem + (size_t)s * kStageBytes;
          const int kg = it.ks0 + ks;
          mbar_expect_tx(&bar_full[s], kStageBytes);
          if (it.kind == 0)
            tma_load_4d(dst, tmap, 0, 2 * kg, 16 * it.a, 0, &bar_full[s]);  // particle groups 2 kg, +1; row groups 16 a..
          else
            tma_load_4d(dst, tmap, 0, 16 * it.a, 2 * kg, 0, &bar_full[s]);  // particle groups 16 a..; row groups 2 kg, +1
          bulk_g2s(dst + kStageA, gB + (size_t)ks * kStageB, kStageB, &bar_full[s]);
        }
      }
      if (*abort_flag) {
        // let the copies in flight land before the CTA can exit
        for (long long k = gs > kStages ? gs - kStages : 0; k < gs; k++)
          if (!mbar_wait(&bar_full[k % kStages], (uint32_t)((k / kStages) & 1), kWaitLimit, nullptr))
            tc_flag_all(cfgs, items, n_items, 8);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer: 22 MMAs per K-step; level u of the accumulator receives digit slice pairs (s, u - s)
    if (lane == 0) {
      long long gs = 0, gc = 0;  // K-steps and chunks consumed so far (all items)
      bool stop = false;
      for (long long n = 0; !stop; n++) {
        const int r = (int)(n % kRing);
        const long long ti0 = kCount ? clock64() : 0;
        const bool have_item = mbar_wait(&bar_item_full[r], (uint32_t)((n / kRing) & 1), wlim, abort_flag);
        if (kCount) c_item += clock64() - ti0;
        if (!have_item) {
          *abort_flag = 1;
          tc_flag_all(cfgs, items, n_items, 64);
          break;
        }
        const int item = item_ring[r];
        mbar_arrive(&bar_item_empty[r]);
        if (item < 0) break;
        const TcItem it = items[item];
        const CfgDev& c = cfgs[it.cfg];
        if (stopped(c)) continue;
        if (kCount) c_items++;
        // density A: K-major, core matrices 128 bytes apart along K and 256 along M; force A: MN-major, 128
        // bytes apart along M (particles) and 2048 along K
        const int mn = it.kind == 0 ? 0 : 1;
        const uint32_t lbo = mn ? 2048u : 128u, sbo = mn ? 128u : 256u;
        for (int ks = 0; ks < it.nks; ks++, gs++) {
          const int s = (int)(gs % kStages);
          const long long use = gs / kStages;
          const bool first = ks % kChunkSteps == 0;
          const bool last = ks % kChunkSteps == kChunkSteps - 1 || ks == it.nks - 1;
          const long long tf0 = kCount ? clock64() : 0;
          const bool full_stage = mbar_wait(&bar_full[s], (uint32_t)(use & 1), wlim, abort_flag);
          if (kCount) c_full += clock64() - tf0;
          if (!full_stage) {
            *abort_flag = 1;
            tc_flag_all(cfgs, items, n_items, 2);
            stop = true;
            break;
          }
          const long long ta0 = kCount ? clock64() : 0;
          const bool acc_free = !(first && gc > 0) || mbar_wait(&bar_acc_empty, (uint32_t)((gc - 1) & 1), wlim, abort_flag);
          if (kCount) {
            c_acc += clock64() - ta0;
            c_ks++;
          }
          if (!acc_free) {
            *abort_flag = 1;
            tc_flag_all(cfgs, items, n_items, 4);
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(smem + (size_t)s * kStageBytes);
          const uint32_t b0 = a0 + kStageA;
          // slice 0 starts every level: levels 0..6 (kHeldLevels) at the first K-step of every second chunk of
          // the item, levels 7..14 at the first K-step of every chunk
          {
            const bool even = ((ks / kChunkSteps) & 1) == 0;
            const uint64_t ad = make_sdesc(a0, lbo, sbo);
            mma_bf16(tbase, ad, make_sdesc(b0), make_idesc(kTileM, kHeldLevels * kTileN, mn), (first && even) ? 0u : 1u);
            mma_bf16(tbase + kHeldLevels * kTileN, ad, make_sdesc(b0 + kHeldLevels * kSliceB),
                     make_idesc(kTileM, (kLevels - kHeldLevels) * kTileN, mn), first ? 0u : 1u);
          }
#pragma unroll
          for (int sl = 1; sl < kDigits; sl++) {
            const int ntot = (kLevels - sl) * kTileN;
            const int n1 = ntot < 256 ? ntot : 256;
            const uint64_t ad = make_sdesc(a0 + sl * kSliceA, lbo, sbo);
            mma_bf16(tbase + sl * kTileN, ad, make_sdesc(b0), make_idesc(kTileM, n1, mn), 1u);
            if (ntot > 256)
              mma_bf16(tbase + sl * kTileN + 256, ad, make_sdesc(b0 + 256 * 32), make_idesc(kTileM, ntot - 256, mn), 1u);
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
      if (!mbar_wait(&bar_drain, 0, kWaitLimit, nullptr)) {
        *abort_flag = 1;
        tc_flag_all(cfgs, items, n_items, 8);
      }
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 and accumulator columns 8 hq .. 8 hq + 7
    const int q = warp & 3, hq = (warp - 2) >> 2;
    const int row = 32 * q + lane;
    const uint32_t trow = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(kEpiCols * hq);
    long long gc = 0;  // chunks read (all items of this CTA)
    bool stop = false;
    for (long long n = 0; !stop; n++) {
      const int r = (int)(n % kRing);
      const bool have = mbar_wait(&bar_item_full[r], (uint32_t)((n / kRing) & 1), wlim, abort_flag);
      if (!__all_sync(0xffffffffu, have)) {
        *abort_flag = 1;
        if (lane == 0) tc_flag_all(cfgs, items, n_items, 128);
        break;
      }
      const int item = item_ring[r];
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_item_empty[r]);
      if (item < 0) break;
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
        const long long te0 = kCount ? clock64() : 0;
        const bool got = mbar_wait(&bar_acc_full, (uint32_t)(gc & 1), wlim, abort_flag);
        const long long te1 = kCount ? clock64() : 0;
        if (kCount) c_eacc += te1 - te0;
        if (!__all_sync(0xffffffffu, got)) {
          *abort_flag = 1;
          if (lane == 0) tc_flag_all(cfgs, items, n_items, 16);
          stop = true;
          break;
        }
        tc_fence_after();
        // levels 0..6 run on over two chunks (their sums stay below 2^24), so they are read after every second
        // chunk and after the item's last; levels 7..14 after every chunk.  The accumulator is released as soon as
        // the last group is in registers, before its conversion.
        const bool full = (ch & 1) || ch == nch - 1;
#pragma unroll
        for (int g = 0; g < 3; g++) {
          if (g == 0 && !full) continue;  // uniform over the CTA
          const int l0 = (g == 1 && !full) ? 2 : 0;
          uint32_t r[5][kEpiCols];  // the group's levels, loaded together, one wait
#pragma unroll
          for (int l = 0; l < 5; l++) {
            if (l < l0) {
#pragma unroll
              for (int i = 0; i < kEpiCols; i++) r[l][i] = 0;  // +0.0f
            } else {
              tmem_ld8(trow + (uint32_t)((5 * g + l) * kTileN), r[l]);
            }
          }
          tmem_ld_wait();
          if (g == 2) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_acc_empty);
            if (kCount) c_eread += clock64() - te1;
          }
          // |x| of level u is at most (u + 1) 2^20 per chunk (u + 1 digit pairs, 256 products of at most 64^2
          // each), twice that for u <= 6: level 0 takes one add; of the others, levels 2, 4, 8, 11, 13 convert on
          // the fp32 pipe and the rest on the conversion unit, which balances the two
#pragma unroll
          for (int i = 0; i < kEpiCols; i++) {
            int32_t v[5];
#pragma unroll
            for (int l = 0; l < 5; l++) {
              const int u = 5 * g + l;
              v[l] = u == 0 ? acc_int_small(r[l][i])
                            : (u == 2 || u == 4 || u == 8 || u == 11 || u == 13) ? acc_int_fma(r[l][i])
                                                                                  : acc_int(r[l][i]);
            }
            // x0 2^28 + x1 2^21 + x2 2^14 + x3 2^7 + x4, with x0 128 + x1 and x2 128 + x3 below 2^31 in magnitude
            const int32_t a = v[0] * 128 + v[1], b = v[2] * 128 + v[3];
            st[g][i] += (long long)a * (1ll << 21) + (long long)b * 128 + v[4];
          }
        }
      }
      if (stop) break;
      const long long tp0 = kCount ? clock64() : 0;
      if (it.kind == 0) {
        // level groups of every output, R' = st0 2^70 + st1 2^35 + st2 (value = R' 2^-110), normalised so that
        // st1, st2 lie in [0, 2^35), and added into the tile's accumulator: integer addition, so the K ranges
        // combine exactly in any order.  The tile's lower groups then stay below (pieces) 2^35 and its top group
        // near R' 2^-70 <= N 2^40, whatever the digit sums of the pieces were.
        unsigned long long* out = reinterpret_cast<unsigned long long*>(c.tc_acc) + (size_t)it.slot * (3 * kTileN * kTileM);
#pragma unroll
        for (int i = 0; i < kEpiCols; i++) {
          const long long c2 = st[2][i] >> 35;
          st[2][i] -= c2 * (1ll << 35);
          st[1][i] += c2;
          const long long c1 = st[1][i] >> 35;
          st[1][i] -= c1 * (1ll << 35);
          st[0][i] += c1;
        }
#pragma unroll
        for (int g = 0; g < 3; g++)
#pragma unroll
          for (int i = 0; i < kEpiCols; i++)
            atomicAdd(out + ((size_t)g * kTileN + kEpiCols * hq + i) * kTileM + row, (unsigned long long)st[g][i]);
      } else {
        // column tile ct: the 16 / d values n1 = (16 / d) ct + i / d, every axis t = i % d of each, as column
        // pairs (Re G, Im G) i = 0, 1, ...; this warp holds pairs 4 hq .. 4 hq + 3.  G~ = R' 2^-110 is taken as
        // R' 2^gs (|.| < 2^126); the top halves of a * G are value 2^(108 + gs), shifted to value 2^ts.
        const int64_t j = (int64_t)it.a * kTileM + row;
        const int d = c.tc_d, npt = 16 / d;
        const int gsh = c.tc_gs, tsh = 108 + c.tc_gs - c.tc_ts;
        __int128 F0 = 0, F1 = 0, F2 = 0, F3 = 0;  // per axis, value 2^ts (at most four terms each)
#pragma unroll
        for (int v = 0; v < kEpiCols / 2; v++) {
          const int i = (kEpiCols / 2) * hq + v;
          const int n1 = npt * it.b + i / d, t = i - (i / d) * d;
          if (i >= npt * d || n1 > c.tc_R1 || j >= c.tc_n) continue;
          q128 gre, gim;
          {
            const __int128 Rr = ((__int128)st[0][2 * v] << 70) + ((__int128)st[1][2 * v] << 35) + (__int128)st[2][2 * v];
            const __int128 Ri =
                ((__int128)st[0][2 * v + 1] << 70) + ((__int128)st[1][2 * v + 1] << 35) + (__int128)st[2][2 * v + 1];
            gre = q128_from_i128(Rr << gsh);
            gim = q128_from_i128(Ri << gsh);
          }
          const fxc a = reinterpret_cast<const fxc*>(c.tc_a1)[(int64_t)n1 * c.tc_nbuf + j];
          uint32_t p[5], r2[5];
          // Im(a G) = Re a Im G + Im a Re G
          smul_top(a.re, gim, p);
          smul_top(a.im, gre, r2);
          const __int128 T =
              (q128_to_i128(q128{{p[1], p[2], p[3], p[4]}}) + q128_to_i128(q128{{r2[1], r2[2], r2[3], r2[4]}})) >> tsh;
          if (t == 0) F0 += T * (__int128)n1;
          else if (t == 1) F1 += T;
          else if (t == 2) F2 += T;
          else F3 += T;
        }
        if (j < c.tc_n) {
          // F = L2 2^88 + L1 2^44 + L0 (L0, L1 in [0, 2^44)): the limbs of all column tiles add up exactly
          const unsigned long long m44 = (1ull << 44) - 1;
          for (int t = 0; t < d; t++) {
            const __int128 F = t == 0 ? F0 : (t == 1 ? F1 : (t == 2 ? F2 : F3));
            unsigned long long* fa = reinterpret_cast<unsigned long long*>(c.tc_facc) + (size_t)t * 3 * c.N + c.tc_j0 + j;
            atomicAdd(fa, (unsigned long long)F & m44);
            atomicAdd(fa + c.N, (unsigned long long)(F >> 44) & m44);
            atomicAdd(fa + 2 * c.N, (unsigned long long)(long long)(F >> 88));
          }
        }
      }
      if (kCount) c_emath += clock64() - tp0;
    }
  }
  unsigned long long* rec = nullptr;
  if (kCount) {
    // one thread of each role writes its own fields; thread 0 the totals after the CTA's last wait
    rec = g_tc_counters[items[0].kind == 0 ? 0 : 1][blockIdx.x % kGcCtas];
    if (warp == 0 && lane == 0) rec[kGcProdWaitStage] = c_prod;
    if (warp == 1 && lane == 0) {
      rec[kGcMmaWaitOperands] = c_full;
      rec[kGcMmaWaitAcc] = c_acc;
      rec[kGcMmaWaitItem] = c_item;
      rec[kGcItems] = c_items;
      rec[kGcKsteps] = c_ks;
      rec[kGcMmaCycles] = clock64() - T0;
    }
    if (warp == 2 && lane == 0) {
      rec[kGcEpiWaitAcc] = c_eacc;
      rec[kGcEpiRead] = c_eread;
      rec[kGcEpiMath] = c_emath;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (kCount && threadIdx.x == 0) {
    rec[kGcCycles] = clock64() - T0;
    rec[kGcT0] = G0;
    rec[kGcT1] = global_ns();
  }
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, kTmemCols);
  }
  // the last CTA out resets the queue for the next launch (every CTA's producer has made its last claim)
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(queue + 1, 1) == (int)gridDim.x - 1) {
      queue[0] = 0;
      queue[1] = 0;
      __threadfence();
    }
  }
}

// ------------------------------------------------------------------------------------------------ finish

namespace {

// per-block partials of the tensor-core density reduction, in the space of one RedPart: Phi as an exact integer
// (units of 2^-220, so every order of summation gives the same bits), max |n~|^2 as dd, max |C|, |S|
struct TcRed {
  u320 phi;
  double a2_hi, a2_lo, cmax;
};
static_assert(sizeof(TcRed) == sizeof(RedPart), "the tensor-core partials reuse the partial buffer");

__device__ __forceinline__ void tc_red_combine(TcRed& a, const TcRed& b) {
  u320_add(a.phi, b.phi);
  if (dd_gt(dd_make(b.a2_hi, b.a2_lo), dd_make(a.a2_hi, a.a2_lo))) {
    a.a2_hi = b.a2_hi;
    a.a2_lo = b.a2_lo;
  }
  a.cmax = fmax(a.cmax, b.cmax);
}

// fixed-order warp tree: lane 0 ends with the combination of lanes 0..31
__device__ __forceinline__ void tc_red_warp(TcRed& v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    TcRed o;
#pragma unroll
    for (int i = 0; i < 5; i++) o.phi.w[i] = __shfl_down_sync(0xffffffffu, v.phi.w[i], off);
    o.a2_hi = __shfl_down_sync(0xffffffffu, v.a2_hi, off);
    o.a2_lo = __shfl_down_sync(0xffffffffu, v.a2_lo, off);
    o.cmax = __shfl_down_sync(0xffffffffu, v.cmax, off);
    if (lane < off) tc_red_combine(v, o);
  }
}

// The scalars of one evaluation from its nb block partials (one block of kFinThreads threads, the same order
// whichever block runs it): Phi, S_max = max |n~|^2 / N, max |C|, |S| and the scale e (2^e > 2 max |C|, |S|).
// The partials are read through L2 (the caller's fence and ticket make every block's write visible).
__device__ __forceinline__ void tc_finalize(const TcRed* blk, int nb, int64_t N, double* scal,
                                            TcRed (&sh)[kFinThreads / 32]) {
  auto load = [&](int i) {
    const unsigned long long* p = reinterpret_cast<const unsigned long long*>(blk + i);
    TcRed r;
#pragma unroll
    for (int k = 0; k < 5; k++) r.phi.w[k] = __ldcg(p + k);
    const double* q = reinterpret_cast<const double*>(p + 5);
    r.a2_hi = __ldcg(q + 0);
    r.a2_lo = __ldcg(q + 1);
    r.cmax = __ldcg(q + 2);
    return r;
  };
  TcRed v;
  u320_zero(v.phi);
  v.a2_hi = v.a2_lo = v.cmax = 0.0;
  if ((int)threadIdx.x < nb) v = load(threadIdx.x);
  for (int i = threadIdx.x + kFinThreads; i < nb; i += kFinThreads) tc_red_combine(v, load(i));
  tc_red_warp(v);
  __syncthreads();  // sh holds the caller's partials
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    v = sh[0];
#pragma unroll
    for (int w = 1; w < kFinThreads / 32; w++) tc_red_combine(v, sh[w]);
    const dd phi = u320_to_dd(v.phi, 220);
    scal[kScPhiHi] = phi.hi;
    scal[kScPhiLo] = phi.lo;
    const dd sm = N > 0 ? dd_div(dd_make(v.a2_hi, v.a2_lo), dd_make((double)N)) : dd_make(0.0);
    scal[kScSmaxHi] = sm.hi;
    scal[kScSmaxLo] = sm.lo;
    scal[kScCmax] = v.cmax;
    scal[kScScaleExp] = v.cmax > 0 ? (double)(ilogb(v.cmax) + 2) : 0.0;
    scal[kScA2MaxHi] = v.a2_hi;
    scal[kScA2MaxLo] = v.a2_lo;
  }
}

}  // namespace

// block map over the tensor-core members (tc_nblk blocks each), 64 threads, a lane pair per (n1, p), p fastest:
// the even lane n~(n1, p), the odd lane n~(n1, -p), from the four real products of the tile accumulator (which the
// even lane clears for the next evaluation once both have read it), as exact Q34.126 values (for the force
// coefficients) and as dd (C, S), with the block's partials: Phi as an exact integer sum of v~ |n~|^2 (|n~|^2 =
// C^2 + S^2 formed exactly, in integer arithmetic rather than on the scarce FP64 pipe), max |n~|^2 and
// max |C|, |S|; the last block to finish reduces the partials to Phi, S_max and the scale.
__global__ void __launch_bounds__(kFinThreads) k_tc_dens_finish(const CfgDev* __restrict__ cfgs,
                                                                const BlockMap* __restrict__ bm) {
  grid_dep_wait();
  const BlockMap m = bm[blockIdx.x];
  const CfgDev& c = cfgs[m.cfg];
  if (stopped(c)) return;  // uniform per block
  TcRed v;
  u320_zero(v.phi);
  v.a2_hi = v.a2_lo = v.cmax = 0.0;
  const int W1 = c.tc_R1 + 1;
  const int64_t idx = ((int64_t)m.blk * kFinThreads + threadIdx.x) >> 1;
  const int neg = threadIdx.x & 1;
  int k = -1, ti = -1, rr = 0, cc = 0;
  bool tr = false;
  double w = 1.0;
  long long P[4][3];  // [2 x + y]: x the cos / sin of w (row), y of a (column)
  long long* acc = nullptr;
  if (idx < (int64_t)W1 * c.tc_nP) {
    // p fastest: a warp's lanes read consecutive accumulator rows (p, cos / sin), contiguous in memory
    const int p = (int)(idx % c.tc_nP), n1 = (int)(idx / c.tc_nP);
    const int64_t ei = (int64_t)p * W1 + n1;  // em is [p][n1][2]
    const int r = 2 * p, col = 2 * n1;
    // the transposed remainder tile holds P_xy(p, n1) at row trRow0 + 2 n1 + y, column 2 (p - trP0) + x
    tr = c.tc_tr && p >= c.tc_trP0;
    // the emit map and the tile map are read together (the tile map entry is in range for every (p, n1))
    const int kp = c.tc_em[ei * 2 + 0], km = c.tc_em[ei * 2 + 1];
    const int tm = c.tc_tilemap[tr ? (c.tc_RT - 1) * c.tc_CTd + (c.tc_CTd - 1) : (r >> 7) * c.tc_CTd + (col >> 5)];
    k = neg ? km : kp;
    if (k >= 0) w = c.wk[k];
    ti = (kp >= 0 || km >= 0) ? tm : -1;
    if (ti >= 0) {
      rr = tr ? c.tc_trRow0 + col : r & 127;
      cc = tr ? 2 * (p - c.tc_trP0) : col & 31;
      acc = c.tc_acc + (size_t)ti * (3 * kTileN * kTileM);
#pragma unroll
      for (int x = 0; x < 2; x++)
#pragma unroll
        for (int y = 0; y < 2; y++)
#pragma unroll
          for (int g = 0; g < 3; g++)
            P[2 * x + y][g] = acc[((size_t)g * kTileN + cc + (tr ? x : y)) * kTileM + rr + (tr ? y : x)];
    }
  }
  __syncwarp();
  if (ti >= 0 && !neg) {
#pragma unroll
    for (int x = 0; x < 2; x++)
#pragma unroll
      for (int y = 0; y < 2; y++)
#pragma unroll
        for (int g = 0; g < 3; g++) acc[((size_t)g * kTileN + cc + (tr ? x : y)) * kTileM + rr + (tr ? y : x)] = 0;
  }
  if (ti >= 0 && k >= 0) {
    // n~(n1, p)  = (P_cc - P_ss) + i (P_cs + P_sc);  n~(n1, -p) = (P_cc + P_ss) + i (P_cs - P_sc)
    FxAcc* part = reinterpret_cast<FxAcc*>(c.part);
    i192 C, S;
    i192_zero(C);
    i192_zero(S);
#pragma unroll
    for (int g = 0; g < 3; g++) {
      const int sh = 70 - 35 * g;
      i192_add_shl(C, (__int128)P[0][g] + (neg ? (__int128)P[3][g] : -(__int128)P[3][g]), sh);
      i192_add_shl(S, (__int128)P[1][g] + (neg ? -(__int128)P[2][g] : (__int128)P[2][g]), sh);
    }
    const dd cd = i192_to_dd(C, 110), sd = i192_to_dd(S, 110);
    c.C_hi[k] = cd.hi;
    c.C_lo[k] = cd.lo;
    c.S_hi[k] = sd.hi;
    c.S_lo[k] = sd.lo;
    // the force coefficients take the weighted value v~(k) n~(k): exact for weight 1, else v~ n~ in dd (relative
    // error 2^-105) rounded to Q34.126
    FxAcc o;
    if (w == 1.0) {
      o.re = i192_to_q160_shl(C, 16);  // value 2^-110 -> Q34.126
      o.im = i192_to_q160_shl(S, 16);
    } else {
      const dd wc = dd_mul_d(cd, w), ws = dd_mul_d(sd, w);
      i192 X, Y;
      i192_zero(X);
      i192_zero(Y);
      i192_add_double_126(X, wc.hi);
      i192_add_double_126(X, wc.lo);
      i192_add_double_126(Y, ws.hi);
      i192_add_double_126(Y, ws.lo);
      o.re = i192_to_q160_shl(X, 0);
      o.im = i192_to_q160_shl(Y, 0);
    }
    part[k] = o;
    // |n~|^2 = (C^2 + S^2) 2^-220 exactly; Phi takes v~ |n~|^2 (rounded to 2^-220 for weights other than 1)
    u320 a2 = u320_sq(C);
    u320_add(a2, u320_sq(S));
    const dd a2d = u320_to_dd(a2, 220);
    v.phi = w == 1.0 ? a2 : u320_mul_weight(a2, w);
    v.a2_hi = a2d.hi;
    v.a2_lo = a2d.lo;
    v.cmax = w * fmax(fabs(cd.hi), fabs(sd.hi));
  }
  tc_red_warp(v);
  __shared__ TcRed sh[kFinThreads / 32];
  __shared__ int last;
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    TcRed a = sh[0];
#pragma unroll
    for (int i = 1; i < kFinThreads / 32; i++) tc_red_combine(a, sh[i]);
    reinterpret_cast<TcRed*>(c.blk)[m.blk] = a;
    // the block that finishes last reduces every block's partial (tc_err[1] counts finished blocks)
    __threadfence();
    last = atomicAdd(c.tc_err + 1, 1) == c.tc_nblk - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    tc_finalize(reinterpret_cast<const TcRed*>(c.blk), c.tc_nblk, c.N, c.scal, sh);
    if (threadIdx.x == 0) c.tc_err[1] = 0;  // for the next evaluation
  }
}

// block map over the tensor-core members (d N / 64 blocks each), 64 threads: F[a][j] from the force limbs (which it clears),
// times 4 pi / L and the power-of-two scale of the coefficients
__global__ void __launch_bounds__(kFinThreads) k_tc_force_finish(const CfgDev* __restrict__ cfgs,
                                                                 const BlockMap* __restrict__ bm) {
  grid_dep_wait();
  const BlockMap m = bm[blockIdx.x];
  const CfgDev& c = cfgs[m.cfg];
  if (stopped(c)) return;
  const int64_t i = (int64_t)m.blk * kFinThreads + threadIdx.x;  // over [a][j]
  if (i >= (int64_t)c.d * c.N) return;
  const int a = (int)(i / c.N);
  const int64_t j = i - (int64_t)a * c.N;
  // sum of the limbs of one axis of the GEMM's force, value X 2^-ts in units of 2^e (axes 2, 3: of 2^(e + bexp))
  auto limbs = [&](int ax) {
    long long* fa = c.tc_facc + (size_t)ax * 3 * c.N + j;
    const long long L0 = fa[0], L1 = fa[c.N], L2 = fa[2 * c.N];
    fa[0] = 0;
    fa[c.N] = 0;
    fa[2 * c.N] = 0;
    i192 X;
    i192_zero(X);
    i192_add_shl(X, (__int128)L0, 0);
    i192_add_shl(X, (__int128)L1, 44);
    i192_add_shl(X, (__int128)L2, 88);
    return X;
  };
  const int e = (int)c.scal[kScScaleExp];
  i192 X = limbs(a);
  int se = e + (a > 0 ? c.tc_bexp : 0);
  if (c.tc_lift) {
    // d = 1 on two lifted axes, n = 2^lift n1 + n2: F = 2^lift F_1 + F_2 = 2^(e + bexp - ts) (X_1 2^(lift - bexp)
    // + X_2), added exactly as integers.  X_1 is non-zero only when some n >= 2^(lift - 1), and then |n2| reaches
    // 2^(lift - 1) - 1, so lift - bexp <= 1 and the sum stays far below 2^150.
    X = i192_shl(X, c.tc_lift - c.tc_bexp);
    X = i192_add(X, limbs(1));
    se = e + c.tc_bexp;
  }
  dd f = dd_mul(i192_to_dd(X, c.tc_ts), c.pref);
  const double sc = pow2(se);
  c.F_hi[i] = f.hi * sc;
  c.F_lo[i] = f.lo * sc;
}

// block map over the tensor-core members (2 d (R1 + 1) nP / 128 blocks each), thread per (column, n1, p), p fastest:
// the force GEMM's coefficient digits of one column (n1, axis t, Re / Im) in both rows (p, cos / sin)
__global__ void __launch_bounds__(128) k_tc_coef(const CfgDev* __restrict__ cfgs, const BlockMap* __restrict__ bm) {
  grid_dep_wait();
  const BlockMap m = bm[blockIdx.x];
  const CfgDev& c = cfgs[m.cfg];
  if (stopped(c)) return;
  const int W1 = c.tc_R1 + 1;
  const int64_t np = (int64_t)W1 * c.tc_nP;
  const int64_t idx = (int64_t)m.blk * blockDim.x + threadIdx.x;
  if (idx >= 2 * c.tc_d * np) return;
  const int qc = (int)(idx / np);  // 2 t + ri: axis t, Re (0) / Im (1) column
  const int t = qc >> 1, ri = qc & 1;
  const int64_t rem = idx - (int64_t)qc * np;
  const int n1 = (int)(rem / c.tc_nP), p = (int)(rem % c.tc_nP);
  const int32_t* em = c.tc_em + ((int64_t)p * W1 + n1) * 2;
  const int kp = em[0], km = em[1];
  const FxAcc* part = reinterpret_cast<const FxAcc*>(c.part);
  const q160 z = q160_zero();
  const q160 Cp = kp >= 0 ? load_q160(&part[kp].re) : z, Sp = kp >= 0 ? load_q160(&part[kp].im) : z;
  const q160 Cm = km >= 0 ? load_q160(&part[km].re) : z, Sm = km >= 0 ? load_q160(&part[km].im) : z;
  const int e = (int)c.scal[kScScaleExp];
  const int32_t pv = c.tc_pvec[p];
  // W = C - i S:  Re U = C+ + C-,  Im U = -(S+ + S-),  Re V = S+ - S-,  Im V = C+ - C-
  //               Re U^a = n_a (C+ - C-), Im U^a = -n_a (S+ - S-), Re V^a = n_a (S+ + S-), Im V^a = n_a (C+ + C-)
  // column Re holds (Re U, Re V) in rows (cos, sin), column Im holds (Im U, Im V); likewise U^a, V^a
  __int128 X0, X1;
  if (t == 0) {
    const int sh = 22 + e;
    if (ri == 0) {
      q160 a = Cp;
      q160_add160(a, Cm);
      X0 = q160_shr_round(a, sh);
      X1 = q160_shr_round(q160_sub160(Sp, Sm), sh);
    } else {
      q160 a = Sp;
      q160_add160(a, Sm);
      X0 = -q160_shr_round(a, sh);
      X1 = q160_shr_round(q160_sub160(Cp, Cm), sh);
    }
  } else {
    int n2, n3, n4;
    unpack_p(pv, c.tc_d, n2, n3, n4);
    const int n = t == 1 ? n2 : (t == 2 ? n3 : n4);
    const int sh = 22 + e + c.tc_bexp;
    if (ri == 0) {
      q160 a = Sp;
      q160_add160(a, Sm);
      X0 = q160_shr_round(q160_mul_int(q160_sub160(Cp, Cm), n), sh);
      X1 = q160_shr_round(q160_mul_int(a, n), sh);
    } else {
      q160 a = Cp;
      q160_add160(a, Cm);
      X0 = -q160_shr_round(q160_mul_int(q160_sub160(Sp, Sm), n), sh);
      X1 = q160_shr_round(q160_mul_int(a, n), sh);
    }
  }
  if (pv == 0) X1 = 0;  // sin(0) = 0 (and every weight n_a is 0)
  const int npt = 16 / c.tc_d;  // n1 values per column tile, all axes of each
  const int ct = n1 / npt;
  const int col = 2 * (c.tc_d * (n1 - ct * npt) + t) + ri;
  const int kk = 2 * p;  // rows (p, cos), (p, sin): adjacent K positions of one core row
  uint8_t* base = c.tc_fB + ((int64_t)ct * c.tc_KSf + (kk >> 4)) * kStageB;
  put_digit_pair(base, kSliceB, slice_off(col, kk & 15), X0, X1);
}

// ------------------------------------------------------------------------------------------------ host side

bool tc_counters_on() { return g_counters_on; }

static cudaError_t tc_dev_alloc(DevBuf* b, size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 16;
  b->bytes = bytes;
  cudaError_t e = cudaMalloc(&b->p, bytes);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(b->p, 0, bytes, st);  // padding rows, columns and K stay zero for good
}

// N <= 2^22: the top level group of a density tile accumulates about N 2^40 (int64), and n~ stays inside Q34.126
bool tc_eligible(const Ctx& c) { return c.d >= 1 && c.d <= 4 && c.N >= 1 && c.N <= (1 << 22) && c.M >= 1; }

int64_t tc_coef_blocks(const Ctx& c) {
  if (!c.tc.on) return 0;
  return (2 * (int64_t)c.tc.d * (c.tc.R1 + 1) * c.tc.nP + 127) / 128;  // a thread per (column, n1, p)
}

int tc_finish_blocks(const Ctx& c) {
  if (!c.tc.on) return 0;
  return (int)((2 * (int64_t)(c.tc.R1 + 1) * c.tc.nP + kFinThreads - 1) / kFinThreads);  // a lane pair per (n1, p)
}

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// (n1, p) of internal wavevector k: p = (n2, n3, n4) of axes 2..d (the components past d are 0).  For d = 1 the
// single index n > 0 is split as n = 2^lift n1 + n2 with n2 in [-2^(lift - 1), 2^(lift - 1)): the phase n s is
// n1 (2^lift s) + n2 s, a wavevector of two lifted axes, and n > 0 exactly when (n1, n2) lies in the two-axis half
// set.
inline void sub_vec(const Ctx& c, int lift, int64_t k, int& n1, int& n2, int& n3, int& n4) {
  const int32_t* n = &c.ks.n_int[(size_t)k * c.d];
  n3 = 0;
  n4 = 0;
  if (c.d == 1) {
    const int64_t B = (int64_t)1 << lift;
    n1 = (int)((n[0] + B / 2) >> lift);
    n2 = (int)(n[0] - B * n1);
    return;
  }
  n1 = n[0];
  n2 = n[1];
  if (c.d >= 3) n3 = n[2];
  if (c.d == 4) n4 = n[3];
}

// d = 1: the split 2^lift minimising the padded work of both GEMMs (rows (n2, cos / sin) in tiles of 128 and
// columns (n1, cos / sin) in tiles of 32 for the density; 8 values of n1 per 32 columns and K in steps of 16
// rows for the force)
int choose_lift(const Ctx& c) {
  int64_t nmax = 1;
  for (int64_t k = 0; k < c.M; k++) nmax = std::max<int64_t>(nmax, c.ks.n_int[k]);
  int best = 4;
  double best_cost = 0;
  for (int lift = 4; lift <= 15; lift++) {  // |n2| <= 2^14 fits the 16-bit field of the packed p
    const int64_t B = (int64_t)1 << lift;
    std::vector<char> seen(B / 2 + 1, 0);
    int64_t nP = 0, R1 = 0;
    for (int64_t k = 0; k < c.M; k++) {
      int n1, n2, n3, n4;
      sub_vec(c, lift, k, n1, n2, n3, n4);
      R1 = std::max<int64_t>(R1, n1);
      const int a = std::abs(n2);
      if (!seen[a]) {
        seen[a] = 1;
        nP++;
      }
    }
    auto pad = [](int64_t x, int64_t m) { return (x + m - 1) / m * m; };
    const double cost = (double)pad(2 * nP, 128) * pad(2 * (R1 + 1), 32) + (double)pad(R1 + 1, 8) * 4 * pad(2 * nP, 16);
    if (lift == 4 || cost < best_cost) {
      best = lift;
      best_cost = cost;
    }
    if (B / 2 > nmax) break;  // every larger split puts the whole set in n1 = 0
  }
  return best;
}
// the canonical half of the sub-vectors: the last non-zero component of p = (n2, n3, n4) is positive, or p = 0
inline bool canonical(int n2, int n3, int n4) { return n4 > 0 || (n4 == 0 && (n3 > 0 || (n3 == 0 && n2 >= 0))); }

struct PVec {
  int n2, n3, n4;
};

}  // namespace

// Tile plan and device buffers of one configuration.  Returns success with t.on = false when the configuration
// does not fit the path's limits (the integer-pipe kernels serve it then).
cudaError_t tc_setup(Ctx* c) {
  TcPlan& t = c->tc;
  t.on = false;
  t.d = 0;
  t.tiles.clear();
  t.tilemap.clear();
  t.em.clear();
  t.pvec.clear();
  t.ks_ct.clear();
  if (!c->tc_requested || !tc_eligible(*c)) return cudaSuccess;
  const int d = c->d == 1 ? 2 : c->d;  // the path's number of axes (d = 1 runs on two lifted axes)
  const int lift = c->d == 1 ? choose_lift(*c) : 0;
  const int64_t M = c->M;
  // canonical sub-vectors present in the set, sorted by |p|^2 (then n4, n3, n2): a prefix of the list is a ball
  int R1 = 0, Rp = 0;
  for (int64_t k = 0; k < M; k++) {
    int n1, n2, n3, n4;
    sub_vec(*c, lift, k, n1, n2, n3, n4);
    R1 = std::max(R1, n1);
    Rp = std::max(Rp, std::max(std::abs(n2), std::max(std::abs(n3), std::abs(n4))));
  }
  // four axes: the packed p has 10-bit fields, and the dense index map below has (2 Rp + 1)^3 entries
  if (d == 4 && Rp > 64) return cudaSuccess;
  // dense index map over the box |n_a| <= Rp of the axes in use
  const int64_t s2 = 2 * Rp + 1, s3 = d >= 3 ? s2 : 1, o3 = d >= 3 ? Rp : 0, o4 = d == 4 ? Rp : 0;
  const int64_t span4 = d == 4 ? s2 : 1;
  std::vector<int32_t> pid((size_t)(s2 * s3 * span4), -1);
  auto pslot = [&](int n2, int n3, int n4) -> int32_t& {
    return pid[(size_t)(((n4 + o4) * s3 + (n3 + o3)) * s2 + (n2 + Rp))];
  };
  // the canonical p of wavevector k (flipping the sign of p when k is (n1, -p)) and whether it was canonical
  auto pcan = [&](int& n2, int& n3, int& n4) {
    const bool can = canonical(n2, n3, n4);
    if (!can) {
      n2 = -n2;
      n3 = -n3;
      n4 = -n4;
    }
    return can;
  };
  std::vector<PVec> plist;
  for (int64_t k = 0; k < M; k++) {
    int n1, n2, n3, n4;
    sub_vec(*c, lift, k, n1, n2, n3, n4);
    pcan(n2, n3, n4);
    int32_t& slot = pslot(n2, n3, n4);
    if (slot < 0) {
      slot = 0;
      plist.push_back({n2, n3, n4});
    }
  }
  std::sort(plist.begin(), plist.end(), [](const PVec& a, const PVec& b) {
    const int ra = a.n2 * a.n2 + a.n3 * a.n3 + a.n4 * a.n4, rb = b.n2 * b.n2 + b.n3 * b.n3 + b.n4 * b.n4;
    if (ra != rb) return ra < rb;
    if (a.n4 != b.n4) return a.n4 < b.n4;
    if (a.n3 != b.n3) return a.n3 < b.n3;
    return a.n2 < b.n2;
  });
  const int nP = (int)plist.size();
  int R2 = 0, R3 = 0, R4 = 0;
  for (int i = 0; i < nP; i++) {
    pslot(plist[i].n2, plist[i].n3, plist[i].n4) = i;
    R2 = std::max(R2, std::abs(plist[i].n2));
    R3 = std::max(R3, std::abs(plist[i].n3));
    R4 = std::max(R4, plist[i].n4);
  }
  // limits: the prep kernel's shared memory, the force epilogue scales
  const size_t prep_smem = (((size_t)nP * 4 + 15) & ~(size_t)15) +
                           (d >= 3 ? (size_t)kPrepStaged * (R2 + 1 + R3 + 1 + (d == 4 ? R4 + 1 : 0)) * sizeof(qent) : 0);
  int lg = 0;
  while ((1ll << lg) < 2ll * nP) lg++;
  int lf = 0;
  while ((1ll << lf) < 4ll * std::max(1, R1) * 2ll * nP) lf++;
  if (prep_smem > kPrepSmemMax || 16 - lg < 1 || 126 - lf < 64 || encode_tiled() == nullptr) return cudaSuccess;
  t.d = d;
  t.lift = lift;
  t.R1 = R1;
  t.Rax[0] = R1;
  t.Rax[1] = R2;
  t.Rax[2] = d >= 3 ? R3 : 0;
  t.Rax[3] = d == 4 ? R4 : 0;
  t.nP = nP;
  t.gs = 16 - lg;  // G~ (|.| <= 2 nP) held as R' 2^gs below 2^126
  t.ts = 126 - lf;  // partial sums of four n1 terms weighted by n1 <= R1, value 2^ts, below 2^126
  t.prep_smem = prep_smem;
  t.pvec.resize(nP);
  for (int i = 0; i < nP; i++) {
    const PVec& v = plist[i];
    t.pvec[i] = d == 4 ? (int32_t)(((uint32_t)v.n2 & 0x3ffu) | (((uint32_t)v.n3 & 0x3ffu) << 10) | ((uint32_t)v.n4 << 20))
                       : (int32_t)(((uint32_t)v.n2 & 0xffffu) | ((uint32_t)v.n3 << 16));
  }
  const int W1 = R1 + 1;
  t.RT = (2 * nP + kTileM - 1) / kTileM;
  t.CTd = (2 * W1 + kTileN - 1) / kTileN;
  t.KSf = (2 * nP + kStepK - 1) / kStepK;
  const int npt = 16 / d;  // force column tile: n1 in [npt ct, npt ct + npt), every axis of each (2 d columns per n1)
  t.CTf = (W1 + npt - 1) / npt;
  t.NPg = (int64_t)t.RT * (kTileM / 8);
  // Transposed remainder tile (two axes).  The last row tile holds rows (p, cos / sin) of the canonical p >= p0
  // only, often a small fraction of its 128 rows, yet it is paired with every column tile its members reach.  When
  // those p fit 32 columns and their n1 fit the rows the force never reads (from the K-step boundary past 2 nP), one
  // tile with the roles swapped covers them all: rows (n1, cos / sin) of a_j(n1), columns (p, cos / sin) of w_j(p).
  t.tr = 0;
  if (d == 2 && t.RT >= 2) {
    const int p0 = (kTileM / 2) * (t.RT - 1);
    const int row0 = (2 * nP + kStepK - 1) / kStepK * kStepK - kTileM * (t.RT - 1);
    int n1max = -1;
    std::vector<char> reach(t.CTd, 0);
    for (int64_t k = 0; k < M; k++) {
      int n1, n2, n3, n4;
      sub_vec(*c, lift, k, n1, n2, n3, n4);
      pcan(n2, n3, n4);
      const int p = pslot(n2, n3, n4);
      if (p >= p0) {
        n1max = std::max(n1max, n1);
        reach[(2 * n1) >> 5] = 1;
      }
    }
    int used = 0;
    for (char r : reach) used += r;
    if (2 * (nP - p0) <= kTileN && row0 + 2 * (n1max + 1) <= kTileM && used >= 2) {
      t.tr = 1;
      t.trP0 = p0;
      t.trRow0 = row0;
      t.trN1 = n1max + 1;
      t.CTd += 1;
    }
  }
  t.bexp = 0;
  while ((1 << t.bexp) <= std::max(R2, std::max(R3, R4))) t.bexp++;
  // emit map: k = (n1, p) -> [p][n1][0], k = (n1, -p) -> [p][n1][1]
  t.em.assign((size_t)nP * W1 * 2, -1);
  t.tilemap.assign((size_t)t.RT * t.CTd, -1);
  std::vector<int> pmax_ct(t.CTf, -1);
  for (int64_t k = 0; k < M; k++) {
    int n1, n2, n3, n4;
    sub_vec(*c, lift, k, n1, n2, n3, n4);
    const bool can = pcan(n2, n3, n4);
    const int p = pslot(n2, n3, n4);
    t.em[((size_t)p * W1 + n1) * 2 + (can ? 0 : 1)] = (int32_t)k;
    if (t.tr && p >= t.trP0)
      t.tilemap[(size_t)(t.RT - 1) * t.CTd + (t.CTd - 1)] = 1;
    else
      t.tilemap[(size_t)((2 * p) >> 7) * t.CTd + ((2 * n1) >> 5)] = 1;
    pmax_ct[n1 / npt] = std::max(pmax_ct[n1 / npt], p);
  }
  for (int i = 0; i < t.RT * t.CTd; i++)
    if (t.tilemap[i] >= 0) {
      t.tilemap[i] = (int32_t)t.tiles.size();
      t.tiles.push_back(i);
    }
  // force K range of each column tile: the rows (p, cos / sin) up to the last p with a set member at one of its n1
  // (p is sorted by |p|: the range of a tile of large n1 is a small disk)
  t.ks_ct.resize(t.CTf);
  for (int ct = 0; ct < t.CTf; ct++) t.ks_ct[ct] = pmax_ct[ct] < 0 ? 0 : (2 * (pmax_ct[ct] + 1) + kStepK - 1) / kStepK;
  // split force K: when the (particle tile, column tile) items of the whole configuration are fewer than the SMs,
  // each column tile's K range is cut into up to fsplit pieces of at least one read-out chunk (their force limbs add
  // up by integer atomics).  The split follows from N and the set alone, not from a chunk, a shard or a batch, so
  // that the truncation of each piece's a_j(n1) G product, and with it every bit of F, is the same in all of them.
  {
    int used = 0;
    for (int ct = 0; ct < t.CTf; ct++) used += t.ks_ct[ct] > 0;
    const int64_t items = (c->N + kTileM - 1) / kTileM * std::max(1, used);
    t.fsplit = (int)std::max<int64_t>(1, std::min<int64_t>(8, std::max(1, c->sm_count) / items));
  }
  const int nt = (int)t.tiles.size();

  t.ntab = kPrepLow + std::max(std::max(R1, R4), std::max(R2, R3)) / kPrepLow + 1;
  // particles per chunk.  The digit tensor, the density B digits, the Q2.126 a_j(n1) and the tables hold one
  // chunk; the density sums run over the chunks into the same exact accumulators and the force rows of a chunk
  // are its own particles, so the results do not depend on the chunking.  By default every particle is one
  // chunk when these buffers fit in 70% of the free device memory.  The chunks cover the context's particles:
  // all N, or its shard.
  {
    const int64_t Np = part_n(c);
    const double bpp = (double)kDigits * t.NPg * 16 + (double)t.CTd * kStageB / kStepK + (double)W1 * sizeof(fxc) +
                       (double)d * t.ntab * sizeof(qent);  // bytes per particle of the chunk buffers
    const int64_t Nr = (Np + kTileM - 1) / kTileM * kTileM;
    int64_t Nc = Nr;
    if (c->tc_chunk_req > 0) {
      Nc = c->tc_chunk_req;
    } else {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && bpp * (double)Nr > 0.7 * (double)fr) {
        const int64_t nch = (int64_t)std::ceil(bpp * (double)Nr / (0.7 * (double)fr));
        Nc = (Np + nch - 1) / nch;
      }
    }
    const int64_t Nmin = (Np + kMaxTcPhases - 1) / kMaxTcPhases;  // at most kMaxTcPhases chunks
    Nc = std::max(Nc, Nmin);
    Nc = std::min((Nc + kTileM - 1) / kTileM * kTileM, Nr);
    t.Nc = Nc;
    t.nchunk = (int)((Np + Nc - 1) / Nc);
  }
  t.KS = t.Nc / kStepK;
  t.PT = (int)(t.Nc / kTileM);
  t.NJ = (int64_t)t.PT * (kTileM / 8);
  cudaStream_t st = c->stream;
  cudaError_t e;
  if ((e = tc_dev_alloc(&t.wT, (size_t)kDigits * t.NPg * t.NJ * 128, st)) != cudaSuccess) return e;
  if ((e = tc_dev_alloc(&t.aB, (size_t)t.CTd * t.KS * kStageB, st)) != cudaSuccess) return e;
  if ((e = tc_dev_alloc(&t.fB, (size_t)t.CTf * t.KSf * kStageB, st)) != cudaSuccess) return e;
  if ((e = tc_dev_alloc(&t.a1, (size_t)W1 * t.Nc * sizeof(fxc), st)) != cudaSuccess) return e;
  if ((e = tc_dev_alloc(&t.tab, (size_t)d * t.Nc * t.ntab * sizeof(qent), st)) != cudaSuccess) return e;
  if ((e = tc_dev_alloc(&t.acc, (size_t)nt * 3 * kTileN * kTileM * 8, st)) != cudaSuccess) return e;
  if ((e = tc_dev_alloc(&t.facc, (size_t)d * 3 * c->N * 8, st)) != cudaSuccess) return e;
  if ((e = tc_dev_alloc(&t.em_d, t.em.size() * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(t.em_d.p, t.em.data(), t.em.size() * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if ((e = tc_dev_alloc(&t.pvec_d, t.pvec.size() * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(t.pvec_d.p, t.pvec.data(), t.pvec.size() * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  if ((e = tc_dev_alloc(&t.tilemap_d, t.tilemap.size() * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(t.tilemap_d.p, t.tilemap.data(), t.tilemap.size() * 4, cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return e;
  if ((e = tc_dev_alloc(&t.err, 16, st)) != cudaSuccess) return e;
  // tensor maps of the digit tensor [slice][row group][particle group][64 bf16]: the density box (two particle
  // groups x sixteen row groups) and the force box (sixteen particle groups x two row groups), all 15 slices
  {
    const cuuint64_t gdim[4] = {64, (cuuint64_t)t.NJ, (cuuint64_t)t.NPg, (cuuint64_t)kDigits};
    const cuuint64_t gstr[3] = {128, (cuuint64_t)t.NJ * 128, (cuuint64_t)t.NJ * (cuuint64_t)t.NPg * 128};
    const cuuint32_t box_d[4] = {64, 2, 16, (cuuint32_t)kDigits}, box_f[4] = {64, 16, 2, (cuuint32_t)kDigits};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(t.tmap_h);
    for (int m = 0; m < 2; m++) {
      const CUresult r = encode_tiled()(&maps[m], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, t.wT.p, gdim, gstr,
                                        m == 0 ? box_d : box_f, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    if ((e = tc_dev_alloc(&t.tmap, 2 * sizeof(CUtensorMap), st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(t.tmap.p, t.tmap_h, 2 * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return e;
    // the host copy must outlive the asynchronous upload
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  }
  t.on = true;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
    cudaFuncSetAttribute(k_tc_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
    cudaFuncSetAttribute(k_tc_prep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPrepSmemMax);
    cudaFuncSetAttribute(k_tc_prep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPrepSmemMax);
    attr = true;
  }
  return cudaGetLastError();
}

void tc_free(Ctx* c) {
  TcPlan& t = c->tc;
  for (DevBuf* b : {&t.wT, &t.aB, &t.fB, &t.a1, &t.tab, &t.acc, &t.facc, &t.em_d, &t.pvec_d, &t.tilemap_d, &t.tmap, &t.err}) {
    if (b->p) cudaFree(b->p);
    b->p = nullptr;
    b->bytes = 0;
  }
  t.on = false;
}

size_t tc_footprint(const Ctx& c) {
  const TcPlan& t = c.tc;
  if (!t.on) return 0;
  size_t b = 0;
  for (const DevBuf* x : {&t.wT, &t.aB, &t.fB, &t.a1, &t.tab, &t.acc, &t.facc, &t.em_d, &t.pvec_d, &t.tilemap_d, &t.tmap})
    b += x->bytes;
  return b;
}

void tc_fill_cfgdev(const Ctx* c, CfgDev* g) {
  const TcPlan& t = c->tc;
  g->tc = t.on ? 1 : 0;
  if (!t.on) return;
  g->tc_d = t.d;
  g->tc_lift = t.lift;
  g->tc_tr = t.tr;
  g->tc_trP0 = t.trP0;
  g->tc_trRow0 = t.trRow0;
  g->tc_trN1 = t.trN1;
  g->tc_R1 = t.R1;
  g->tc_nP = t.nP;
  for (int a = 0; a < 4; a++) g->tc_Rax[a] = t.Rax[a];
  g->tc_RT = t.RT;
  g->tc_CTd = t.CTd;
  g->tc_PT = t.PT;
  g->tc_KSf = t.KSf;
  g->tc_CTf = t.CTf;
  g->tc_bexp = t.bexp;
  g->tc_KS = t.KS;
  g->tc_NJ = t.NJ;
  g->tc_NPg = t.NPg;
  g->tc_j0 = part_p0(c);  // chunk 0 (tc_chunk_cfgdev for the others)
  g->tc_n = std::min<int64_t>(part_n(c), t.Nc);
  g->tc_nbuf = t.Nc;
  g->tc_wT = (uint8_t*)t.wT.p;
  g->tc_aB = (uint8_t*)t.aB.p;
  g->tc_fB = (uint8_t*)t.fB.p;
  g->tc_a1 = t.a1.p;
  g->tc_tab = t.tab.p;
  g->tc_ntab = t.ntab;
  g->tc_acc = (long long*)t.acc.p;
  g->tc_facc = (long long*)t.facc.p;
  g->tc_nblk = tc_finish_blocks(*c);
  g->tc_em = (const int32_t*)t.em_d.p;
  g->tc_pvec = (const int32_t*)t.pvec_d.p;
  g->tc_tilemap = (const int32_t*)t.tilemap_d.p;
  g->tc_tmap = t.tmap.p;
  g->tc_err = (int*)t.err.p;
  g->tc_gs = t.gs;
  g->tc_ts = t.ts;
  g->psplit[SSH_FX] = 1;
}

int tc_chunks(const Ctx* c) { return c->tc.on ? c->tc.nchunk : 0; }

long long* tc_acc_ptr(const Ctx* c) { return c->tc.on ? reinterpret_cast<long long*>(c->tc.acc.p) : nullptr; }
int64_t tc_acc_words(const Ctx* c) { return c->tc.on ? (int64_t)c->tc.tiles.size() * 3 * kTileN * kTileM : 0; }

static int64_t chunk_len(const Ctx* c, int ch) { return std::min<int64_t>(c->tc.Nc, part_n(c) - (int64_t)ch * c->tc.Nc); }

void tc_chunk_cfgdev(const Ctx* c, int ch, CfgDev* g) {
  g->tc_j0 = part_p0(c) + (int64_t)ch * c->tc.Nc;
  g->tc_n = chunk_len(c, ch);
}

// density K-steps (tiles x K-steps) of one chunk
int64_t tc_density_steps(const Ctx* c, int ch) {
  return c->tc.on ? (int64_t)c->tc.tiles.size() * ((chunk_len(c, ch) + kStepK - 1) / kStepK) : 0;
}

// blocks (128 threads) of the tables kernel for one chunk: two threads per (axis, particle)
int64_t tc_table_blocks(const Ctx* c, int ch) { return (2 * (int64_t)c->tc.d * chunk_len(c, ch) + 127) / 128; }

// preparation items of one chunk (cfg: its descriptor in the engine), the heavier w items first.  w items of
// three or four axes cover 16 particles (their powers fill shared memory); a table item covers enough groups of 8 particles for 128
// (entry, group) lane pairs, at most 128 particles.  They reach the chunk's last K-step boundary, so that stale
// digits of an earlier, longer chunk never enter the density sums.
void tc_prep_items(const Ctx* c, int cfg, int ch, std::vector<TwItem>& prep) {
  const TcPlan& t = c->tc;
  const int64_t npad = (chunk_len(c, ch) + kStepK - 1) / kStepK * kStepK;
  for (int kind = 1; kind >= 0; kind--) {
    const int count = kind == 0 ? t.R1 + 1 : t.nP;
    const bool staged = kind == 1 && t.d >= 3;
    int ng = staged ? kPrepStaged / 8 : 1;
    if (!staged)
      while (ng < kPrepTable / 8 && ng * count < kPrepThreads / 2) ng *= 2;
    for (int64_t j = 0; j < npad; j += 8 * ng) prep.push_back({cfg, kind | (staged ? 1 << 8 : 0) | (ng << 9), j});
  }
}

// GEMM items of one chunk; pieces: the density pieces this chunk should be cut into (about its share of the SMs)
void tc_gemm_items(const Ctx* c, int cfg, int ch, int64_t pieces, std::vector<TcItem>& dens, std::vector<TcItem>& force) {
  const TcPlan& t = c->tc;
  const int64_t n = chunk_len(c, ch);
  const int64_t KS = (n + kStepK - 1) / kStepK;
  // density pieces.  The column tiles of a row tile read the same rows of w, so their pieces share K ranges and
  // sit next to each other in the list: CTAs claim them together and the second read of each w stage hits L2.
  // Each row tile splits uniformly into `split` K ranges (at most one per read-out chunk); when the tiles do not
  // divide the pieces and the pieces are long (128 K-steps and more), the K-steps of the row tiles are laid end to
  // end and cut every `len` steps instead, so that every SM gets about the same work (a cut also falls at each row
  // tile's end).  A piece holds at most 1024 read-outs, so the int64 level groups (below 2^52 per read-out)
  // cannot overflow.
  const int64_t nt = (int64_t)t.tiles.size();
  const int64_t total = nt * KS;
  const int64_t want = std::max<int64_t>(1, pieces);
  const int64_t len = std::min<int64_t>(1024 * kChunkSteps, std::max<int64_t>(1, (total + want - 1) / want));
  const bool cross = want > nt && want % nt != 0 && len >= 8 * kChunkSteps;
  int64_t split = std::max<int64_t>(1, std::min<int64_t>((KS + kChunkSteps - 1) / kChunkSteps, want / nt));
  split = std::max<int64_t>(split, (KS + 1024 * kChunkSteps - 1) / (1024 * kChunkSteps));
  auto emit = [&](int ti0, int ti1, int64_t k0, int64_t k1) {  // one piece per column tile of the row tile
    for (int ti = ti0; ti < ti1; ti++)
      dens.push_back({cfg, 0, t.tiles[ti] / t.CTd, t.tiles[ti] % t.CTd, (int32_t)k0, (int32_t)(k1 - k0), ti, 0});
  };
  int64_t g0 = 0;  // K-steps of the row tiles before this one (cut grid)
  for (int ti0 = 0; ti0 < (int)nt;) {
    int ti1 = ti0;  // tiles are listed row tile by row tile
    while (ti1 < (int)nt && t.tiles[ti1] / t.CTd == t.tiles[ti0] / t.CTd) ti1++;
    if (cross) {
      for (int64_t k0 = 0; k0 < KS;) {  // cut where the global K-step g0 + k reaches a multiple of len
        const int64_t k1 = std::min<int64_t>(KS, k0 + (len - (g0 + k0) % len));
        emit(ti0, ti1, k0, k1);
        k0 = k1;
      }
      g0 += KS;
    } else {
      for (int64_t sp = 0; sp < split; sp++) {
        const int64_t k0 = KS * sp / split, k1 = KS * (sp + 1) / split;
        if (k1 > k0) emit(ti0, ti1, k0, k1);
      }
    }
    ti0 = ti1;
  }
  // force items: particle tile x column tile, with the K range of the column tile (the coefficients beyond are
  // zero), particle-tile-major: the column tiles of one particle tile are claimed together from the queue and
  // read the particle tile's digits from L2 once they are in
  const int PT = (int)((n + kTileM - 1) / kTileM);
  for (int pt = 0; pt < PT; pt++)
    for (int ct = 0; ct < t.CTf; ct++) {
      const int ks = t.ks_ct[ct];
      const int sp = std::max(1, std::min(t.fsplit, ks / kChunkSteps));  // pieces of at least one read-out chunk
      for (int i = 0; i < sp; i++) {
        const int k0 = (int)((int64_t)ks * i / sp), k1 = (int)((int64_t)ks * (i + 1) / sp);
        if (k1 > k0) force.push_back({cfg, 1, pt, ct, k0, k1 - k0, ct, 0});
      }
    }
}

size_t tc_gemm_smem() { return kGemmSmem; }

cudaError_t tc_launch_force_finish(const EngineView& v, cudaStream_t st, Prof* prof) {
  if (v.ntc_list == 0) return cudaSuccess;
  prof_begin(prof, st, kKTcFinish);
  cudaError_t le = launch_pdl(k_tc_force_finish, dim3((unsigned)v.ntc_bm_ff), dim3(kFinThreads), 0, st, v.cfgs, v.tc_bm_ff);
  if (le != cudaSuccess) return le;
  prof_end(prof, st);
  return cudaGetLastError();
}

// prep4: the last items of the range, those of four-axis members (their own kernel instance); one profiler record
// covers both launches
static cudaError_t launch_tables_prep(const EngineView& v, int tab_off, int tab_n, int prep_off, int prep_n, int prep4,
                                      cudaStream_t st, Prof* prof) {
  if (tab_n > 0) {
    prof_begin(prof, st, kKTcTables);
    const cudaError_t le =
        launch_pdl(k_tc_tables, dim3((unsigned)tab_n), dim3(128), 0, st, v.cfgs, v.tc_bm_tab + tab_off);
    if (le != cudaSuccess) return le;
    prof_end(prof, st);
  }
  if (prep_n > 0) {
    prof_begin(prof, st, kKTcPrep);
    if (prep_n > prep4) {
      const cudaError_t le = launch_pdl(k_tc_prep<false>, dim3((unsigned)(prep_n - prep4)), dim3(kPrepThreads),
                                        v.tc_prep_smem, st, v.cfgs, v.tc_prep + prep_off);
      if (le != cudaSuccess) return le;
    }
    if (prep4 > 0) {
      const cudaError_t le = launch_pdl(k_tc_prep<true>, dim3((unsigned)prep4), dim3(kPrepThreads), v.tc_prep_smem, st,
                                        v.cfgs, v.tc_prep + prep_off + (prep_n - prep4));
      if (le != cudaSuccess) return le;
    }
    prof_end(prof, st);
  }
  return cudaSuccess;
}

// chunk by chunk: tables, preparation, density GEMM (into the exact tile accumulators); then the finish
cudaError_t tc_launch_density(const EngineView& v, cudaStream_t st, Prof* prof) {
  const cudaError_t le = tc_launch_density_gemms(v, st, prof);
  if (le != cudaSuccess) return le;
  return tc_launch_dens_finish(v, st, prof);
}

cudaError_t tc_launch_density_gemms(const EngineView& v, cudaStream_t st, Prof* prof) {
  if (v.ntc_list == 0) return cudaSuccess;
  for (int ph = 0; ph < v.ntc_phase; ph++) {
    const TcPhase& P = v.tc_ph[ph];
    cudaError_t le = launch_tables_prep(v, P.tab_off, P.tab_n, P.prep_off, P.prep_n, P.prep4, st, prof);
    if (le != cudaSuccess) return le;
    if (P.dens_n > 0) {
      prof_begin(prof, st, kKTcDens);
      le = launch_pdl(g_counters_on ? k_tc_gemm<true> : k_tc_gemm<false>, dim3((unsigned)std::min(P.dens_n, v.sm_count)),
                      dim3(kGemmThreads), kGemmSmem, st,
                      v.cfgs, v.tc_dens + P.dens_off, P.dens_n, v.counters + 2);
      if (le != cudaSuccess) return le;
      prof_end(prof, st);
    }
  }
  return cudaGetLastError();
}

cudaError_t tc_launch_dens_finish(const EngineView& v, cudaStream_t st, Prof* prof) {
  if (v.ntc_list == 0) return cudaSuccess;
  prof_begin(prof, st, kKTcFinish);
  const cudaError_t le =
      launch_pdl(k_tc_dens_finish, dim3((unsigned)v.ntc_bm_fin), dim3(kFinThreads), 0, st, v.cfgs, v.tc_bm_fin);
  if (le != cudaSuccess) return le;
  prof_end(prof, st);
  return cudaGetLastError();
}

// the coefficients, then chunk by chunk in reverse order (the last chunk's digits are still in the buffers): the
// preparation again where needed, and the force GEMM
cudaError_t tc_launch_force(const EngineView& v, cudaStream_t st, Prof* prof) {
  if (v.ntc_list == 0) return cudaSuccess;
  prof_begin(prof, st, kKTcCoef);
  cudaError_t le = launch_pdl(k_tc_coef, dim3((unsigned)v.ntc_bm_coef), dim3(128), 0, st, v.cfgs, v.tc_bm_coef);
  if (le != cudaSuccess) return le;
  prof_end(prof, st);
  for (int ph = v.ntc_phase - 1; ph >= 0; ph--) {
    const TcPhase& P = v.tc_ph[ph];
    le = launch_tables_prep(v, P.rtab_off, P.rtab_n, P.rprep_off, P.rprep_n, P.rprep4, st, prof);
    if (le != cudaSuccess) return le;
    if (P.force_n > 0) {
      prof_begin(prof, st, kKTcForce);
      le = launch_pdl(g_counters_on ? k_tc_gemm<true> : k_tc_gemm<false>, dim3((unsigned)std::min(P.force_n, v.sm_count)),
                      dim3(kGemmThreads), kGemmSmem, st,
                      v.cfgs, v.tc_force + P.force_off, P.force_n, v.counters + 4);
      if (le != cudaSuccess) return le;
      prof_end(prof, st);
    }
  }
  return cudaGetLastError();
}

}  // namespace ssh

// The limit of the tensor-core GEMM's waits on work, in clock cycles, on one device (0: the default, about one
// second at the maximum clock).  A wait that runs out records SSH_ETIMEOUT for the evaluation; this makes that
// path testable with a limit too short for any real wait.
extern "C" ssh_status ssh_gemm_counters(int device, int enable) {
  using namespace ssh;
  int cur = 0;
  cudaError_t e = cudaGetDevice(&cur);
  if (e == cudaSuccess && cur != device) e = cudaSetDevice(device);
  if (e == cudaSuccess && enable) {
    static unsigned long long zero[2 * kGcCtas * kGcFields];
    e = cudaMemcpyToSymbol(g_tc_counters, zero, sizeof zero);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (cur != device) cudaSetDevice(cur);
  if (e != cudaSuccess) {
    ssh::set_error(std::string("ssh_gemm_counters: ") + cudaGetErrorString(e));
    return SSH_ECUDA;
  }
  g_counters_on = enable != 0;
  return SSH_OK;
}

extern "C" ssh_status ssh_gemm_counters_read(int device, uint64_t* out) {
  using namespace ssh;
  if (!out) {
    ssh::set_error("ssh_gemm_counters_read: NULL output");
    return SSH_EINVAL;
  }
  int cur = 0;
  cudaError_t e = cudaGetDevice(&cur);
  if (e == cudaSuccess && cur != device) e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(out, g_tc_counters, sizeof(g_tc_counters));
  if (cur != device) cudaSetDevice(cur);
  if (e != cudaSuccess) {
    ssh::set_error(std::string("ssh_gemm_counters_read: ") + cudaGetErrorString(e));
    return SSH_ECUDA;
  }
  return SSH_OK;
}

extern "C" ssh_status ssh_set_wait_limit(int device, int64_t cycles) {
  if (cycles < 0) {
    ssh::set_error("ssh_set_wait_limit: negative limit");
    return SSH_EINVAL;
  }
  int cur = 0;
  cudaError_t e = cudaGetDevice(&cur);
  if (e == cudaSuccess && cur != device) e = cudaSetDevice(device);
  const long long v = cycles == 0 ? ssh::kWaitLimit : (long long)cycles;
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(ssh::g_tc_wait_limit, &v, sizeof v);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (cur != device) cudaSetDevice(cur);
  if (e != cudaSuccess) {
    ssh::set_error(std::string("ssh_set_wait_limit: ") + cudaGetErrorString(e));
    return SSH_ECUDA;
  }
  return SSH_OK;
}
