// fx.cuh -- 128-bit fixed-point arithmetic on the integer pipes, the B300 form of "dd precision".
//
// On this GPU the FP64 pipe issues about 1.6 FMA per clock per SM while the integer multiply-add pipe
// issues 64 and the ALU pipes 128, so the sums the paper carries in double-double arithmetic (Simulations)
// are carried in the integer units instead:
//   * positions are unsigned Q0.128 fractions of the box (s = u / 2^128), so the phase of k = 2 pi n / L,
//     t = n.s mod 1, is an exact integer product that wraps modulo 2^128 -- argument reduction is free;
//   * phasors, tables and scaled densities are signed two's-complement Q2.126 (value = X / 2^126,
//     range [-2, 2), resolution 2^-126 ~ 1.2e-38), four little-endian 32-bit limbs;
//   * sums are five-limb Q34.126 accumulators: exact, so every reduction order gives bit-identical sums.
// mul126(a, b) = (a * b) >> 126 from a truncated 128 x 128 product: the partial products below limb 3
// are dropped, so the result is low by at most 12 units of 2^-126.
#pragma once
#include <stdint.h>

#include "dd.cuh"

struct __align__(16) q128 {
  uint32_t w[4];
};
struct q160 {
  uint32_t w[5];
};

__device__ __forceinline__ q128 q128_zero() { q128 r; r.w[0] = r.w[1] = r.w[2] = r.w[3] = 0u; return r; }
__device__ __forceinline__ q160 q160_zero() { q160 r; r.w[0] = r.w[1] = r.w[2] = r.w[3] = r.w[4] = 0u; return r; }

__device__ __forceinline__ q128 q128_add(const q128& a, const q128& b) {
  q128 r;
  asm("add.cc.u32 %0, %4, %8;\n\t"
      "addc.cc.u32 %1, %5, %9;\n\t"
      "addc.cc.u32 %2, %6, %10;\n\t"
      "addc.u32 %3, %7, %11;"
      : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3])
      : "r"(a.w[0]), "r"(a.w[1]), "r"(a.w[2]), "r"(a.w[3]), "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]));
  return r;
}

__device__ __forceinline__ q128 q128_sub(const q128& a, const q128& b) {
  q128 r;
  asm("sub.cc.u32 %0, %4, %8;\n\t"
      "subc.cc.u32 %1, %5, %9;\n\t"
      "subc.cc.u32 %2, %6, %10;\n\t"
      "subc.u32 %3, %7, %11;"
      : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3])
      : "r"(a.w[0]), "r"(a.w[1]), "r"(a.w[2]), "r"(a.w[3]), "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]));
  return r;
}

__device__ __forceinline__ q128 q128_neg(const q128& a) { return q128_sub(q128_zero(), a); }

// acc += sign-extended a
__device__ __forceinline__ void q160_add(q160& acc, const q128& a) {
  uint32_t sx = (uint32_t)((int32_t)a.w[3] >> 31);
  asm("add.cc.u32 %0, %0, %5;\n\t"
      "addc.cc.u32 %1, %1, %6;\n\t"
      "addc.cc.u32 %2, %2, %7;\n\t"
      "addc.cc.u32 %3, %3, %8;\n\t"
      "addc.u32 %4, %4, %9;"
      : "+r"(acc.w[0]), "+r"(acc.w[1]), "+r"(acc.w[2]), "+r"(acc.w[3]), "+r"(acc.w[4])
      : "r"(a.w[0]), "r"(a.w[1]), "r"(a.w[2]), "r"(a.w[3]), "r"(sx));
}

__device__ __forceinline__ void q160_add160(q160& acc, const q160& a) {
  asm("add.cc.u32 %0, %0, %5;\n\t"
      "addc.cc.u32 %1, %1, %6;\n\t"
      "addc.cc.u32 %2, %2, %7;\n\t"
      "addc.cc.u32 %3, %3, %8;\n\t"
      "addc.u32 %4, %4, %9;"
      : "+r"(acc.w[0]), "+r"(acc.w[1]), "+r"(acc.w[2]), "+r"(acc.w[3]), "+r"(acc.w[4])
      : "r"(a.w[0]), "r"(a.w[1]), "r"(a.w[2]), "r"(a.w[3]), "r"(a.w[4]));
}

__device__ __forceinline__ q160 q160_sub160(const q160& a, const q160& b) {
  q160 r;
  asm("sub.cc.u32 %0, %5, %10;\n\t"
      "subc.cc.u32 %1, %6, %11;\n\t"
      "subc.cc.u32 %2, %7, %12;\n\t"
      "subc.cc.u32 %3, %8, %13;\n\t"
      "subc.u32 %4, %9, %14;"
      : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3]), "=r"(r.w[4])
      : "r"(a.w[0]), "r"(a.w[1]), "r"(a.w[2]), "r"(a.w[3]), "r"(a.w[4]), "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]),
        "r"(b.w[3]), "r"(b.w[4]));
  return r;
}

// acc * k for a small signed integer k (|acc * k| < 2^159), exact.
__device__ __forceinline__ q160 q160_mul_int(const q160& a, int32_t k) {
  uint32_t m = (uint32_t)(k < 0 ? -k : k);
  q160 r;
  asm("mul.lo.u32 %0, %5, %10;\n\t"
      "mul.hi.u32 %1, %5, %10;\n\t"
      "mad.lo.cc.u32 %1, %6, %10, %1;\n\t"
      "madc.hi.u32 %2, %6, %10, 0;\n\t"
      "mad.lo.cc.u32 %2, %7, %10, %2;\n\t"
      "madc.hi.u32 %3, %7, %10, 0;\n\t"
      "mad.lo.cc.u32 %3, %8, %10, %3;\n\t"
      "madc.hi.u32 %4, %8, %10, 0;\n\t"
      "mad.lo.u32 %4, %9, %10, %4;"
      : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3]), "=r"(r.w[4])
      : "r"(a.w[0]), "r"(a.w[1]), "r"(a.w[2]), "r"(a.w[3]), "r"(a.w[4]), "r"(m));
  // the unsigned product of the two's-complement bit pattern is correct modulo 2^160
  if (k < 0) r = q160_sub160(q160_zero(), r);
  return r;
}

// Limbs 3..7 (r[0] = limb 3) of the unsigned 256-bit product a * b, dropping the partial products of
// limbs 0..2 (so r[1..4] is low by at most 3).  20 multiply-adds on the IMAD pipe.
__device__ __forceinline__ void umul_top(const q128& a, const q128& b, uint32_t r[5]) {
  asm("mul.lo.u32 %0, %5, %12;\n\t"
      "mul.hi.u32 %1, %5, %12;\n\t"
      // row 1: a1 * (b2, b3)
      "mad.lo.cc.u32 %0, %6, %11, %0;\n\t"
      "madc.lo.cc.u32 %1, %6, %12, %1;\n\t"
      "addc.u32 %2, 0, 0;\n\t"
      "mad.hi.cc.u32 %1, %6, %11, %1;\n\t"
      "madc.hi.cc.u32 %2, %6, %12, %2;\n\t"
      "addc.u32 %3, 0, 0;\n\t"
      // row 2: a2 * (b1, b2, b3)
      "mad.lo.cc.u32 %0, %7, %10, %0;\n\t"
      "madc.lo.cc.u32 %1, %7, %11, %1;\n\t"
      "madc.lo.cc.u32 %2, %7, %12, %2;\n\t"
      "addc.u32 %3, %3, 0;\n\t"
      "mad.hi.cc.u32 %1, %7, %10, %1;\n\t"
      "madc.hi.cc.u32 %2, %7, %11, %2;\n\t"
      "madc.hi.cc.u32 %3, %7, %12, %3;\n\t"
      "addc.u32 %4, 0, 0;\n\t"
      // row 3: a3 * (b0, b1, b2, b3)
      "mad.lo.cc.u32 %0, %8, %9, %0;\n\t"
      "madc.lo.cc.u32 %1, %8, %10, %1;\n\t"
      "madc.lo.cc.u32 %2, %8, %11, %2;\n\t"
      "madc.lo.cc.u32 %3, %8, %12, %3;\n\t"
      "addc.u32 %4, %4, 0;\n\t"
      "mad.hi.cc.u32 %1, %8, %9, %1;\n\t"
      "madc.hi.cc.u32 %2, %8, %10, %2;\n\t"
      "madc.hi.cc.u32 %3, %8, %11, %3;\n\t"
      "madc.hi.u32 %4, %8, %12, %4;"
      : "=&r"(r[0]), "=&r"(r[1]), "=&r"(r[2]), "=&r"(r[3]), "=&r"(r[4])
      : "r"(a.w[0]), "r"(a.w[1]), "r"(a.w[2]), "r"(a.w[3]), "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]));
}

// Signed correction of the top half: for two's-complement a, b the signed product's bits 128..255 are
// the unsigned ones minus (a < 0 ? b : 0) minus (b < 0 ? a : 0), modulo 2^128.
__device__ __forceinline__ void smul_top(const q128& a, const q128& b, uint32_t r[5]) {
  umul_top(a, b, r);
  uint32_t ma = (uint32_t)((int32_t)a.w[3] >> 31), mb = (uint32_t)((int32_t)b.w[3] >> 31);
  asm("sub.cc.u32 %0, %0, %4;\n\t"
      "subc.cc.u32 %1, %1, %5;\n\t"
      "subc.cc.u32 %2, %2, %6;\n\t"
      "subc.u32 %3, %3, %7;"
      : "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4])
      : "r"(b.w[0] & ma), "r"(b.w[1] & ma), "r"(b.w[2] & ma), "r"(b.w[3] & ma));
  asm("sub.cc.u32 %0, %0, %4;\n\t"
      "subc.cc.u32 %1, %1, %5;\n\t"
      "subc.cc.u32 %2, %2, %6;\n\t"
      "subc.u32 %3, %3, %7;"
      : "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4])
      : "r"(a.w[0] & mb), "r"(a.w[1] & mb), "r"(a.w[2] & mb), "r"(a.w[3] & mb));
}

// Q2.126 x Q2.126 -> Q2.126: bits 126..253 of the signed product.
__device__ __forceinline__ q128 mul126(const q128& a, const q128& b) {
  uint32_t r[5];
  smul_top(a, b, r);
  q128 o;
  o.w[0] = __funnelshift_l(r[0], r[1], 2);
  o.w[1] = __funnelshift_l(r[1], r[2], 2);
  o.w[2] = __funnelshift_l(r[2], r[3], 2);
  o.w[3] = __funnelshift_l(r[3], r[4], 2);
  return o;
}

// complex Q2.126
struct fxc {
  q128 re, im;
};

// complex Q34.126 accumulator (one partial or final n~(k))
struct FxAcc {
  q160 re, im;
};

__device__ __forceinline__ fxc fxc_mul(const fxc& a, const fxc& b) {
  fxc z;
  z.re = q128_sub(mul126(a.re, b.re), mul126(a.im, b.im));
  z.im = q128_add(mul126(a.re, b.im), mul126(a.im, b.re));
  return z;
}

__device__ __forceinline__ fxc fxc_conj(const fxc& a) {
  fxc z;
  z.re = a.re;
  z.im = q128_neg(a.im);
  return z;
}

// One as Q2.126.
__device__ __forceinline__ q128 q126_one() {
  q128 r = q128_zero();
  r.w[3] = 0x40000000u;
  return r;
}

// Exact conversions.  x * 2^shift as a signed 128-bit integer, truncated toward -infinity (|x| < 2^(127-shift)).
__device__ __forceinline__ __int128 d2i128_scaled(double x, int shift) {
  if (x == 0.0) return 0;
  int e;
  double m = frexp(x, &e);  // x = m 2^e, 0.5 <= |m| < 1
  long long mant = (long long)ldexp(m, 53);  // exact, |mant| < 2^53
  int sh = e - 53 + shift;
  __int128 v = (__int128)mant;
  if (sh >= 0) return v << sh;
  if (sh <= -64) return mant < 0 ? (__int128)-1 : (__int128)0;
  return v >> (-sh);  // arithmetic shift: floor
}

__device__ __forceinline__ q128 q128_from_i128(__int128 v) {
  unsigned __int128 u = (unsigned __int128)v;
  q128 r;
  r.w[0] = (uint32_t)u;
  r.w[1] = (uint32_t)(u >> 32);
  r.w[2] = (uint32_t)(u >> 64);
  r.w[3] = (uint32_t)(u >> 96);
  return r;
}

// Fractional position (hi + lo, any real; only the value mod 1 matters) as an unsigned Q0.128 turn.
__device__ __forceinline__ q128 turns_from_dd(double hi, double lo) {
  // remove the integer part exactly (hi - floor(hi) can round for small negative hi): f + e = hi - floor(hi)
  dd f = two_sum(hi, -floor(hi));
  if (f.hi >= 1.0) f.hi -= 1.0;  // f.hi = 1 exactly when e < 0; one turn is zero modulo 2^128
  // f.hi * 2^128 can exceed the signed range: scale by 2^127, then double in unsigned (wrapping) arithmetic
  unsigned __int128 v = (unsigned __int128)d2i128_scaled(f.hi, 127) * 2u + (unsigned __int128)d2i128_scaled(f.lo, 128) +
                        (unsigned __int128)d2i128_scaled(lo, 128);
  return q128_from_i128((__int128)v);
}

// dd value x (|x| < 2) as Q2.126.
__device__ __forceinline__ q128 q126_from_dd(double hi, double lo) {
  return q128_from_i128(d2i128_scaled(hi, 126) + d2i128_scaled(lo, 126));
}

// Five-limb Q34.126 accumulator to a double-double value (exact pieces, accurate dd sums).
__device__ __forceinline__ void q160_to_dd(const q160& a, double* hi, double* lo) {
  double p4 = ldexp((double)(int32_t)a.w[4], 128 - 126);
  double p3 = ldexp((double)a.w[3], 96 - 126);
  double p2 = ldexp((double)a.w[2], 64 - 126);
  double p1 = ldexp((double)a.w[1], 32 - 126);
  double p0 = ldexp((double)a.w[0], -126);
  dd s = dd_make(p4, 0.0);
  s = dd_add_d(s, p3);
  s = dd_add_d(s, p2);
  s = dd_add_d(s, p1);
  s = dd_add_d(s, p0);
  *hi = s.hi;
  *lo = s.lo;
}

// e^{2 pi i t} for an unsigned Q0.128 turn t, as complex Q2.126.  t = c1 2^-8 + c2 2^-16 + r, r < 2^-16:
// table A[c1] * table B[c2] * (cos, sin)(2 pi r) with the Taylor series to theta^8 (theta < 1e-4).
// tab_a / tab_b: [256][8] limbs (cos then sin, Q2.126); pi_q: pi 2^125; inv_fact[n]: 1/n! in Q2.126.
__device__ __forceinline__ fxc fx_sincos_turns(const q128& t, const uint32_t (*tab_a)[8], const uint32_t (*tab_b)[8],
                                               const q128& pi_q, const uint32_t (*inv_fact)[4]) {
  uint32_t c1 = t.w[3] >> 24, c2 = (t.w[3] >> 16) & 255u;
  q128 r = t;
  r.w[3] &= 0xFFFFu;
  q128 th = mul126(r, pi_q);  // 2 pi r as Q2.126 (r, pi_q both non-negative)
  q128 t2 = mul126(th, th);
  auto C = [&](int n) { q128 v; v.w[0] = inv_fact[n][0]; v.w[1] = inv_fact[n][1]; v.w[2] = inv_fact[n][2]; v.w[3] = inv_fact[n][3]; return v; };
  // sin = th (1 - t2 (1/3! - t2 (1/5! - t2 / 7!)))
  q128 ps = q128_sub(C(5), mul126(C(7), t2));
  ps = q128_sub(C(3), mul126(ps, t2));
  ps = q128_sub(q126_one(), mul126(ps, t2));
  q128 sn = mul126(ps, th);
  // cos = 1 - t2 (1/2! - t2 (1/4! - t2 (1/6! - t2 / 8!)))
  q128 pc = q128_sub(C(6), mul126(C(8), t2));
  pc = q128_sub(C(4), mul126(pc, t2));
  pc = q128_sub(C(2), mul126(pc, t2));
  pc = q128_sub(q126_one(), mul126(pc, t2));
  fxc e;
  e.re = pc;
  e.im = sn;
  fxc a, b;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    a.re.w[i] = tab_a[c1][i];
    a.im.w[i] = tab_a[c1][4 + i];
    b.re.w[i] = tab_b[c2][i];
    b.im.w[i] = tab_b[c2][4 + i];
  }
  return fxc_mul(fxc_mul(a, b), e);
}

// ---------------------------------------------------------------------------------------------------------------
// First-quadrant form of a unit phasor, for the density kernel's inner loop.  z = i^q (c + i s) with c, s >= 0 as
// unsigned Q1.127 (value = X / 2^127), and cs = c + s for the three-product complex multiply; the quadrant q
// (0..3) lives in the two low bits of cs (an error of at most 3 * 2^-127 in cs).  Products of such values are the
// top halves of unsigned 256-bit products, already in Q2.126: no sign correction and no shift.
struct __align__(16) qent {
  q128 c, s, cs;
};

__device__ __forceinline__ q128 q128_shl1(const q128& a) {
  q128 r;
  r.w[3] = __funnelshift_l(a.w[2], a.w[3], 1);
  r.w[2] = __funnelshift_l(a.w[1], a.w[2], 1);
  r.w[1] = __funnelshift_l(a.w[0], a.w[1], 1);
  r.w[0] = a.w[0] << 1;
  return r;
}

// signed Q2.126 phasor (|z| ~ 1) -> first-quadrant form
__device__ __forceinline__ qent to_quadrant(const fxc& z) {
  const bool xn = (int32_t)z.re.w[3] < 0, yn = (int32_t)z.im.w[3] < 0;
  const uint32_t q = xn ? (yn ? 2u : 1u) : (yn ? 3u : 0u);
  q128 c, s;
  switch (q) {  // rotate by i^-q: both components become non-negative
    case 0: c = z.re; s = z.im; break;
    case 1: c = z.im; s = q128_neg(z.re); break;
    case 2: c = q128_neg(z.re); s = q128_neg(z.im); break;
    default: c = q128_neg(z.im); s = z.re; break;
  }
  qent e;
  e.c = q128_shl1(c);
  e.s = q128_shl1(s);
  e.cs = q128_add(e.c, e.s);
  e.cs.w[0] = (e.cs.w[0] & ~3u) | q;
  return e;
}

// Top 128 bits (limbs 4..7) of the unsigned 256-bit product a * b from 16 multiply-adds in carry chains: the high
// halves of the limb-3 column and everything above it.  The dropped low halves of column 3 and all lower columns
// sum to less than 7 * 2^128, so the result is low by at most 8 units of its last place (8 * 2^-126 in Q2.126).
__device__ __forceinline__ q128 umulhi(const q128& a, const q128& b) {
  q128 o;
  asm("mul.hi.u32 %0, %4, %11;\n\t"
      "mad.hi.cc.u32 %0, %5, %10, %0;\n\t"
      "addc.u32 %1, 0, 0;\n\t"
      "mad.hi.cc.u32 %0, %6, %9, %0;\n\t"
      "addc.u32 %1, %1, 0;\n\t"
      "mad.hi.cc.u32 %0, %7, %8, %0;\n\t"
      "addc.u32 %1, %1, 0;\n\t"
      // column 4: a1 b3, a2 b2, a3 b1
      "mad.lo.cc.u32 %0, %5, %11, %0;\n\t"
      "madc.hi.cc.u32 %1, %5, %11, %1;\n\t"
      "addc.u32 %2, 0, 0;\n\t"
      "mad.lo.cc.u32 %0, %6, %10, %0;\n\t"
      "madc.hi.cc.u32 %1, %6, %10, %1;\n\t"
      "addc.u32 %2, %2, 0;\n\t"
      "mad.lo.cc.u32 %0, %7, %9, %0;\n\t"
      "madc.hi.cc.u32 %1, %7, %9, %1;\n\t"
      "addc.u32 %2, %2, 0;\n\t"
      // column 5: a2 b3, a3 b2
      "mad.lo.cc.u32 %1, %6, %11, %1;\n\t"
      "madc.hi.cc.u32 %2, %6, %11, %2;\n\t"
      "addc.u32 %3, 0, 0;\n\t"
      "mad.lo.cc.u32 %1, %7, %10, %1;\n\t"
      "madc.hi.cc.u32 %2, %7, %10, %2;\n\t"
      "addc.u32 %3, %3, 0;\n\t"
      // column 6: a3 b3
      "mad.lo.cc.u32 %2, %7, %11, %2;\n\t"
      "madc.hi.u32 %3, %7, %11, %3;"
      : "=&r"(o.w[0]), "=&r"(o.w[1]), "=&r"(o.w[2]), "=&r"(o.w[3])
      : "r"(a.w[0]), "r"(a.w[1]), "r"(a.w[2]), "r"(a.w[3]), "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]));
  return o;
}

// acc += (negate ? ~a : a), sign-extended to 160 bits; ~a = -a - 2^-126, the caller counts the missing units.
__device__ __forceinline__ void q160_add_xor(q160& acc, const q128& a, uint32_t m) {
  q128 x;
  x.w[0] = a.w[0] ^ m;
  x.w[1] = a.w[1] ^ m;
  x.w[2] = a.w[2] ^ m;
  x.w[3] = a.w[3] ^ m;
  q160_add(acc, x);
}

// acc += k (a small non-negative count of units of 2^-126)
__device__ __forceinline__ void q160_add_units(q160& acc, uint32_t k) {
  asm("add.cc.u32 %0, %0, %5;\n\t"
      "addc.cc.u32 %1, %1, 0;\n\t"
      "addc.cc.u32 %2, %2, 0;\n\t"
      "addc.cc.u32 %3, %3, 0;\n\t"
      "addc.u32 %4, %4, 0;"
      : "+r"(acc.w[0]), "+r"(acc.w[1]), "+r"(acc.w[2]), "+r"(acc.w[3]), "+r"(acc.w[4])
      : "r"(k));
}

// z * b for first-quadrant phasors, renormalised to the first quadrant: three unsigned products give
// re = c1 c2 - s1 s2 and im = (c1 + s1)(c2 + s2) - c1 c2 - s1 s2 >= 0 (clamped at 0); if re < 0 the result is rotated by -i
// (c, s) = (im, -re) and the quadrant advances.  The Q2.126 results are doubled back to Q1.127.
__device__ __forceinline__ qent qmul(const qent& z, const qent& b) {
  const q128 p1 = umulhi(z.c, b.c), p2 = umulhi(z.s, b.s), p3 = umulhi(z.cs, b.cs);
  const q128 re = q128_sub(p1, p2);
  q128 im = q128_sub(q128_sub(p3, p1), p2);
  // im = c1 s2 + s1 c2 >= 0 exactly; each truncated top half is up to 8 units low, so on the real axis (both
  // factors inexact) the computed value can fall a few units below 0 and would wrap: it is 0 within its error
  if ((int32_t)im.w[3] < 0) im = q128_zero();
  uint32_t q = (z.cs.w[0] + b.cs.w[0]) & 3u;
  const bool neg = (int32_t)re.w[3] < 0;
  const q128 nre = q128_neg(re);
  q128 c, s;
#pragma unroll
  for (int w = 0; w < 4; w++) {
    c.w[w] = neg ? im.w[w] : re.w[w];
    s.w[w] = neg ? nre.w[w] : im.w[w];
  }
  q = (q + (neg ? 1u : 0u)) & 3u;
  qent r;
  r.c = q128_shl1(c);
  r.s = q128_shl1(s);
  r.cs = q128_add(r.c, r.s);
  r.cs.w[0] = (r.cs.w[0] & ~3u) | q;
  return r;
}

// Sign-magnitude Q1.127 of a Q2.126 value with |x| < 1/2: the magnitude doubled, the sign in bit 127.
__device__ __forceinline__ q128 q127_signmag(const q128& x) {
  const bool neg = (int32_t)x.w[3] < 0;
  q128 m = q128_shl1(neg ? q128_neg(x) : x);
  if (neg) m.w[3] |= 0x80000000u;
  return m;
}
