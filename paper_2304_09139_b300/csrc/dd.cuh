// dd.cuh -- double-double ("double-word") arithmetic for host and device.
//
// The paper evaluates the energy and force in double-double arithmetic (Simulations);
// a dd value is an unevaluated sum hi + lo of two doubles with |lo| <= ulp(hi)/2, about 106 significant
// bits.  The building blocks follow the published algorithms:
//   two_sum        Knuth's TwoSum, 6 flops, exact: a + b = s + e
//   fast_two_sum   Dekker's Fast2Sum (|a| >= |b|), 3 flops, exact
//   two_prod       product with FMA, 2 flops, exact: a * b = p + e
//   dd_add         Joldes-Muller-Popescu 2017 "AccurateDWPlusDW", 20 flops, relative error <= 3u^2
//   dd_add_sloppy  the same paper's "SloppyDWPlusDW", 11 flops, normwise error (used for same-order sums)
//   dd_mul         DW x DW with FMA (the same paper's algorithm without the lo*lo term), 8 flops
//   dd_mul_d       DW x double with FMA, 5 flops
// and a sincos of a phase given in turns (dd_sincos_turns) built from two 256-entry dd tables and a
// Taylor series on a remainder below 2^-16 turns.  The phase is reduced exactly (a turn is 1), which is
// the dd argument reduction of k.r: with fractional positions s = r / L, k.r_j = 2 pi n.s_j.
#pragma once
#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#define SSH_HD __host__ __device__ __forceinline__
#else
#define SSH_HD inline
#endif

#ifdef __CUDACC__
struct __align__(16) dd {
#else
struct alignas(16) dd {
#endif
  double hi, lo;
};

SSH_HD dd dd_make(double h, double l = 0.0) { dd r; r.hi = h; r.lo = l; return r; }

SSH_HD dd two_sum(double a, double b) {
  double s = a + b;
  double ap = s - b;
  double bp = s - ap;
  double e = (a - ap) + (b - bp);
  return dd_make(s, e);
}

SSH_HD dd fast_two_sum(double a, double b) {
  double s = a + b;
  double e = b - (s - a);
  return dd_make(s, e);
}

SSH_HD dd two_prod(double a, double b) {
  double p = a * b;
  double e = fma(a, b, -p);
  return dd_make(p, e);
}

SSH_HD dd dd_add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  dd t = two_sum(x.lo, y.lo);
  double c = s.lo + t.hi;
  dd v = fast_two_sum(s.hi, c);
  double w = t.lo + v.lo;
  return fast_two_sum(v.hi, w);
}

SSH_HD dd dd_add_sloppy(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  double v = x.lo + y.lo;
  double w = s.lo + v;
  return fast_two_sum(s.hi, w);
}

SSH_HD dd dd_neg(dd x) { return dd_make(-x.hi, -x.lo); }
SSH_HD dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }

SSH_HD dd dd_add_d(dd x, double y) {
  dd s = two_sum(x.hi, y);
  double v = x.lo + s.lo;
  return fast_two_sum(s.hi, v);
}

SSH_HD dd dd_mul(dd x, dd y) {
  dd c = two_prod(x.hi, y.hi);
  double t = x.hi * y.lo;
  double c2 = fma(x.lo, y.hi, t);
  double c3 = c.lo + c2;
  return fast_two_sum(c.hi, c3);
}

SSH_HD dd dd_mul_d(dd x, double y) {
  dd c = two_prod(x.hi, y);
  double c3 = fma(x.lo, y, c.lo);
  return fast_two_sum(c.hi, c3);
}

SSH_HD dd dd_sqr(dd x) { return dd_mul(x, x); }

// x / y by one Newton correction of the double quotient (relative error ~ 2^-104); host set-up only.
SSH_HD dd dd_div(dd x, dd y) {
  double q1 = x.hi / y.hi;
  dd r = dd_sub(x, dd_mul_d(y, q1));
  double q2 = r.hi / y.hi;
  r = dd_sub(r, dd_mul_d(y, q2));
  double q3 = r.hi / y.hi;
  dd q = fast_two_sum(q1, q2);
  return dd_add_d(q, q3);
}

SSH_HD double dd_to_d(dd x) { return x.hi + x.lo; }

// x - floor(x) for a normalised dd: a value in [0, 1).  The integer part is removed with TwoSum, which is
// exact even when x.hi is a small negative number (there hi - floor(hi) = hi + 1 would round).  The result
// may have hi = 1.0 with lo < 0 (a value just below one).
SSH_HD dd dd_frac(dd x) {
  double fh = floor(x.hi);
  dd r = two_sum(x.hi, -fh);  // exact
  r = dd_add_d(r, x.lo);
  if (r.hi < 0.0 || (r.hi == 0.0 && r.lo < 0.0)) r = dd_add_d(r, 1.0);
  if (r.hi > 1.0 || (r.hi == 1.0 && r.lo >= 0.0)) r = dd_add_d(r, -1.0);
  return r;
}

// frac(m (sh + sl)) in turns for an integer m: m * sh is split exactly with TwoProd, its integer part is
// removed exactly, and m * sl (below 2^-53 |m sh|) is added.  The phase of k = 2 pi n / L at fractional
// position s is the sum of these over the axes.
SSH_HD dd dd_turns_times(int m, double sh, double sl) {
  dd p = two_prod((double)m, sh);
  dd t = dd_frac(p);
  return dd_add_d(t, (double)m * sl);
}

SSH_HD int dd_lt(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
SSH_HD int dd_gt(dd a, dd b) { return dd_lt(b, a); }

// complex dd
struct ddc {
  dd re, im;
};

SSH_HD ddc ddc_make(dd r, dd i) { ddc z; z.re = r; z.im = i; return z; }
SSH_HD ddc ddc_conj(ddc z) { return ddc_make(z.re, dd_neg(z.im)); }

SSH_HD ddc ddc_mul(ddc a, ddc b) {
  dd rr = dd_mul(a.re, b.re), ii = dd_mul(a.im, b.im);
  dd ri = dd_mul(a.re, b.im), ir = dd_mul(a.im, b.re);
  return ddc_make(dd_add(rr, dd_neg(ii)), dd_add(ri, ir));
}

SSH_HD ddc ddc_add(ddc a, ddc b) { return ddc_make(dd_add(a.re, b.re), dd_add(a.im, b.im)); }

// e^{2 pi i t} for t in turns (any real dd; only frac(t) matters).  Tables hold e^{2 pi i c/2^8} and
// e^{2 pi i c/2^16} for c = 0..255 as dd pairs [cos.hi, cos.lo, sin.hi, sin.lo]; inv_fact[n] = 1/n!;
// two_pi = 2 pi as dd.  Remainder |r| < 2^-16 turns, theta = 2 pi r, |theta| < 1e-4: sin needs terms
// to theta^7 and cos to theta^8 for an error below 2^-110.
SSH_HD ddc dd_sincos_turns_tab(dd t, const double (*tab_a)[4], const double (*tab_b)[4],
                               const double (*inv_fact)[2], const double* two_pi) {
  t = dd_frac(t);
  double x1 = t.hi * 256.0;
  int c1 = (int)floor(x1);
  if (c1 > 255) c1 = 255;
  if (c1 < 0) c1 = 0;
  dd r1 = dd_make(t.hi - (double)c1 * (1.0 / 256.0), t.lo);  // exact subtraction
  r1 = fast_two_sum(r1.hi, r1.lo);
  double x2 = r1.hi * 65536.0;
  int c2 = (int)floor(x2);
  if (c2 > 255) c2 = 255;
  if (c2 < 0) c2 = 0;
  dd r = dd_make(r1.hi - (double)c2 * (1.0 / 65536.0), r1.lo);
  r = fast_two_sum(r.hi, r.lo);
  dd th = dd_mul(r, dd_make(two_pi[0], two_pi[1]));
  dd t2 = dd_sqr(th);
  // sin: th * (1 - t2/3! + t2^2/5! - t2^3/7!)
  dd ps = dd_neg(dd_make(inv_fact[7][0], inv_fact[7][1]));
  ps = dd_add(dd_mul(ps, t2), dd_make(inv_fact[5][0], inv_fact[5][1]));
  ps = dd_add(dd_mul(ps, t2), dd_neg(dd_make(inv_fact[3][0], inv_fact[3][1])));
  ps = dd_add_d(dd_mul(ps, t2), 1.0);
  dd sn = dd_mul(ps, th);
  // cos: 1 - t2/2! + t2^2/4! - t2^3/6! + t2^4/8!
  dd pc = dd_make(inv_fact[8][0], inv_fact[8][1]);
  pc = dd_add(dd_mul(pc, t2), dd_neg(dd_make(inv_fact[6][0], inv_fact[6][1])));
  pc = dd_add(dd_mul(pc, t2), dd_make(inv_fact[4][0], inv_fact[4][1]));
  pc = dd_add(dd_mul(pc, t2), dd_neg(dd_make(inv_fact[2][0], inv_fact[2][1])));
  pc = dd_add_d(dd_mul(pc, t2), 1.0);
  ddc e = ddc_make(pc, sn);
  const double* a = tab_a[c1];
  const double* b = tab_b[c2];
  ddc za = ddc_make(dd_make(a[0], a[1]), dd_make(a[2], a[3]));
  ddc zb = ddc_make(dd_make(b[0], b[1]), dd_make(b[2], b[3]));
  return ddc_mul(ddc_mul(za, zb), e);
}
