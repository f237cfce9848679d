/*
 * oracle.c -- plain, slow, obviously-correct CPU oracle for the stealthy-hyperuniform
 * collective-coordinate energy, its force, and the FIRE quench (arXiv:2304.09139).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, import or call this file:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm use it.
 * It shares no code, header, table or constant generator with the CUDA library.
 *
 * Arithmetic: IEEE binary128 (__float128, libquadmath), one sincosq per (k, particle) pair, sums in
 * index order.  Every function follows a definition in the paper:
 *   k-set            -- reciprocal lattice k = 2*pi*n/L of the periodic box, inversion symmetry leaves
 *                       M independent vectors, chi = M / (d (N-1))          (Definitions, Eq. for chi)
 *   n~(k)            -- collective density, sum_j exp(i k.r_j)             (Eq. ntilde)
 *   Phi, S(k), S_max -- Phi = sum over the half-space of |n~(k)|^2 (constant term dropped, eps0 = 1),
 *                       S(k) = |n~(k)|^2 / N, S_max = max S(k)              (Eqs. energy, structurefactor, smax)
 *   F_j              -- F_j = -grad_j Phi                                   (Eq. force); also at chosen
 *                       particles from given (C, S), for checks of large systems
 *   weights          -- a general non-negative v~(k) per wavevector (the paper's v~(k) > 0 that selects
 *                       ground states): Phi = sum v~ |n~|^2, F = -grad Phi; S(k) is unweighted (Eqs. energy, force)
 *   FIRE             -- Bitzek et al. 2006 structural relaxation, the minimiser the paper uses (Simulations)
 *
 * Conventions (readings of the paper, restated here so the file stands alone):
 *   * positions are fractional, s = r/L in [0,1), given as a double-double pair (hi, lo) per coordinate,
 *     row-major [N][d]; the pair is lifted to binary128 exactly (hi + lo).
 *   * the exponent sign is +: C_k = sum_j cos(2 pi n.s_j), S_k = sum_j sin(2 pi n.s_j).  |n~|, Phi and F
 *     do not depend on the sign; only the sign of S_k is convention.
 *   * with C, S as above, F_{j,a} = (4 pi / L) sum_k n_a [C_k sin(th_jk) - S_k cos(th_jk)],
 *     th_jk = 2 pi n_k.s_j: the half-space sum of Eq. force with eps0 = 1 and v~ = eps0 L^d.
 *   * half-space H: n != 0 whose first non-zero component is positive.  Order: by |n|^2, then
 *     lexicographically on the signed components.  chi mode keeps the first M = round-half-even(chi d (N-1));
 *     K mode keeps every n with |n|^2 <= (K L / 2 pi)^2 (1 + 1e-12).
 * Outputs of binary128 values are returned as double-double pairs (hi = nearest double, lo = rest).
 */
#include <math.h>
#include <quadmath.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __float128 q_t;

static void q_to_dd(q_t x, double *hi, double *lo) {
  double h = (double)x;
  *hi = h;
  *lo = (double)(x - (q_t)h);
}

/* ---------------------------------------------------------------- k-set (Definitions) */

typedef struct {
  int64_t norm2;
  int32_t c[4];
} kvec_t;

static int g_sort_d; /* dimension used by the comparator (the oracle is not re-entrant here) */

static int kvec_cmp(const void *pa, const void *pb) {
  const kvec_t *a = (const kvec_t *)pa, *b = (const kvec_t *)pb;
  if (a->norm2 != b->norm2) return a->norm2 < b->norm2 ? -1 : 1;
  for (int i = 0; i < g_sort_d; i++)
    if (a->c[i] != b->c[i]) return a->c[i] < b->c[i] ? -1 : 1;
  return 0;
}

static int in_half_space(const int32_t *c, int d) {
  for (int i = 0; i < d; i++) {
    if (c[i] > 0) return 1;
    if (c[i] < 0) return 0;
  }
  return 0; /* n = 0 is excluded */
}

/* Enumerate H intersect {|n|^2 <= r2max}; returns count, fills *out (malloc'd, caller frees). */
static int64_t enumerate_half_ball(int d, int64_t r2max, kvec_t **out) {
  int64_t R = 0;
  while ((R + 1) * (R + 1) <= r2max) R++;
  int64_t side = 2 * R + 1, total = 1;
  for (int i = 0; i < d; i++) total *= side;
  kvec_t *v = (kvec_t *)malloc(sizeof(kvec_t) * (size_t)(total > 0 ? total : 1));
  int64_t cnt = 0;
  for (int64_t idx = 0; idx < total; idx++) {
    int64_t rem = idx, n2 = 0;
    kvec_t k;
    memset(&k, 0, sizeof k);
    for (int i = d - 1; i >= 0; i--) {
      k.c[i] = (int32_t)(rem % side - R);
      rem /= side;
      n2 += (int64_t)k.c[i] * k.c[i];
    }
    if (n2 > r2max || !in_half_space(k.c, d)) continue;
    k.norm2 = n2;
    v[cnt++] = k;
  }
  *out = v;
  return cnt;
}

/* M for chi mode: round-half-even of chi * d * (N - 1), evaluated in double. */
int64_t oracle_chi_to_m(int d, int64_t N, double chi) {
  double x = chi * (double)d * (double)(N - 1);
  return (int64_t)nearbyint(x); /* default rounding mode: to nearest, ties to even */
}

/*
 * Build the k-set.  Exactly one of chi > 0 (chi mode) or K > 0 (K mode).
 * n_out: capacity cap rows of d int32 (row-major), may be NULL to query M only.
 * Returns 0 on success, -1 on bad arguments, -2 if cap is too small.
 */
int oracle_kset(int d, int64_t N, double L, double chi, double K, int64_t cap, int32_t *n_out, int64_t *M_out) {
  if (d < 1 || d > 4 || N < 1 || !(L > 0)) return -1;
  if ((chi > 0) == (K > 0)) return -1;
  kvec_t *v = NULL;
  int64_t cnt = 0, M = 0;
  if (K > 0) {
    long double rr = (long double)K * (long double)L / (2.0L * 3.141592653589793238462643383279502884L);
    long double lim = rr * rr * (1.0L + 1e-12L);
    int64_t r2max = (int64_t)floorl(lim);
    cnt = enumerate_half_ball(d, r2max, &v);
    M = cnt;
  } else {
    M = oracle_chi_to_m(d, N, chi);
    if (M < 0) return -1;
    int64_t r2 = 1;
    for (;;) {
      free(v);
      cnt = enumerate_half_ball(d, r2, &v);
      if (cnt >= M) break;
      r2 *= 2;
    }
  }
  g_sort_d = d;
  qsort(v, (size_t)cnt, sizeof(kvec_t), kvec_cmp);
  *M_out = M;
  if (n_out) {
    if (cap < M) { free(v); return -2; }
    for (int64_t m = 0; m < M; m++)
      for (int i = 0; i < d; i++) n_out[m * d + i] = v[m].c[i];
  }
  free(v);
  return 0;
}

/* ---------------------------------------------------------------- n~(k), Phi, F (Eqs. ntilde, energy, force) */

static const q_t Q_2PI = 2 * M_PIq;

/* Phase in turns, t = frac(n . s), with s lifted exactly from (hi, lo).  The hi and lo sums are kept
 * apart because n_a * hi is exact in binary128 and so is the integer part removed from it. */
static q_t phase_turns(int d, const int32_t *n, const double *s_hi, const double *s_lo) {
  q_t th = 0, tl = 0;
  for (int a = 0; a < d; a++) {
    th += (q_t)n[a] * (q_t)s_hi[a];
    if (s_lo) tl += (q_t)n[a] * (q_t)s_lo[a];
  }
  th -= floorq(th);
  q_t t = th + tl;
  t -= floorq(t);
  return t;
}

static void cos_sin_turns(q_t t, q_t *c, q_t *s) {
  if (t >= 0.5Q) t -= 1; /* argument in [-1/2, 1/2) turns */
  sincosq(Q_2PI * t, s, c);
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

/* C_k and S_k in binary128 (internal form). */
static void ntilde_q(int d, int64_t N, const double *s_hi, const double *s_lo, int64_t M, const int32_t *n,
                     q_t *C, q_t *S) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < M; k++) {
    q_t c_sum = 0, s_sum = 0;
    for (int64_t j = 0; j < N; j++) {
      q_t c, s;
      q_t t = phase_turns(d, n + k * d, s_hi + j * d, s_lo ? s_lo + j * d : NULL);
      cos_sin_turns(t, &c, &s);
      c_sum += c;
      s_sum += s;
    }
    C[k] = c_sum;
    S[k] = s_sum;
  }
}

/* C_k, S_k as (hi, lo) pairs: C_out[2k], C_out[2k+1]. */
int oracle_ntilde(int d, int64_t N, const double *s_hi, const double *s_lo, int64_t M, const int32_t *n,
                  double *C_out, double *S_out, int nthreads) {
  if (d < 1 || d > 4 || N < 0 || M < 0) return -1;
  set_threads(nthreads);
  q_t *C = (q_t *)malloc(sizeof(q_t) * (size_t)(M > 0 ? M : 1));
  q_t *S = (q_t *)malloc(sizeof(q_t) * (size_t)(M > 0 ? M : 1));
  ntilde_q(d, N, s_hi, s_lo, M, n, C, S);
  for (int64_t k = 0; k < M; k++) {
    q_to_dd(C[k], &C_out[2 * k], &C_out[2 * k + 1]);
    q_to_dd(S[k], &S_out[2 * k], &S_out[2 * k + 1]);
  }
  free(C);
  free(S);
  return 0;
}

/* Phi, S_max and F.  Any output pointer may be NULL.  F_out is [N][d][2] (hi, lo).
 * Sum orders: Phi over k ascending; F_j over k ascending; each C_k over j ascending. */
/* Phi, S_max, F with per-wavevector weights w (NULL: every weight 1) */
int oracle_phi_grad_w(int d, int64_t N, double L, const double *s_hi, const double *s_lo, int64_t M,
                      const int32_t *n, const double *w, double *phi, double *smax, double *F_out, double *C_out,
                      double *S_out, int nthreads) {
  if (d < 1 || d > 4 || N < 0 || M < 0 || !(L > 0)) return -1;
  set_threads(nthreads);
  q_t *C = (q_t *)malloc(sizeof(q_t) * (size_t)(M > 0 ? M : 1));
  q_t *S = (q_t *)malloc(sizeof(q_t) * (size_t)(M > 0 ? M : 1));
  ntilde_q(d, N, s_hi, s_lo, M, n, C, S);
  q_t P = 0, smx = 0;
  for (int64_t k = 0; k < M; k++) {
    q_t a2 = C[k] * C[k] + S[k] * S[k];
    P += (w ? (q_t)w[k] : (q_t)1) * a2;
    q_t sk = N > 0 ? a2 / (q_t)N : 0;
    if (sk > smx) smx = sk;
  }
  if (phi) q_to_dd(P, &phi[0], &phi[1]);
  if (smax) q_to_dd(smx, &smax[0], &smax[1]);
  if (C_out)
    for (int64_t k = 0; k < M; k++) q_to_dd(C[k], &C_out[2 * k], &C_out[2 * k + 1]);
  if (S_out)
    for (int64_t k = 0; k < M; k++) q_to_dd(S[k], &S_out[2 * k], &S_out[2 * k + 1]);
  if (F_out) {
    const q_t pref = 2 * Q_2PI / (q_t)L; /* 4 pi / L */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < N; j++) {
      q_t f[4] = {0, 0, 0, 0};
      for (int64_t k = 0; k < M; k++) {
        q_t c, s;
        q_t t = phase_turns(d, n + k * d, s_hi + j * d, s_lo ? s_lo + j * d : NULL);
        cos_sin_turns(t, &c, &s);
        q_t t2 = (w ? (q_t)w[k] : (q_t)1) * (C[k] * s - S[k] * c);
        for (int a = 0; a < d; a++) f[a] += (q_t)n[k * d + a] * t2;
      }
      for (int a = 0; a < d; a++) q_to_dd(pref * f[a], &F_out[(j * d + a) * 2], &F_out[(j * d + a) * 2 + 1]);
    }
  }
  free(C);
  free(S);
  return 0;
}

/* F_{j,a} = (4 pi / L) sum_k v~_k n_a [C_k sin(th_jk) - S_k cos(th_jk)] (Eq. force) at P given particles, from given
 * collective densities C_k + i S_k (dd pairs, lifted exactly to binary128) instead of the particles' own: the
 * force on those particles inside a configuration whose n~(k) is (C, S).  The per-pair sum is the one of
 * oracle_phi_grad_w, k ascending.  w may be NULL (every weight 1).  F_out is [P][d][2] (hi, lo). */
int oracle_force_at(int d, int64_t P, double L, const double *s_hi, const double *s_lo, int64_t M, const int32_t *n,
                    const double *C_in, const double *S_in, const double *w, double *F_out, int nthreads) {
  if (d < 1 || d > 4 || P < 0 || M < 0 || !(L > 0)) return -1;
  set_threads(nthreads);
  const q_t pref = 2 * Q_2PI / (q_t)L; /* 4 pi / L */
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < P; j++) {
    q_t f[4] = {0, 0, 0, 0};
    for (int64_t k = 0; k < M; k++) {
      q_t c, s;
      q_t t = phase_turns(d, n + k * d, s_hi + j * d, s_lo ? s_lo + j * d : NULL);
      cos_sin_turns(t, &c, &s);
      const q_t Ck = (q_t)C_in[2 * k] + (q_t)C_in[2 * k + 1];
      const q_t Sk = (q_t)S_in[2 * k] + (q_t)S_in[2 * k + 1];
      q_t t2 = (w ? (q_t)w[k] : (q_t)1) * (Ck * s - Sk * c);
      for (int a = 0; a < d; a++) f[a] += (q_t)n[k * d + a] * t2;
    }
    for (int a = 0; a < d; a++) q_to_dd(pref * f[a], &F_out[(j * d + a) * 2], &F_out[(j * d + a) * 2 + 1]);
  }
  return 0;
}

int oracle_phi_grad(int d, int64_t N, double L, const double *s_hi, const double *s_lo, int64_t M,
                    const int32_t *n, double *phi, double *smax, double *F_out, double *C_out, double *S_out,
                    int nthreads) {
  return oracle_phi_grad_w(d, N, L, s_hi, s_lo, M, n, NULL, phi, smax, F_out, C_out, S_out, nthreads);
}

/* ---------------------------------------------------------------- post-processing (Eq. tau; Fig. S1) */

/* Shell averages of S(k) = |n~(k)|^2 / N (Eq. structurefactor) and the truncated order metric of Eq. tau, from
 * the particles' own n~ (binary128 throughout).
 *   Shells: with integers nbins >= 1 and n2max >= 1, edge E_b = ceil(b^2 n2max / nbins^2) (b = 0..nbins, exact
 *   integer arithmetic); shell b < nbins - 1 holds the wavevectors with E_b <= |n|^2 < E_(b+1), the last shell
 *   E_(nbins-1) <= |n|^2 <= n2max.  So shell b covers |n| in [b R / nbins, (b + 1) R / nbins), R^2 = n2max, and
 *   |k| = 2 pi |n| / L.  Wavevectors beyond n2max are in no shell.  counts[b] is the shell's population and
 *   mean_out[2b], mean_out[2b+1] the (hi, lo) pair of its mean S (0 for an empty shell).
 *   tau: the integral over k of [S(k) - 1]^2 taken as the lattice sum over every wavevector of the set and its
 *   mirror -k, each cell of volume (2 pi / L)^d, divided by (2 pi D)^d rho^2 with D = 1 / K and rho = N / L^d:
 *   tau = 2 (K L)^d / N^2 sum_k [S(k) - 1]^2.  The sum runs in index order. */
int oracle_structure_factor(int d, int64_t N, double L, const double *s_hi, const double *s_lo, int64_t M,
                            const int32_t *n, int nbins, int64_t n2max, double K, int64_t *counts, double *mean_out,
                            double *tau_out, int nthreads) {
  if (d < 1 || d > 4 || N < 1 || M < 0 || !(L > 0) || nbins < 1 || n2max < 1 || !(K > 0)) return -1;
  set_threads(nthreads);
  q_t *C = (q_t *)malloc(sizeof(q_t) * (size_t)(M > 0 ? M : 1));
  q_t *S = (q_t *)malloc(sizeof(q_t) * (size_t)(M > 0 ? M : 1));
  q_t *sum = (q_t *)calloc((size_t)nbins, sizeof(q_t));
  int64_t *E = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nbins + 1));
  ntilde_q(d, N, s_hi, s_lo, M, n, C, S);
  const unsigned __int128 den = (unsigned __int128)nbins * (unsigned __int128)nbins;
  for (int b = 0; b <= nbins; b++) {
    const unsigned __int128 num = (unsigned __int128)b * (unsigned __int128)b * (unsigned __int128)n2max;
    E[b] = (int64_t)((num + den - 1) / den);
  }
  for (int b = 0; b < nbins; b++) counts[b] = 0;
  q_t t2 = 0;
  for (int64_t k = 0; k < M; k++) {
    int64_t m = 0;
    for (int a = 0; a < d; a++) m += (int64_t)n[k * d + a] * (int64_t)n[k * d + a];
    const q_t sk = (C[k] * C[k] + S[k] * S[k]) / (q_t)N;
    t2 += (sk - 1) * (sk - 1);
    if (m > n2max) continue;
    int b = 0;
    while (b + 1 < nbins && m >= E[b + 1]) b++;   /* linear search: the oracle is not fast, only plain */
    counts[b]++;
    sum[b] += sk;
  }
  for (int b = 0; b < nbins; b++) {
    const q_t mean = counts[b] > 0 ? sum[b] / (q_t)counts[b] : 0;
    q_to_dd(mean, &mean_out[2 * b], &mean_out[2 * b + 1]);
  }
  q_t kl = 1;
  for (int a = 0; a < d; a++) kl *= (q_t)K * (q_t)L;
  q_to_dd(2 * kl * t2 / ((q_t)N * (q_t)N), &tau_out[0], &tau_out[1]);
  free(C);
  free(S);
  free(sum);
  free(E);
  return 0;
}

/* g_2(r) from pair counts (the supplement's Fig. S1b): counts[b] of ordered pairs (i < n_ref, j != i) at distances
 * in [b w, (b + 1) w), w = r_max / nbins, divided by the count an ideal gas of the same density gives in that shell,
 * n_ref (N - 1) / L^d times the shell's volume v_d ((b + 1)^d - b^d) w^d, v_d = pi^(d/2) / Gamma(d/2 + 1) the volume
 * of the unit ball (2, pi, 4 pi / 3, pi^2 / 2 for d = 1..4).  r_out[b] = (b + 1/2) w. */
int oracle_g2(int d, int64_t N, double L, int64_t n_ref, double r_max, int nbins, const uint64_t *counts,
              double *r_out, double *g_out) {
  if (d < 1 || d > 4 || N < 2 || !(L > 0) || n_ref < 1 || !(r_max > 0) || nbins < 1) return -1;
  const q_t vd[5] = {0, 2, M_PIq, 4 * M_PIq / 3, M_PIq * M_PIq / 2};
  const q_t w = (q_t)r_max / (q_t)nbins;
  q_t ld = 1, wd = 1;
  for (int a = 0; a < d; a++) {
    ld *= (q_t)L;
    wd *= w;
  }
  const q_t dens = (q_t)n_ref * (q_t)(N - 1) / ld;
  for (int b = 0; b < nbins; b++) {
    q_t lo = 1, hi = 1;
    for (int a = 0; a < d; a++) {
      lo *= (q_t)b;
      hi *= (q_t)(b + 1);
    }
    const q_t ideal = dens * vd[d] * (hi - lo) * wd;
    r_out[b] = (double)(((q_t)b + 0.5Q) * w);
    g_out[b] = (double)((q_t)counts[b] / ideal);
  }
  return 0;
}

/* ---------------------------------------------------------------- FIRE (Bitzek et al. 2006) */

/*
 * FIRE as published: MD with semi-implicit Euler and unit mass, plus the velocity-mixing rules
 *   P = F.v;  v <- (1-alpha) v + alpha |v| F/|F|;
 *   P > 0 for more than n_min steps in a row: dt <- min(dt f_inc, dt_max), alpha <- alpha f_alpha;
 *   P <= 0: dt <- dt f_dec, v <- 0, alpha <- alpha_start.
 * Energy guard (the reading taken for the paper's stopping rule, Phi at its machine-precision floor): a step that
 * raises Phi is undone, dt <- dt f_dec, v <- 0, alpha <- alpha_start.
 * Stop when S_max <= smax_target (status 0) or after max_steps (status 1).
 * Positions are in/out as fractional (hi, lo) pairs; the minimiser works on r = L s in binary128.
 */
typedef struct {
  double dt0, dt_max, alpha_start, f_alpha, f_inc, f_dec;
  int n_min;
  int64_t max_steps;
  double smax_target;
} oracle_fire_params;

int oracle_fire(int d, int64_t N, double L, double *s_hi, double *s_lo, int64_t M, const int32_t *n,
                const oracle_fire_params *p, int64_t *steps_out, double *smax_out, double *phi_out,
                int nthreads) {
  if (d < 1 || d > 4 || N < 1 || M < 0 || !(L > 0)) return -1;
  set_threads(nthreads);
  int64_t nd = N * d;
  q_t *x = (q_t *)calloc((size_t)nd, sizeof(q_t)), *v = (q_t *)calloc((size_t)nd, sizeof(q_t));
  q_t *F = (q_t *)calloc((size_t)nd, sizeof(q_t)), *xs = (q_t *)calloc((size_t)nd, sizeof(q_t));
  q_t *Fs = (q_t *)calloc((size_t)nd, sizeof(q_t));
  double *hh = (double *)malloc(sizeof(double) * (size_t)nd), *ll = (double *)malloc(sizeof(double) * (size_t)nd);
  double *Fd = (double *)malloc(sizeof(double) * (size_t)nd * 2);
  for (int64_t i = 0; i < nd; i++) x[i] = ((q_t)s_hi[i] + (q_t)s_lo[i]) * (q_t)L;
  q_t dt = p->dt0, alpha = p->alpha_start, phi = 0, phi_s = 0, smx = 0;
  int64_t n_pos = 0, step = 0;
  int status = 1;
  /* evaluate at the start */
  for (int64_t i = 0; i < nd; i++) {
    q_t s = x[i] / (q_t)L;
    s -= floorq(s);
    q_to_dd(s, &hh[i], &ll[i]);
  }
  double ph[2], sm[2];
  oracle_phi_grad(d, N, L, hh, ll, M, n, ph, sm, Fd, NULL, NULL, nthreads);
  phi = (q_t)ph[0] + (q_t)ph[1];
  smx = (q_t)sm[0] + (q_t)sm[1];
  for (int64_t i = 0; i < nd; i++) F[i] = (q_t)Fd[2 * i] + (q_t)Fd[2 * i + 1];
  for (step = 0; step < p->max_steps; step++) {
    if (smx <= (q_t)p->smax_target) { status = 0; break; }
    /* FIRE mixing and adaptation, using F at the current positions and v from the previous step */
    q_t P = 0, fn = 0, vn = 0;
    for (int64_t i = 0; i < nd; i++) { P += F[i] * v[i]; fn += F[i] * F[i]; vn += v[i] * v[i]; }
    if (P > 0) {
      q_t scale = fn > 0 ? sqrtq(vn) / sqrtq(fn) : 0;
      for (int64_t i = 0; i < nd; i++) v[i] = (1 - alpha) * v[i] + alpha * scale * F[i];
      if (n_pos > p->n_min) {
        dt = dt * (q_t)p->f_inc;
        if (dt > (q_t)p->dt_max) dt = p->dt_max;
        alpha *= (q_t)p->f_alpha;
      }
      n_pos++;
    } else {
      for (int64_t i = 0; i < nd; i++) v[i] = 0;
      dt *= (q_t)p->f_dec;
      alpha = p->alpha_start;
      n_pos = 0;
    }
    /* semi-implicit Euler with unit mass */
    memcpy(xs, x, sizeof(q_t) * (size_t)nd);
    memcpy(Fs, F, sizeof(q_t) * (size_t)nd);
    phi_s = phi;
    for (int64_t i = 0; i < nd; i++) { v[i] += dt * F[i]; x[i] += dt * v[i]; }
    for (int64_t i = 0; i < nd; i++) {
      q_t s = x[i] / (q_t)L;
      s -= floorq(s);
      q_to_dd(s, &hh[i], &ll[i]);
    }
    oracle_phi_grad(d, N, L, hh, ll, M, n, ph, sm, Fd, NULL, NULL, nthreads);
    q_t phi_new = (q_t)ph[0] + (q_t)ph[1];
    if (phi_new > phi_s) { /* energy guard: undo the step */
      memcpy(x, xs, sizeof(q_t) * (size_t)nd);
      memcpy(F, Fs, sizeof(q_t) * (size_t)nd);
      for (int64_t i = 0; i < nd; i++) v[i] = 0;
      dt *= (q_t)p->f_dec;
      alpha = p->alpha_start;
      n_pos = 0;
      continue;
    }
    phi = phi_new;
    smx = (q_t)sm[0] + (q_t)sm[1];
    for (int64_t i = 0; i < nd; i++) F[i] = (q_t)Fd[2 * i] + (q_t)Fd[2 * i + 1];
  }
  if (status == 1 && smx <= (q_t)p->smax_target) status = 0;
  for (int64_t i = 0; i < nd; i++) {
    q_t s = x[i] / (q_t)L;
    s -= floorq(s);
    q_to_dd(s, &s_hi[i], &s_lo[i]);
  }
  *steps_out = step;
  smax_out[0] = (double)smx;
  smax_out[1] = (double)(smx - (q_t)smax_out[0]);
  phi_out[0] = (double)phi;
  phi_out[1] = (double)(phi - (q_t)phi_out[0]);
  free(x); free(v); free(F); free(xs); free(Fs); free(hh); free(ll); free(Fd);
  return status;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
