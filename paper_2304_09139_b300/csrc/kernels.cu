// kernels.cu -- the Phi + force hot path (Eqs. ntilde, energy, smax, force of arXiv:2304.09139) on sm_103a.
//
// One evaluation is seven launches; every kernel serves any number of configurations (a batch), each described
// by a CfgDev.  The two hot kernels are persistent: their CTAs pull (configuration, tile) items from a queue
// sorted largest-first.  The light kernels take the configuration from blockIdx.y.
//   k_twiddle     per-particle power tables T[row][j] = e^{2 pi i m s_{j,axis}} for the rows of the
//                 table layout (prefix components, high and low digit of the last component)
//   k_ntilde      n~(k) = sum_j e^{2 pi i n.s_j}: a thread owns up to 4 consecutive k of one column; a
//                 block stages, per chunk of particles, the products G = prod_prefix T * T_hi and the 32
//                 low-digit rows in shared memory, so each (k, particle) pair costs one complex multiply
//                 and one accumulate.  Particle splits write partial sums.
//   k_nt_reduce   fixed-order sum of the partials, |n~|^2, per-block Phi / max partials
//   k_finalize    Phi, S_max, and the power-of-two scale of (C, S) for the fixed-point force
//   k_coef        (C_k, S_k) in the arithmetic of the force kernel
//   k_force       F_j = (4 pi / L) sum_k n [C sin(th) - S cos(th)]: a thread owns a particle and walks the
//                 columns; along a column the phase advances by one multiply with T_lo[1]; per column the
//                 sums A = sum w, B = sum A give sum (n_lo + i) w = n_lo A + (len A - B)
//   k_f_reduce    fixed-order sum over column splits, scaling to physical units
// Every reduction has a fixed order, so results are bitwise reproducible run to run.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "fx.cuh"
#include "reduce.cuh"
#include "ssh_internal.h"

#define SSH_TABLE_QUAL __device__
#include "gen/tables.h"

namespace ssh {

// ------------------------------------------------------------------------------------------------ policies

struct PolF64 {
  using Tab = double2;  // (cos, sin)
  using Ph = double2;
  struct Acc { double re, im; };
  using Real = double;
  using RAcc = double;
  using Coef = double2;  // (C, S)
  static constexpr int kIdx = SSH_FP64;
  static __device__ __forceinline__ Ph load(const Tab* p) { return __ldg(p); }
  static __device__ __forceinline__ Ph one() { return make_double2(1.0, 0.0); }
  static __device__ __forceinline__ Ph mul(const Ph& a, const Ph& b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
  }
  static __device__ __forceinline__ void acc_zero(Acc& a) { a.re = 0; a.im = 0; }
  static __device__ __forceinline__ void acc_add(Acc& a, const Ph& z) { a.re += z.x; a.im += z.y; }
  static __device__ __forceinline__ void acc_add_acc(Acc& a, const Acc& b) { a.re += b.re; a.im += b.im; }
  static __device__ __forceinline__ void acc_to_dd(const Acc& a, dd* c, dd* s) { *c = dd_make(a.re); *s = dd_make(a.im); }
  static __device__ __forceinline__ Real w(const Coef& c, const Ph& z) { return fma(c.x, z.y, -c.y * z.x); }
  static __device__ __forceinline__ void rzero(RAcc& a) { a = 0; }
  static __device__ __forceinline__ void radd(RAcc& a, const Real& x) { a += x; }
  static __device__ __forceinline__ void radd_r(RAcc& a, const RAcc& x) { a += x; }
  static __device__ __forceinline__ RAcc rmul_int(const RAcc& a, int k) { return a * (double)k; }
  static __device__ __forceinline__ RAcc rsub(const RAcc& a, const RAcc& b) { return a - b; }
  static __device__ __forceinline__ dd r_to_dd(const RAcc& a) { return dd_make(a); }
  static __device__ __forceinline__ Coef make_coef(dd c, dd s, int /*e*/) { return make_double2(c.hi + c.lo, s.hi + s.lo); }
  static __device__ __forceinline__ Tab phasor(int32_t m, double sh, double sl) {
    double p = (double)m * sh;
    double e = fma((double)m, sh, -p);
    double t = (p - floor(p)) + (e + (double)m * sl);
    double sv, cv;
    sincospi(2.0 * t, &sv, &cv);
    return make_double2(cv, sv);
  }
};

struct PolDD {
  using Tab = ddc;
  using Ph = ddc;
  using Acc = ddc;
  using Real = dd;
  using RAcc = dd;
  using Coef = ddc;  // (C, S)
  static constexpr int kIdx = SSH_DD;
  static __device__ __forceinline__ Ph load(const Tab* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 a = __ldg(q), b = __ldg(q + 1);
    return ddc_make(dd_make(a.x, a.y), dd_make(b.x, b.y));
  }
  static __device__ __forceinline__ Ph one() { return ddc_make(dd_make(1.0), dd_make(0.0)); }
  static __device__ __forceinline__ Ph mul(const Ph& a, const Ph& b) { return ddc_mul(a, b); }
  static __device__ __forceinline__ void acc_zero(Acc& a) { a = ddc_make(dd_make(0.0), dd_make(0.0)); }
  static __device__ __forceinline__ void acc_add(Acc& a, const Ph& z) { a = ddc_add(a, z); }
  static __device__ __forceinline__ void acc_add_acc(Acc& a, const Acc& b) { a = ddc_add(a, b); }
  static __device__ __forceinline__ void acc_to_dd(const Acc& a, dd* c, dd* s) { *c = a.re; *s = a.im; }
  static __device__ __forceinline__ Real w(const Coef& c, const Ph& z) {
    return dd_add(dd_mul(c.re, z.im), dd_neg(dd_mul(c.im, z.re)));
  }
  static __device__ __forceinline__ void rzero(RAcc& a) { a = dd_make(0.0); }
  static __device__ __forceinline__ void radd(RAcc& a, const Real& x) { a = dd_add(a, x); }
  static __device__ __forceinline__ void radd_r(RAcc& a, const RAcc& x) { a = dd_add(a, x); }
  static __device__ __forceinline__ RAcc rmul_int(const RAcc& a, int k) { return dd_mul_d(a, (double)k); }
  static __device__ __forceinline__ RAcc rsub(const RAcc& a, const RAcc& b) { return dd_sub(a, b); }
  static __device__ __forceinline__ dd r_to_dd(const RAcc& a) { return a; }
  static __device__ __forceinline__ Coef make_coef(dd c, dd s, int /*e*/) { return ddc_make(c, s); }
  static __device__ __forceinline__ Tab phasor(int32_t m, double sh, double sl) {
    dd t = dd_turns_times(m, sh, sl);
    return dd_sincos_turns_tab(t, SSH_DD_TAB_A, SSH_DD_TAB_B, SSH_DD_INV_FACT, SSH_DD_2PI);
  }
};

struct PolFX {
  using Tab = fxc;
  using Ph = fxc;
  using Acc = FxAcc;
  using Real = q128;
  using RAcc = q160;
  using Coef = fxc;  // (C, S) * 2^-e in Q2.126
  static constexpr int kIdx = SSH_FX;
  static __device__ __forceinline__ Ph load(const Tab* p) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
    uint4 a = __ldg(q), b = __ldg(q + 1);
    fxc z;
    z.re.w[0] = a.x; z.re.w[1] = a.y; z.re.w[2] = a.z; z.re.w[3] = a.w;
    z.im.w[0] = b.x; z.im.w[1] = b.y; z.im.w[2] = b.z; z.im.w[3] = b.w;
    return z;
  }
  static __device__ __forceinline__ Ph one() { fxc z; z.re = q126_one(); z.im = q128_zero(); return z; }
  static __device__ __forceinline__ Ph mul(const Ph& a, const Ph& b) { return fxc_mul(a, b); }
  static __device__ __forceinline__ void acc_zero(Acc& a) { a.re = q160_zero(); a.im = q160_zero(); }
  static __device__ __forceinline__ void acc_add(Acc& a, const Ph& z) { q160_add(a.re, z.re); q160_add(a.im, z.im); }
  static __device__ __forceinline__ void acc_add_acc(Acc& a, const Acc& b) { q160_add160(a.re, b.re); q160_add160(a.im, b.im); }
  static __device__ __forceinline__ void acc_to_dd(const Acc& a, dd* c, dd* s) {
    q160_to_dd(a.re, &c->hi, &c->lo);
    q160_to_dd(a.im, &s->hi, &s->lo);
  }
  static __device__ __forceinline__ Real w(const Coef& c, const Ph& z) {
    return q128_sub(mul126(c.re, z.im), mul126(c.im, z.re));
  }
  static __device__ __forceinline__ void rzero(RAcc& a) { a = q160_zero(); }
  static __device__ __forceinline__ void radd(RAcc& a, const Real& x) { q160_add(a, x); }
  static __device__ __forceinline__ void radd_r(RAcc& a, const RAcc& x) { q160_add160(a, x); }
  static __device__ __forceinline__ RAcc rmul_int(const RAcc& a, int k) { return q160_mul_int(a, k); }
  static __device__ __forceinline__ RAcc rsub(const RAcc& a, const RAcc& b) { return q160_sub160(a, b); }
  static __device__ __forceinline__ dd r_to_dd(const RAcc& a) { dd r; q160_to_dd(a, &r.hi, &r.lo); return r; }
  // (C, S) 2^-e (|.| < 1/2) as sign-magnitude Q1.127 for the fixed-point force kernel
  static __device__ __forceinline__ Coef make_coef(dd c, dd s, int e) {
    fxc z;
    z.re = q127_signmag(q126_from_dd(ldexp(c.hi, -e), ldexp(c.lo, -e)));
    z.im = q127_signmag(q126_from_dd(ldexp(s.hi, -e), ldexp(s.lo, -e)));
    return z;
  }
  static __device__ __forceinline__ Tab phasor(int32_t m, double sh, double sl) {
    q128 u = turns_from_dd(sh, sl);
    unsigned __int128 uu = ((unsigned __int128)u.w[3] << 96) | ((unsigned __int128)u.w[2] << 64) |
                           ((unsigned __int128)u.w[1] << 32) | (unsigned __int128)u.w[0];
    unsigned __int128 t = uu * (unsigned __int128)(__int128)m;  // exact phase modulo one turn
    q128 tq = q128_from_i128((__int128)t);
    q128 piq;
#pragma unroll
    for (int i = 0; i < 4; i++) piq.w[i] = SSH_FX_PI_Q3_125[i];
    return fx_sincos_turns(tq, SSH_FX_TAB_A, SSH_FX_TAB_B, piq, SSH_FX_INV_FACT);
  }
};


__device__ __forceinline__ bool stopped(const CfgDev& c) { return c.run && *c.run; }

// ------------------------------------------------------------------------------------------------ kernels

template <class P>
__global__ void __launch_bounds__(kTwThreads) k_twiddle(const CfgDev* __restrict__ cfgs, const TwItem* __restrict__ items) {
  const TwItem it = items[blockIdx.x];
  const CfgDev& c = cfgs[it.cfg];
  if (stopped(c)) return;  // a finished minimisation turns these launches into no-ops
  const int64_t idx = it.start + threadIdx.x;
  if (idx >= (int64_t)c.nrows * c.Npad) return;
  const int row = (int)(idx / c.Npad);
  const int64_t j = idx - (int64_t)row * c.Npad;
  typename P::Tab v;
  if (j < c.N) {
    const TabRow r = c.rows[row];
    v = P::phasor(r.m, c.s_hi[r.axis * c.N + j], c.s_lo[r.axis * c.N + j]);
  } else {
    v = P::one();
  }
  reinterpret_cast<typename P::Tab*>(c.tab)[idx] = v;
}

// Persistent: each CTA takes (configuration, k-block, particle split) items until the queue is empty.
template <class P>
__global__ void __launch_bounds__(kNtThreads) k_ntilde(const CfgDev* __restrict__ cfgs, const NtItem* __restrict__ items,
                                                       int n_items, int* __restrict__ queue) {
  using Tab = typename P::Tab;
  using Ph = typename P::Ph;
  constexpr int prec = P::kIdx;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  Tab* sm = reinterpret_cast<Tab*>(smem_raw);
  for (;;) {
    __syncthreads();  // the previous item is finished with shared memory and s_item
    if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int ii = s_item;
    if (ii >= n_items) return;
    const NtItem it = items[ii];
    const CfgDev& c = cfgs[it.cfg];
    if (stopped(c)) continue;
    const Tab* __restrict__ tab = reinterpret_cast<const Tab*>(c.tab);
    const int64_t ld = c.Npad;
    const NtBlock blk = c.blocks[it.blk];
    const int64_t plen = c.plen[prec];
    const int pchunk = c.pchunk[prec];
    const int64_t j_begin = (int64_t)it.ps * plen;
    const int64_t j_end = min(c.N, j_begin + plen);
    const int nrow = blk.ng + kDigit;
    const int stride = nrow | 1;
    const bool active = (int)threadIdx.x < blk.nslots;
    NtSlot sl;
    if (active) sl = c.slots[blk.slot0 + threadIdx.x];
    else { sl.k0 = 0; sl.cnt = 0; sl.g = 0; sl.r0 = 0; }
    typename P::Acc acc[kSlotK];
#pragma unroll
    for (int i = 0; i < kSlotK; i++) P::acc_zero(acc[i]);
    for (int64_t j0 = j_begin; j0 < j_end; j0 += pchunk) {
      const int pc = (int)min((int64_t)pchunk, j_end - j0);
      __syncthreads();
      for (int idx = threadIdx.x; idx < nrow * pc; idx += blockDim.x) {
        const int row = idx / pc, jj = idx - row * pc;
        const int64_t j = j0 + jj;
        Ph v;
        if (row < blk.ng) {
          const int32_t* gr = c.g_rows + (int64_t)(blk.g0 + row) * kMaxDim;
          v = P::load(tab + (int64_t)gr[kMaxDim - 1] * ld + j);
#pragma unroll
          for (int a = 0; a < kMaxDim - 1; a++)
            if (gr[a] >= 0) v = P::mul(v, P::load(tab + (int64_t)gr[a] * ld + j));
        } else {
          v = P::load(tab + (int64_t)(c.lo_base + row - blk.ng) * ld + j);
        }
        sm[jj * stride + row] = v;
      }
      __syncthreads();
      if (active) {
        for (int jj = 0; jj < pc; jj++) {
          const Tab* rp = sm + jj * stride;
          const Ph G = rp[sl.g];
          const Tab* lp = rp + blk.ng + sl.r0;
#pragma unroll
          for (int i = 0; i < kSlotK; i++) {
            if (i < sl.cnt) P::acc_add(acc[i], P::mul(G, lp[i]));
          }
        }
      }
    }
    if (active) {
      typename P::Acc* part = reinterpret_cast<typename P::Acc*>(c.part) + (int64_t)it.ps * c.M;
#pragma unroll
      for (int i = 0; i < kSlotK; i++)
        if (i < sl.cnt) part[sl.k0 + i] = acc[i];
    }
  }
}

// ---- fixed-point density kernel: first-quadrant phasors, three unsigned products per pair
// Shared memory per particle: ng G entries (48 B each), then the 32 low-digit entries with a 16-byte skew every
// fourth entry (entry r at 48 r + 16 (r / 4)), so the 4-strided reads of a warp fall on distinct banks; the
// per-particle stride is 16 mod 128 bytes so that staging stores spread over the banks too.
__host__ __device__ __forceinline__ int fx_lo_off(int r) { return 48 * r + 16 * (r >> 2); }
__host__ __device__ __forceinline__ int fx_particle_bytes(int ng) {
  int b = 48 * ng + 48 * kDigit + 16 * (kDigit / 4);
  return b + (((16 - b % 128) % 128) + 128) % 128;
}

__global__ void __launch_bounds__(kNtThreads) k_ntilde_fx(const CfgDev* __restrict__ cfgs, const NtItem* __restrict__ items,
                                                          int n_items, int* __restrict__ queue) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int ii = s_item;
    if (ii >= n_items) return;
    const NtItem it = items[ii];
    const CfgDev& c = cfgs[it.cfg];
    if (stopped(c)) continue;
    const fxc* __restrict__ tab = reinterpret_cast<const fxc*>(c.tab);
    const int64_t ld = c.Npad;
    const NtBlock blk = c.blocks[it.blk];
    const int64_t plen = c.plen[SSH_FX];
    const int pchunk = c.pchunk[SSH_FX];
    const int64_t j_begin = (int64_t)it.ps * plen;
    const int64_t j_end = min(c.N, j_begin + plen);
    const int nrow = blk.ng + kDigit;
    const int pbytes = fx_particle_bytes(blk.ng);
    const int lo_base_b = 48 * blk.ng;
    const bool active = (int)threadIdx.x < blk.nslots;
    NtSlot sl;
    if (active) sl = c.slots[blk.slot0 + threadIdx.x];
    else { sl.k0 = 0; sl.cnt = 0; sl.g = 0; sl.r0 = 0; }
    q160 accC[kSlotK], accS[kSlotK];
    uint32_t cntC[kSlotK], cntS[kSlotK];
#pragma unroll
    for (int i = 0; i < kSlotK; i++) {
      accC[i] = q160_zero();
      accS[i] = q160_zero();
      cntC[i] = 0;
      cntS[i] = 0;
    }
    for (int64_t j0 = j_begin; j0 < j_end; j0 += pchunk) {
      const int pc = (int)min((int64_t)pchunk, j_end - j0);
      __syncthreads();
      for (int idx = threadIdx.x; idx < nrow * pc; idx += blockDim.x) {
        const int row = idx / pc, jj = idx - row * pc;
        const int64_t j = j0 + jj;
        fxc v;
        int off;
        if (row < blk.ng) {
          const int32_t* gr = c.g_rows + (int64_t)(blk.g0 + row) * kMaxDim;
          v = PolFX::load(tab + (int64_t)gr[kMaxDim - 1] * ld + j);
#pragma unroll
          for (int a = 0; a < kMaxDim - 1; a++)
            if (gr[a] >= 0) v = fxc_mul(v, PolFX::load(tab + (int64_t)gr[a] * ld + j));
          off = 48 * row;
        } else {
          v = PolFX::load(tab + (int64_t)(c.lo_base + row - blk.ng) * ld + j);
          off = lo_base_b + fx_lo_off(row - blk.ng);
        }
        *reinterpret_cast<qent*>(smem_raw + jj * pbytes + off) = to_quadrant(v);
      }
      __syncthreads();
      if (active) {
        for (int jj = 0; jj < pc; jj++) {
          const unsigned char* base = smem_raw + jj * pbytes;
          const qent G = *reinterpret_cast<const qent*>(base + 48 * sl.g);
          const uint32_t qG = G.cs.w[0];
#pragma unroll
          for (int i = 0; i < kSlotK; i++) {
            if (i < sl.cnt) {
              const qent T = *reinterpret_cast<const qent*>(base + lo_base_b + fx_lo_off(sl.r0 + i));
              const q128 p1 = umulhi(G.c, T.c), p2 = umulhi(G.s, T.s), p3 = umulhi(G.cs, T.cs);
              const q128 re = q128_sub(p1, p2);
              const q128 im = q128_sub(q128_sub(p3, p1), p2);
              const uint32_t q = (qG + T.cs.w[0]) & 3u;
              const bool sw = q & 1u;
              q128 a, b;
#pragma unroll
              for (int w = 0; w < 4; w++) {
                a.w[w] = sw ? im.w[w] : re.w[w];
                b.w[w] = sw ? re.w[w] : im.w[w];
              }
              const uint32_t mC = 0u - (((q >> 1) ^ q) & 1u), mS = 0u - (q >> 1);
              q160_add_xor(accC[i], a, mC);
              q160_add_xor(accS[i], b, mS);
              cntC[i] += mC & 1u;
              cntS[i] += mS & 1u;
            }
          }
        }
      }
    }
    if (active) {
      FxAcc* part = reinterpret_cast<FxAcc*>(c.part) + (int64_t)it.ps * c.M;
#pragma unroll
      for (int i = 0; i < kSlotK; i++) {
        if (i < sl.cnt) {
          FxAcc o;
          o.re = accC[i];
          o.im = accS[i];
          q160_add_units(o.re, cntC[i]);  // the +1 units of each one's-complement negation
          q160_add_units(o.im, cntS[i]);
          part[sl.k0 + i] = o;
        }
      }
    }
  }
}

constexpr int kRedThreads = 256;

__device__ __forceinline__ void block_reduce(RedPart& v, RedPart* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      RedPart o = sh[threadIdx.x + s];
      RedPart m = sh[threadIdx.x];
      red_combine(m, o);
      sh[threadIdx.x] = m;
    }
    __syncthreads();
  }
  v = sh[0];
}

// grid (k blocks, configurations of this precision)
template <class P>
__global__ void __launch_bounds__(kRedThreads) k_nt_reduce(const CfgDev* __restrict__ cfgs, const int* __restrict__ list) {
  const CfgDev& c = cfgs[list[blockIdx.y]];
  if (stopped(c) || (int)blockIdx.x >= c.nblk) return;  // uniform per block
  if (P::kIdx == SSH_FX && c.tc) return;                 // the tensor-core finish kernel did this
  __shared__ RedPart sh[kRedThreads];
  const int64_t k = (int64_t)blockIdx.x * kRedThreads + threadIdx.x;
  const int64_t M = c.M;
  const typename P::Acc* part = reinterpret_cast<const typename P::Acc*>(c.part);
  RedPart v = {0, 0, 0, 0, 0, 0, 0, 0};
  if (k < M) {
    typename P::Acc a = part[k];
    for (int p = 1; p < c.psplit[P::kIdx]; p++) P::acc_add_acc(a, part[(int64_t)p * M + k]);
    dd cc, ss;
    P::acc_to_dd(a, &cc, &ss);
    c.C_hi[k] = cc.hi;
    c.C_lo[k] = cc.lo;
    c.S_hi[k] = ss.hi;
    c.S_lo[k] = ss.lo;
    dd a2 = dd_add(dd_sqr(cc), dd_sqr(ss));
    const double w = c.wk[k];  // Phi and the force coefficients carry the weight; S_max does not
    const dd wa2 = w == 1.0 ? a2 : dd_mul_d(a2, w);
    v.phi_hi = wa2.hi;
    v.phi_lo = wa2.lo;
    v.a2max_hi = a2.hi;
    v.a2max_lo = a2.lo;
    v.cmax = w * fmax(fabs(cc.hi), fabs(ss.hi));
  }
  block_reduce(v, sh);
  if (threadIdx.x == 0) reinterpret_cast<RedPart*>(c.blk)[blockIdx.x] = v;
}

// scal[kScPhiHi..] as listed in ssh_internal.h.  Scale exponent e: |C|, |S| < 2^(e-1).  Grid (1, configs).
// Fixed order: thread t combines partials t, t + 256, ...; then warp shuffle trees and one pass over the warps.
constexpr int kFinalizeThreads = 64;
__global__ void __launch_bounds__(kFinalizeThreads) k_finalize(const CfgDev* __restrict__ cfgs,
                                                               const int* __restrict__ list, int prec) {
  grid_dep_wait();
  const CfgDev& c = cfgs[list[blockIdx.y]];
  // tensor-core members finalise fixed-point evaluations in the last block of their density finish
  if (stopped(c) || (prec == SSH_FX && c.tc)) return;
  __shared__ RedPart sh[kFinalizeThreads / 32];
  finalize_block<kFinalizeThreads>(reinterpret_cast<const RedPart*>(c.blk), c.nblk, c.N, c.scal, sh);
}

template <class P>
__global__ void k_coef(const CfgDev* __restrict__ cfgs, const int* __restrict__ list) {
  const CfgDev& c = cfgs[list[blockIdx.y]];
  if (stopped(c) || (P::kIdx == SSH_FX && c.tc)) return;  // the tensor-core path builds its own coefficients
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= c.M) return;
  const int e = (int)c.scal[kScScaleExp];
  const double w = c.wk[k];
  dd C = dd_make(c.C_hi[k], c.C_lo[k]), S = dd_make(c.S_hi[k], c.S_lo[k]);
  if (w != 1.0) {
    C = dd_mul_d(C, w);
    S = dd_mul_d(S, w);
  }
  reinterpret_cast<typename P::Coef*>(c.coef)[k] = P::make_coef(C, S, e);
}

__device__ __forceinline__ int floordiv_d(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Persistent: each CTA takes (configuration, particle block, column split) items until the queue is empty.
template <class P>
__global__ void __launch_bounds__(kForceThreads) k_force(const CfgDev* __restrict__ cfgs, const FItem* __restrict__ items,
                                                         int n_items, int* __restrict__ queue) {
  using Ph = typename P::Ph;
  using RAcc = typename P::RAcc;
  __shared__ int s_item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int ii = s_item;
    if (ii >= n_items) return;
    const FItem it = items[ii];
    const CfgDev& c = cfgs[it.cfg];
    if (stopped(c)) continue;
    const typename P::Tab* __restrict__ tab = reinterpret_cast<const typename P::Tab*>(c.tab);
    const typename P::Coef* __restrict__ coef = reinterpret_cast<const typename P::Coef*>(c.coef);
    const int64_t ld = c.Npad, N = c.N;
    const int d = c.d;
    const int64_t j = (int64_t)it.pb * kForceThreads + threadIdx.x;
    const int64_t jj = j < N ? j : N - 1;
    const Ph b = P::load(tab + (int64_t)(c.lo_base + 1) * ld + jj);
    RAcc F[kMaxDim];
#pragma unroll
    for (int a = 0; a < kMaxDim; a++) P::rzero(F[a]);
    const int c_end = c.fsplit[it.ks + 1];
    for (int ci = c.fsplit[it.ks]; ci < c_end; ci++) {
      const FCol col = c.cols[ci];
      Ph G = P::one();
      const bool hasG = d > 1;
#pragma unroll
      for (int a = 0; a < kMaxDim - 1; a++) {
        if (a + 1 < d) {
          Ph t = P::load(tab + (int64_t)col.rows[a] * ld + jj);
          G = a > 0 ? P::mul(G, t) : t;
        }
      }
      int q = floordiv_d(col.nlo, kDigit);
      int r = col.nlo - q * kDigit;
      Ph th = P::load(tab + (int64_t)(c.hi_base + q - c.qmin) * ld + jj);
      Ph z = hasG ? P::mul(G, th) : th;
      if (r != 0) z = P::mul(z, P::load(tab + (int64_t)(c.lo_base + r) * ld + jj));
      RAcc A, B;
      P::rzero(A);
      P::rzero(B);
      for (int i = 0; i < col.len; i++) {
        if (i > 0) {
          if (++r == kDigit) {  // re-anchor at each digit boundary
            r = 0;
            q++;
            th = P::load(tab + (int64_t)(c.hi_base + q - c.qmin) * ld + jj);
            z = hasG ? P::mul(G, th) : th;
          } else {
            z = P::mul(z, b);
          }
        }
        const typename P::Coef cf = coef[col.k0 + i];
        P::radd(A, P::w(cf, z));
        P::radd_r(B, A);
      }
      const RAcc last = P::rsub(P::rmul_int(A, col.nlo + col.len), B);
#pragma unroll
      for (int a = 0; a < kMaxDim; a++) {
        if (a + 1 < d) P::radd_r(F[a], P::rmul_int(A, col.pre[a < kMaxDim - 1 ? a : 0]));
        else if (a + 1 == d) P::radd_r(F[a], last);
      }
    }
    if (j < N) {
      RAcc* fpart = reinterpret_cast<RAcc*>(c.fpart);
#pragma unroll
      for (int a = 0; a < kMaxDim; a++)
        if (a < d) fpart[((int64_t)it.ks * d + a) * N + j] = F[a];
    }
  }
}

// ---- fixed-point force kernel: phase recurrence and coefficient products on first-quadrant unsigned values
// With z = i^q (c + i s) and conj(n~) = C - i S, w = Im(conj(n~) z) is
//   q = 0: C s - S c,   q = 1: S s + C c,   q = 2: -C s + S c,   q = 3: -S s - C c,
// i.e. +-X s +- Y c with (X, Y) = (C, S) for even q and (S, C) for odd q: two unsigned products of the
// sign-magnitude coefficients.  Negations are one's complements whose missing units are counted (cntA for
// A = sum w, cntB for B = sum A) and added exactly at the end of the column.
// at most 96 registers, so that five CTAs fit an SM (the persistent launch runs five per SM)
__global__ void __launch_bounds__(kForceThreads, 5) k_force_fx(const CfgDev* __restrict__ cfgs, const FItem* __restrict__ items,
                                                            int n_items, int* __restrict__ queue) {
  __shared__ int s_item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int ii = s_item;
    if (ii >= n_items) return;
    const FItem it = items[ii];
    const CfgDev& c = cfgs[it.cfg];
    if (stopped(c)) continue;
    const fxc* __restrict__ tab = reinterpret_cast<const fxc*>(c.tab);
    const uint4* __restrict__ coef = reinterpret_cast<const uint4*>(c.coef);
    const int64_t ld = c.Npad, N = c.N;
    const int d = c.d;
    const int64_t j = (int64_t)it.pb * kForceThreads + threadIdx.x;
    const int64_t jj = j < N ? j : N - 1;
    const qent bq = to_quadrant(PolFX::load(tab + (int64_t)(c.lo_base + 1) * ld + jj));
    q160 F[kMaxDim];
#pragma unroll
    for (int a = 0; a < kMaxDim; a++) F[a] = q160_zero();
    const int c_end = c.fsplit[it.ks + 1];
    for (int ci = c.fsplit[it.ks]; ci < c_end; ci++) {
      const FCol col = c.cols[ci];
      fxc G = PolFX::one();
      const bool hasG = d > 1;
#pragma unroll
      for (int a = 0; a < kMaxDim - 1; a++) {
        if (a + 1 < d) {
          fxc t = PolFX::load(tab + (int64_t)col.rows[a] * ld + jj);
          G = a > 0 ? fxc_mul(G, t) : t;
        }
      }
      int q = floordiv_d(col.nlo, kDigit);
      int r = col.nlo - q * kDigit;
      fxc zs = PolFX::load(tab + (int64_t)(c.hi_base + q - c.qmin) * ld + jj);
      if (hasG) zs = fxc_mul(G, zs);
      if (r != 0) zs = fxc_mul(zs, PolFX::load(tab + (int64_t)(c.lo_base + r) * ld + jj));
      qent z = to_quadrant(zs);
      q160 A = q160_zero(), B = q160_zero();
      uint32_t cntA = 0, cntB = 0;
      for (int i = 0; i < col.len; i++) {
        if (i > 0) {
          if (++r == kDigit) {  // re-anchor at each digit boundary
            r = 0;
            q++;
            zs = PolFX::load(tab + (int64_t)(c.hi_base + q - c.qmin) * ld + jj);
            if (hasG) zs = fxc_mul(G, zs);
            z = to_quadrant(zs);
          } else {
            z = qmul(z, bq);
          }
        }
        const uint4 cr = __ldg(coef + 2 * (col.k0 + i)), sr = __ldg(coef + 2 * (col.k0 + i) + 1);
        const uint32_t qz = z.cs.w[0] & 3u;
        const bool odd = qz & 1u;
        q128 X, Y;
        X.w[0] = odd ? sr.x : cr.x;  Y.w[0] = odd ? cr.x : sr.x;
        X.w[1] = odd ? sr.y : cr.y;  Y.w[1] = odd ? cr.y : sr.y;
        X.w[2] = odd ? sr.z : cr.z;  Y.w[2] = odd ? cr.z : sr.z;
        X.w[3] = odd ? sr.w : cr.w;  Y.w[3] = odd ? cr.w : sr.w;
        const uint32_t sX = X.w[3] >> 31, sY = Y.w[3] >> 31;
        X.w[3] &= 0x7FFFFFFFu;
        Y.w[3] &= 0x7FFFFFFFu;
        const uint32_t negA = (qz >> 1) ^ sX;                      // sign of the X s term
        const uint32_t negB = (((qz ^ (qz >> 1)) & 1u) ^ 1u) ^ sY;  // sign of the Y c term
        const q128 pa = umulhi(X, z.s), pb = umulhi(Y, z.c);
        q160_add_xor(A, pa, 0u - negA);
        q160_add_xor(A, pb, 0u - negB);
        cntA += negA + negB;
        q160_add160(B, A);
        cntB += cntA;
      }
      q160_add_units(A, cntA);
      q160_add_units(B, cntB);
      const q160 last = q160_sub160(q160_mul_int(A, col.nlo + col.len), B);
#pragma unroll
      for (int a = 0; a < kMaxDim; a++) {
        if (a + 1 < d) q160_add160(F[a], q160_mul_int(A, col.pre[a < kMaxDim - 1 ? a : 0]));
        else if (a + 1 == d) q160_add160(F[a], last);
      }
    }
    if (j < N) {
      q160* fpart = reinterpret_cast<q160*>(c.fpart);
#pragma unroll
      for (int a = 0; a < kMaxDim; a++)
        if (a < d) fpart[((int64_t)it.ks * d + a) * N + j] = F[a];
    }
  }
}

// grid (coordinate blocks, configurations of this precision)
template <class P>
__global__ void k_f_reduce(const CfgDev* __restrict__ cfgs, const int* __restrict__ list) {
  const CfgDev& c = cfgs[list[blockIdx.y]];
  if (stopped(c)) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over d * N, [a][j]
  const int64_t nd = (int64_t)c.d * c.N;
  if (i >= nd) return;
  if (P::kIdx == SSH_FX && c.tc) return;  // the tensor-core force finish kernel did this
  const typename P::RAcc* fpart = reinterpret_cast<const typename P::RAcc*>(c.fpart);
  typename P::RAcc s = fpart[i];
  for (int k = 1; k < c.ksplit; k++) P::radd_r(s, fpart[(int64_t)k * nd + i]);
  dd f = dd_mul(P::r_to_dd(s), c.pref);
  const int e = P::kIdx == SSH_FX ? (int)c.scal[kScScaleExp] : 0;
  c.F_hi[i] = ldexp(f.hi, e);
  c.F_lo[i] = ldexp(f.lo, e);
}

// ------------------------------------------------------------------------------------------------ host side

static size_t tab_bytes(int prec) { return prec == SSH_FP64 ? 16 : 32; }

// Launch shape of one configuration (depends on that configuration only, so its arithmetic -- and therefore
// its result -- is the same alone and in any batch).
void setup_launch(Ctx* c) {
  const int nblocks = (int)c->nt.blocks.size();
  const int target = c->sm_count * 2;
  for (int prec = 0; prec < 3; prec++) {
    Launch& L = c->launch[prec];
    int stride = (c->nt.max_ng + kDigit) | 1;
    L.nt_stride = stride;
    size_t budget = 96 * 1024;
    const size_t per_particle = prec == SSH_FX ? (size_t)fx_particle_bytes(c->nt.max_ng) : (size_t)stride * tab_bytes(prec);
    int pchunk = (int)(budget / per_particle);
    pchunk = std::max(8, std::min(64, pchunk & ~7));
    L.nt_pchunk = pchunk;
    L.nt_smem = (size_t)pchunk * per_particle;
    int ps = nblocks > 0 ? (target + nblocks - 1) / nblocks : 1;
    int64_t max_ps = std::max<int64_t>(1, c->N / pchunk);
    L.nt_psplit = (int)std::max<int64_t>(1, std::min<int64_t>(ps, max_ps));
    // force items: enough (configuration, particle block, column split) tiles to keep every SM busy with several
    // resident CTAs of the persistent kernel
    int pblocks = (int)((c->N + kForceThreads - 1) / kForceThreads);
    int kspl = (8 * c->sm_count + pblocks - 1) / pblocks;
    kspl = std::max(1, std::min(kspl, (int)c->fp.cols.size()));
    L.f_ksplit = kspl;
  }
}

template <class P>
static cudaError_t launch_prec(const EngineView& v, bool want_force, cudaStream_t st, Prof* prof) {
  if (v.nlist == 0) return cudaSuccess;
  if (v.ntw > 0) {
    prof_begin(prof, st, kKTwiddle);
    k_twiddle<P><<<(unsigned)v.ntw, kTwThreads, 0, st>>>(v.cfgs, v.tw);
    prof_end(prof, st);
  }
  if constexpr (P::kIdx == SSH_FX) {
    cudaError_t te = tc_launch_density(v, st, prof);
    if (te != cudaSuccess) return te;
  }
  if (v.nnt > 0) {
    cudaMemsetAsync(v.counters, 0, sizeof(int), st);
    const int grid = std::min(v.nnt, 2 * v.sm_count);
    prof_begin(prof, st, kKNtilde);
    if constexpr (P::kIdx == SSH_FX)
      k_ntilde_fx<<<grid, kNtThreads, v.nt_smem, st>>>(v.cfgs, v.nt, v.nnt, v.counters);
    else
      k_ntilde<P><<<grid, kNtThreads, v.nt_smem, st>>>(v.cfgs, v.nt, v.nnt, v.counters);
    prof_end(prof, st);
  }
  if (v.nlist > v.ntc_list) {
    const dim3 gr((unsigned)std::max(1, v.maxblk), (unsigned)v.nlist);
    prof_begin(prof, st, kKNtReduce);
    k_nt_reduce<P><<<gr, kRedThreads, 0, st>>>(v.cfgs, v.list);
    prof_end(prof, st);
  }
  if (P::kIdx != SSH_FX || v.nlist > v.ntc_list) {
    prof_begin(prof, st, kKFinalize);
    cudaError_t le =
        launch_pdl(k_finalize, dim3(1, (unsigned)v.nlist), dim3(kFinalizeThreads), 0, st, v.cfgs, v.list, (int)P::kIdx);
    if (le != cudaSuccess) return le;
    prof_end(prof, st);
  }
  if (want_force) {
    if (v.nlist > v.ntc_list) {  // members that use these coefficients (the tensor-core path builds its own)
      const dim3 gc((unsigned)std::max<int64_t>(1, (v.maxM + 255) / 256), (unsigned)v.nlist);
      prof_begin(prof, st, kKCoef);
      k_coef<P><<<gc, 256, 0, st>>>(v.cfgs, v.list);
      prof_end(prof, st);
    }
    if constexpr (P::kIdx == SSH_FX) {
      cudaError_t te = tc_launch_force(v, st, prof);
      if (te != cudaSuccess) return te;
    }
    if (v.nfi > 0) {
      cudaMemsetAsync(v.counters + 1, 0, sizeof(int), st);
      const int grid = std::min(v.nfi, 5 * v.sm_count);
      prof_begin(prof, st, kKForce);
      if constexpr (P::kIdx == SSH_FX)
        k_force_fx<<<grid, kForceThreads, 0, st>>>(v.cfgs, v.fi, v.nfi, v.counters + 1);
      else
        k_force<P><<<grid, kForceThreads, 0, st>>>(v.cfgs, v.fi, v.nfi, v.counters + 1);
      prof_end(prof, st);
    }
    if (v.nlist > v.ntc_list) {
      const dim3 gf((unsigned)std::max<int64_t>(1, (v.maxND + 255) / 256), (unsigned)v.nlist);
      prof_begin(prof, st, kKFReduce);
      k_f_reduce<P><<<gf, 256, 0, st>>>(v.cfgs, v.list);
      prof_end(prof, st);
    }
    if constexpr (P::kIdx == SSH_FX) {
      cudaError_t te = tc_launch_force_finish(v, st, prof);
      if (te != cudaSuccess) return te;
    }
  }
  return cudaGetLastError();
}

cudaError_t engine_eval(const Engine* e, int prec, bool want_force, cudaStream_t st, Prof* prof) {
  switch (prec) {
    case SSH_FP64: return launch_prec<PolF64>(e->view[prec], want_force, st, prof);
    case SSH_DD: return launch_prec<PolDD>(e->view[prec], want_force, st, prof);
    case SSH_FX: return launch_prec<PolFX>(e->view[prec], want_force, st, prof);
    default: return cudaErrorInvalidValue;
  }
}

// dynamic shared memory above 48 KB is opted into once, never inside a stream capture
void kernels_set_attributes(size_t smem_max) {
  cudaFuncSetAttribute(k_ntilde<PolF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
  cudaFuncSetAttribute(k_ntilde<PolDD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
  cudaFuncSetAttribute(k_ntilde<PolFX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
  cudaFuncSetAttribute(k_ntilde_fx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
}

// ------------------------------------------------------------------------------------------------ profiler

void prof_begin(Prof* p, cudaStream_t st, int id) {
  if (!p || !p->on) return;
  ProfRec r;
  r.id = id;
  if (!p->pool.empty()) { r.e0 = p->pool.back(); p->pool.pop_back(); }
  else cudaEventCreate(&r.e0);
  if (!p->pool.empty()) { r.e1 = p->pool.back(); p->pool.pop_back(); }
  else cudaEventCreate(&r.e1);
  cudaEventRecord(r.e0, st);
  p->pending.push_back(r);
}

void prof_end(Prof* p, cudaStream_t st) {
  if (!p || !p->on || p->pending.empty()) return;
  cudaEventRecord(p->pending.back().e1, st);
}

cudaError_t prof_collect(Prof* p, cudaStream_t st) {
  if (p->pending.empty()) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  for (ProfRec& r : p->pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
      p->ms[r.id] += ms;
      p->launches[r.id] += 1;
    }
    p->pool.push_back(r.e0);
    p->pool.push_back(r.e1);
  }
  p->pending.clear();
  return cudaSuccess;
}

// ------------------------------------------------------------------------------------------------ buffers

static cudaError_t dev_alloc(DevBuf* b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  b->bytes = bytes;
  return cudaMalloc(&b->p, bytes);
}

template <class T>
static cudaError_t upload(DevBuf* b, const std::vector<T>& v, cudaStream_t st) {
  cudaError_t e = dev_alloc(b, sizeof(T) * std::max<size_t>(1, v.size()));
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpyAsync(b->p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st);
}

// Plans and buffers of one configuration, then its own single-member engine.
cudaError_t plan_upload(Ctx* c) {
  cudaStream_t st = c->stream;
  cudaError_t e;
  setup_launch(c);
  // column split for the force kernel: equal numbers of wavevectors per split, the same for every precision
  int ks = 1;
  for (int p = 0; p < 3; p++) ks = std::max(ks, c->launch[p].f_ksplit);
  for (int p = 0; p < 3; p++) c->launch[p].f_ksplit = ks;
  c->f_split.assign(ks + 1, 0);
  {
    int ncol = (int)c->fp.cols.size();
    int64_t per = (c->M + ks - 1) / std::max(1, ks);
    int ci = 0;
    for (int s = 1; s < ks; s++) {
      int64_t target = per * s;
      while (ci < ncol && c->fp.cols[ci].k0 < target) ci++;
      c->f_split[s] = ci;
    }
    c->f_split[ks] = ncol;
  }
  if ((e = upload(&c->rows, c->tl.rows, st)) != cudaSuccess) return e;
  if ((e = upload(&c->slots, c->nt.slots, st)) != cudaSuccess) return e;
  if ((e = upload(&c->blocks, c->nt.blocks, st)) != cudaSuccess) return e;
  if ((e = upload(&c->grows, c->nt.g_rows, st)) != cudaSuccess) return e;
  if ((e = upload(&c->cols, c->fp.cols, st)) != cudaSuccess) return e;
  if ((e = upload(&c->fsplit, c->f_split, st)) != cudaSuccess) return e;
  size_t nd = (size_t)c->d * c->N;
  if ((e = dev_alloc(&c->s_hi, nd * 8)) != cudaSuccess) return e;
  if ((e = dev_alloc(&c->s_lo, nd * 8)) != cudaSuccess) return e;
  if ((e = dev_alloc(&c->tab, (size_t)c->tl.rows.size() * c->Npad * kTabBytes)) != cudaSuccess) return e;
  int max_ps = 1;
  for (int p = 0; p < 3; p++) max_ps = std::max(max_ps, c->launch[p].nt_psplit);
  if ((e = dev_alloc(&c->part, (size_t)max_ps * c->M * kAccBytes)) != cudaSuccess) return e;
  for (DevBuf* b : {&c->C_hi, &c->C_lo, &c->S_hi, &c->S_lo})
    if ((e = dev_alloc(b, (size_t)c->M * 8)) != cudaSuccess) return e;
  {
    const std::vector<double> ones((size_t)std::max<int64_t>(c->M, 1), 1.0);
    if ((e = dev_alloc(&c->wk, ones.size() * 8)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(c->wk.p, ones.data(), ones.size() * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;  // the host vector goes out of scope
    c->wmax = 1.0;
  }
  if ((e = dev_alloc(&c->coef, (size_t)c->M * kTabBytes)) != cudaSuccess) return e;
  if ((e = tc_setup(c)) != cudaSuccess) return e;
  c->n_red_blocks = (int)((c->M + kRedThreads - 1) / kRedThreads);
  if ((e = dev_alloc(&c->blk, (size_t)std::max(std::max(1, c->n_red_blocks), tc_finish_blocks(*c)) * sizeof(RedPart))) !=
      cudaSuccess)
    return e;
  if ((e = dev_alloc(&c->scal, sizeof(double) * kScCount)) != cudaSuccess) return e;
  if ((e = dev_alloc(&c->fpart, (size_t)ks * nd * kRAccBytes)) != cudaSuccess) return e;
  if ((e = dev_alloc(&c->F_hi, nd * 8)) != cudaSuccess) return e;
  if ((e = dev_alloc(&c->F_lo, nd * 8)) != cudaSuccess) return e;
  cudaMemsetAsync(c->scal.p, 0, sizeof(double) * kScCount, st);
  cudaMemsetAsync(c->F_hi.p, 0, nd * 8, st);
  cudaMemsetAsync(c->F_lo.p, 0, nd * 8, st);
  size_t smem_max = 0;
  for (int p = 0; p < 3; p++) smem_max = std::max(smem_max, c->launch[p].nt_smem);
  kernels_set_attributes(std::max<size_t>(smem_max, 96 * 1024));
  c->eng = new Engine();
  if ((e = engine_build(c->eng, {c}, {-1}, false, st)) != cudaSuccess) return e;
  return cudaGetLastError();
}

size_t device_footprint(const Ctx& c) {
  const size_t nd = (size_t)c.d * c.N;
  int max_ps = 1;
  for (int p = 0; p < 3; p++) max_ps = std::max(max_ps, c.launch[p].nt_psplit);
  size_t b = 0;
  b += (size_t)c.tl.rows.size() * c.Npad * kTabBytes;         // power tables
  b += (size_t)max_ps * c.M * kAccBytes;                       // density partials
  b += (size_t)c.M * (4 * 8 + kTabBytes);                      // C, S, coefficients
  b += (size_t)c.launch[0].f_ksplit * nd * kRAccBytes;         // force partials
  b += nd * 8 * (4 + 6);                                       // positions, force, velocity, undo copies
  b += c.nt.slots.size() * sizeof(NtSlot) + c.nt.g_rows.size() * 4 + c.fp.cols.size() * sizeof(FCol);
  b += c.tl.rows.size() * sizeof(TabRow) + 64 * 1024;          // small buffers and allocation granularity
  b += tc_footprint(c);                                        // tensor-core digit slices and partials
  return b;
}

cudaError_t eval_phi_grad(Ctx* c, int prec, bool want_force) {
  return engine_eval(c->eng, prec, want_force, c->stream, &c->prof);
}

}  // namespace ssh
