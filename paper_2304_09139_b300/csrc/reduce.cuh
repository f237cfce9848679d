// reduce.cuh -- per-block partials of the density reduction (Phi, max |n~|^2, max |C|, |S|), shared by the
// integer-pipe and tensor-core paths.
#pragma once
#include "dd.cuh"
#include "ssh_internal.h"

namespace ssh {

struct RedPart {  // per-block partials of the density reduction
  double phi_hi, phi_lo, a2max_hi, a2max_lo, cmax, pad0, pad1, pad2;
};

__device__ __forceinline__ void red_combine(RedPart& a, const RedPart& b) {
  // Phi is a sum of non-negative terms: the two-sum form without the low-word two-sum is accurate to ~2^-104
  dd s = dd_add_sloppy(dd_make(a.phi_hi, a.phi_lo), dd_make(b.phi_hi, b.phi_lo));
  a.phi_hi = s.hi;
  a.phi_lo = s.lo;
  if (dd_gt(dd_make(b.a2max_hi, b.a2max_lo), dd_make(a.a2max_hi, a.a2max_lo))) {
    a.a2max_hi = b.a2max_hi;
    a.a2max_lo = b.a2max_lo;
  }
  a.cmax = fmax(a.cmax, b.cmax);
}

// fixed-order warp reduction (lane 0 ends with the combination of lanes 0..31 in a fixed tree); only the lanes
// that keep a result combine, so the tree costs 31 combines (FP64 work is scarce on this part)
__device__ __forceinline__ void red_warp(RedPart& v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    RedPart o;
    o.phi_hi = __shfl_down_sync(0xffffffffu, v.phi_hi, off);
    o.phi_lo = __shfl_down_sync(0xffffffffu, v.phi_lo, off);
    o.a2max_hi = __shfl_down_sync(0xffffffffu, v.a2max_hi, off);
    o.a2max_lo = __shfl_down_sync(0xffffffffu, v.a2max_lo, off);
    o.cmax = __shfl_down_sync(0xffffffffu, v.cmax, off);
    if (lane < off) red_combine(v, o);
  }
}

// The scalars of one evaluation from its nb block partials, by one block of kThreads threads: lane-strided
// combination in block order, a fixed warp tree, then the warps in order (the same order whichever block runs
// it); thread 0 writes Phi, S_max = max |n~|^2 / N, max |C|, |S| and the power-of-two scale e of (C, S)
// (2^e > 2 max |C|, |S|).  The partials are read through L2, so a block of the kernel that wrote them may run it
// once every block's write is visible (fence + ticket).
template <int kThreads>
__device__ __forceinline__ void finalize_block(const RedPart* blk, int nb, int64_t N, double* scal,
                                               RedPart (&sh)[kThreads / 32]) {
  auto load = [&](int i) {
    const double* p = reinterpret_cast<const double*>(blk + i);
    RedPart r;
    r.phi_hi = __ldcg(p + 0);
    r.phi_lo = __ldcg(p + 1);
    r.a2max_hi = __ldcg(p + 2);
    r.a2max_lo = __ldcg(p + 3);
    r.cmax = __ldcg(p + 4);
    r.pad0 = r.pad1 = r.pad2 = 0;
    return r;
  };
  RedPart v = {0, 0, 0, 0, 0, 0, 0, 0};
  if ((int)threadIdx.x < nb) v = load(threadIdx.x);
  for (int i = threadIdx.x + kThreads; i < nb; i += kThreads) red_combine(v, load(i));
  red_warp(v);
  __syncthreads();  // sh may hold the caller's earlier partials
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    v = sh[0];
#pragma unroll
    for (int w = 1; w < kThreads / 32; w++) red_combine(v, sh[w]);
    scal[kScPhiHi] = v.phi_hi;
    scal[kScPhiLo] = v.phi_lo;
    dd sm = N > 0 ? dd_div(dd_make(v.a2max_hi, v.a2max_lo), dd_make((double)N)) : dd_make(0.0);
    scal[kScSmaxHi] = sm.hi;
    scal[kScSmaxLo] = sm.lo;
    scal[kScCmax] = v.cmax;
    scal[kScScaleExp] = v.cmax > 0 ? (double)(ilogb(v.cmax) + 2) : 0.0;
    scal[kScA2MaxHi] = v.a2max_hi;
    scal[kScA2MaxLo] = v.a2max_lo;
  }
}

}  // namespace ssh
