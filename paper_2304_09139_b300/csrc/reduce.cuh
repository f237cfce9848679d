// reduce.cuh -- per-block partials of the density reduction (Phi, max |n~|^2, max |C|, |S|), shared by the
// integer-pipe and tensor-core paths.
#pragma once
#include "dd.cuh"

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

}  // namespace ssh
