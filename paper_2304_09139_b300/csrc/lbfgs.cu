// lbfgs.cu -- limited-memory BFGS with a backtracking (Armijo) line search, on the device, as an alternative
// minimiser to FIRE for the collective-coordinate energy (the paper quenches with "various minimizers"; FIRE is
// the one it names).  Positions stay double-double and fractional; the gradient with respect to the fractional
// positions is G = dPhi/ds = -L F; the history pairs s_k = x_{k+1} - x_k (minimum image) and y_k = G_{k+1} - G_k
// are kept in binary64.
//
// The direction p = -H G uses the compact representation of the inverse L-BFGS matrix (Byrd, Nocedal and
// Schnabel 1994, Theorem 2.2): with S = [s_i], Y = [y_i] (oldest first), R the upper triangle of S^T Y, D its
// diagonal and gamma = s^T y / y^T y of the newest pair,
//   H G = gamma G + S w1 + gamma Y w2,   t = R^-1 (S^T G),   w2 = -t,   w1 = R^-T ((D + gamma Y^T Y) t - gamma Y^T G),
// so one iteration needs the dot products of the new pair with the history and of G with every pair (one pass
// over the coordinates), a small triangular solve, and one pass forming p: two passes, however long the history,
// instead of the two-loop recursion's 2m dependent reductions.
//
// One step of a member (the host launches these only when a member minimises with L-BFGS; every kernel skips
// the FIRE members and finished runs):
//   k_lb_dir     if a new direction is due: p, G.p, max |p|, |G|^2, max |G|; the step length alpha
//   k_lb_trial   saves the accepted state (positions, force) and moves to x + alpha p (steepest descent when the
//                history holds no usable pair)
//   ... evaluation of Phi, S_max and F at the trial positions ...
//   k_lb_accept  Armijo test Phi(x + alpha p) <= Phi(x) + c1 alpha G.p (+ the evaluation-error margin of the
//                energy guard); accept, or halve alpha and restore (k_fire_restore); stop rules as FIRE's
//   k_lb_pairs   after an accepted step: the new pair and every dot product (block partials, the last block
//                reduces them in block order and solves for t and w1)
// Every reduction has a fixed order, so a member's run is bit-identical alone and in a batch.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "dd.cuh"
#include "ssh_internal.h"

namespace ssh {

namespace {

// FP64 arithmetic on this part has a 64-cycle dependent latency (16 times FP32's): every sum here is a shallow
// tree over independent partial sums rather than a long chain
constexpr int kLbThreads = 128;
constexpr int kLbWarps = kLbThreads / 32;
constexpr double kArmijo = 1e-4;

__device__ __forceinline__ FireState* lb_state(const CfgDev& c) { return reinterpret_cast<FireState*>(c.fs); }

__device__ __forceinline__ bool lb_running(const CfgDev& c) {
  const FireState* fs = lb_state(c);
  return fs->method == kMethodLbfgs && fs->status == kFsRunning;
}

// minimum-image difference of two fractional coordinates in [0, 1), as binary64
__device__ __forceinline__ double frac_diff(double ah, double al, double bh, double bl) {
  double d = (ah - bh) + (al - bl);
  if (d > 0.5) d -= 1.0;
  else if (d < -0.5) d += 1.0;
  return d;
}

// block sum of kV values per thread: a fixed shuffle tree per warp, then the warps in order; the block's totals
// land in out[0..kV) (shared memory), written by the first kV threads
template <int kV>
__device__ __forceinline__ void block_sum(double (&v)[kV], double (*sh)[kV], double* out) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int q = 0; q < kV; q++) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int q = 0; q < kV; q++) sh[threadIdx.x >> 5][q] = v[q];
  __syncthreads();
  for (int q = threadIdx.x; q < kV; q += kLbThreads) {
    double a = 0.0;
#pragma unroll
    for (int w = 0; w < kLbWarps; w++) a += sh[w][q];
    out[q] = a;
  }
  __syncthreads();
}

// column sums over nb block partials (stride kLbPartStride) into out[0..nv): warp w takes the columns q = w mod
// kLbWarps, its lanes stride over the blocks, then a shuffle tree; max instead of sum for columns >= nsum
__device__ __forceinline__ void column_sums(const double* part, int nb, int nv, int nsum, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = warp; q < nv; q += kLbWarps) {
    const bool mx = q >= nsum;
    double a = 0.0;
    for (int b = lane; b < nb; b += 32) {
      const double x = __ldcg(part + (int64_t)b * kLbPartStride + q);
      a = mx ? fmax(a, x) : a + x;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_down_sync(0xffffffffu, a, off);
      a = mx ? fmax(a, o) : a + o;
    }
    if (lane == 0) out[q] = a;
  }
  __syncthreads();
}

// ticket of the last block of a member's pass (counter in the member's matrix block); true in every thread
__device__ __forceinline__ bool last_block(int* counter, int nblocks) {
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1) == nblocks - 1;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

}  // namespace

// Block map: nb_fire blocks of kLbThreads per member.  A new direction when one is due.
__global__ void __launch_bounds__(kLbThreads) k_lb_dir(const CfgDev* __restrict__ cfgs, const BlockMap* __restrict__ bm) {
  grid_dep_wait();
  const BlockMap mb = bm[blockIdx.x];
  const CfgDev& c = cfgs[mb.cfg];
  if (!lb_running(c)) return;
  FireState* fs = lb_state(c);
  if (!fs->lb_need_dir) return;
  LbMat* L = reinterpret_cast<LbMat*>(c.lb_mat);
  const int64_t nd = (int64_t)c.d * c.N;
  const int cnt = fs->lb_sd ? 0 : fs->lb_count, m = kLbMaxPairs;
  double w1[kLbMaxPairs], tt[kLbMaxPairs];
  int slot[kLbMaxPairs];
#pragma unroll
  for (int q = 0; q < kLbMaxPairs; q++) {
    slot[q] = (fs->lb_head + 1 - cnt + q + 2 * m) % m;  // chronological q -> ring slot
    w1[q] = q < cnt ? L->w1[q] : 0.0;
    tt[q] = q < cnt ? L->t[q] : 0.0;
  }
  const double gamma = fs->lb_gamma;
  // partials: G.p, |G|^2 (sums), max |p|, max |G|
  double v[2] = {0.0, 0.0};
  double pm = 0.0, gm = 0.0;
  for (int64_t i = (int64_t)mb.blk * kLbThreads + threadIdx.x; i < nd; i += (int64_t)c.nb_fire * kLbThreads) {
    const double g = c.lb_G[i];
    double p = -gamma * g;
    // every slot is loaded (unused ones carry zero coefficients), so the loads issue together
    double sv[kLbMaxPairs], yv[kLbMaxPairs];
#pragma unroll
    for (int q = 0; q < kLbMaxPairs; q++) {
      sv[q] = c.lb_S[(int64_t)slot[q] * nd + i];
      yv[q] = c.lb_Y[(int64_t)slot[q] * nd + i];
    }
    double acc[4] = {0.0, 0.0, 0.0, 0.0};  // four independent partial sums: a shallow dependent chain
#pragma unroll
    for (int q = 0; q < kLbMaxPairs; q++) acc[q & 3] += gamma * tt[q] * yv[q] - w1[q] * sv[q];
    p += (acc[0] + acc[1]) + (acc[2] + acc[3]);
    c.lb_P[i] = p;
    v[0] += g * p;
    v[1] += g * g;
    pm = fmax(pm, fabs(p));
    gm = fmax(gm, fabs(g));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    pm = fmax(pm, __shfl_down_sync(0xffffffffu, pm, off));
    gm = fmax(gm, __shfl_down_sync(0xffffffffu, gm, off));
  }
  __shared__ double sh[kLbWarps][2], shm[kLbWarps][2], tot[2];
  if ((threadIdx.x & 31) == 0) {
    shm[threadIdx.x >> 5][0] = pm;
    shm[threadIdx.x >> 5][1] = gm;
  }
  block_sum<2>(v, sh, tot);
  double* part = c.lb_part + (int64_t)mb.blk * kLbPartStride;
  if (threadIdx.x == 0) {
    for (int w = 1; w < kLbWarps; w++) {
      pm = fmax(pm, shm[w][0]);
      gm = fmax(gm, shm[w][1]);
    }
    part[0] = tot[0];
    part[1] = tot[1];
    part[2] = pm;
    part[3] = gm;
  }
  if (!last_block(&L->ticket_dir, c.nb_fire)) return;
  __shared__ double col[4];
  column_sums(c.lb_part, c.nb_fire, 4, 2, col);
  if (threadIdx.x != 0) return;
  const double gp = col[0], g2 = col[1], pmax = col[2], gmax = col[3];
  L->ticket_dir = 0;
  if (cnt > 0 && !(gp < 0)) {  // not a descent direction: drop the history, steepest descent
    fs->lb_count = 0;
    fs->lb_sd = 1;
  }
  if (fs->lb_sd) {
    fs->lb_gp = -g2;
    fs->lb_alpha = gmax > 0 ? fs->lb_dmax / gmax : 0.0;  // the largest component moves dmax
  } else {
    fs->lb_gp = gp;
    fs->lb_alpha = pmax > fs->lb_dmax ? fs->lb_dmax / pmax : 1.0;  // the quasi-Newton step, capped
  }
  fs->lb_need_dir = 0;
}

// Block map: d N / 64 blocks per member.  Save the accepted state and move to the trial point.
__global__ void k_lb_trial(const CfgDev* __restrict__ cfgs, const BlockMap* __restrict__ bm) {
  grid_dep_wait();
  const BlockMap mb = bm[blockIdx.x];
  const CfgDev& c = cfgs[mb.cfg];
  if (!lb_running(c)) return;
  const FireState* fs = lb_state(c);
  const int64_t i = (int64_t)mb.blk * blockDim.x + threadIdx.x;
  if (i >= (int64_t)c.d * c.N) return;
  const double step = fs->lb_alpha * (fs->lb_sd ? -c.lb_G[i] : c.lb_P[i]);
  dd s = dd_make(c.s_hi[i], c.s_lo[i]);
  c.bs_hi[i] = s.hi;
  c.bs_lo[i] = s.lo;
  c.bF_hi[i] = c.F_hi[i];
  c.bF_lo[i] = c.F_lo[i];
  s = dd_frac(dd_add_d(s, step));
  c.s_hi[i] = s.hi;
  c.s_lo[i] = s.lo;
}

// One thread per member: the Armijo test of the trial, and the stop rules.
__global__ void k_lb_accept(const CfgDev* __restrict__ cfgs, const int* __restrict__ all, int n) {
  grid_dep_wait();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const CfgDev& c = cfgs[all[t]];
  if (!lb_running(c)) return;
  FireState* fs = lb_state(c);
  const dd phi = dd_make(c.scal[kScPhiHi], c.scal[kScPhiLo]);
  const dd smx = dd_make(c.scal[kScSmaxHi], c.scal[kScSmaxLo]);
  fs->step++;
  fs->stage_step++;
  if (tc_failed(c)) {  // incomplete sums: undo the trial and stop the run
    fs->status = kFsDevErr;
    fs->rejected_now = 1;
    fs->lb_accepted = 0;
    return;
  }
  if (!isfinite(phi.hi) || !isfinite(smx.hi)) {
    fs->status = kFsNan;
    fs->rejected_now = 1;
    fs->lb_accepted = 0;
    return;
  }
  const dd phi_acc = dd_make(fs->phi_hi, fs->phi_lo);
  const double margin = fs->phi_tol * sqrt(fmax(phi_acc.hi, 0.0));
  // sufficient decrease (the gradient is with respect to fractional positions; alpha p is the fractional move)
  const double bound = kArmijo * fs->lb_alpha * fs->lb_gp + margin;
  if (dd_gt(phi, dd_add_d(phi_acc, bound))) {
    fs->rejected_now = 1;
    fs->rejected++;
    fs->lb_accepted = 0;
    fs->lb_alpha *= 0.5;
    if (++fs->lb_backtracks > 60) {
      // the direction does not descend within the evaluation's resolution: restart from steepest descent
      fs->lb_count = 0;
      fs->lb_sd = 1;
      fs->lb_need_dir = 1;
      fs->lb_backtracks = 0;
    }
  } else {
    fs->rejected_now = 0;
    fs->lb_accepted = 1;
    fs->lb_backtracks = 0;
    fs->phi_hi = phi.hi;
    fs->phi_lo = phi.lo;
    fs->smax_hi = smx.hi;
    fs->smax_lo = smx.lo;
  }
  const double sm = fs->smax_hi + fs->smax_lo;
  if (sm <= fs->target) {
    fs->status = kFsConverged;
  } else if (fs->step >= fs->max_steps) {
    fs->status = kFsMaxSteps;
  } else {
    if (sm < 0.5 * fs->best_smax) {
      fs->best_smax = sm;
      fs->best_step = fs->stage_step;
    }
    if (fs->stage_floor > 0 && sm <= fs->stage_floor) fs->status = kFsStageDone;
    else if (fs->stage_step - fs->best_step > fs->stall_window) fs->status = kFsStageDone;
  }
}

// Block map: nb_fire blocks of kLbThreads per member.  After an accepted step: the new pair (s, y), G at the new
// point, and the dot products s_j.y, s.y_j, y_j.y, s_j.G, y_j.G; the last block updates S^T Y and Y^T Y and
// solves for the direction's coefficients.
__global__ void __launch_bounds__(kLbThreads) k_lb_pairs(const CfgDev* __restrict__ cfgs, const BlockMap* __restrict__ bm) {
  grid_dep_wait();
  const BlockMap mb = bm[blockIdx.x];
  const CfgDev& c = cfgs[mb.cfg];
  FireState* fs = lb_state(c);
  if (fs->method != kMethodLbfgs || !fs->lb_accepted) return;  // also after a converging step: harmless
  LbMat* L = reinterpret_cast<LbMat*>(c.lb_mat);
  const int64_t nd = (int64_t)c.d * c.N;
  const int m = kLbMaxPairs;
  const int h = (fs->lb_head + 1) % m;  // slot of the candidate pair
  const double Lbox = c.L;
  constexpr int kV = 5 * kLbMaxPairs + 1;  // five dot products per slot, then s.s of the new pair
  double v[kV];
#pragma unroll
  for (int q = 0; q < kV; q++) v[q] = 0.0;
  for (int64_t i = (int64_t)mb.blk * kLbThreads + threadIdx.x; i < nd; i += (int64_t)c.nb_fire * kLbThreads) {
    const double sn = frac_diff(c.s_hi[i], c.s_lo[i], c.bs_hi[i], c.bs_lo[i]);
    const double gn = -Lbox * c.F_hi[i];
    const double yn = gn - c.lb_G[i];
    c.lb_S[(int64_t)h * nd + i] = sn;
    c.lb_Y[(int64_t)h * nd + i] = yn;
    c.lb_G[i] = gn;
#pragma unroll
    for (int j = 0; j < kLbMaxPairs; j++) {
      const double sj = j == h ? sn : c.lb_S[(int64_t)j * nd + i];
      const double yj = j == h ? yn : c.lb_Y[(int64_t)j * nd + i];
      v[5 * j + 0] += sj * yn;  // s_j . y_new
      v[5 * j + 1] += sn * yj;  // s_new . y_j
      v[5 * j + 2] += yj * yn;  // y_j . y_new
      v[5 * j + 3] += sj * gn;  // s_j . G
      v[5 * j + 4] += yj * gn;  // y_j . G
    }
    v[5 * kLbMaxPairs] += sn * sn;
  }
  __shared__ double sh[kLbWarps][kV], btot[kV];
  block_sum<kV>(v, sh, btot);
  for (int q = threadIdx.x; q < kV; q += kLbThreads) c.lb_part[(int64_t)mb.blk * kLbPartStride + q] = btot[q];
  if (!last_block(&L->ticket_pairs, c.nb_fire)) return;
  __shared__ double cols[kV];
  column_sums(c.lb_part, c.nb_fire, kV, kV, cols);
  // S^T Y and Y^T Y into shared memory (the lanes together), the small solve then reads shared memory only
  __shared__ double sStY[kLbMaxPairs][kLbMaxPairs], sYtY[kLbMaxPairs][kLbMaxPairs];
  for (int q = threadIdx.x; q < kLbMaxPairs * kLbMaxPairs; q += kLbThreads) {
    sStY[q / kLbMaxPairs][q % kLbMaxPairs] = L->StY[q / kLbMaxPairs][q % kLbMaxPairs];
    sYtY[q / kLbMaxPairs][q % kLbMaxPairs] = L->YtY[q / kLbMaxPairs][q % kLbMaxPairs];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  L->ticket_pairs = 0;
  const double* tot = cols;
  fs->lb_accepted = 0;
  fs->lb_need_dir = 1;
  const double sy = tot[5 * h + 0], yy = tot[5 * h + 2], ss = tot[5 * kLbMaxPairs];
  // keep the pair only with positive curvature (s and y not nearly orthogonal)
  if (yy > 0 && ss > 0 && sy > 1e-10 * sqrt(ss * yy)) {
    for (int j = 0; j < m; j++) {
      sStY[h][j] = L->StY[h][j] = tot[5 * j + 1];  // s_h . y_j
      sStY[j][h] = L->StY[j][h] = tot[5 * j + 0];  // s_j . y_h
      sYtY[h][j] = sYtY[j][h] = L->YtY[h][j] = L->YtY[j][h] = tot[5 * j + 2];
    }
    sStY[h][h] = L->StY[h][h] = sy;
    fs->lb_head = h;
    fs->lb_count = fs->lb_count < m ? fs->lb_count + 1 : m;
    fs->lb_gamma = sy / yy;
    fs->lb_sd = 0;
  }
  const int cnt = fs->lb_count;
  if (cnt == 0) {
    fs->lb_sd = 1;
    return;
  }
  // chronological order q = 0 (oldest) .. cnt - 1 (newest)
  int slot[kLbMaxPairs];
  for (int q = 0; q < cnt; q++) slot[q] = (fs->lb_head + 1 - cnt + q + 2 * m) % m;
  double a[kLbMaxPairs], b[kLbMaxPairs], t[kLbMaxPairs], z[kLbMaxPairs], w[kLbMaxPairs];
  for (int q = 0; q < cnt; q++) {
    a[q] = tot[5 * slot[q] + 3];
    b[q] = tot[5 * slot[q] + 4];
  }
  const double gamma = fs->lb_gamma;
  double rd[kLbMaxPairs];  // reciprocals of the diagonal of R (positive: pairs are kept only with s.y > 0)
  for (int q = 0; q < cnt; q++) rd[q] = 1.0 / sStY[slot[q]][slot[q]];
  // t = R^-1 a (R upper triangular, R[q][r] = s_q . y_r for q <= r)
  for (int q = cnt - 1; q >= 0; q--) {
    double a0 = a[q], a1 = 0.0;
    for (int r = q + 1; r < cnt; r++) {
      if ((r - q) & 1) a0 -= sStY[slot[q]][slot[r]] * t[r];
      else a1 -= sStY[slot[q]][slot[r]] * t[r];
    }
    t[q] = (a0 + a1) * rd[q];
  }
  // z = (D + gamma Y^T Y) t - gamma b;  w1 = R^-T z
  for (int q = 0; q < cnt; q++) {
    double acc = sStY[slot[q]][slot[q]] * t[q] - gamma * b[q];
    for (int r = 0; r < cnt; r++) acc += gamma * sYtY[slot[q]][slot[r]] * t[r];
    z[q] = acc;
  }
  for (int q = 0; q < cnt; q++) {
    double a0 = z[q], a1 = 0.0;
    for (int r = 0; r < q; r++) {
      if (r & 1) a1 -= sStY[slot[r]][slot[q]] * w[r];
      else a0 -= sStY[slot[r]][slot[q]] * w[r];
    }
    w[q] = (a0 + a1) * rd[q];
  }
  for (int q = 0; q < cnt; q++) {
    L->t[q] = t[q];
    L->w1[q] = w[q];
  }
}

// Stage start of L-BFGS members (elementwise, after the stage's evaluation): G at the start positions.
__global__ void k_lb_stage_g(const CfgDev* __restrict__ cfgs, const int* __restrict__ idx) {
  const CfgDev& c = cfgs[idx[blockIdx.y]];
  if (lb_state(c)->method != kMethodLbfgs) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)c.d * c.N) return;
  c.lb_G[i] = -c.L * c.F_hi[i];
}

// ------------------------------------------------------------------------------------------------ host

cudaError_t lbfgs_pre(const Engine* e, cudaStream_t st) {
  const CfgDev* cfgs = e->view[0].cfgs;
  cudaError_t le = launch_pdl(k_lb_dir, dim3((unsigned)e->nbm_dots), dim3(kLbThreads), 0, st, cfgs, e->bm_dots);
  if (le == cudaSuccess) le = launch_pdl(k_lb_trial, dim3((unsigned)e->nbm_nd), dim3(64), 0, st, cfgs, e->bm_nd);
  return le;
}

cudaError_t lbfgs_post_accept(const Engine* e, cudaStream_t st) {
  const CfgDev* cfgs = e->view[0].cfgs;
  return launch_pdl(k_lb_accept, dim3((unsigned)((e->nall + 127) / 128)), dim3(128), 0, st, cfgs, e->all, e->nall);
}

cudaError_t lbfgs_post_pairs(const Engine* e, cudaStream_t st) {
  const CfgDev* cfgs = e->view[0].cfgs;
  return launch_pdl(k_lb_pairs, dim3((unsigned)e->nbm_dots), dim3(kLbThreads), 0, st, cfgs, e->bm_dots);
}

cudaError_t lbfgs_stage_g(const CfgDev* cfgs, int64_t maxND, const int* d_idx, int n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_lb_stage_g<<<dim3((unsigned)std::max<int64_t>(1, (maxND + 255) / 256), (unsigned)n), 256, 0, st>>>(cfgs, d_idx);
  return cudaGetLastError();
}

}  // namespace ssh
