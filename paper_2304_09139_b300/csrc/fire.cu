// fire.cu -- the paper's minimiser (Simulations: FIRE, Bitzek et al. 2006) kept on the device, for one
// configuration or for every member of a batch at once.
//
// One step, for the force F and energy Phi at the accepted positions and the velocity v of the last step:
//   k_fire_dots     P = F.v, |F|^2, |v|^2 (partials per chunk of 2048 particles of an axis, fixed order; a shard
//                   computes its chunks' partials and the caller sums them, k_fire_dots_part / k_fire_control);
//                   the last block of a member applies
//                   the FIRE rules: P > 0 -> v <- (1-a) v + a |v| F/|F|; after more than n_min such steps
//                   dt <- min(dt f_inc, dt_max), a <- a f_alpha;  P <= 0 -> v <- 0, dt <- dt f_dec, a <- a_start
//   k_fire_move     semi-implicit Euler with unit mass: v <- v + dt F, r <- r + dt v (dd, wrapped into the box);
//                   the accepted positions and force are kept for a possible undo
//   (Phi + force at the new positions: the evaluation kernels of each member's current precision)
//   k_fire_accept   energy guard: Phi_new > Phi -> reject (dt <- dt f_dec, v <- 0, a <- a_start) and undo;
//                   convergence S_max <= target; step cap; the precision stage ends when S_max falls below the
//                   stage floor or has not halved in stall_window steps
//   k_fire_restore  the undo of a rejected step
// Every kernel first reads its member's device status word and skips the member when its run has ended, so a
// captured chunk of steps costs nothing for converged members.  The host replays a CUDA graph of
// kFireGraphSteps steps and reads the status words between chunks; they are the only per-chunk copy.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>

#include "ssh_internal.h"

namespace ssh {

constexpr int kFireThreads = 256;
constexpr int kFireGraphSteps = 8;

__device__ __forceinline__ FireState* fstate(const CfgDev& c) { return reinterpret_cast<FireState*>(c.fs); }

// Partial sums P = F.v, |F|^2, |v|^2 (high words) of dot chunk q of member c: axis a = q / nq1, particles
// [jb kDotChunk, (jb + 1) kDotChunk) (q = a nq1 + jb), each thread over a fixed stride, then a fixed tree.  The
// chunking depends on N alone, so a chunk's partial is the same whichever launch or shard computes it.  Every
// thread of the block calls it; thread 0 returns the three sums.
__device__ void dots_chunk(const CfgDev& c, int64_t q, double (*sh)[kFireThreads], double out[3]) {
  const int64_t nq1 = (c.N + kDotChunk - 1) / kDotChunk;
  const int a = (int)(q / nq1);
  const int64_t j0 = (q - (int64_t)a * nq1) * kDotChunk, j1 = min(c.N, j0 + kDotChunk);
  double p = 0, f2 = 0, v2 = 0;
  for (int64_t j = j0 + threadIdx.x; j < j1; j += kFireThreads) {
    const int64_t i = (int64_t)a * c.N + j;
    const double f = c.F_hi[i], w = c.v_hi[i];
    p = fma(f, w, p);
    f2 = fma(f, f, f2);
    v2 = fma(w, w, v2);
  }
  sh[0][threadIdx.x] = p;
  sh[1][threadIdx.x] = f2;
  sh[2][threadIdx.x] = v2;
  __syncthreads();
  for (int st = kFireThreads / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
      for (int r = 0; r < 3; r++) sh[r][threadIdx.x] += sh[r][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int r = 0; r < 3; r++) out[r] = sh[r][0];
  __syncthreads();
}

// The FIRE controls of a step from the chunk partials part[3][nq], summed by one warp (lane-strided in chunk order,
// then a fixed shuffle tree): mixing, velocity reset, dt and alpha (Bitzek et al. 2006).
__device__ void dots_control(FireState* fs, const double* part, int64_t nq, int lane) {
  // the state the rules read, loaded before the sums so that the loads overlap (one latency, not a chain)
  const double alpha = fs->alpha, dt = fs->dt, f_inc = fs->f_inc, dt_max = fs->dt_max, f_alpha = fs->f_alpha,
               f_dec = fs->f_dec, alpha_start = fs->alpha_start;
  const long long n_pos = fs->n_pos, n_min = fs->n_min;
  double P = 0, f2 = 0, v2 = 0;
  for (int64_t b = lane; b < nq; b += 32) {
    P += part[b];
    f2 += part[nq + b];
    v2 += part[2 * nq + b];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    P += __shfl_down_sync(0xffffffffu, P, off);
    f2 += __shfl_down_sync(0xffffffffu, f2, off);
    v2 += __shfl_down_sync(0xffffffffu, v2, off);
  }
  if (lane != 0) return;
  fs->dots_ticket = 0;  // for the next step
  if (P > 0) {
    fs->zero_v = 0;
    fs->cv = 1.0 - alpha;
    fs->cf = f2 > 0 ? alpha * sqrt(v2) / sqrt(f2) : 0.0;
    if (n_pos > n_min) {
      fs->dt = fmin(dt * f_inc, dt_max);
      fs->alpha = alpha * f_alpha;
    }
    fs->n_pos = n_pos + 1;
  } else {
    fs->zero_v = 1;
    fs->cv = 0;
    fs->cf = 0;
    fs->dt = dt * f_dec;
    fs->alpha = alpha_start;
    fs->n_pos = 0;
  }
}

// block map: nb_fire blocks per member, each over the dot chunks q = blk, blk + nb_fire, ...; the last block of a
// member to finish applies the FIRE controls from every chunk's partials
__global__ void __launch_bounds__(kFireThreads) k_fire_dots(const CfgDev* __restrict__ cfgs,
                                                            const BlockMap* __restrict__ bm) {
  grid_dep_wait();
  const BlockMap m = bm[blockIdx.x];
  const CfgDev& c = cfgs[m.cfg];
  FireState* fs = fstate(c);
  if (fs->status || fs->method != kMethodFire) return;  // uniform over the member's blocks
  __shared__ double sh[3][kFireThreads];
  __shared__ int last;
  for (int64_t q = m.blk; q < c.n_dchunk; q += c.nb_fire) {
    double r[3];
    dots_chunk(c, q, sh, r);
    if (threadIdx.x == 0)
      for (int k = 0; k < 3; k++) c.fdots[k * c.n_dchunk + q] = r[k];
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&fs->dots_ticket, 1) == c.nb_fire - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x >= 32) return;
  __threadfence();
  dots_control(fs, c.fdots, c.n_dchunk, threadIdx.x);
}

// A shard's half of k_fire_dots: every chunk's partials into out[3][n_dchunk] (exactly 0 for chunks of particles
// outside the shard, whose force and velocity stay 0), for the caller to sum over the shards.  One member.
__global__ void __launch_bounds__(kFireThreads) k_fire_dots_part(const CfgDev* __restrict__ cfgs,
                                                                 const BlockMap* __restrict__ bm, double* out) {
  grid_dep_wait();
  const BlockMap m = bm[blockIdx.x];
  const CfgDev& c = cfgs[m.cfg];
  const FireState* fs = fstate(c);
  if (fs->status || fs->method != kMethodFire) return;
  __shared__ double sh[3][kFireThreads];
  for (int64_t q = m.blk; q < c.n_dchunk; q += c.nb_fire) {
    double r[3];
    dots_chunk(c, q, sh, r);
    if (threadIdx.x == 0)
      for (int k = 0; k < 3; k++) out[k * c.n_dchunk + q] = r[k];
  }
}

// The other half: the FIRE controls from the partials summed over every shard (one warp, one member)
__global__ void k_fire_control(const CfgDev* __restrict__ cfgs, const double* __restrict__ tot) {
  grid_dep_wait();
  const CfgDev& c = cfgs[0];
  FireState* fs = fstate(c);
  if (fs->status || fs->method != kMethodFire) return;
  dots_control(fs, tot, c.n_dchunk, threadIdx.x);
}

// block map: d N / 64 blocks per member
__global__ void k_fire_move(const CfgDev* __restrict__ cfgs, const BlockMap* __restrict__ bm) {
  grid_dep_wait();
  const BlockMap m = bm[blockIdx.x];
  const CfgDev& c = cfgs[m.cfg];
  const FireState* fs = fstate(c);
  if (fs->status || fs->method != kMethodFire) return;
  const int64_t i = (int64_t)m.blk * blockDim.x + threadIdx.x;
  if (i >= (int64_t)c.d * c.N) return;
  const double cv = fs->cv, cf = fs->cf, dt = fs->dt;
  const int zero_v = fs->zero_v;
  dd F = dd_make(c.F_hi[i], c.F_lo[i]);
  // the mixing and the Euler velocity step in one: v <- cv v + (cf + dt) F (v <- dt F after a reset), which saves
  // a dd product and a dd sum on the FP64 pipe
  const dd v = zero_v ? dd_mul_d(F, dt) : dd_add(dd_mul_d(dd_make(c.v_hi[i], c.v_lo[i]), cv), dd_mul_d(F, cf + dt));
  c.v_hi[i] = v.hi;
  c.v_lo[i] = v.lo;
  dd s = dd_make(c.s_hi[i], c.s_lo[i]);
  c.bs_hi[i] = s.hi;
  c.bs_lo[i] = s.lo;
  c.bF_hi[i] = F.hi;
  c.bF_lo[i] = F.lo;
  s = dd_frac(dd_add(s, dd_mul(dd_mul_d(v, dt), c.inv_L)));
  c.s_hi[i] = s.hi;
  c.s_lo[i] = s.lo;
}

// one thread per member
__global__ void k_fire_accept(const CfgDev* __restrict__ cfgs, const int* __restrict__ all, int n) {
  grid_dep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const CfgDev& c = cfgs[all[i]];
  FireState* fs = fstate(c);
  if (fs->status || fs->method != kMethodFire) return;
  // every input is loaded up front, so that the loads overlap (one latency, not a chain of them)
  const dd phi = dd_make(c.scal[kScPhiHi], c.scal[kScPhiLo]);
  const dd smx = dd_make(c.scal[kScSmaxHi], c.scal[kScSmaxLo]);
  const long long step = fs->step + 1, stage_step = fs->stage_step + 1, max_steps = fs->max_steps,
                  best_step0 = fs->best_step, stall_window = fs->stall_window;
  const dd phi_acc = dd_make(fs->phi_hi, fs->phi_lo);
  const double smax_hi0 = fs->smax_hi, smax_lo0 = fs->smax_lo, phi_tol = fs->phi_tol, target = fs->target,
               best_smax0 = fs->best_smax, stage_floor = fs->stage_floor;
  const bool failed = tc_failed(c);
  fs->step = step;
  fs->stage_step = stage_step;
  if (failed) {  // incomplete sums: undo the step and stop the run
    fs->status = kFsDevErr;
    fs->rejected_now = 1;
    return;
  }
  if (!isfinite(phi.hi) || !isfinite(smx.hi)) {
    fs->status = kFsNan;
    fs->rejected_now = 1;
    return;
  }
  // uphill beyond the evaluation's own error bound: reject (FIRE's uphill reset, with dt halved)
  const double margin = phi_tol * sqrt(fmax(phi_acc.hi, 0.0));
  double sm;
  if (dd_gt(phi, dd_add_d(phi_acc, margin))) {
    const double dt = fs->dt, f_dec = fs->f_dec, alpha_start = fs->alpha_start;
    const long long rejected = fs->rejected;
    fs->rejected_now = 1;
    fs->rejected = rejected + 1;
    fs->dt = dt * f_dec;
    fs->alpha = alpha_start;
    fs->n_pos = 0;
    sm = smax_hi0 + smax_lo0;
  } else {
    fs->rejected_now = 0;
    fs->phi_hi = phi.hi;
    fs->phi_lo = phi.lo;
    fs->smax_hi = smx.hi;
    fs->smax_lo = smx.lo;
    sm = smx.hi + smx.lo;
  }
  if (sm <= target) {
    fs->status = kFsConverged;
  } else if (step >= max_steps) {
    fs->status = kFsMaxSteps;
  } else {
    long long best_step = best_step0;
    if (sm < 0.5 * best_smax0) {
      fs->best_smax = sm;
      fs->best_step = stage_step;
      best_step = stage_step;
    }
    if (stage_floor > 0 && sm <= stage_floor) fs->status = kFsStageDone;
    else if (stage_step - best_step > stall_window) fs->status = kFsStageDone;
  }
}

// Undo of a rejected step.  Runs whatever the status, so the state the host reads is the accepted one; a
// repeated undo restores the same saved copy again.  Block map: d N / 64 blocks per member.
__global__ void k_fire_restore(const CfgDev* __restrict__ cfgs, const BlockMap* __restrict__ bm) {
  grid_dep_wait();
  const BlockMap m = bm[blockIdx.x];
  const CfgDev& c = cfgs[m.cfg];
  if (!fstate(c)->rejected_now) return;
  const int64_t i = (int64_t)m.blk * blockDim.x + threadIdx.x;
  if (i >= (int64_t)c.d * c.N) return;
  c.s_hi[i] = c.bs_hi[i];
  c.s_lo[i] = c.bs_lo[i];
  c.F_hi[i] = c.bF_hi[i];
  c.F_lo[i] = c.bF_lo[i];
  c.v_hi[i] = 0.0;
  c.v_lo[i] = 0.0;
}

// New stage for members idx[0..n): the accepted energy, S_max and force are those of the stage's precision at the
// current positions (already in scal / F).  first[t]: a new run (parameters and counters; v is zeroed apart).
__global__ void k_fire_stage_init(const CfgDev* __restrict__ cfgs, const int* __restrict__ idx, int n,
                                  const FireState* __restrict__ params, const int* __restrict__ first) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const CfgDev& c = cfgs[idx[t]];
  FireState* fs = fstate(c);
  const FireState& prm = params[t];
  if (first[t]) {
    *fs = prm;
    fs->step = 0;
    fs->rejected = 0;
  }
  // every stage restarts FIRE: v = 0 (k_fire_zero_v), dt = dt0, alpha = alpha_start, no downhill run yet
  fs->dt = prm.dt;
  fs->alpha = prm.alpha_start;
  fs->n_pos = 0;
  fs->zero_v = 0;
  fs->phi_tol = prm.phi_tol;
  fs->status = kFsRunning;
  fs->rejected_now = 0;
  fs->stage_step = 0;
  fs->stage = prm.stage;
  fs->phi_hi = c.scal[kScPhiHi];
  fs->phi_lo = c.scal[kScPhiLo];
  fs->smax_hi = c.scal[kScSmaxHi];
  fs->smax_lo = c.scal[kScSmaxLo];
  fs->best_smax = fs->smax_hi + fs->smax_lo;
  fs->best_step = 0;
  fs->stage_floor = prm.stage_floor;
  fs->stall_window = prm.stall_window;
  fs->dots_ticket = 0;
  // L-BFGS restarts every stage too: no history, steepest descent first; no particle moves more than a tenth of
  // the mean spacing in one step
  fs->method = prm.method;
  fs->lb_count = 0;
  fs->lb_head = kLbMaxPairs - 1;
  fs->lb_need_dir = 1;
  fs->lb_accepted = 0;
  fs->lb_sd = 1;
  fs->lb_backtracks = 0;
  fs->lb_alpha = 0.0;
  fs->lb_gp = 0.0;
  fs->lb_gamma = 1.0;
  fs->lb_dmax = 0.1 / pow((double)c.N, 1.0 / c.d);
  double sm = fs->best_smax;
  if (tc_failed(c)) fs->status = kFsDevErr;
  else if (!isfinite(sm) || !isfinite(fs->phi_hi)) fs->status = kFsNan;
  else if (sm <= fs->target) fs->status = kFsConverged;
  else if (fs->stage_floor > 0 && sm <= fs->stage_floor) fs->status = kFsStageDone;
}

// v = 0 for the members idx[t] (every stage start); grid (coordinate blocks, n)
__global__ void k_fire_zero_v(const CfgDev* __restrict__ cfgs, const int* __restrict__ idx, const int* __restrict__ first) {
  (void)first;
  const CfgDev& c = cfgs[idx[blockIdx.y]];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)c.d * c.N) return;
  c.v_hi[i] = 0.0;
  c.v_lo[i] = 0.0;
}

// ------------------------------------------------------------------------------------------------ host

struct FireBufs {
  DevBuf v_hi, v_lo, bs_hi, bs_lo, bF_hi, bF_lo, part, fs;
  DevBuf lb_S, lb_Y, lb_G, lb_P, lb_part, lb_mat;  // L-BFGS history, gradient, direction, partials, matrices
  int method = kMethodFire;                         // minimiser the cached step graphs were captured for
  DevBuf init_idx, init_prm, init_first;  // arguments of k_fire_stage_init (single context)
  FireState* h_fs = nullptr;               // pinned
  Engine* eng[3] = {nullptr, nullptr, nullptr};             // this context alone, minimising in precision p
  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};   // kFireGraphSteps steps
  cudaGraphExec_t graph1[3] = {nullptr, nullptr, nullptr};  // one step
  int nb = 0;
  bool begun = false;
};

cudaError_t fire_alloc(Ctx* c) {
  if (c->fire) return cudaSuccess;
  FireBufs* f = new FireBufs();
  size_t nd = (size_t)c->d * c->N;
  cudaError_t e = cudaSuccess;
  for (DevBuf* b : {&f->v_hi, &f->v_lo, &f->bs_hi, &f->bs_lo, &f->bF_hi, &f->bF_lo}) {
    b->bytes = std::max<size_t>(nd * 8, 16);
    if (e == cudaSuccess) e = cudaMalloc(&b->p, b->bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->p, 0, b->bytes, c->stream);
  }
  f->nb = (int)std::max<int64_t>(1, std::min<int64_t>(256, ((int64_t)nd + kFireThreads - 1) / kFireThreads));
  f->part.bytes = sizeof(double) * 3 * dot_chunks(c->d, c->N);
  if (e == cudaSuccess) e = cudaMalloc(&f->part.p, f->part.bytes);
  f->lb_S.bytes = f->lb_Y.bytes = std::max<size_t>((size_t)kLbMaxPairs * nd * 8, 16);
  f->lb_G.bytes = f->lb_P.bytes = std::max<size_t>(nd * 8, 16);
  f->lb_part.bytes = sizeof(double) * kLbPartStride * f->nb;
  f->lb_mat.bytes = sizeof(LbMat);
  for (DevBuf* b : {&f->lb_S, &f->lb_Y, &f->lb_G, &f->lb_P, &f->lb_part, &f->lb_mat}) {
    if (e == cudaSuccess) e = cudaMalloc(&b->p, b->bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->p, 0, b->bytes, c->stream);
  }
  f->fs.bytes = sizeof(FireState);
  if (e == cudaSuccess) e = cudaMalloc(&f->fs.p, f->fs.bytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->fs.p, 0, f->fs.bytes, c->stream);
  for (DevBuf* b : {&f->init_idx, &f->init_prm, &f->init_first}) {
    b->bytes = sizeof(FireState);
    if (e == cudaSuccess) e = cudaMalloc(&b->p, b->bytes);
  }
  if (e == cudaSuccess) e = cudaMallocHost(&f->h_fs, sizeof(FireState));
  c->fire = f;
  // the context's own engine now carries the minimiser pointers too (still without a status word)
  eval_graphs_reset(c);
  if (e == cudaSuccess) e = engine_build(c->eng, {c}, {-1}, false, c->stream);
  return e;
}

void fire_fill_cfgdev(const Ctx* c, CfgDev* g) {
  const FireBufs* f = c->fire;
  g->fs = f->fs.p;
  g->v_hi = (double*)f->v_hi.p;
  g->v_lo = (double*)f->v_lo.p;
  g->bs_hi = (double*)f->bs_hi.p;
  g->bs_lo = (double*)f->bs_lo.p;
  g->bF_hi = (double*)f->bF_hi.p;
  g->bF_lo = (double*)f->bF_lo.p;
  g->fdots = (double*)f->part.p;
  g->n_dchunk = (int)dot_chunks(c->d, c->N);
  g->nb_fire = f->nb;
  g->lb_S = (double*)f->lb_S.p;
  g->lb_Y = (double*)f->lb_Y.p;
  g->lb_G = (double*)f->lb_G.p;
  g->lb_P = (double*)f->lb_P.p;
  g->lb_part = (double*)f->lb_part.p;
  g->lb_mat = f->lb_mat.p;
  g->run = &reinterpret_cast<FireState*>(f->fs.p)->status;
}

void fire_free(Ctx* c) {
  FireBufs* f = c->fire;
  if (!f) return;
  for (DevBuf* b : {&f->v_hi, &f->v_lo, &f->bs_hi, &f->bs_lo, &f->bF_hi, &f->bF_lo, &f->part, &f->fs, &f->init_idx,
                    &f->init_prm, &f->init_first, &f->lb_S, &f->lb_Y, &f->lb_G, &f->lb_P, &f->lb_part, &f->lb_mat})
    if (b->p) cudaFree(b->p);
  if (f->h_fs) cudaFreeHost(f->h_fs);
  for (int p = 0; p < 3; p++) {
    if (f->graph[p]) cudaGraphExecDestroy(f->graph[p]);
    if (f->graph1[p]) cudaGraphExecDestroy(f->graph1[p]);
    if (f->eng[p]) {
      engine_free(f->eng[p]);
      delete f->eng[p];
    }
  }
  delete f;
  c->fire = nullptr;
}

FireState fire_params(const ssh_min_params* p) {
  FireState prm;
  memset(&prm, 0, sizeof prm);
  prm.dt = p->dt0;
  prm.alpha = p->alpha_start;
  prm.dt_max = p->dt_max;
  prm.alpha_start = p->alpha_start;
  prm.f_alpha = p->f_alpha;
  prm.f_inc = p->f_inc;
  prm.f_dec = p->f_dec;
  prm.n_min = p->n_min;
  prm.max_steps = p->max_steps;
  prm.target = p->smax_target;
  prm.stage_floor = 0.0;
  prm.stall_window = p->stall_window[0];
  prm.method = p->method == SSH_MIN_LBFGS ? kMethodLbfgs : kMethodFire;
  return prm;
}

// Phi = sum_k |n~_k|^2 with every n~ off by at most eps N: |dPhi| <= 2 eps N sum |n~| + M (eps N)^2, below
// 2 eps N sqrt(M Phi) + M (eps N)^2; with weights v~(k), sum_k v~ |n~|^2, it is below 2 eps N sqrt(M max v~ Phi).  eps: 2^-100 for the tensor-core digits and for double-double, 2^-120 for
// the integer-pipe fixed point; FP64 keeps the strict test (its steps are rejected on any rise).
double fire_phi_tol(const Ctx* c, int prec) {
  double eps = 0.0;
  if (prec == SSH_FX) eps = c->tc.on ? 0x1p-100 : 0x1p-120;
  else if (prec == SSH_DD) eps = 0x1p-100;
  return 2.0 * eps * (double)c->N * sqrt((double)c->M * c->wmax);
}

// One FIRE step of every member of e as stream work.
cudaError_t fire_step_engine(const Engine* e, cudaStream_t st, Prof* prof) {
  if (e->nall == 0) return cudaSuccess;
  const CfgDev* cfgs = e->view[0].cfgs;
  // element-wise kernels in 64-thread blocks, so that one configuration spreads over every SM (their dd
  // arithmetic runs on the FP64 pipe, a few lanes per SM on this part)
  const unsigned gt = (unsigned)((e->nall + 127) / 128);
  prof_begin(prof, st, kKFire);
  if (e->nbm_dots == 0 || e->nbm_nd == 0) return cudaErrorInvalidValue;  // members without minimiser buffers
  const bool fire = e->methods & (1 << kMethodFire), lbfgs = e->methods & (1 << kMethodLbfgs);
  cudaError_t le = cudaSuccess;
  if (fire) {
    le = launch_pdl(k_fire_dots, dim3((unsigned)e->nbm_dots), dim3(kFireThreads), 0, st, cfgs, e->bm_dots);
    if (le == cudaSuccess) le = launch_pdl(k_fire_move, dim3((unsigned)e->nbm_nd), dim3(64), 0, st, cfgs, e->bm_nd);
  }
  if (lbfgs && le == cudaSuccess) le = lbfgs_pre(e, st);
  if (le != cudaSuccess) return le;
  prof_end(prof, st);
  for (int p = 0; p < 3; p++) {
    if (e->view[p].nlist == 0) continue;
    cudaError_t err = engine_eval(e, p, true, st, prof);
    if (err != cudaSuccess) return err;
  }
  prof_begin(prof, st, kKFire);
  if (fire) le = launch_pdl(k_fire_accept, dim3(gt), dim3(128), 0, st, cfgs, e->all, e->nall);
  if (lbfgs && le == cudaSuccess) le = lbfgs_post_accept(e, st);
  if (le == cudaSuccess) le = launch_pdl(k_fire_restore, dim3((unsigned)e->nbm_nd), dim3(64), 0, st, cfgs, e->bm_nd);
  if (lbfgs && le == cudaSuccess) le = lbfgs_post_pairs(e, st);
  if (le != cudaSuccess) return le;
  prof_end(prof, st);
  return cudaGetLastError();
}

static cudaError_t stage_init_launch(const CfgDev* cfgs, int64_t maxND, const int* d_idx, int n, const FireState* d_prm,
                                     const int* d_first, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_fire_zero_v<<<dim3((unsigned)std::max<int64_t>(1, (maxND + 255) / 256), (unsigned)n), 256, 0, st>>>(cfgs, d_idx,
                                                                                                       d_first);
  k_fire_stage_init<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(cfgs, d_idx, n, d_prm, d_first);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = lbfgs_stage_g(cfgs, maxND, d_idx, n, st);  // L-BFGS members: G at the start
  return e;
}

cudaError_t fire_stage_init_engine(const Engine* e, const std::vector<int>& idx, const std::vector<FireState>& params,
                                   const std::vector<int>& first, cudaStream_t st) {
  const int n = (int)idx.size();
  if (n == 0) return cudaSuccess;
  // small, short-lived argument arrays (batch and server set-up, never inside a capture)
  void *di = nullptr, *dp = nullptr, *df = nullptr;
  cudaError_t err = cudaMalloc(&di, sizeof(int) * n);
  if (err == cudaSuccess) err = cudaMalloc(&dp, sizeof(FireState) * n);
  if (err == cudaSuccess) err = cudaMalloc(&df, sizeof(int) * n);
  if (err == cudaSuccess) err = cudaMemcpyAsync(di, idx.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = cudaMemcpyAsync(dp, params.data(), sizeof(FireState) * n, cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = cudaMemcpyAsync(df, first.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess)
    err = stage_init_launch(e->view[0].cfgs, e->maxND_all, (const int*)di, n, (const FireState*)dp, (const int*)df, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);  // the host vectors and the arrays are released below
  cudaFree(di);
  cudaFree(dp);
  cudaFree(df);
  return err;
}

// ---- single context

static cudaError_t fire_engine(Ctx* c, int prec, Engine** out) {
  FireBufs* f = c->fire;
  if (!f->eng[prec]) {
    f->eng[prec] = new Engine();
    cudaError_t e = engine_build(f->eng[prec], {c}, {prec}, true, c->stream);
    if (e != cudaSuccess) return e;
  }
  f->eng[prec]->methods = 1 << f->method;
  *out = f->eng[prec];
  return cudaSuccess;
}

// the minimiser of the next run; the step graphs captured for the other one are dropped
static void fire_set_method(Ctx* c, int method) {
  FireBufs* f = c->fire;
  if (f->method == method) return;
  for (int p = 0; p < 3; p++) {
    if (f->graph[p]) cudaGraphExecDestroy(f->graph[p]);
    if (f->graph1[p]) cudaGraphExecDestroy(f->graph1[p]);
    f->graph[p] = f->graph1[p] = nullptr;
  }
  f->method = method;
}

static cudaError_t fire_graph(Ctx* c, int prec, cudaGraphExec_t* out, int steps = kFireGraphSteps) {
  FireBufs* f = c->fire;
  cudaGraphExec_t* slot = steps == 1 ? &f->graph1[prec] : &f->graph[prec];
  if (*slot) { *out = *slot; return cudaSuccess; }
  Engine* E = nullptr;
  cudaError_t e = fire_engine(c, prec, &E);
  if (e != cudaSuccess) return e;
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  for (int s = 0; s < steps && e == cudaSuccess; s++) e = fire_step_engine(E, c->stream, nullptr);
  cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(slot, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e == cudaSuccess) *out = *slot;
  return e;
}

// Start (first = 1) or continue a run in precision prec: Phi, S_max and F at the current positions, then the
// stage initialisation.
static cudaError_t single_stage_start(Ctx* c, int prec, const FireState& prm, int first) {
  FireBufs* f = c->fire;
  cudaStream_t st = c->stream;
  cudaError_t e = engine_eval(c->eng, prec, true, st, nullptr);  // no status word: always evaluates
  Engine* E = nullptr;
  if (e == cudaSuccess) e = fire_engine(c, prec, &E);
  int idx = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->init_idx.p, &idx, sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->init_prm.p, &prm, sizeof(FireState), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->init_first.p, &first, sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = stage_init_launch(E->view[0].cfgs, E->maxND_all, (const int*)f->init_idx.p, 1, (const FireState*)f->init_prm.p,
                          (const int*)f->init_first.p, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host arguments above live on this stack frame
  return e;
}

cudaError_t fire_engine_for(Ctx* c, int prec, Engine** out) { return fire_engine(c, prec, out); }

bool fire_begun(const Ctx* c) { return c->fire && c->fire->begun; }

cudaError_t fire_dots_partials(const Engine* e, double* out, cudaStream_t st) {
  if (e->nall != 1 || e->nbm_dots == 0) return cudaErrorInvalidValue;
  return launch_pdl(k_fire_dots_part, dim3((unsigned)e->nbm_dots), dim3(kFireThreads), 0, st, e->view[0].cfgs, e->bm_dots,
                    out);
}

cudaError_t fire_control_move(const Engine* e, const double* tot, cudaStream_t st) {
  if (e->nall != 1 || e->nbm_nd == 0) return cudaErrorInvalidValue;
  const CfgDev* cfgs = e->view[0].cfgs;
  cudaError_t le = launch_pdl(k_fire_control, dim3(1), dim3(32), 0, st, cfgs, tot);
  if (le == cudaSuccess) le = launch_pdl(k_fire_move, dim3((unsigned)e->nbm_nd), dim3(64), 0, st, cfgs, e->bm_nd);
  return le;
}

cudaError_t fire_accept_restore(const Engine* e, cudaStream_t st) {
  const CfgDev* cfgs = e->view[0].cfgs;
  const unsigned gt = (unsigned)((e->nall + 127) / 128);
  cudaError_t le = launch_pdl(k_fire_accept, dim3(gt), dim3(128), 0, st, cfgs, e->all, e->nall);
  if (le == cudaSuccess) le = launch_pdl(k_fire_restore, dim3((unsigned)e->nbm_nd), dim3(64), 0, st, cfgs, e->bm_nd);
  return le;
}

// A FIRE run from the Phi, S_max and F already in the context (a shard's exchanged evaluation): the stage start of
// fire_begin without its evaluation.  One fixed-point stage, FIRE only.
ssh_status fire_begin_from_results(Ctx* c, const ssh_min_params* p) {
  cudaError_t e = fire_alloc(c);
  if (e != cudaSuccess) { set_error(std::string("shard FIRE begin: allocation: ") + cudaGetErrorString(e)); return SSH_ENOMEM; }
  FireState prm = fire_params(p);
  fire_set_method(c, prm.method);
  prm.stage = 0;
  prm.phi_tol = fire_phi_tol(c, SSH_FX);
  FireBufs* f = c->fire;
  cudaStream_t st = c->stream;
  Engine* E = nullptr;
  e = fire_engine(c, SSH_FX, &E);
  int idx = 0, first = 1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->init_idx.p, &idx, sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->init_prm.p, &prm, sizeof(FireState), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f->init_first.p, &first, sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = stage_init_launch(E->view[0].cfgs, E->maxND_all, (const int*)f->init_idx.p, 1, (const FireState*)f->init_prm.p,
                          (const int*)f->init_first.p, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host arguments above live on this stack frame
  if (e != cudaSuccess) { set_error(std::string("shard FIRE begin: ") + cudaGetErrorString(e)); return SSH_ECUDA; }
  f->begun = true;
  return SSH_OK;
}

ssh_status fire_begin(Ctx* c, const ssh_min_params* p) {
  cudaError_t e = fire_alloc(c);
  if (e != cudaSuccess) { set_error(std::string("ssh_fire_begin: allocation: ") + cudaGetErrorString(e)); return SSH_ENOMEM; }
  FireState prm = fire_params(p);
  fire_set_method(c, prm.method);
  prm.stage = 0;
  prm.phi_tol = fire_phi_tol(c, p->stage_prec[0]);
  e = single_stage_start(c, p->stage_prec[0], prm, 1);
  if (e != cudaSuccess) { set_error(std::string("ssh_fire_begin: ") + cudaGetErrorString(e)); return SSH_ECUDA; }
  c->fire->begun = true;
  return SSH_OK;
}

ssh_status fire_steps(Ctx* c, int prec, int64_t nsteps) {
  if (!c->fire || !c->fire->begun) { set_error("ssh_fire_steps: call ssh_fire_begin first"); return SSH_EINVAL; }
  cudaError_t e = cudaSuccess;
  // profiling, or the GEMM's counting instance: direct launches, so every kernel of the step carries its own events
  // and a captured graph keeps no counting instance
  if (c->prof.on || tc_counters_on()) {
    Engine* E = nullptr;
    e = fire_engine(c, prec, &E);
    for (int64_t i = 0; e == cudaSuccess && i < nsteps; i++) e = fire_step_engine(E, c->stream, &c->prof);
    if (e != cudaSuccess) { set_error(std::string("ssh_fire_steps: ") + cudaGetErrorString(e)); return SSH_ECUDA; }
    return SSH_OK;
  }
  cudaGraphExec_t g8 = nullptr, g1 = nullptr;
  if (nsteps >= kFireGraphSteps) e = fire_graph(c, prec, &g8);
  if (e == cudaSuccess && nsteps % kFireGraphSteps) e = fire_graph(c, prec, &g1, 1);
  for (int64_t i = 0; e == cudaSuccess && i + kFireGraphSteps <= nsteps; i += kFireGraphSteps) e = cudaGraphLaunch(g8, c->stream);
  for (int64_t i = 0; e == cudaSuccess && i < nsteps % kFireGraphSteps; i++) e = cudaGraphLaunch(g1, c->stream);
  if (e != cudaSuccess) { set_error(std::string("ssh_fire_steps: ") + cudaGetErrorString(e)); return SSH_ECUDA; }
  return SSH_OK;
}

ssh_status fs_status_code(int status) {
  switch (status) {
    case kFsConverged: return SSH_OK;
    case kFsNan: return SSH_ENAN;
    case kFsDevErr: return SSH_ETIMEOUT;
    default: return SSH_ENOTCONV;
  }
}

ssh_status fire_state(Ctx* c, ssh_min_result* r, int* dev_status) {
  if (!c->fire || !c->fire->begun) { set_error("ssh_fire_state: call ssh_fire_begin first"); return SSH_EINVAL; }
  FireBufs* f = c->fire;
  cudaError_t e = cudaMemcpyAsync(f->h_fs, f->fs.p, sizeof(FireState), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) { set_error(std::string("ssh_fire_state: ") + cudaGetErrorString(e)); return SSH_ECUDA; }
  const FireState& h = *f->h_fs;
  if (r) {
    memset(r, 0, sizeof *r);
    r->steps = h.step;
    r->rejected = h.rejected;
    r->smax[0] = h.smax_hi;
    r->smax[1] = h.smax_lo;
    r->phi[0] = h.phi_hi;
    r->phi[1] = h.phi_lo;
    r->dt = h.dt;
    r->status = fs_status_code(h.status);
  }
  if (h.status == kFsDevErr && c->tc.on) {
    cudaMemsetAsync(c->tc.err.p, 0, sizeof(int), c->stream);  // reported here: clear for later evaluations
    set_error("ssh_fire_state: a bounded wait of a tensor-core kernel gave up; the step was undone");
  }
  if (dev_status) *dev_status = h.status;
  return SSH_OK;
}

ssh_status minimize(Ctx* c, const ssh_min_params* p, ssh_min_result* res) {
  auto t0 = std::chrono::steady_clock::now();
  cudaError_t e = fire_alloc(c);
  if (e != cudaSuccess) {
    set_error(std::string("ssh_minimize: allocation: ") + cudaGetErrorString(e));
    return SSH_ENOMEM;
  }
  FireBufs* f = c->fire;
  cudaStream_t st = c->stream;
  FireState prm = fire_params(p);
  fire_set_method(c, prm.method);
  ssh_min_result r;
  memset(&r, 0, sizeof r);
  r.status = SSH_ENOTCONV;
  int final_status = kFsStageDone;
  const int64_t chunk_graphs = std::max<int64_t>(1, p->chunk / kFireGraphSteps);
  // the device stops at max_steps; the host gives up a little after that in case the status never changes
  const int64_t max_chunks = p->max_steps / (chunk_graphs * kFireGraphSteps) + 4;
  for (int s = 0; s < p->n_stages; s++) {
    const int prec = p->stage_prec[s];
    auto ts = std::chrono::steady_clock::now();
    prm.stage = s;
    prm.stage_floor = s + 1 < p->n_stages ? p->stage_floor[s] : 0.0;
    prm.stall_window = p->stall_window[s];
    prm.phi_tol = fire_phi_tol(c, prec);
    e = single_stage_start(c, prec, prm, s == 0);
    cudaGraphExec_t g = nullptr;
    if (e == cudaSuccess) e = fire_graph(c, prec, &g);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->h_fs, f->fs.p, sizeof(FireState), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error(std::string("ssh_minimize: ") + cudaGetErrorString(e));
      return SSH_ECUDA;
    }
    const long long steps_before = f->h_fs->step;
    int status = f->h_fs->status;
    int64_t chunks = 0;
    while (status == kFsRunning) {
      for (int64_t q = 0; q < chunk_graphs && e == cudaSuccess; q++) e = cudaGraphLaunch(g, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(f->h_fs, f->fs.p, sizeof(FireState), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        set_error(std::string("ssh_minimize: ") + cudaGetErrorString(e));
        return SSH_ECUDA;
      }
      status = f->h_fs->status;
      double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (status == kFsRunning && ((p->max_seconds > 0 && el > p->max_seconds) || ++chunks > max_chunks)) {
        status = -1;  // wall limit, or a status word that stopped moving
        break;
      }
    }
    r.stage_steps[s] = f->h_fs->step - steps_before;
    r.stage_wall_s[s] = std::chrono::duration<double>(std::chrono::steady_clock::now() - ts).count();
    r.stages_used = s + 1;
    r.final_prec = prec;
    final_status = status;
    if (status != kFsStageDone) break;
  }
  const FireState& h = *f->h_fs;
  r.steps = h.step;
  r.rejected = h.rejected;
  r.smax[0] = h.smax_hi;
  r.smax[1] = h.smax_lo;
  r.phi[0] = h.phi_hi;
  r.phi[1] = h.phi_lo;
  r.dt = h.dt;
  r.wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  c->have_result = false;  // device result buffers hold the last trial, not necessarily the accepted state
  ssh_status out;
  switch (final_status) {
    case kFsConverged: out = SSH_OK; break;
    case kFsNan: out = SSH_ENAN; set_error("ssh_minimize: non-finite energy"); break;
    case kFsDevErr:
      out = SSH_ETIMEOUT;
      if (c->tc.on) cudaMemsetAsync(c->tc.err.p, 0, sizeof(int), st);  // reported here: clear it
      set_error("ssh_minimize: a bounded wait of a tensor-core kernel gave up; the last step was undone");
      break;
    case -1: out = SSH_ETIMEOUT; set_error("ssh_minimize: wall-time limit reached"); break;
    default: out = SSH_ENOTCONV; set_error("ssh_minimize: step cap or stall above the S_max target"); break;
  }
  r.status = out;
  if (res) *res = r;
  return out;
}

}  // namespace ssh
