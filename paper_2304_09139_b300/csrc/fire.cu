// fire.cu -- the paper's minimiser (Simulations: FIRE, Bitzek et al. 2006) kept on the device.
//
// One step, for the force F and energy Phi at the accepted positions and the velocity v of the last step:
//   k_fire_dots     P = F.v, |F|^2, |v|^2 (per-block partials, fixed order)
//   k_fire_ctrl     FIRE rules: P > 0 -> v <- (1-a) v + a |v| F/|F|; after more than n_min such steps
//                   dt <- min(dt f_inc, dt_max), a <- a f_alpha;  P <= 0 -> v <- 0, dt <- dt f_dec, a <- a_start
//   k_fire_move     semi-implicit Euler with unit mass: v <- v + dt F, r <- r + dt v (dd, wrapped into the box);
//                   the accepted positions and force are kept for a possible undo
//   (Phi + force at the new positions: the seven evaluation kernels)
//   k_fire_accept   energy guard: Phi_new > Phi -> reject (dt <- dt f_dec, v <- 0, a <- a_start) and undo;
//                   convergence S_max <= target; step cap; the precision stage ends when S_max falls below the
//                   stage floor or has not halved in stall_window steps
//   k_fire_restore  the undo of a rejected step
// Every kernel first reads the device status word and returns when the run has ended, so a captured chunk
// of steps costs nothing after convergence.  The host replays a CUDA graph of kFireGraphSteps steps per
// precision and reads the status word between chunks; the status word is the only per-chunk copy.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>

#include "ssh_internal.h"

namespace ssh {

enum { kFsRunning = 0, kFsConverged = 1, kFsNan = 2, kFsStageDone = 3, kFsMaxSteps = 4 };
constexpr int kFireThreads = 256;
constexpr int kFireGraphSteps = 8;

struct FireState {
  int status;
  int rejected_now;
  int zero_v;
  int pad0;
  double dt, alpha, cv, cf;
  long long n_pos, step, stage_step, rejected;
  double phi_hi, phi_lo, smax_hi, smax_lo;
  double best_smax;
  long long best_step;
  // parameters
  double dt_max, alpha_start, f_alpha, f_inc, f_dec;
  long long n_min, stall_window, max_steps;
  double target, stage_floor;
};

__global__ void __launch_bounds__(kFireThreads) k_fire_dots(const FireState* __restrict__ fs, int64_t nd,
                                                            const double* __restrict__ F, const double* __restrict__ v,
                                                            double* __restrict__ part) {
  if (fs->status) return;
  __shared__ double sh[3][kFireThreads];
  double p = 0, f2 = 0, v2 = 0;
  for (int64_t i = (int64_t)blockIdx.x * kFireThreads + threadIdx.x; i < nd; i += (int64_t)gridDim.x * kFireThreads) {
    double f = F[i], w = v[i];
    p = fma(f, w, p);
    f2 = fma(f, f, f2);
    v2 = fma(w, w, v2);
  }
  sh[0][threadIdx.x] = p;
  sh[1][threadIdx.x] = f2;
  sh[2][threadIdx.x] = v2;
  __syncthreads();
  for (int s = kFireThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int q = 0; q < 3; q++) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; q++) part[q * gridDim.x + blockIdx.x] = sh[q][0];
}

__global__ void k_fire_ctrl(FireState* fs, const double* __restrict__ part, int nb) {
  if (fs->status) return;
  double P = 0, f2 = 0, v2 = 0;
  for (int b = 0; b < nb; b++) {  // fixed order
    P += part[b];
    f2 += part[nb + b];
    v2 += part[2 * nb + b];
  }
  if (P > 0) {
    fs->zero_v = 0;
    fs->cv = 1.0 - fs->alpha;
    fs->cf = f2 > 0 ? fs->alpha * sqrt(v2) / sqrt(f2) : 0.0;
    if (fs->n_pos > fs->n_min) {
      fs->dt = fmin(fs->dt * fs->f_inc, fs->dt_max);
      fs->alpha *= fs->f_alpha;
    }
    fs->n_pos++;
  } else {
    fs->zero_v = 1;
    fs->cv = 0;
    fs->cf = 0;
    fs->dt *= fs->f_dec;
    fs->alpha = fs->alpha_start;
    fs->n_pos = 0;
  }
}

__global__ void k_fire_move(const FireState* __restrict__ fs, int64_t nd, double* s_hi, double* s_lo, double* v_hi,
                            double* v_lo, const double* __restrict__ F_hi, const double* __restrict__ F_lo,
                            double* bs_hi, double* bs_lo, double* bF_hi, double* bF_lo, dd inv_L) {
  if (fs->status) return;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  dd F = dd_make(F_hi[i], F_lo[i]);
  dd v = fs->zero_v ? dd_make(0.0) : dd_add(dd_mul_d(dd_make(v_hi[i], v_lo[i]), fs->cv), dd_mul_d(F, fs->cf));
  v = dd_add(v, dd_mul_d(F, fs->dt));
  v_hi[i] = v.hi;
  v_lo[i] = v.lo;
  dd s = dd_make(s_hi[i], s_lo[i]);
  bs_hi[i] = s.hi;
  bs_lo[i] = s.lo;
  bF_hi[i] = F.hi;
  bF_lo[i] = F.lo;
  s = dd_frac(dd_add(s, dd_mul(dd_mul_d(v, fs->dt), inv_L)));
  s_hi[i] = s.hi;
  s_lo[i] = s.lo;
}

__global__ void k_fire_accept(FireState* fs, const double* __restrict__ scal) {
  if (fs->status) return;
  dd phi = dd_make(scal[kScPhiHi], scal[kScPhiLo]);
  dd smx = dd_make(scal[kScSmaxHi], scal[kScSmaxLo]);
  fs->step++;
  fs->stage_step++;
  if (!isfinite(phi.hi) || !isfinite(smx.hi)) {
    fs->status = kFsNan;
    fs->rejected_now = 1;
    return;
  }
  if (dd_gt(phi, dd_make(fs->phi_hi, fs->phi_lo))) {
    fs->rejected_now = 1;
    fs->rejected++;
    fs->dt *= fs->f_dec;
    fs->alpha = fs->alpha_start;
    fs->n_pos = 0;
  } else {
    fs->rejected_now = 0;
    fs->phi_hi = phi.hi;
    fs->phi_lo = phi.lo;
    fs->smax_hi = smx.hi;
    fs->smax_lo = smx.lo;
  }
  double sm = fs->smax_hi + fs->smax_lo;
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

// Undo of a rejected step.  Runs whatever the status, so the state the host reads is the accepted one; a
// repeated undo restores the same saved copy again.
__global__ void k_fire_restore(const FireState* __restrict__ fs, int64_t nd, double* s_hi, double* s_lo, double* v_hi,
                               double* v_lo, double* F_hi, double* F_lo, const double* __restrict__ bs_hi,
                               const double* __restrict__ bs_lo, const double* __restrict__ bF_hi,
                               const double* __restrict__ bF_lo) {
  if (!fs->rejected_now) return;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  s_hi[i] = bs_hi[i];
  s_lo[i] = bs_lo[i];
  F_hi[i] = bF_hi[i];
  F_lo[i] = bF_lo[i];
  v_hi[i] = 0.0;
  v_lo[i] = 0.0;
}

// New stage: the accepted energy, S_max and force are those of this precision at the current positions.
__global__ void k_fire_stage_init(FireState* fs, const double* __restrict__ scal, int first, FireState params) {
  if (first) {
    *fs = params;
    fs->step = 0;
    fs->rejected = 0;
    fs->n_pos = 0;
  }
  fs->status = kFsRunning;
  fs->rejected_now = 0;
  fs->stage_step = 0;
  fs->phi_hi = scal[kScPhiHi];
  fs->phi_lo = scal[kScPhiLo];
  fs->smax_hi = scal[kScSmaxHi];
  fs->smax_lo = scal[kScSmaxLo];
  fs->best_smax = fs->smax_hi + fs->smax_lo;
  fs->best_step = 0;
  fs->stage_floor = params.stage_floor;
  fs->stall_window = params.stall_window;
  double sm = fs->best_smax;
  if (!isfinite(sm) || !isfinite(fs->phi_hi)) fs->status = kFsNan;
  else if (sm <= fs->target) fs->status = kFsConverged;
  else if (fs->stage_floor > 0 && sm <= fs->stage_floor) fs->status = kFsStageDone;
}

// ------------------------------------------------------------------------------------------------ host

struct FireBufs {
  DevBuf v_hi, v_lo, bs_hi, bs_lo, bF_hi, bF_lo, part, fs;
  FireState* h_fs = nullptr;  // pinned
  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};   // kFireGraphSteps steps
  cudaGraphExec_t graph1[3] = {nullptr, nullptr, nullptr};  // one step
  int nb = 0;
  bool begun = false;
};

static cudaError_t fire_alloc(Ctx* c) {
  if (c->fire) return cudaSuccess;
  FireBufs* f = new FireBufs();
  size_t nd = (size_t)c->d * c->N;
  cudaError_t e = cudaSuccess;
  for (DevBuf* b : {&f->v_hi, &f->v_lo, &f->bs_hi, &f->bs_lo, &f->bF_hi, &f->bF_lo}) {
    b->bytes = nd * 8;
    if (e == cudaSuccess) e = cudaMalloc(&b->p, b->bytes);
  }
  f->nb = (int)std::min<int64_t>(256, ((int64_t)nd + kFireThreads - 1) / kFireThreads);
  f->part.bytes = sizeof(double) * 3 * f->nb;
  if (e == cudaSuccess) e = cudaMalloc(&f->part.p, f->part.bytes);
  f->fs.bytes = sizeof(FireState);
  if (e == cudaSuccess) e = cudaMalloc(&f->fs.p, f->fs.bytes);
  if (e == cudaSuccess) e = cudaMallocHost(&f->h_fs, sizeof(FireState));
  c->fire = f;
  return e;
}

void fire_free(Ctx* c) {
  FireBufs* f = c->fire;
  if (!f) return;
  for (DevBuf* b : {&f->v_hi, &f->v_lo, &f->bs_hi, &f->bs_lo, &f->bF_hi, &f->bF_lo, &f->part, &f->fs})
    if (b->p) cudaFree(b->p);
  if (f->h_fs) cudaFreeHost(f->h_fs);
  for (int p = 0; p < 3; p++) {
    if (f->graph[p]) cudaGraphExecDestroy(f->graph[p]);
    if (f->graph1[p]) cudaGraphExecDestroy(f->graph1[p]);
  }
  delete f;
  c->fire = nullptr;
}

// One FIRE step as stream work (captured into a graph by the caller).
static cudaError_t fire_step(Ctx* c, int prec) {
  FireBufs* f = c->fire;
  cudaStream_t st = c->stream;
  const int64_t nd = (int64_t)c->d * c->N;
  FireState* fs = (FireState*)f->fs.p;
  prof_begin(c, kKFire);
  k_fire_dots<<<f->nb, kFireThreads, 0, st>>>(fs, nd, (const double*)c->F_hi.p, (const double*)f->v_hi.p,
                                              (double*)f->part.p);
  k_fire_ctrl<<<1, 1, 0, st>>>(fs, (const double*)f->part.p, f->nb);
  const unsigned g = (unsigned)((nd + 255) / 256);
  k_fire_move<<<g, 256, 0, st>>>(fs, nd, (double*)c->s_hi.p, (double*)c->s_lo.p, (double*)f->v_hi.p,
                                 (double*)f->v_lo.p, (const double*)c->F_hi.p, (const double*)c->F_lo.p,
                                 (double*)f->bs_hi.p, (double*)f->bs_lo.p, (double*)f->bF_hi.p, (double*)f->bF_lo.p,
                                 c->inv_L);
  prof_end(c);
  c->run_flag = &fs->status;
  cudaError_t e = eval_phi_grad(c, prec, true);
  c->run_flag = nullptr;
  if (e != cudaSuccess) return e;
  prof_begin(c, kKFire);
  k_fire_accept<<<1, 1, 0, st>>>(fs, (const double*)c->scal.p);
  k_fire_restore<<<g, 256, 0, st>>>(fs, nd, (double*)c->s_hi.p, (double*)c->s_lo.p, (double*)f->v_hi.p,
                                    (double*)f->v_lo.p, (double*)c->F_hi.p, (double*)c->F_lo.p,
                                    (const double*)f->bs_hi.p, (const double*)f->bs_lo.p,
                                    (const double*)f->bF_hi.p, (const double*)f->bF_lo.p);
  prof_end(c);
  return cudaGetLastError();
}

static cudaError_t fire_graph(Ctx* c, int prec, cudaGraphExec_t* out, int steps = kFireGraphSteps) {
  FireBufs* f = c->fire;
  cudaGraphExec_t* slot = steps == 1 ? &f->graph1[prec] : &f->graph[prec];
  if (*slot) { *out = *slot; return cudaSuccess; }
  bool prof = c->prof.on;
  c->prof.on = false;  // no profiler events inside a capture
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  for (int s = 0; s < steps && e == cudaSuccess; s++) e = fire_step(c, prec);
  cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
  c->prof.on = prof;
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(slot, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e == cudaSuccess) *out = *slot;
  return e;
}

static FireState params_to_state(const ssh_min_params* p) {
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
  return prm;
}

// Stepper: state from the current positions in the first stage's precision (v = 0).
ssh_status fire_begin(Ctx* c, const ssh_min_params* p) {
  cudaError_t e = fire_alloc(c);
  if (e != cudaSuccess) { set_error(std::string("ssh_fire_begin: allocation: ") + cudaGetErrorString(e)); return SSH_ENOMEM; }
  FireBufs* f = c->fire;
  cudaStream_t st = c->stream;
  const int64_t nd = (int64_t)c->d * c->N;
  cudaMemsetAsync(f->v_hi.p, 0, nd * 8, st);
  cudaMemsetAsync(f->v_lo.p, 0, nd * 8, st);
  e = eval_phi_grad(c, p->stage_prec[0], true);
  if (e == cudaSuccess) {
    k_fire_stage_init<<<1, 1, 0, st>>>((FireState*)f->fs.p, (const double*)c->scal.p, 1, params_to_state(p));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) { set_error(std::string("ssh_fire_begin: ") + cudaGetErrorString(e)); return SSH_ECUDA; }
  f->begun = true;
  return SSH_OK;
}

// Enqueue exactly nsteps FIRE steps in precision prec (no host synchronisation).
ssh_status fire_steps(Ctx* c, int prec, int64_t nsteps) {
  if (!c->fire || !c->fire->begun) { set_error("ssh_fire_steps: call ssh_fire_begin first"); return SSH_EINVAL; }
  cudaGraphExec_t g8 = nullptr, g1 = nullptr;
  cudaError_t e = cudaSuccess;
  if (c->prof.on) {  // profiling: direct launches, so every kernel of the step carries its own events
    for (int64_t i = 0; e == cudaSuccess && i < nsteps; i++) e = fire_step(c, prec);
    if (e != cudaSuccess) { set_error(std::string("ssh_fire_steps: ") + cudaGetErrorString(e)); return SSH_ECUDA; }
    return SSH_OK;
  }
  if (nsteps >= kFireGraphSteps) e = fire_graph(c, prec, &g8);
  if (e == cudaSuccess && nsteps % kFireGraphSteps) e = fire_graph(c, prec, &g1, 1);
  for (int64_t i = 0; e == cudaSuccess && i + kFireGraphSteps <= nsteps; i += kFireGraphSteps) e = cudaGraphLaunch(g8, c->stream);
  for (int64_t i = 0; e == cudaSuccess && i < nsteps % kFireGraphSteps; i++) e = cudaGraphLaunch(g1, c->stream);
  if (e != cudaSuccess) { set_error(std::string("ssh_fire_steps: ") + cudaGetErrorString(e)); return SSH_ECUDA; }
  return SSH_OK;
}

// Read the stepper state (synchronises the stream).  Returns the device status word in *dev_status.
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
    r->status = h.status == kFsConverged ? SSH_OK : h.status == kFsNan ? SSH_ENAN : SSH_ENOTCONV;
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
  const int64_t nd = (int64_t)c->d * c->N;
  cudaMemsetAsync(f->v_hi.p, 0, nd * 8, st);
  cudaMemsetAsync(f->v_lo.p, 0, nd * 8, st);
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
  ssh_min_result r;
  memset(&r, 0, sizeof r);
  r.status = SSH_ENOTCONV;
  int final_status = kFsStageDone;
  FireState* fs = (FireState*)f->fs.p;
  const int64_t chunk_graphs = std::max<int64_t>(1, p->chunk / kFireGraphSteps);
  // the device stops at max_steps; the host gives up a little after that in case the status never changes
  const int64_t max_chunks = p->max_steps / (chunk_graphs * kFireGraphSteps) + 4;
  for (int s = 0; s < p->n_stages; s++) {
    const int prec = p->stage_prec[s];
    auto ts = std::chrono::steady_clock::now();
    prm.stage_floor = s + 1 < p->n_stages ? p->stage_floor[s] : 0.0;
    prm.stall_window = p->stall_window[s];
    // Phi and F of this precision at the current positions
    e = eval_phi_grad(c, prec, true);
    if (e == cudaSuccess) {
      k_fire_stage_init<<<1, 1, 0, st>>>(fs, (const double*)c->scal.p, s == 0, prm);
      e = cudaGetLastError();
    }
    cudaGraphExec_t g = nullptr;
    if (e == cudaSuccess) e = fire_graph(c, prec, &g);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->h_fs, fs, sizeof(FireState), cudaMemcpyDeviceToHost, st);
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
      if (e == cudaSuccess) e = cudaMemcpyAsync(f->h_fs, fs, sizeof(FireState), cudaMemcpyDeviceToHost, st);
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
    case -1: out = SSH_ETIMEOUT; set_error("ssh_minimize: wall-time limit reached"); break;
    default: out = SSH_ENOTCONV; set_error("ssh_minimize: step cap or stall above the S_max target"); break;
  }
  r.status = out;
  if (res) *res = r;
  return out;
}

}  // namespace ssh
