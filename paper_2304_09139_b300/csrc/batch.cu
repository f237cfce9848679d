// batch.cu -- many configurations on one GPU: a batch that evaluates and minimises all its members through the
// same persistent launches, and a server that admits ensemble requests into such a batch while it runs.
//
// Runner: the active members, each with its minimiser parameters and current precision stage.  A chunk is a
// CUDA graph of kGraphSteps batched FIRE steps (re-captured when membership or a member's precision changes),
// replayed until the chunk length is reached; then the host gathers every member's status word in one copy,
// moves members whose stage ended to their next precision (re-evaluating Phi, S_max and F there), and retires
// members that converged, failed or hit their step cap.  A member's arithmetic depends on that member alone, and
// a member whose run has ended is skipped by every kernel, so a configuration follows the same trajectory alone
// and in any mix: results are bit-identical.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cstring>
#include "ssh_internal.h"

namespace ssh {

constexpr int kGraphSteps = 4;

__global__ void k_gather_fs(const CfgDev* __restrict__ cfgs, int n, FireState* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = *reinterpret_cast<const FireState*>(cfgs[i].fs);
}

struct Member {
  ssh_ctx* h = nullptr;
  ssh_min_params p;
  int stage = 0;
  bool done = false;
  uint64_t ticket = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  double stage_t0 = 0;
  ssh_min_result res;
  long long stage_step0 = 0;
  int want_positions = 0;
  int64_t work = 0;  // M N pairs of one evaluation
};

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static ssh_status fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return SSH_ECUDA;
}

struct Runner {
  int device = 0;
  EngineTune tune;  // the batch's work decomposition (ssh_batch_autotune)
  cudaStream_t st = nullptr;
  std::vector<Member> act;
  Engine eng;
  bool dirty = true;
  cudaGraphExec_t graph = nullptr;
  DevBuf gather;
  FireState* h_fs = nullptr;
  int h_cap = 0;
  Prof* prof = nullptr;

  ~Runner() {
    if (graph) cudaGraphExecDestroy(graph);
    engine_free(&eng);
    if (gather.p) cudaFree(gather.p);
    if (h_fs) cudaFreeHost(h_fs);
  }

  // Phi, S_max, F of members idx in their current stage precision, then their stage initialisation.
  cudaError_t start_stage(const std::vector<int>& idx, bool first) {
    if (idx.empty()) return cudaSuccess;
    std::vector<Ctx*> ms;
    std::vector<int> precs;
    std::vector<FireState> prm;
    std::vector<int> firsts, local;
    for (size_t t = 0; t < idx.size(); t++) {
      Member& m = act[idx[t]];
      ms.push_back(&m.h->c);
      precs.push_back(m.p.stage_prec[m.stage]);
      FireState f = fire_params(&m.p);
      f.stage = m.stage;
      f.stage_floor = m.stage + 1 < m.p.n_stages ? m.p.stage_floor[m.stage] : 0.0;
      f.stall_window = m.p.stall_window[m.stage];
      f.phi_tol = fire_phi_tol(&m.h->c, m.p.stage_prec[m.stage]);
      prm.push_back(f);
      firsts.push_back(first ? 1 : 0);
      local.push_back((int)t);
      m.stage_t0 = now_s();
    }
    Engine tmp;
    tmp.tune = tune;
    cudaError_t e = engine_build(&tmp, ms, precs, false, st);
    for (int p = 0; p < 3 && e == cudaSuccess; p++)
      if (tmp.view[p].nlist) e = engine_eval(&tmp, p, true, st, prof);
    if (e == cudaSuccess) e = fire_stage_init_engine(&tmp, local, prm, firsts, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    engine_free(&tmp);
    dirty = true;
    return e;
  }

  cudaError_t add(std::vector<Member>& fresh) {
    std::vector<int> idx;
    for (Member& m : fresh) {
      cudaError_t e = fire_alloc(&m.h->c);
      if (e != cudaSuccess) return e;
      m.stage = 0;
      m.t_admit = now_s();
      memset(&m.res, 0, sizeof m.res);
      act.push_back(m);
      idx.push_back((int)act.size() - 1);
    }
    return start_stage(idx, true);
  }

  cudaError_t rebuild() {
    std::vector<Ctx*> ms;
    std::vector<int> precs;
    for (Member& m : act) {
      ms.push_back(&m.h->c);
      precs.push_back(m.p.stage_prec[m.stage]);
    }
    eng.tune = tune;
    cudaError_t e = engine_build(&eng, ms, precs, true, st);
    eng.methods = 0;
    for (Member& m : act) eng.methods |= 1 << (m.p.method == SSH_MIN_LBFGS ? kMethodLbfgs : kMethodFire);
    if (act.empty()) eng.methods = 1 << kMethodFire;
    if (graph) {
      cudaGraphExecDestroy(graph);
      graph = nullptr;
    }
    if (e == cudaSuccess && !act.empty() && !(prof && prof->on) && !tc_counters_on()) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
      for (int s = 0; s < kGraphSteps && e == cudaSuccess; s++) e = fire_step_engine(&eng, st, nullptr);
      cudaError_t e2 = cudaStreamEndCapture(st, &g);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&graph, g, 0);
      if (g) cudaGraphDestroy(g);
    }
    if ((int)act.size() > h_cap) {
      if (gather.p) cudaFree(gather.p);
      if (h_fs) cudaFreeHost(h_fs);
      h_cap = std::max<int>(64, 2 * (int)act.size());
      gather.bytes = sizeof(FireState) * h_cap;
      if (e == cudaSuccess) e = cudaMalloc(&gather.p, gather.bytes);
      if (e == cudaSuccess) e = cudaMallocHost(&h_fs, sizeof(FireState) * h_cap);
    }
    dirty = false;
    return e;
  }

  // Enqueue `steps` batched steps without any host check (the stepper used for timing).
  cudaError_t launch_steps(int64_t steps) {
    cudaError_t e = cudaSuccess;
    if (act.empty()) return e;
    if (dirty) e = rebuild();
    if (graph) {
      for (int64_t s = 0; s + kGraphSteps <= steps && e == cudaSuccess; s += kGraphSteps) e = cudaGraphLaunch(graph, st);
      for (int64_t s = steps - steps % kGraphSteps; s < steps && e == cudaSuccess; s++) e = fire_step_engine(&eng, st, prof);
    } else {
      for (int64_t s = 0; s < steps && e == cudaSuccess; s++) e = fire_step_engine(&eng, st, prof);
    }
    return e;
  }

  // Run `steps` batched steps, then update stages.  Members that ended are moved to `finished`.
  cudaError_t chunk(int64_t steps, std::vector<Member>& finished) {
    cudaError_t e = cudaSuccess;
    if (act.empty()) return e;
    if (dirty) e = rebuild();
    if (e != cudaSuccess) return e;
    if (graph) {
      for (int64_t s = 0; s < steps && e == cudaSuccess; s += kGraphSteps) e = cudaGraphLaunch(graph, st);
    } else {
      for (int64_t s = 0; s < steps && e == cudaSuccess; s++) e = fire_step_engine(&eng, st, prof);
    }
    const int n = (int)act.size();
    if (e == cudaSuccess) {
      k_gather_fs<<<(n + 127) / 128, 128, 0, st>>>(eng.view[0].cfgs, n, (FireState*)gather.p);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_fs, gather.p, sizeof(FireState) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    std::vector<int> next_stage;
    for (int i = 0; i < n; i++) {
      Member& m = act[i];
      const FireState& f = h_fs[i];
      if (f.status == kFsRunning) continue;
      m.res.stage_steps[m.stage] = f.step - m.stage_step0;
      m.res.stage_wall_s[m.stage] = now_s() - m.stage_t0;
      if (f.status == kFsStageDone && m.stage + 1 < m.p.n_stages) {
        m.stage++;
        m.stage_step0 = f.step;
        next_stage.push_back(i);
        continue;
      }
      m.done = true;
      m.t_done = now_s();
      m.res.steps = f.step;
      m.res.rejected = f.rejected;
      m.res.smax[0] = f.smax_hi;
      m.res.smax[1] = f.smax_lo;
      m.res.phi[0] = f.phi_hi;
      m.res.phi[1] = f.phi_lo;
      m.res.dt = f.dt;
      m.res.final_prec = m.p.stage_prec[m.stage];
      m.res.stages_used = m.stage + 1;
      m.res.wall_s = m.t_done - m.t_admit;
      m.res.status = fs_status_code(f.status);
      if (f.status == kFsDevErr && m.h->c.tc.on) cudaMemsetAsync(m.h->c.tc.err.p, 0, sizeof(int), st);
    }
    if (!next_stage.empty()) e = start_stage(next_stage, false);
    std::vector<Member> keep;
    for (Member& m : act) {
      if (m.done) finished.push_back(m);
      else keep.push_back(m);
    }
    if (keep.size() != act.size()) {
      act.swap(keep);
      dirty = true;
    }
    return e;
  }
};

}  // namespace ssh

using ssh::Member;
using ssh::Runner;
using ssh::set_error;

// ------------------------------------------------------------------------------------------------ batch

struct ssh_batch {
  int device = 0;
  int fx_impl = 0;  // members' ssh_opts.fx_impl
  cudaStream_t stream = nullptr;
  std::vector<ssh_ctx*> members;
  std::vector<ssh_min_result> results;
  ssh::Prof prof;
  Runner* stepper = nullptr;  // ssh_batch_begin / ssh_batch_steps
  ssh::EngineTune tune;       // ssh_batch_autotune's choice (defaults until then)
};

extern "C" {

ssh_status ssh_batch_create(const ssh_opts* opts, ssh_batch** out) {
  if (!out) { set_error("ssh_batch_create: out is NULL"); return SSH_EINVAL; }
  if (opts && (opts->shard_first != 0 || opts->shard_count != 0)) {
    set_error("ssh_batch_create: batch members hold every particle (no shard fields)");
    return SSH_EINVAL;
  }
  ssh_batch* b = new (std::nothrow) ssh_batch();
  if (!b) { set_error("ssh_batch_create: out of host memory"); return SSH_ENOMEM; }
  b->device = opts ? opts->device : 0;
  b->fx_impl = opts ? opts->fx_impl : 0;
  cudaError_t e = cudaSetDevice(b->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { delete b; return ssh::fail(e, "ssh_batch_create"); }
  *out = b;
  return SSH_OK;
}

void ssh_batch_destroy(ssh_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  delete b->stepper;
  for (ssh_ctx* h : b->members) ssh_destroy(h);
  for (ssh::ProfRec& r : b->prof.pending) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
  for (cudaEvent_t ev : b->prof.pool) cudaEventDestroy(ev);
  cudaStreamDestroy(b->stream);
  delete b;
}

ssh_status ssh_batch_add(ssh_batch* b, int d, int64_t N, double L, double chi, double K, const double* s_hi,
                         const double* s_lo, int* slot) {
  if (!b || !s_hi) { set_error("ssh_batch_add: NULL argument"); return SSH_EINVAL; }
  ssh_opts o;
  memset(&o, 0, sizeof o);
  o.device = b->device;
  o.fx_impl = b->fx_impl;
  ssh_ctx* h = nullptr;
  ssh_status s = ssh_create(d, N, L, chi, K, &o, &h);
  if (s != SSH_OK) return s;
  s = ssh_set_stream(h, b->stream);
  if (s == SSH_OK) s = ssh_set_positions_frac(h, s_hi, s_lo);
  if (s != SSH_OK) { ssh_destroy(h); return s; }
  b->members.push_back(h);
  ssh_min_result z;
  memset(&z, 0, sizeof z);
  b->results.push_back(z);
  if (slot) *slot = (int)b->members.size() - 1;
  return SSH_OK;
}

ssh_status ssh_batch_size(const ssh_batch* b, int* n, int64_t* pairs) {
  if (!b) { set_error("ssh_batch_size: NULL batch"); return SSH_EINVAL; }
  if (n) *n = (int)b->members.size();
  if (pairs) {
    int64_t t = 0;
    for (ssh_ctx* h : b->members) t += h->c.M * h->c.N;
    *pairs = t;
  }
  return SSH_OK;
}

ssh_status ssh_batch_member(ssh_batch* b, int slot, ssh_ctx** ctx) {
  if (!b || !ctx || slot < 0 || slot >= (int)b->members.size()) { set_error("ssh_batch_member: bad slot"); return SSH_EINVAL; }
  *ctx = b->members[slot];
  return SSH_OK;
}

ssh_status ssh_batch_eval(ssh_batch* b, int prec, int want_force) {
  if (!b || prec < SSH_FP64 || prec > SSH_FX) { set_error("ssh_batch_eval: bad arguments"); return SSH_EINVAL; }
  cudaSetDevice(b->device);
  std::vector<ssh::Ctx*> ms;
  std::vector<int> precs;
  for (ssh_ctx* h : b->members) {
    if (!h->c.have_positions) { set_error("ssh_batch_eval: a member has no positions"); return SSH_EINVAL; }
    ms.push_back(&h->c);
    precs.push_back(prec);
  }
  ssh::Engine e;
  e.tune = b->tune;
  cudaError_t err = ssh::engine_build(&e, ms, precs, false, b->stream);
  if (err == cudaSuccess) err = ssh::engine_eval(&e, prec, want_force != 0, b->stream, &b->prof);
  if (err == cudaSuccess) err = cudaStreamSynchronize(b->stream);
  ssh::engine_free(&e);
  if (err != cudaSuccess) return ssh::fail(err, "ssh_batch_eval");
  for (ssh_ctx* h : b->members) {
    h->c.have_result = true;
    h->c.last_prec = prec;
    h->c.last_force = want_force != 0;
  }
  return SSH_OK;
}

// The batch autotuner: times the evaluation of every member together under each candidate work decomposition of
// the tensor-core GEMMs (density pieces at 50, 100, 200, 400% of each member's SM share; force items in bundles or
// one by one), keeps the fastest, and remembers it per member shape set for the rest of the process.  The
// decomposition changes only the order of exact integer sums, so results are the same bit for bit.
namespace {
std::mutex g_tune_mu;
std::map<std::string, ssh::EngineTune> g_tune_cache;
}  // namespace

ssh_status ssh_batch_autotune(ssh_batch* b, int prec, int reps, ssh_tune* out) {
  if (!b || prec < SSH_FP64 || prec > SSH_FX || reps < 1 || reps > 1000) {
    set_error("ssh_batch_autotune: bad arguments");
    return SSH_EINVAL;
  }
  cudaSetDevice(b->device);
  std::vector<ssh::Ctx*> ms;
  std::vector<int> precs;
  std::vector<std::string> shapes;
  for (ssh_ctx* h : b->members) {
    if (!h->c.have_positions) { set_error("ssh_batch_autotune: a member has no positions"); return SSH_EINVAL; }
    ms.push_back(&h->c);
    precs.push_back(prec);
    shapes.push_back(std::to_string(h->c.d) + "/" + std::to_string(h->c.N) + "/" + std::to_string(h->c.M) + "/" +
                     std::to_string(h->c.tc.on ? h->c.tc.nchunk : 0));
  }
  if (ms.empty()) { set_error("ssh_batch_autotune: empty batch"); return SSH_EINVAL; }
  std::sort(shapes.begin(), shapes.end());
  std::string key = std::to_string(b->device) + "/" + std::to_string(prec);
  for (const std::string& x : shapes) key += ";" + x;
  ssh_tune rep;
  memset(&rep, 0, sizeof rep);
  // mean time of one evaluation (Phi, S_max, F) under a decomposition: one untimed, then reps timed
  auto time_it = [&](const ssh::EngineTune& t, double* ms_out) -> cudaError_t {
    ssh::Engine e;
    e.tune = t;
    cudaError_t err = ssh::engine_build(&e, ms, precs, false, b->stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) err = ssh::engine_eval(&e, prec, true, b->stream, nullptr);
    if (err == cudaSuccess) err = cudaEventRecord(e0, b->stream);
    for (int r = 0; r < reps && err == cudaSuccess; r++) err = ssh::engine_eval(&e, prec, true, b->stream, nullptr);
    if (err == cudaSuccess) err = cudaEventRecord(e1, b->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float msf = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&msf, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ssh::engine_free(&e);
    *ms_out = (double)msf / reps;
    return err;
  };
  ssh::EngineTune best;
  bool cached = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      best = it->second;
      cached = true;
    }
  }
  cudaError_t err = cudaSuccess;
  if (cached) {
    err = time_it(ssh::EngineTune(), &rep.ms_default);
    if (err == cudaSuccess) err = time_it(best, &rep.ms_tuned);
  } else {
    static const int kPct[4] = {50, 100, 200, 400};
    double best_ms = 0.0;
    for (int fb = 1; fb >= 0 && err == cudaSuccess; fb--)
      for (int pi = 0; pi < 4 && err == cudaSuccess; pi++) {
        ssh::EngineTune t;
        t.dens_pct = kPct[pi];
        t.force_bundle = fb;
        double msv = 0.0;
        err = time_it(t, &msv);
        rep.candidates++;
        if (err != cudaSuccess) break;
        if (t.dens_pct == 100 && t.force_bundle == 1) rep.ms_default = msv;
        if (rep.candidates == 1 || msv < best_ms) {
          best_ms = msv;
          best = t;
        }
      }
    rep.ms_tuned = best_ms;
    if (err == cudaSuccess) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[key] = best;
    }
  }
  if (err != cudaSuccess) return ssh::fail(err, "ssh_batch_autotune");
  b->tune = best;
  if (b->stepper) {
    b->stepper->tune = best;
    b->stepper->dirty = true;  // the next chunk of steps rebuilds its engine and graph with it
  }
  rep.dens_pieces_pct = best.dens_pct;
  rep.force_bundles = best.force_bundle;
  if (out) *out = rep;
  return SSH_OK;
}

// Minimise every member to completion through batched steps (the same FIRE step, stages and stopping rules as
// ssh_minimize, per member).
ssh_status ssh_batch_minimize(ssh_batch* b, const ssh_min_params* pin, int64_t chunk_steps, double max_seconds,
                              ssh_min_result* results) {
  if (!b) { set_error("ssh_batch_minimize: NULL batch"); return SSH_EINVAL; }
  cudaSetDevice(b->device);
  Runner r;
  r.tune = b->tune;
  r.device = b->device;
  r.st = b->stream;
  r.prof = b->prof.on ? &b->prof : nullptr;
  std::vector<Member> fresh;
  for (size_t i = 0; i < b->members.size(); i++) {
    Member m;
    m.h = b->members[i];
    if (!m.h->c.have_positions) { set_error("ssh_batch_minimize: a member has no positions"); return SSH_EINVAL; }
    ssh_status s = ssh::complete_params(m.h, pin, &m.p);
    if (s != SSH_OK) return s;
    m.ticket = i;
    fresh.push_back(m);
  }
  const double t0 = ssh::now_s();
  cudaError_t e = r.add(fresh);
  if (e != cudaSuccess) return ssh::fail(e, "ssh_batch_minimize: start");
  std::vector<Member> finished;
  const int64_t chunk = chunk_steps > 0 ? chunk_steps : 32;
  ssh_status out = SSH_OK;
  while (!r.act.empty()) {
    e = r.chunk(chunk, finished);
    if (e != cudaSuccess) return ssh::fail(e, "ssh_batch_minimize");
    if (max_seconds > 0 && ssh::now_s() - t0 > max_seconds && !r.act.empty()) {
      set_error("ssh_batch_minimize: wall-time limit reached");
      out = SSH_ETIMEOUT;
      for (Member& m : r.act) {
        m.res.status = SSH_ETIMEOUT;
        finished.push_back(m);
      }
      break;
    }
  }
  for (Member& m : finished) {
    b->results[m.ticket] = m.res;
    if (results) results[m.ticket] = m.res;
    if (m.res.status != SSH_OK && out == SSH_OK) out = (ssh_status)m.res.status;
    m.h->c.have_result = false;
  }
  if (out != SSH_OK && out != SSH_ETIMEOUT) set_error("ssh_batch_minimize: some members did not converge");
  return out;
}

ssh_status ssh_batch_begin(ssh_batch* b, const ssh_min_params* pin) {
  if (!b) { set_error("ssh_batch_begin: NULL batch"); return SSH_EINVAL; }
  cudaSetDevice(b->device);
  delete b->stepper;
  b->stepper = new Runner();
  b->stepper->tune = b->tune;
  b->stepper->device = b->device;
  b->stepper->st = b->stream;
  std::vector<Member> fresh;
  for (size_t i = 0; i < b->members.size(); i++) {
    Member m;
    m.h = b->members[i];
    if (!m.h->c.have_positions) { set_error("ssh_batch_begin: a member has no positions"); return SSH_EINVAL; }
    ssh_status s = ssh::complete_params(m.h, pin, &m.p);
    if (s != SSH_OK) return s;
    m.ticket = i;
    fresh.push_back(m);
  }
  cudaError_t e = b->stepper->add(fresh);
  if (e != cudaSuccess) return ssh::fail(e, "ssh_batch_begin");
  return SSH_OK;
}

ssh_status ssh_batch_steps(ssh_batch* b, int64_t nsteps) {
  if (!b || !b->stepper || nsteps < 0) { set_error("ssh_batch_steps: call ssh_batch_begin first"); return SSH_EINVAL; }
  cudaSetDevice(b->device);
  b->stepper->prof = b->prof.on ? &b->prof : nullptr;
  if (b->prof.on) b->stepper->dirty = true;  // profiling: direct launches carry per-kernel events
  cudaError_t e = b->stepper->launch_steps(nsteps);
  if (e != cudaSuccess) return ssh::fail(e, "ssh_batch_steps");
  return SSH_OK;
}

ssh_status ssh_batch_prof_enable(ssh_batch* b, int on) {
  if (!b) { set_error("ssh_batch_prof_enable: NULL batch"); return SSH_EINVAL; }
  cudaSetDevice(b->device);
  ssh::prof_collect(&b->prof, b->stream);
  b->prof.on = on != 0;
  for (int i = 0; i < ssh::kKCount; i++) { b->prof.ms[i] = 0; b->prof.launches[i] = 0; }
  return SSH_OK;
}

ssh_status ssh_batch_prof_read(ssh_batch* b, int n, double* ms, int64_t* launches) {
  if (!b || n < 0) { set_error("ssh_batch_prof_read: bad arguments"); return SSH_EINVAL; }
  cudaSetDevice(b->device);
  cudaError_t e = ssh::prof_collect(&b->prof, b->stream);
  if (e != cudaSuccess) return ssh::fail(e, "ssh_batch_prof_read");
  for (int i = 0; i < n && i < ssh::kKCount; i++) {
    if (ms) ms[i] = b->prof.ms[i];
    if (launches) launches[i] = b->prof.launches[i];
  }
  return SSH_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------ server

namespace {

struct Pending {
  uint64_t ticket;
  int d;
  int64_t N;
  double L, chi, K;
  std::vector<double> s_hi, s_lo;
  ssh_min_params p;
  bool has_params;
  int want_positions;
  double t_submit;
  size_t footprint;
  int64_t work;
};

struct Done {
  ssh_result r;
  std::vector<double> s_hi, s_lo;
};

}  // namespace

struct ssh_server {
  ssh_server_opts o;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Pending> queue;
  std::map<uint64_t, Done> done;
  std::map<uint64_t, int> state;  // 0 queued, 1 running, 2 done, 3 cancelled
  std::map<uint64_t, size_t> foot;
  uint64_t next_ticket = 1;
  size_t used = 0;
  bool stop = false;
  std::thread worker;
  double t0 = 0;
  ssh_server_stats stats;
  std::string worker_error;
};

static size_t estimate_footprint(int d, int64_t N, double L, double chi, double K, int sm_count, int64_t* work) {
  ssh::Ctx c;
  c.d = d;
  c.N = N;
  c.L = L;
  c.sm_count = sm_count;
  if (ssh::build_kset(d, N, L, chi, K, &c.ks) != 0) return 0;
  c.M = c.ks.M;
  c.tl = ssh::build_table_layout(c.ks);
  c.nt = ssh::build_nt_plan(c.ks, c.tl);
  c.fp = ssh::build_f_plan(c.ks, c.tl);
  c.Npad = (N + 31) / 32 * 32;
  ssh::setup_launch(&c);
  int ks = 1;
  for (int p = 0; p < 3; p++) ks = std::max(ks, c.launch[p].f_ksplit);
  for (int p = 0; p < 3; p++) c.launch[p].f_ksplit = ks;
  if (work) *work = c.M * c.N;
  return ssh::device_footprint(c);
}

static void server_loop(ssh_server* sv) {
  cudaSetDevice(sv->o.device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  Runner r;
  r.device = sv->o.device;
  r.st = st;
  const int64_t chunk = sv->o.chunk_steps > 0 ? sv->o.chunk_steps : 32;
  int64_t steps_now = chunk;
  for (;;) {
    std::vector<Pending> admit;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      if (r.act.empty())
        sv->cv.wait_for(lk, std::chrono::milliseconds(20), [&] { return sv->stop || !sv->queue.empty(); });
      if (sv->stop) break;
      // admission while a slot is free, the footprint fits the HBM budget and the batch's pairs per step stay
      // within max_pairs_per_step (a request that exceeds a limit alone is admitted into an empty batch)
      int64_t pairs = 0;
      for (Member& m : r.act) pairs += m.work;
      while (!sv->queue.empty() && (int)(r.act.size() + admit.size()) < sv->o.max_slots) {
        size_t pick = 0;  // FIFO: the oldest; smallest-work-first: the least M N (oldest among equals)
        if (sv->o.policy == 0)
          for (size_t i = 1; i < sv->queue.size(); i++)
            if (sv->queue[i].work < sv->queue[pick].work) pick = i;
        Pending& q = sv->queue[pick];
        if (sv->state[q.ticket] == 3) { sv->queue.erase(sv->queue.begin() + pick); continue; }
        const bool empty = r.act.empty() && admit.empty();
        if (!empty && (sv->used + q.footprint > (size_t)sv->o.hbm_budget_bytes ||
                       pairs + q.work > sv->o.max_pairs_per_step))
          break;
        sv->used += q.footprint;
        pairs += q.work;
        sv->foot[q.ticket] = q.footprint;
        sv->state[q.ticket] = 1;
        admit.push_back(std::move(q));
        sv->queue.erase(sv->queue.begin() + pick);
      }
    }
    std::vector<Member> fresh;
    for (Pending& q : admit) {
      Member m;
      ssh_opts o;
      memset(&o, 0, sizeof o);
      o.device = sv->o.device;
      o.fx_impl = sv->o.fx_impl;
      ssh_status s = ssh_create(q.d, q.N, q.L, q.chi, q.K, &o, &m.h);
      if (s == SSH_OK) s = ssh_set_stream(m.h, st);
      if (s == SSH_OK) s = ssh_set_positions_frac(m.h, q.s_hi.data(), q.s_lo.empty() ? nullptr : q.s_lo.data());
      if (s == SSH_OK) s = ssh::complete_params(m.h, q.has_params ? &q.p : nullptr, &m.p);
      m.ticket = q.ticket;
      m.t_submit = q.t_submit;
      if (s != SSH_OK) {
        std::lock_guard<std::mutex> lk(sv->mu);
        Done dn;
        memset(&dn.r, 0, sizeof dn.r);
        dn.r.status = s;
        dn.r.t_submit = q.t_submit - sv->t0;
        dn.r.t_done = ssh::now_s() - sv->t0;
        sv->done[q.ticket] = dn;
        sv->state[q.ticket] = 2;
        sv->used -= sv->foot[q.ticket];
        if (m.h) ssh_destroy(m.h);
        continue;
      }
      m.want_positions = q.want_positions;
      m.work = q.work;
      fresh.push_back(m);
    }
    cudaError_t e = cudaSuccess;
    if (!fresh.empty()) e = r.add(fresh);
    std::vector<Member> finished;
    if (e == cudaSuccess && !r.act.empty()) {
      const double tc = ssh::now_s();
      e = r.chunk(steps_now, finished);
      // chunk length adapts so that admissions and retirements happen about every target_chunk seconds
      const double per_step = (ssh::now_s() - tc) / (double)steps_now;
      int64_t want = per_step > 0 ? (int64_t)(0.1 / per_step) : chunk;
      steps_now = std::max<int64_t>(4, std::min<int64_t>(chunk, (want + 3) / 4 * 4));
    }
    if (e != cudaSuccess) {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->worker_error = cudaGetErrorString(e);
      sv->stop = true;
      break;
    }
    for (Member& m : finished) {
      Done dn;
      memset(&dn.r, 0, sizeof dn.r);
      dn.r.status = m.res.status;
      dn.r.steps = m.res.steps;
      dn.r.rejected = m.res.rejected;
      dn.r.smax[0] = m.res.smax[0];
      dn.r.smax[1] = m.res.smax[1];
      dn.r.phi[0] = m.res.phi[0];
      dn.r.phi[1] = m.res.phi[1];
      dn.r.final_prec = m.res.final_prec;
      dn.r.t_submit = m.t_submit - sv->t0;
      dn.r.t_admit = m.t_admit - sv->t0;
      dn.r.t_done = m.t_done - sv->t0;
      const int want_pos = m.want_positions;
      if (want_pos) {
        size_t nd = (size_t)m.h->c.d * m.h->c.N;
        dn.s_hi.resize(nd);
        dn.s_lo.resize(nd);
        ssh_get_positions_frac(m.h, dn.s_hi.data(), dn.s_lo.data());
      }
      dn.r.has_positions = want_pos ? 1 : 0;
      ssh_destroy(m.h);
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->used -= sv->foot[m.ticket];
      sv->done[m.ticket] = std::move(dn);
      sv->state[m.ticket] = 2;
      sv->stats.completed++;
      if (dn.r.status == SSH_OK) sv->stats.converged++;
    }
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stats.running = (int64_t)r.act.size();
      sv->stats.queued = (int64_t)sv->queue.size();
      sv->stats.hbm_used_bytes = (int64_t)sv->used;
    }
  }
  for (Member& m : r.act) ssh_destroy(m.h);
  r.act.clear();
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
}

extern "C" {

ssh_status ssh_server_create(const ssh_server_opts* opts, ssh_server** out) {
  if (!out) { set_error("ssh_server_create: out is NULL"); return SSH_EINVAL; }
  ssh_server* sv = new (std::nothrow) ssh_server();
  if (!sv) { set_error("ssh_server_create: out of host memory"); return SSH_ENOMEM; }
  memset(&sv->o, 0, sizeof sv->o);
  if (opts) sv->o = *opts;
  if (sv->o.max_slots <= 0) sv->o.max_slots = 256;
  if (sv->o.hbm_budget_bytes <= 0) sv->o.hbm_budget_bytes = (int64_t)64 << 30;
  if (sv->o.chunk_steps <= 0) sv->o.chunk_steps = 32;
  if (sv->o.max_pairs_per_step <= 0) sv->o.max_pairs_per_step = (int64_t)1 << 28;
  cudaError_t e = cudaSetDevice(sv->o.device);
  if (e != cudaSuccess) { delete sv; return ssh::fail(e, "ssh_server_create"); }
  memset(&sv->stats, 0, sizeof sv->stats);
  sv->t0 = ssh::now_s();
  sv->worker = std::thread(server_loop, sv);
  *out = sv;
  return SSH_OK;
}

void ssh_server_destroy(ssh_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  delete sv;
}

ssh_status ssh_submit(ssh_server* sv, const ssh_request* q, uint64_t* ticket) {
  if (!sv || !q || !ticket || !q->s_hi) { set_error("ssh_submit: NULL argument"); return SSH_EINVAL; }
  if (q->d < 1 || q->d > ssh::kMaxDim || q->N < 1 || !(q->L > 0)) { set_error("ssh_submit: bad configuration"); return SSH_EINVAL; }
  int sm = 148;
  cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, sv->o.device);
  int64_t work = 0;
  size_t fp = estimate_footprint(q->d, q->N, q->L, q->chi, q->K, sm, &work);
  if (fp == 0) { set_error("ssh_submit: could not build the wavevector set"); return SSH_EINVAL; }
  if ((int64_t)fp > sv->o.hbm_budget_bytes) { set_error("ssh_submit: request larger than the HBM budget"); return SSH_EINVAL; }
  Pending p;
  p.d = q->d;
  p.N = q->N;
  p.L = q->L;
  p.chi = q->chi;
  p.K = q->K;
  size_t nd = (size_t)q->d * q->N;
  p.s_hi.assign(q->s_hi, q->s_hi + nd);
  if (q->s_lo) p.s_lo.assign(q->s_lo, q->s_lo + nd);
  p.has_params = q->params != nullptr;
  if (q->params) p.p = *q->params;
  p.want_positions = q->want_positions;
  p.t_submit = ssh::now_s();
  p.footprint = fp;
  p.work = std::max<int64_t>(1, work);
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stop) { set_error("ssh_submit: server stopped: " + sv->worker_error); return SSH_ECUDA; }
  p.ticket = sv->next_ticket++;
  sv->state[p.ticket] = 0;
  *ticket = p.ticket;
  sv->queue.push_back(std::move(p));
  sv->stats.submitted++;
  sv->cv.notify_all();
  return SSH_OK;
}

ssh_status ssh_poll(ssh_server* sv, uint64_t ticket, ssh_result* out) {
  if (!sv) { set_error("ssh_poll: NULL server"); return SSH_EINVAL; }
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->state.find(ticket);
  if (it == sv->state.end()) { set_error("ssh_poll: unknown ticket"); return SSH_ENOTFOUND; }
  if (it->second == 3) { set_error("ssh_poll: cancelled"); return SSH_ENOTFOUND; }
  if (it->second != 2) {
    if (sv->stop) { set_error("ssh_poll: server stopped: " + sv->worker_error); return SSH_ECUDA; }
    return SSH_EBUSY;
  }
  if (out) *out = sv->done[ticket].r;
  return SSH_OK;
}

ssh_status ssh_result_positions(ssh_server* sv, uint64_t ticket, double* s_hi, double* s_lo) {
  if (!sv) { set_error("ssh_result_positions: NULL server"); return SSH_EINVAL; }
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->done.find(ticket);
  if (it == sv->done.end()) { set_error("ssh_result_positions: no result for this ticket"); return SSH_ENOTFOUND; }
  if (!it->second.r.has_positions) { set_error("ssh_result_positions: positions were not requested"); return SSH_EINVAL; }
  if (s_hi) memcpy(s_hi, it->second.s_hi.data(), sizeof(double) * it->second.s_hi.size());
  if (s_lo) memcpy(s_lo, it->second.s_lo.data(), sizeof(double) * it->second.s_lo.size());
  return SSH_OK;
}

ssh_status ssh_release(ssh_server* sv, uint64_t ticket) {
  if (!sv) { set_error("ssh_release: NULL server"); return SSH_EINVAL; }
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->state.find(ticket);
  if (it == sv->state.end() || it->second != 2) { set_error("ssh_release: no finished request with this ticket"); return SSH_ENOTFOUND; }
  sv->done.erase(ticket);
  sv->state.erase(it);
  return SSH_OK;
}

ssh_status ssh_cancel(ssh_server* sv, uint64_t ticket) {
  if (!sv) { set_error("ssh_cancel: NULL server"); return SSH_EINVAL; }
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->state.find(ticket);
  if (it == sv->state.end()) { set_error("ssh_cancel: unknown ticket"); return SSH_ENOTFOUND; }
  if (it->second != 0) { set_error("ssh_cancel: already admitted or finished"); return SSH_EBUSY; }
  it->second = 3;
  return SSH_OK;
}

ssh_status ssh_server_get_stats(ssh_server* sv, ssh_server_stats* out) {
  if (!sv || !out) { set_error("ssh_server_get_stats: NULL argument"); return SSH_EINVAL; }
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->stats;
  return SSH_OK;
}

}  // extern "C"
