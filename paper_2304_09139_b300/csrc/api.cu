// api.cu -- the extern "C" boundary (include/ssh.h): validation, host<->device copies, dispatch.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "ssh_internal.h"

#define SSH_TABLE_QUAL static
#include "gen/tables.h"


namespace ssh {
static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
}  // namespace ssh

using ssh::set_error;

static ssh_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return SSH_ECUDA;
}

#define SSH_CUDA(call, what)                         \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

static void free_buf(ssh::DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

namespace ssh {

void eval_graphs_reset(Ctx* c) {
  for (auto& row : c->eval_graph)
    for (cudaGraphExec_t& g : row) {
      if (g) cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

}  // namespace ssh

// One evaluation: replays a CUDA graph of the context engine's launches (captured at the first call for this
// precision), which removes the host launch gaps; with the profiler on, or when the stream is itself being captured
// by the caller, the kernels are launched directly.
static cudaError_t eval_replayed(ssh::Ctx& c, int prec, bool want_force) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(c.stream, &cs);
  if (e != cudaSuccess) return e;
  if (c.prof.on || ssh::tc_counters_on() || cs != cudaStreamCaptureStatusNone) return ssh::eval_phi_grad(&c, prec, want_force);
  cudaGraphExec_t& g = c.eval_graph[prec][want_force ? 1 : 0];
  if (!g) {
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    e = ssh::eval_phi_grad(&c, prec, want_force);
    const cudaError_t e2 = cudaStreamEndCapture(c.stream, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g = nullptr;
      return e;
    }
  }
  return cudaGraphLaunch(g, c.stream);
}

extern "C" {

const char* ssh_version(void) { return "ssh 0.1 sm_103a"; }

const char* ssh_last_error(void) { return ssh::g_err.c_str(); }

// The context of a built wavevector set (ks moves in); argument checks of d, N, L and the set done by the caller.
static ssh_status create_from(int d, int64_t N, double L, ssh::KSet&& ks, const ssh_opts* opts, ssh_ctx** out) {
  ssh_ctx* h = new (std::nothrow) ssh_ctx();
  if (!h) { set_error("ssh_create: out of host memory"); return SSH_ENOMEM; }
  ssh::Ctx& c = h->c;
  c.d = d;
  c.N = N;
  c.L = L;
  c.device = opts ? opts->device : 0;
  const int fx_impl = opts ? opts->fx_impl : SSH_FX_AUTO;
  if (fx_impl < SSH_FX_AUTO || fx_impl > SSH_FX_TENSOR) { delete h; set_error("ssh_create: bad fx_impl"); return SSH_EINVAL; }
  c.tc_requested = fx_impl == SSH_FX_TENSOR || (fx_impl == SSH_FX_AUTO && SSH_FX_AUTO_TENSOR);
  c.tc_chunk_req = opts ? opts->tc_chunk : 0;
  if (c.tc_chunk_req < 0) { delete h; set_error("ssh_create: tc_chunk must be >= 0"); return SSH_EINVAL; }
  const int64_t sp0 = opts ? opts->shard_first : 0, spn = opts ? opts->shard_count : 0;
  if (sp0 != 0 || spn != 0) {
    // a particle shard: aligned to the dot-product chunks, so that every chunk's partial sums belong to one shard
    if (sp0 < 0 || spn < 1 || sp0 + spn > N || sp0 % ssh::kDotChunk != 0 ||
        (sp0 + spn < N && spn % ssh::kDotChunk != 0)) {
      delete h;
      set_error("ssh_create: a shard [shard_first, shard_first + shard_count) must lie in [0, N), start on a multiple "
                "of 2048 and hold a multiple of 2048 particles unless it ends at N");
      return SSH_EINVAL;
    }
    c.shard_p0 = sp0;
    c.shard_n = spn;
  }
  c.ks = std::move(ks);
  c.M = c.ks.M;
  if (c.M > (int64_t)1 << 30) { delete h; set_error("ssh_create: M too large"); return SSH_EINVAL; }
  c.tl = ssh::build_table_layout(c.ks);
  c.nt = ssh::build_nt_plan(c.ks, c.tl);
  c.fp = ssh::build_f_plan(c.ks, c.tl);
  c.Npad = (N + 31) / 32 * 32;
  // 4 pi / L as dd
  dd four_pi = dd_make(2.0 * SSH_DD_2PI[0], 2.0 * SSH_DD_2PI[1]);
  c.pref = dd_div(four_pi, dd_make(L));
  c.inv_L = dd_div(dd_make(1.0), dd_make(L));
  cudaError_t e = cudaSetDevice(c.device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { delete h; return cuda_fail(e, "ssh_create: device/stream"); }
  c.own_stream = true;
  cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, c.device);
  e = ssh::plan_upload(&c);
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_stage, sizeof(double) * (2 * (size_t)d * N + ssh::kPackTail));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->stage_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) {
    ssh_destroy(h);
    return e == cudaErrorMemoryAllocation ? (set_error("ssh_create: out of device memory"), SSH_ENOMEM)
                                          : cuda_fail(e, "ssh_create: set-up");
  }
  if (c.shard_n > 0 && !c.tc.on) {
    ssh_destroy(h);
    set_error("ssh_create: a particle shard needs the tensor-core fixed-point path (a set within its limits)");
    return SSH_EINVAL;
  }
  *out = h;
  return SSH_OK;
}

// A shard context's evaluations need the other shards' densities: they run through ssh_shard_* only.
static bool whole(const ssh::Ctx& c, const char* fn) {
  if (c.shard_n == 0) return true;
  set_error(std::string(fn) + ": a particle-shard context evaluates and minimises through ssh_shard_*");
  return false;
}

static bool check_dnl(const char* fn, int d, int64_t N, double L) {
  if (d < 1 || d > ssh::kMaxDim) { set_error(std::string(fn) + ": d must be 1..4"); return false; }
  if (N < 1 || N > (int64_t)1 << 31) { set_error(std::string(fn) + ": N must be in [1, 2^31]"); return false; }
  if (!(L > 0) || !isfinite(L)) { set_error(std::string(fn) + ": L must be positive and finite"); return false; }
  return true;
}

static bool check_mode(const char* fn, double chi, double K) {
  if (!isfinite(chi) || !isfinite(K) || chi < 0 || K < 0 || (chi > 0) == (K > 0)) {
    set_error(std::string(fn) + ": give exactly one of chi > 0 or K > 0");
    return false;
  }
  if (chi >= 1.0) { set_error(std::string(fn) + ": chi must be < 1"); return false; }
  return true;
}

ssh_status ssh_create(int d, int64_t N, double L, double chi, double K, const ssh_opts* opts, ssh_ctx** out) {
  if (!out) { set_error("ssh_create: out is NULL"); return SSH_EINVAL; }
  *out = nullptr;
  if (!check_dnl("ssh_create", d, N, L) || !check_mode("ssh_create", chi, K)) return SSH_EINVAL;
  ssh::KSet ks;
  if (ssh::build_kset(d, N, L, chi, K, &ks) != 0) {
    set_error("ssh_create: could not build the wavevector set");
    return SSH_EINVAL;
  }
  return create_from(d, N, L, std::move(ks), opts, out);
}

ssh_status ssh_create_kset(int d, int64_t N, double L, int64_t M, const int32_t* n, const ssh_opts* opts, ssh_ctx** out) {
  if (!out) { set_error("ssh_create_kset: out is NULL"); return SSH_EINVAL; }
  *out = nullptr;
  if (!check_dnl("ssh_create_kset", d, N, L)) return SSH_EINVAL;
  if (M < 1 || M > (int64_t)1 << 30 || !n) { set_error("ssh_create_kset: need 1 <= M <= 2^30 vectors"); return SSH_EINVAL; }
  ssh::KSet ks;
  if (ssh::build_kset_list(d, M, n, L, &ks) != 0) {
    set_error("ssh_create_kset: the vectors must be distinct, in the half space (first non-zero component > 0), "
              "with |n_a| <= 32767");
    return SSH_EINVAL;
  }
  return create_from(d, N, L, std::move(ks), opts, out);
}

ssh_status ssh_kset_build_region(int d, int64_t N, double L, double chi, double K, const int32_t* w, int64_t cap,
                                 int32_t* n, int64_t* M) {
  if (!check_dnl("ssh_kset_build_region", d, N, L) || !check_mode("ssh_kset_build_region", chi, K)) return SSH_EINVAL;
  std::vector<int32_t> v;
  if (ssh::kset_region(d, N, L, chi, K, w, &v) != 0) {
    set_error("ssh_kset_build_region: bad arguments (axis weights must be integers in [1, 2^20])");
    return SSH_EINVAL;
  }
  const int64_t m = (int64_t)v.size() / d;
  if (M) *M = m;
  if (n) {
    if (cap < m) { set_error("ssh_kset_build_region: buffer too small"); return SSH_EINVAL; }
    if (m > 0) memcpy(n, v.data(), sizeof(int32_t) * v.size());
  }
  return SSH_OK;
}

void ssh_destroy(ssh_ctx* h) {
  if (!h) return;
  ssh::Ctx& c = h->c;
  cudaSetDevice(c.device);
  if (c.stream) cudaStreamSynchronize(c.stream);
  ssh::fire_free(&c);
  ssh::eval_graphs_reset(&c);
  if (c.eng) {
    ssh::engine_free(c.eng);
    delete c.eng;
    c.eng = nullptr;
  }
  ssh::tc_free(&c);
  for (ssh::DevBuf* b : {&c.s_hi, &c.s_lo, &c.rows, &c.slots, &c.blocks, &c.grows, &c.cols, &c.fsplit, &c.tab, &c.part,
                         &c.C_hi, &c.C_lo, &c.S_hi, &c.S_lo, &c.wk, &c.coef, &c.blk, &c.scal, &c.fpart, &c.F_hi, &c.F_lo})
    free_buf(*b);
  free_buf(h->d_pack);
  if (h->h_stage) cudaFreeHost(h->h_stage);
  if (h->stage_done) cudaEventDestroy(h->stage_done);
  for (ssh::ProfRec& r : c.prof.pending) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
  for (cudaEvent_t ev : c.prof.pool) cudaEventDestroy(ev);
  if (c.own_stream && c.stream) cudaStreamDestroy(c.stream);
  delete h;
}

ssh_status ssh_get_dims(const ssh_ctx* h, int* d, int64_t* N, int64_t* M, double* L) {
  if (!h) { set_error("ssh_get_dims: NULL context"); return SSH_EINVAL; }
  if (d) *d = h->c.d;
  if (N) *N = h->c.N;
  if (M) *M = h->c.M;
  if (L) *L = h->c.L;
  return SSH_OK;
}

ssh_status ssh_get_fx_impl(const ssh_ctx* h, int* impl) {
  if (!h || !impl) { set_error("ssh_get_fx_impl: NULL argument"); return SSH_EINVAL; }
  *impl = h->c.tc.on ? SSH_FX_TENSOR : SSH_FX_INTEGER;
  return SSH_OK;
}

ssh_status ssh_set_weights(ssh_ctx* h, const double* w) {
  if (!h) { set_error("ssh_set_weights: NULL context"); return SSH_EINVAL; }
  ssh::Ctx& c = h->c;
  const int64_t M = c.M;
  if (M == 0) return SSH_OK;
  std::vector<double> wi((size_t)M, 1.0);  // internal order
  double wmax = 1.0;
  if (w) {
    wmax = 0.0;
    for (int64_t k = 0; k < M; k++) {
      const double x = w[c.ks.int2pub[k]];
      if (!(x >= 0.0 && x <= 1024.0)) { set_error("ssh_set_weights: weights must be finite, in [0, 1024]"); return SSH_EINVAL; }
      wi[k] = x;
      wmax = std::max(wmax, x);
    }
  }
  cudaSetDevice(c.device);
  SSH_CUDA(cudaMemcpyAsync(c.wk.p, wi.data(), sizeof(double) * M, cudaMemcpyHostToDevice, c.stream), "ssh_set_weights");
  SSH_CUDA(cudaStreamSynchronize(c.stream), "ssh_set_weights");  // the host vector goes out of scope
  c.wmax = wmax;
  c.have_result = false;
  return SSH_OK;
}

ssh_status ssh_get_tc_chunks(const ssh_ctx* h, int* nchunk, int64_t* chunk) {
  if (!h) { set_error("ssh_get_tc_chunks: null context"); return SSH_EINVAL; }
  if (nchunk) *nchunk = h->c.tc.on ? h->c.tc.nchunk : 0;
  if (chunk) *chunk = h->c.tc.on ? h->c.tc.Nc : 0;
  return SSH_OK;
}

ssh_status ssh_get_tc_plan(const ssh_ctx* h, int* row_tiles, int* col_tiles, int* tiles, int* transposed) {
  if (!h) { set_error("ssh_get_tc_plan: null context"); return SSH_EINVAL; }
  const ssh::TcPlan& t = h->c.tc;
  if (row_tiles) *row_tiles = t.on ? t.RT : 0;
  if (col_tiles) *col_tiles = t.on ? t.CTd : 0;
  if (tiles) *tiles = t.on ? (int)t.tiles.size() : 0;
  if (transposed) *transposed = t.on ? t.tr : 0;
  return SSH_OK;
}

ssh_status ssh_get_kset(const ssh_ctx* h, int64_t* M, int32_t* n) {
  if (!h) { set_error("ssh_get_kset: NULL context"); return SSH_EINVAL; }
  if (M) *M = h->c.M;
  if (n && h->c.M > 0) memcpy(n, h->c.ks.n_pub.data(), sizeof(int32_t) * h->c.ks.n_pub.size());
  return SSH_OK;
}

ssh_status ssh_kset_build(int d, int64_t N, double L, double chi, double K, int64_t cap, int32_t* n, int64_t* M) {
  ssh::KSet ks;
  if (ssh::build_kset(d, N, L, chi, K, &ks) != 0) { set_error("ssh_kset_build: bad arguments"); return SSH_EINVAL; }
  if (M) *M = ks.M;
  if (n) {
    if (cap < ks.M) { set_error("ssh_kset_build: buffer too small"); return SSH_EINVAL; }
    if (ks.M > 0) memcpy(n, ks.n_pub.data(), sizeof(int32_t) * ks.n_pub.size());
  }
  return SSH_OK;
}

ssh_status ssh_set_stream(ssh_ctx* h, void* stream) {
  if (!h) { set_error("ssh_set_stream: NULL context"); return SSH_EINVAL; }
  ssh::Ctx& c = h->c;
  cudaSetDevice(c.device);
  SSH_CUDA(cudaStreamSynchronize(c.stream), "ssh_set_stream: sync old stream");
  if (stream) {
    if (c.own_stream) { cudaStreamDestroy(c.stream); c.own_stream = false; }
    c.stream = (cudaStream_t)stream;
  } else if (!c.own_stream) {
    SSH_CUDA(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking), "ssh_set_stream: create");
    c.own_stream = true;
  }
  return SSH_OK;
}

ssh_status ssh_sync(ssh_ctx* h) {
  if (!h) { set_error("ssh_sync: NULL context"); return SSH_EINVAL; }
  cudaSetDevice(h->c.device);
  SSH_CUDA(cudaStreamSynchronize(h->c.stream), "ssh_sync");
  return SSH_OK;
}

// s (fractional, any real) -> [0, 1) as dd, SoA staging [a][j].
// True when every s_hi is in [+0, 1) (sign bit clear, exponent below that of 1.0; NaN, infinities and -0 fail)
// and every s_lo is a zero of either sign: such values are their own fractions.  Branch-free bit tests.
static bool frac_all_plain(const double* s_hi, const double* s_lo, int64_t n) {
  uint64_t bad = 0;
  for (int64_t i = 0; i < n; i++) {
    uint64_t u;
    memcpy(&u, s_hi + i, sizeof u);
    bad |= (uint64_t)((u >> 52) >= 0x3ff);
  }
  if (s_lo)
    for (int64_t i = 0; i < n; i++) {
      uint64_t u;
      memcpy(&u, s_lo + i, sizeof u);
      bad |= u << 1;
    }
  return bad == 0;
}

static ssh_status stage_and_upload(ssh_ctx* h, const double* s_hi, const double* s_lo, bool physical) {
  ssh::Ctx& c = h->c;
  const int64_t N = c.N;
  const int d = c.d;
  double* hs = h->h_stage;
  double* ls = h->h_stage + (size_t)d * N;
  cudaSetDevice(c.device);
  // the previous upload from the staging buffer must have landed before it is rewritten
  SSH_CUDA(cudaEventSynchronize(h->stage_done), "upload positions");
  if (!physical && frac_all_plain(s_hi, s_lo, (int64_t)d * N)) {
    // every value is its own fraction: the staging is a transposed copy, and the low words are zeroed on the
    // device instead of being copied
    for (int a = 0; a < d; a++) {
      double* o = hs + (size_t)a * N;
      const double* in = s_hi + a;
      for (int64_t j = 0; j < N; j++) o[j] = in[j * d];
    }
    SSH_CUDA(cudaMemcpyAsync(c.s_hi.p, hs, sizeof(double) * d * N, cudaMemcpyHostToDevice, c.stream), "upload positions");
    SSH_CUDA(cudaMemsetAsync(c.s_lo.p, 0, sizeof(double) * d * N, c.stream), "upload positions");
    SSH_CUDA(cudaEventRecord(h->stage_done, c.stream), "upload positions");
    c.have_positions = true;
    c.have_result = false;
    return SSH_OK;
  } else {
    dd Ld = dd_make(c.L);
    for (int64_t j = 0; j < N; j++) {
      for (int a = 0; a < d; a++) {
        double hi = s_hi[j * d + a], lo = s_lo ? s_lo[j * d + a] : 0.0;
        if (!physical && hi >= 0.0 && hi < 1.0 && lo == 0.0) {
          // already in [0, 1) with a zero low word: its own fraction (+ 0.0 turns -0 into +0, as the full path does)
          hs[a * N + j] = hi + 0.0;
          ls[a * N + j] = 0.0;
          continue;
        }
        if (!isfinite(hi) || !isfinite(lo)) {
          set_error("positions contain a non-finite value");
          return SSH_ENAN;
        }
        dd v = two_sum(hi, lo);
        if (physical) v = dd_div(v, Ld);
        v = dd_frac(v);
        hs[a * N + j] = v.hi;
        ls[a * N + j] = v.lo;
      }
    }
  }
  SSH_CUDA(cudaMemcpyAsync(c.s_hi.p, hs, sizeof(double) * d * N, cudaMemcpyHostToDevice, c.stream), "upload positions");
  SSH_CUDA(cudaMemcpyAsync(c.s_lo.p, ls, sizeof(double) * d * N, cudaMemcpyHostToDevice, c.stream), "upload positions");
  // no wait here: downloads into the staging buffer are ordered after these copies on the stream, and the next
  // upload waits for this event before it rewrites the buffer
  SSH_CUDA(cudaEventRecord(h->stage_done, c.stream), "upload positions");
  c.have_positions = true;
  c.have_result = false;
  return SSH_OK;
}

ssh_status ssh_set_positions(ssh_ctx* h, const double* r_hi, const double* r_lo) {
  if (!h || !r_hi) { set_error("ssh_set_positions: NULL argument"); return SSH_EINVAL; }
  return stage_and_upload(h, r_hi, r_lo, true);
}

ssh_status ssh_set_positions_frac(ssh_ctx* h, const double* s_hi, const double* s_lo) {
  if (!h || !s_hi) { set_error("ssh_set_positions_frac: NULL argument"); return SSH_EINVAL; }
  return stage_and_upload(h, s_hi, s_lo, false);
}

ssh_status ssh_get_positions_frac(ssh_ctx* h, double* s_hi, double* s_lo) {
  if (!h) { set_error("ssh_get_positions_frac: NULL context"); return SSH_EINVAL; }
  ssh::Ctx& c = h->c;
  if (!c.have_positions) { set_error("ssh_get_positions_frac: no positions set"); return SSH_EINVAL; }
  const int64_t N = c.N;
  const int d = c.d;
  double* hs = h->h_stage;
  double* ls = h->h_stage + (size_t)d * N;
  cudaSetDevice(c.device);
  SSH_CUDA(cudaMemcpyAsync(hs, c.s_hi.p, sizeof(double) * d * N, cudaMemcpyDeviceToHost, c.stream), "download positions");
  SSH_CUDA(cudaMemcpyAsync(ls, c.s_lo.p, sizeof(double) * d * N, cudaMemcpyDeviceToHost, c.stream), "download positions");
  SSH_CUDA(cudaStreamSynchronize(c.stream), "download positions");
  for (int64_t j = 0; j < N; j++)
    for (int a = 0; a < d; a++) {
      if (s_hi) s_hi[j * d + a] = hs[a * N + j];
      if (s_lo) s_lo[j * d + a] = ls[a * N + j];
    }
  return SSH_OK;
}

ssh_status ssh_get_positions(ssh_ctx* h, double* r_hi, double* r_lo) {
  if (!h) { set_error("ssh_get_positions: NULL context"); return SSH_EINVAL; }
  ssh::Ctx& c = h->c;
  const int64_t nd = (int64_t)c.d * c.N;
  std::vector<double> hi((size_t)nd), lo((size_t)nd);
  const ssh_status st = ssh_get_positions_frac(h, hi.data(), lo.data());
  if (st != SSH_OK) return st;
  for (int64_t i = 0; i < nd; i++) {
    const dd r = dd_mul_d(dd_make(hi[i], lo[i]), c.L);
    if (r_hi) r_hi[i] = r.hi;
    if (r_lo) r_lo[i] = r.lo;
  }
  return SSH_OK;
}

ssh_status ssh_eval(ssh_ctx* h, int prec, int want_force) {
  if (!h) { set_error("ssh_eval: NULL context"); return SSH_EINVAL; }
  ssh::Ctx& c = h->c;
  if (prec < SSH_FP64 || prec > SSH_FX) { set_error("ssh_eval: unknown precision"); return SSH_EINVAL; }
  if (!c.have_positions) { set_error("ssh_eval: no positions set"); return SSH_EINVAL; }
  if (!whole(c, "ssh_eval")) return SSH_EINVAL;
  cudaSetDevice(c.device);
  cudaError_t e = eval_replayed(c, prec, want_force != 0);
  if (e != cudaSuccess) return cuda_fail(e, "ssh_eval: launch");
  c.have_result = true;
  c.last_prec = prec;
  c.last_force = want_force != 0;
  return SSH_OK;
}

// The results of an evaluation in one block for a single download: the scalars and the status words {any
// non-finite F_hi, the tensor-core status} first, then F_hi and F_lo turned from the device's axis-major [a][j] to
// the caller's [j][a] (nd = d N values each, or none).  The first status word is only ever set here; the host
// clears it after a call that found it set.
__global__ void k_pack_results(const double* __restrict__ F_hi, const double* __restrict__ F_lo,
                               const double* __restrict__ scal, const int* __restrict__ tc_err, int64_t N, int d,
                               int64_t nd, double* __restrict__ out) {
  int* status = reinterpret_cast<int*>(out + ssh::kScCount);
  double* f = out + ssh::kPackTail;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nd) {
    const int64_t j = i / d;
    const int a = (int)(i - j * d);
    const double fh = F_hi[a * N + j];
    f[i] = fh;
    f[nd + i] = F_lo[a * N + j];
    if (!isfinite(fh)) status[0] = 1;
  }
  if (i < ssh::kScCount) out[i] = scal[i];
  if (i == 0) status[1] = tc_err ? *tc_err : 0;
}

ssh_status ssh_get_results(ssh_ctx* h, double phi[2], double smax[2], double* F_hi, double* F_lo) {
  if (!h) { set_error("ssh_get_results: NULL context"); return SSH_EINVAL; }
  ssh::Ctx& c = h->c;
  if (!c.have_result) { set_error("ssh_get_results: no evaluation yet"); return SSH_EINVAL; }
  if ((F_hi || F_lo) && !c.last_force) { set_error("ssh_get_results: last evaluation had no force"); return SSH_EINVAL; }
  cudaSetDevice(c.device);
  const int64_t N = c.N;
  const int d = c.d;
  const int64_t nd = (F_hi || F_lo) ? (int64_t)d * N : 0;
  const size_t full = sizeof(double) * (2 * (size_t)d * N + ssh::kPackTail);
  if (!h->d_pack.p) {
    SSH_CUDA(cudaMalloc(&h->d_pack.p, full), "ssh_get_results: results buffer");
    h->d_pack.bytes = full;
    SSH_CUDA(cudaMemsetAsync(h->d_pack.p, 0, sizeof(double) * ssh::kPackTail, c.stream), "ssh_get_results");
  }
  // one kernel packs the scalars, the status words and the force (in the caller's layout); one copy brings them
  double* dp = reinterpret_cast<double*>(h->d_pack.p);
  const int64_t work = std::max<int64_t>(nd, ssh::kScCount);
  k_pack_results<<<(unsigned)((work + 255) / 256), 256, 0, c.stream>>>(
      (const double*)c.F_hi.p, (const double*)c.F_lo.p, (const double*)c.scal.p, c.tc.on ? (const int*)c.tc.err.p : nullptr,
      N, d, nd, dp);
  SSH_CUDA(cudaGetLastError(), "ssh_get_results: pack");
  double* hp = h->h_stage;
  SSH_CUDA(cudaMemcpyAsync(hp, dp, sizeof(double) * (ssh::kPackTail + 2 * nd), cudaMemcpyDeviceToHost, c.stream),
           "download results");
  SSH_CUDA(cudaStreamSynchronize(c.stream), "ssh_get_results");
  const double* sc = hp;
  int status[2];
  memcpy(status, sc + ssh::kScCount, sizeof status);
  if (status[0] != 0) cudaMemsetAsync(dp + ssh::kScCount, 0, sizeof(int), c.stream);  // for the next call
  if (status[1] != 0) {
    // a bounded wait inside a tensor-core kernel gave up: the results of that evaluation are not valid
    cudaMemsetAsync(c.tc.err.p, 0, sizeof(int), c.stream);
    set_error("tensor-core kernel: a bounded wait gave up (status " + std::to_string(status[1]) + ")");
    return SSH_ETIMEOUT;
  }
  if (phi) { phi[0] = sc[ssh::kScPhiHi]; phi[1] = sc[ssh::kScPhiLo]; }
  if (smax) { smax[0] = sc[ssh::kScSmaxHi]; smax[1] = sc[ssh::kScSmaxLo]; }
  bool bad = !isfinite(sc[ssh::kScPhiHi]) || !isfinite(sc[ssh::kScSmaxHi]);
  if (nd) {
    if (F_hi) memcpy(F_hi, hp + ssh::kPackTail, sizeof(double) * nd);
    if (F_lo) memcpy(F_lo, hp + ssh::kPackTail + nd, sizeof(double) * nd);
    bad = bad || status[0] != 0;
  }
  if (bad) { set_error("non-finite energy, S_max or force"); return SSH_ENAN; }
  return SSH_OK;
}

ssh_status ssh_energy_grad(ssh_ctx* h, int prec, double phi[2], double smax[2], double* F_hi, double* F_lo) {
  ssh_status s = ssh_eval(h, prec, (F_hi || F_lo) ? 1 : 0);
  if (s != SSH_OK) return s;
  return ssh_get_results(h, phi, smax, F_hi, F_lo);
}

ssh_status ssh_get_ntilde(ssh_ctx* h, double* C_hi, double* C_lo, double* S_hi, double* S_lo) {
  if (!h) { set_error("ssh_get_ntilde: NULL context"); return SSH_EINVAL; }
  ssh::Ctx& c = h->c;
  if (!c.have_result) { set_error("ssh_get_ntilde: no evaluation yet"); return SSH_EINVAL; }
  const int64_t M = c.M;
  if (M == 0) return SSH_OK;
  std::vector<double> buf((size_t)4 * M);
  cudaSetDevice(c.device);
  const ssh::DevBuf* src[4] = {&c.C_hi, &c.C_lo, &c.S_hi, &c.S_lo};
  for (int i = 0; i < 4; i++)
    SSH_CUDA(cudaMemcpyAsync(buf.data() + (size_t)i * M, src[i]->p, sizeof(double) * M, cudaMemcpyDeviceToHost, c.stream),
             "download n~");
  SSH_CUDA(cudaStreamSynchronize(c.stream), "download n~");
  double* dst[4] = {C_hi, C_lo, S_hi, S_lo};
  for (int i = 0; i < 4; i++) {
    if (!dst[i]) continue;
    for (int64_t k = 0; k < M; k++) dst[i][c.ks.int2pub[k]] = buf[(size_t)i * M + k];
  }
  return SSH_OK;
}

ssh_status ssh_min_defaults(const ssh_ctx* h, ssh_min_params* p) {
  if (!h || !p) { set_error("ssh_min_defaults: NULL argument"); return SSH_EINVAL; }
  const ssh::Ctx& c = h->c;
  memset(p, 0, sizeof *p);
  double k2 = c.ks.k2max > 0 ? c.ks.k2max : 1.0;
  p->dt_max = 1.0 / sqrt(2.0 * (double)c.N * k2);
  p->dt0 = p->dt_max / 10.0;
  p->alpha_start = 0.1;
  p->f_alpha = 0.99;
  p->f_inc = 1.1;
  p->f_dec = 0.5;
  p->n_min = 5;
  // The paper's cheap FP64 stage only pays where FP64 is fast.  On this part the tensor-core fixed-point step
  // is several times faster than an FP64 step, so a tensor-core context quenches in fixed point throughout.
  p->n_stages = c.tc.on ? 1 : 2;
  p->stage_prec[0] = c.tc.on ? SSH_FX : SSH_FP64;
  p->stage_prec[1] = SSH_FX;
  p->stage_prec[2] = SSH_FX;
  p->stage_floor[0] = 1e-24;
  // stall windows 0: by the stage's precision (complete_params), whatever ladder the caller sets
  p->stall_window[0] = 0;
  p->stall_window[1] = 0;
  p->stall_window[2] = 0;
  p->max_steps = 200000;
  p->smax_target = 1e-36;
  p->chunk = 64;
  p->max_seconds = 0;
  return SSH_OK;
}

}  // extern "C"

ssh_status ssh::complete_params(const ssh_ctx* h, const ssh_min_params* pin, ssh_min_params* out) {
  ssh_min_params d;
  ssh_min_defaults(h, &d);
  ssh_min_params p = pin ? *pin : d;
  // zero fields take defaults
  if (p.dt_max <= 0) p.dt_max = d.dt_max;
  if (p.dt0 <= 0) p.dt0 = std::min(d.dt0, p.dt_max);
  if (p.alpha_start <= 0) p.alpha_start = d.alpha_start;
  if (p.f_alpha <= 0) p.f_alpha = d.f_alpha;
  if (p.f_inc <= 0) p.f_inc = d.f_inc;
  if (p.f_dec <= 0) p.f_dec = d.f_dec;
  if (p.n_min <= 0) p.n_min = d.n_min;
  if (p.n_stages <= 0) {
    p.n_stages = d.n_stages;
    for (int i = 0; i < 3; i++) { p.stage_prec[i] = d.stage_prec[i]; p.stage_floor[i] = d.stage_floor[i]; }
  }
  // an FP64 stage reaches its rounding floor quickly and hands over after 200 steps without halving; a dd or
  // fixed-point stage is the last word on the quench and keeps going for 5000 (slow d = 1 quenches need it)
  for (int i = 0; i < 3; i++)
    if (p.stall_window[i] <= 0) p.stall_window[i] = p.stage_prec[i] == SSH_FP64 ? 200 : 5000;
  if (p.max_steps <= 0) p.max_steps = d.max_steps;
  if (p.smax_target <= 0) p.smax_target = d.smax_target;
  if (p.chunk <= 0) p.chunk = d.chunk;
  if (p.n_stages > 3 || !(p.dt0 > 0) || !(p.dt_max >= p.dt0) || !(p.f_dec < 1) || !(p.f_inc >= 1) ||
      !(p.alpha_start < 1) || !(p.f_alpha <= 1)) {
    set_error("ssh_minimize: inconsistent parameters");
    return SSH_EINVAL;
  }
  for (int i = 0; i < p.n_stages; i++)
    if (p.stage_prec[i] < SSH_FP64 || p.stage_prec[i] > SSH_FX) {
      set_error("ssh_minimize: unknown stage precision");
      return SSH_EINVAL;
    }
  *out = p;
  return SSH_OK;
}

extern "C" {

ssh_status ssh_minimize(ssh_ctx* h, const ssh_min_params* pin, ssh_min_result* res) {
  if (!h) { set_error("ssh_minimize: NULL context"); return SSH_EINVAL; }
  ssh::Ctx& c = h->c;
  if (!c.have_positions) { set_error("ssh_minimize: no positions set"); return SSH_EINVAL; }
  if (!whole(c, "ssh_minimize")) return SSH_EINVAL;
  ssh_min_params p;
  ssh_status st = ssh::complete_params(h, pin, &p);
  if (st != SSH_OK) return st;
  cudaSetDevice(c.device);
  return ssh::minimize(&c, &p, res);
}

ssh_status ssh_fire_begin(ssh_ctx* h, const ssh_min_params* pin) {
  if (!h) { set_error("ssh_fire_begin: NULL context"); return SSH_EINVAL; }
  ssh::Ctx& c = h->c;
  if (!c.have_positions) { set_error("ssh_fire_begin: no positions set"); return SSH_EINVAL; }
  if (!whole(c, "ssh_fire_begin")) return SSH_EINVAL;
  ssh_min_params p;
  ssh_status st = ssh::complete_params(h, pin, &p);
  if (st != SSH_OK) return st;
  cudaSetDevice(c.device);
  return ssh::fire_begin(&c, &p);
}

ssh_status ssh_fire_steps(ssh_ctx* h, int prec, int64_t nsteps) {
  if (!h || prec < SSH_FP64 || prec > SSH_FX || nsteps < 0) { set_error("ssh_fire_steps: bad arguments"); return SSH_EINVAL; }
  if (!whole(h->c, "ssh_fire_steps")) return SSH_EINVAL;
  cudaSetDevice(h->c.device);
  return ssh::fire_steps(&h->c, prec, nsteps);
}

ssh_status ssh_fire_state(ssh_ctx* h, ssh_min_result* res, int* running) {
  if (!h) { set_error("ssh_fire_state: NULL context"); return SSH_EINVAL; }
  cudaSetDevice(h->c.device);
  int st = 0;
  ssh_status s = ssh::fire_state(&h->c, res, &st);
  if (running) *running = st == 0;
  return s;
}

ssh_status ssh_prof_enable(ssh_ctx* h, int on) {
  if (!h) { set_error("ssh_prof_enable: NULL context"); return SSH_EINVAL; }
  ssh::Ctx& c = h->c;
  cudaSetDevice(c.device);
  cudaError_t e = ssh::prof_collect(&c.prof, c.stream);
  if (e != cudaSuccess) return cuda_fail(e, "ssh_prof_enable");
  c.prof.on = on != 0;
  for (int i = 0; i < ssh::kKCount; i++) { c.prof.ms[i] = 0; c.prof.launches[i] = 0; }
  return SSH_OK;
}

ssh_status ssh_prof_read(ssh_ctx* h, int n, double* ms, int64_t* launches) {
  if (!h || n < 0) { set_error("ssh_prof_read: bad arguments"); return SSH_EINVAL; }
  ssh::Ctx& c = h->c;
  cudaSetDevice(c.device);
  cudaError_t e = ssh::prof_collect(&c.prof, c.stream);
  if (e != cudaSuccess) return cuda_fail(e, "ssh_prof_read");
  for (int i = 0; i < n && i < ssh::kKCount; i++) {
    if (ms) ms[i] = c.prof.ms[i];
    if (launches) launches[i] = c.prof.launches[i];
  }
  return SSH_OK;
}

}  // extern "C"
