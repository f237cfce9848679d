// shard.cu -- one configuration's particles split into shards, one per GPU, with the exchanges left to the caller.
//
// Both sums of a step are reductions over the particles (Simulations), so a shard evaluates n~ over its own
// particles and the shards' partial sums add up to the whole configuration's.  On the tensor-core path the partial
// sums are the exact integer level groups of the density GEMM's tile accumulators, so adding them (an all-reduce
// of int64 words, in any order) gives every shard the very accumulators one unsharded context would hold; the
// density finish, the force coefficients and each shard's own forces then follow bit for bit.  A FIRE step has
// one more exchange: the dot products F.v, F.F, v.v, as partial sums per chunk of 2048 particles of an axis (the
// shard boundaries lie on chunk boundaries, so each chunk's partial belongs to one shard and the element-wise sum
// over shards reproduces the unsharded partials exactly).  A step is therefore
//   ssh_shard_step_dots  -> exchange (binary64 sum) -> ssh_shard_step_move  -> exchange (int64 sum)
//                        -> ssh_shard_step_finish
// and every shard takes the same acceptance, stop and stage decisions.  Nothing here talks to another GPU: the
// caller moves the buffers (NCCL all-reduce, or a sum in one process), on the context's stream or after ssh_sync.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "ssh_internal.h"

using ssh::Ctx;
using ssh::set_error;

namespace {

bool shard_ctx(const ssh_ctx* h, const char* fn) {
  if (!h) {
    set_error(std::string(fn) + ": NULL context");
    return false;
  }
  if (h->c.shard_n == 0 || !h->c.tc.on) {
    set_error(std::string(fn) + ": not a particle-shard context (ssh_opts.shard_count)");
    return false;
  }
  return true;
}

ssh_status fail(cudaError_t e, const char* fn) {
  set_error(std::string(fn) + ": " + cudaGetErrorString(e));
  return SSH_ECUDA;
}

// zero the tile accumulators, run the density GEMMs of the shard's chunks into them, copy them out
cudaError_t density_out(Ctx& c, const ssh::EngineView& v, int64_t* out) {
  long long* acc = ssh::tc_acc_ptr(&c);
  const size_t bytes = sizeof(long long) * (size_t)ssh::tc_acc_words(&c);
  cudaError_t e = cudaMemsetAsync(acc, 0, bytes, c.stream);
  if (e == cudaSuccess) e = ssh::tc_launch_density_gemms(v, c.stream, &c.prof);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, acc, bytes, cudaMemcpyDeviceToDevice, c.stream);
  return e;
}

// the summed accumulators back in place, then the density finish (Phi, S_max, n~, the scale) and the force
cudaError_t finish_in(Ctx& c, const ssh::EngineView& v, const int64_t* tot, bool want_force) {
  long long* acc = ssh::tc_acc_ptr(&c);
  const size_t bytes = sizeof(long long) * (size_t)ssh::tc_acc_words(&c);
  cudaError_t e = cudaMemcpyAsync(acc, tot, bytes, cudaMemcpyDeviceToDevice, c.stream);
  if (e == cudaSuccess) e = ssh::tc_launch_dens_finish(v, c.stream, &c.prof);
  if (e == cudaSuccess && want_force) e = ssh::tc_launch_force(v, c.stream, &c.prof);
  if (e == cudaSuccess && want_force) e = ssh::tc_launch_force_finish(v, c.stream, &c.prof);
  return e;
}

bool fire_running(const ssh_ctx* h, const char* fn) {
  if (!ssh::fire_begun(&h->c)) {
    set_error(std::string(fn) + ": call ssh_shard_fire_begin first");
    return false;
  }
  return true;
}

}  // namespace

extern "C" {

ssh_status ssh_shard_words(const ssh_ctx* h, int64_t* dens_words, int64_t* dots_words) {
  if (!shard_ctx(h, "ssh_shard_words")) return SSH_EINVAL;
  if (dens_words) *dens_words = ssh::tc_acc_words(&h->c);
  if (dots_words) *dots_words = 3 * ssh::dot_chunks(h->c.d, h->c.N);
  return SSH_OK;
}

ssh_status ssh_shard_density(ssh_ctx* h, int64_t* dens_out) {
  if (!shard_ctx(h, "ssh_shard_density")) return SSH_EINVAL;
  Ctx& c = h->c;
  if (!c.have_positions || !dens_out) {
    set_error("ssh_shard_density: no positions set, or a NULL buffer");
    return SSH_EINVAL;
  }
  cudaSetDevice(c.device);
  const cudaError_t e = density_out(c, c.eng->view[SSH_FX], dens_out);
  return e == cudaSuccess ? SSH_OK : fail(e, "ssh_shard_density");
}

ssh_status ssh_shard_finish(ssh_ctx* h, const int64_t* dens_total, int want_force) {
  if (!shard_ctx(h, "ssh_shard_finish")) return SSH_EINVAL;
  Ctx& c = h->c;
  if (!c.have_positions || !dens_total) {
    set_error("ssh_shard_finish: no positions set, or a NULL buffer");
    return SSH_EINVAL;
  }
  cudaSetDevice(c.device);
  const cudaError_t e = finish_in(c, c.eng->view[SSH_FX], dens_total, want_force != 0);
  if (e != cudaSuccess) return fail(e, "ssh_shard_finish");
  c.have_result = true;
  c.last_prec = SSH_FX;
  c.last_force = want_force != 0;
  return SSH_OK;
}

ssh_status ssh_shard_fire_begin(ssh_ctx* h, const ssh_min_params* pin) {
  if (!shard_ctx(h, "ssh_shard_fire_begin")) return SSH_EINVAL;
  Ctx& c = h->c;
  if (!c.have_result || !c.last_force || c.last_prec != SSH_FX) {
    set_error("ssh_shard_fire_begin: needs the results of an ssh_shard_finish with the force");
    return SSH_EINVAL;
  }
  ssh_min_params p;
  ssh_status st = ssh::complete_params(h, pin, &p);
  if (st != SSH_OK) return st;
  if (p.method != SSH_MIN_FIRE || p.n_stages != 1 || p.stage_prec[0] != SSH_FX) {
    set_error("ssh_shard_fire_begin: sharded runs are FIRE in one fixed-point stage");
    return SSH_EINVAL;
  }
  cudaSetDevice(c.device);
  return ssh::fire_begin_from_results(&c, &p);
}

ssh_status ssh_shard_step_dots(ssh_ctx* h, double* dots_out) {
  if (!shard_ctx(h, "ssh_shard_step_dots") || !fire_running(h, "ssh_shard_step_dots")) return SSH_EINVAL;
  if (!dots_out) { set_error("ssh_shard_step_dots: NULL buffer"); return SSH_EINVAL; }
  Ctx& c = h->c;
  cudaSetDevice(c.device);
  ssh::Engine* E = nullptr;
  cudaError_t e = ssh::fire_engine_for(&c, SSH_FX, &E);
  if (e == cudaSuccess) e = ssh::fire_dots_partials(E, dots_out, c.stream);
  return e == cudaSuccess ? SSH_OK : fail(e, "ssh_shard_step_dots");
}

ssh_status ssh_shard_step_move(ssh_ctx* h, const double* dots_total, int64_t* dens_out) {
  if (!shard_ctx(h, "ssh_shard_step_move") || !fire_running(h, "ssh_shard_step_move")) return SSH_EINVAL;
  if (!dots_total || !dens_out) { set_error("ssh_shard_step_move: NULL buffer"); return SSH_EINVAL; }
  Ctx& c = h->c;
  cudaSetDevice(c.device);
  ssh::Engine* E = nullptr;
  cudaError_t e = ssh::fire_engine_for(&c, SSH_FX, &E);
  if (e == cudaSuccess) e = ssh::fire_control_move(E, dots_total, c.stream);
  if (e == cudaSuccess) e = density_out(c, E->view[SSH_FX], dens_out);
  return e == cudaSuccess ? SSH_OK : fail(e, "ssh_shard_step_move");
}

ssh_status ssh_shard_step_finish(ssh_ctx* h, const int64_t* dens_total) {
  if (!shard_ctx(h, "ssh_shard_step_finish") || !fire_running(h, "ssh_shard_step_finish")) return SSH_EINVAL;
  if (!dens_total) { set_error("ssh_shard_step_finish: NULL buffer"); return SSH_EINVAL; }
  Ctx& c = h->c;
  cudaSetDevice(c.device);
  ssh::Engine* E = nullptr;
  cudaError_t e = ssh::fire_engine_for(&c, SSH_FX, &E);
  if (e == cudaSuccess) e = finish_in(c, E->view[SSH_FX], dens_total, true);
  if (e == cudaSuccess) e = ssh::fire_accept_restore(E, c.stream);
  if (e != cudaSuccess) return fail(e, "ssh_shard_step_finish");
  c.have_result = false;  // as after ssh_fire_steps: the result buffers hold the last trial
  return SSH_OK;
}

}  // extern "C"
