// pipes.cu -- measured instruction rates of the pipes this library's arithmetics run on.
//
// The roofline denominators of the FP64 (double-double) and integer (fixed-point) kernels are instruction rates,
// not bytes or tensor FLOPs, and the part's nominal figures are not a measurement.  ssh_pipe_rate times a kernel
// that keeps every SM busy with independent chains of one operation and reports operations per second:
//   SSH_PIPE_FP64_FMA  fma.rn.f64                                 (the dd kernels' pipe)
//   SSH_PIPE_FP32_FMA  fma.rn.f32
//   SSH_PIPE_IMAD      mad.lo.u32 (32-bit integer multiply-add)     (the fixed-point kernels' pipe)
//   SSH_PIPE_IMAD_HI   mad.hi.u32 (high half of the 64-bit product, plus an addend)
//   SSH_PIPE_DD_CMAC   one complex double-double multiply and complex add (ddc_mul + ddc_add of dd.cuh)
//   SSH_PIPE_FX_CMUL   one product of first-quadrant 128-bit fixed-point phasors (qmul of fx.cuh)
// Each thread runs kChains independent chains so that the pipe, not the latency of one chain, limits the rate;
// the grid is 8 CTAs of 256 threads per SM.  Results feed a conditional store, so no chain is optimised away.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "dd.cuh"
#include "fx.cuh"
#include "ssh_internal.h"

namespace {

constexpr int kPipeThreads = 256;
constexpr int kPipeCtasPerSm = 8;

template <int KIND>
struct PipeOp;

template <>
struct PipeOp<SSH_PIPE_FP64_FMA> {
  static constexpr int kChains = 8, kUnroll = 8;
  double v[kChains];
  __device__ void init(uint32_t t) {
#pragma unroll
    for (int i = 0; i < kChains; i++) v[i] = 1.0 + 1e-9 * (double)(t + i);
  }
  __device__ void step(double b, double c) {
#pragma unroll
    for (int i = 0; i < kChains; i++) v[i] = fma(v[i], b, c);
  }
  __device__ double result() const {
    double s = 0;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += v[i];
    return s;
  }
};

template <>
struct PipeOp<SSH_PIPE_FP32_FMA> {
  static constexpr int kChains = 8, kUnroll = 8;
  float v[kChains];
  __device__ void init(uint32_t t) {
#pragma unroll
    for (int i = 0; i < kChains; i++) v[i] = 1.0f + 1e-6f * (float)(t + i);
  }
  __device__ void step(double b, double c) {
    const float fb = (float)b, fc = (float)c;
#pragma unroll
    for (int i = 0; i < kChains; i++) v[i] = fmaf(v[i], fb, fc);
  }
  __device__ double result() const {
    double s = 0;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += v[i];
    return s;
  }
};

template <>
struct PipeOp<SSH_PIPE_IMAD> {
  static constexpr int kChains = 8, kUnroll = 8;
  uint32_t v[kChains];
  uint32_t m = 0, a = 0;
  __device__ void init(uint32_t t) {
#pragma unroll
    for (int i = 0; i < kChains; i++) v[i] = t * 2654435761u + (uint32_t)i;
    m = 0x9E3779B1u ^ t;
    a = 0x7F4A7C15u + t;
  }
  __device__ void step(double, double) {
#pragma unroll
    for (int i = 0; i < kChains; i++) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(v[i]) : "r"(m), "r"(a));
  }
  __device__ double result() const {
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kChains; i++) s ^= v[i];
    return (double)s;
  }
};

template <>
struct PipeOp<SSH_PIPE_IMAD_HI> {
  static constexpr int kChains = 8, kUnroll = 8;
  uint32_t v[kChains];
  uint32_t m = 0, a = 0;
  __device__ void init(uint32_t t) {
#pragma unroll
    for (int i = 0; i < kChains; i++) v[i] = t * 2654435761u + (uint32_t)i;
    m = 0x9E3779B1u ^ t;
    a = 0x7F4A7C15u + t;
  }
  __device__ void step(double, double) {
#pragma unroll
    for (int i = 0; i < kChains; i++) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(v[i]) : "r"(m), "r"(a));
  }
  __device__ double result() const {
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kChains; i++) s ^= v[i];
    return (double)s;
  }
};

template <>
struct PipeOp<SSH_PIPE_DD_CMAC> {
  static constexpr int kChains = 2, kUnroll = 2;
  ddc acc[kChains], z[kChains];
  __device__ void init(uint32_t t) {
#pragma unroll
    for (int i = 0; i < kChains; i++) {
      const double x = 1e-3 * (double)((t + i) & 1023);
      z[i] = ddc_make(dd_make(cos(x), 1e-20), dd_make(sin(x), -1e-20));
      acc[i] = ddc_make(dd_make(0.0), dd_make(0.0));
    }
  }
  __device__ void step(double, double) {
#pragma unroll
    for (int i = 0; i < kChains; i++) {
      z[i] = ddc_mul(z[i], z[i ^ 1]);
      acc[i] = ddc_add(acc[i], z[i]);
    }
  }
  __device__ double result() const {
    double s = 0;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += acc[i].re.hi + acc[i].im.lo;
    return s;
  }
};

template <>
struct PipeOp<SSH_PIPE_FX_CMUL> {
  static constexpr int kChains = 2, kUnroll = 2;
  qent z[kChains], b;
  __device__ void init(uint32_t t) {
#pragma unroll
    for (int i = 0; i < kChains; i++) {
#pragma unroll
      for (int w = 0; w < 4; w++) {
        z[i].c.w[w] = 0x6A09E667u + 977u * (t + i + w);
        z[i].s.w[w] = 0x3C6EF372u + 131u * (t + i + w);
      }
      z[i].c.w[3] &= 0x7FFFFFFFu;
      z[i].s.w[3] &= 0x3FFFFFFFu;
      z[i].cs = q128_add(z[i].c, z[i].s);
    }
    b = z[0];
  }
  __device__ void step(double, double) {
#pragma unroll
    for (int i = 0; i < kChains; i++) z[i] = qmul(z[i], b);
  }
  __device__ double result() const {
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kChains; i++) s ^= z[i].c.w[3] ^ z[i].s.w[0] ^ z[i].cs.w[0];
    return (double)s;
  }
};

template <int KIND>
__global__ void __launch_bounds__(kPipeThreads) k_pipe(long long iters, double b, double c, long long key, double* sink) {
  PipeOp<KIND> op;
  op.init(blockIdx.x * kPipeThreads + threadIdx.x);
  for (long long it = 0; it < iters; it++) {
#pragma unroll
    for (int u = 0; u < PipeOp<KIND>::kUnroll; u++) op.step(b, c);
  }
  // a store under a condition the compiler cannot decide (key is a run-time value that no result matches in
  // practice) keeps every chain live; a constant there would let it prove the store dead and drop the work
  const double r = op.result();
  if (__double_as_longlong(r) == key) sink[0] = r;
}

template <int KIND>
cudaError_t time_pipe(int sms, long long iters, double* sink, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
  if (e == cudaSuccess) {
    k_pipe<KIND><<<sms * kPipeCtasPerSm, kPipeThreads>>>(iters, 0.9999999, 1e-7, 0x7ff4dead5eed1234ll, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

// Operations per second of one kind: a short run sizes the timed run to about 100 ms, which is timed three times
// (the best is kept: the clock ramps during the first).
template <int KIND>
cudaError_t pipe_rate(int sms, double* sink, double* per_s, double* ms_out) {
  float ms = 0;
  long long iters = 64;
  cudaError_t e = time_pipe<KIND>(sms, iters, sink, &ms);
  for (int g = 0; e == cudaSuccess && ms < 10.0f && g < 10; g++) {
    iters *= 4;
    e = time_pipe<KIND>(sms, iters, sink, &ms);
  }
  if (e != cudaSuccess) return e;
  if (ms < 10.0f) return cudaErrorUnknown;  // the work did not scale with the iterations: no rate to report
  iters = (long long)((double)iters * 100.0 / (double)ms) + 1;
  float best = 0;
  for (int r = 0; r < 3 && e == cudaSuccess; r++) {
    e = time_pipe<KIND>(sms, iters, sink, &ms);
    if (r == 0 || ms < best) best = ms;
  }
  if (e != cudaSuccess) return e;
  const double ops = (double)sms * kPipeCtasPerSm * kPipeThreads * (double)iters * PipeOp<KIND>::kUnroll *
                     PipeOp<KIND>::kChains;
  *per_s = ops / (best * 1e-3);
  *ms_out = best;
  return cudaSuccess;
}

}  // namespace

extern "C" ssh_status ssh_pipe_rate(int device, int kind, double* ops_per_s, double* ms) {
  if (!ops_per_s || kind < 0 || kind > SSH_PIPE_FX_CMUL) {
    ssh::set_error("ssh_pipe_rate: bad arguments");
    return SSH_EINVAL;
  }
  int cur = 0;
  cudaError_t e = cudaGetDevice(&cur);
  if (e == cudaSuccess && cur != device) e = cudaSetDevice(device);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  double* sink = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(double));
  double r = 0, t = 0;
  if (e == cudaSuccess) {
    switch (kind) {
      case SSH_PIPE_FP64_FMA: e = pipe_rate<SSH_PIPE_FP64_FMA>(sms, sink, &r, &t); break;
      case SSH_PIPE_FP32_FMA: e = pipe_rate<SSH_PIPE_FP32_FMA>(sms, sink, &r, &t); break;
      case SSH_PIPE_IMAD: e = pipe_rate<SSH_PIPE_IMAD>(sms, sink, &r, &t); break;
      case SSH_PIPE_IMAD_HI: e = pipe_rate<SSH_PIPE_IMAD_HI>(sms, sink, &r, &t); break;
      case SSH_PIPE_DD_CMAC: e = pipe_rate<SSH_PIPE_DD_CMAC>(sms, sink, &r, &t); break;
      default: e = pipe_rate<SSH_PIPE_FX_CMUL>(sms, sink, &r, &t); break;
    }
  }
  if (sink) cudaFree(sink);
  if (cur != device) cudaSetDevice(cur);
  if (e != cudaSuccess) {
    ssh::set_error(std::string("ssh_pipe_rate: ") + cudaGetErrorString(e));
    return SSH_ECUDA;
  }
  *ops_per_s = r;
  if (ms) *ms = t;
  return SSH_OK;
}
