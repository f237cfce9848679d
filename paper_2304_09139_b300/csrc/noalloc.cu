// noalloc.cu -- an allocation-free variant of the collective-density kernel, for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at all: a host program that hands all of a GPU's memory to another
// framework's pool or arena at start-up (a foreign cudaMalloc then fails, or fragments the pool and escapes its
// accounting), and real-time or embedded loops that must not allocate after start-up (cudaMalloc and cudaFree
// can synchronise the device and take unbounded time).  For them ssh_ntilde_noalloc computes n~(k) = C + i S
// with caller-owned inputs and outputs and keeps its working memory in the fixed device array below instead of
// allocating.
//
// The array g_noalloc_scratch (kNoAllocScratchBytes = 8 MiB) exists once per device in every process that
// loads the library and is held until the process exits.  It holds the positions converted to Q0.128
// turns (N d 16 bytes) followed by the per-particle-split partial sums (splits x M x 40 bytes); calls whose
// N d 16 + M 40 exceeds it are rejected with SSH_EINVAL.  All calls on a device share the one array and it
// keeps the last call's contents: every slot a call reads is written earlier in that same call, so nothing
// has to start at zero, but two calls whose kernels overlap on the GPU (different streams, or different
// host threads) race on the array and corrupt each other's results.  Serialise such calls.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "fx.cuh"
#include "ssh_internal.h"

#define SSH_TABLE_QUAL __device__
#include "gen/tables.h"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;
constexpr int kNoAllocThreads = 128;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NaAcc {
  q160 re, im;
};

// Host-side device address of g_noalloc_scratch and the device's SM count, looked up once per device.
std::mutex g_na_mutex;
void* g_na_ptr[kNoAllocMaxDevices] = {nullptr};
int g_na_sms[kNoAllocMaxDevices] = {0};

__global__ void k_na_turns(int64_t nd, const double* __restrict__ s_hi, const double* __restrict__ s_lo,
                           q128* __restrict__ u) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  u[i] = turns_from_dd(s_hi[i], s_lo ? s_lo[i] : 0.0);
}

// One thread per wavevector, one grid row per particle split: e^{2 pi i n.s_j} from the exact Q0.128 phase
// and the table + Taylor sincos, summed exactly in Q34.126.
__global__ void __launch_bounds__(kNoAllocThreads) k_na_ntilde(int d, int64_t N, int64_t M, const q128* __restrict__ u,
                                                               const int32_t* __restrict__ n, int64_t plen,
                                                               NaAcc* __restrict__ part) {
  const int64_t k = (int64_t)blockIdx.x * kNoAllocThreads + threadIdx.x;
  if (k >= M) return;
  int32_t nk[ssh::kMaxDim] = {0, 0, 0, 0};
#pragma unroll
  for (int a = 0; a < ssh::kMaxDim; a++)
    if (a < d) nk[a] = n[k * d + a];
  q128 piq;
#pragma unroll
  for (int i = 0; i < 4; i++) piq.w[i] = SSH_FX_PI_Q3_125[i];
  NaAcc acc;
  acc.re = q160_zero();
  acc.im = q160_zero();
  const int64_t j0 = (int64_t)blockIdx.y * plen, j1 = min(N, j0 + plen);
  for (int64_t j = j0; j < j1; j++) {
    unsigned __int128 t = 0;
#pragma unroll
    for (int a = 0; a < ssh::kMaxDim; a++) {
      if (a < d) {
        q128 v = u[j * d + a];
        unsigned __int128 w = ((unsigned __int128)v.w[3] << 96) | ((unsigned __int128)v.w[2] << 64) |
                              ((unsigned __int128)v.w[1] << 32) | (unsigned __int128)v.w[0];
        t += w * (unsigned __int128)(__int128)nk[a];  // exact modulo one turn
      }
    }
    fxc z = fx_sincos_turns(q128_from_i128((__int128)t), SSH_FX_TAB_A, SSH_FX_TAB_B, piq, SSH_FX_INV_FACT);
    q160_add(acc.re, z.re);
    q160_add(acc.im, z.im);
  }
  part[(int64_t)blockIdx.y * M + k] = acc;
}

__global__ void k_na_reduce(int64_t M, int psplit, const NaAcc* __restrict__ part, double* C_hi, double* C_lo,
                            double* S_hi, double* S_lo) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  NaAcc a = part[k];
  for (int p = 1; p < psplit; p++) {
    q160_add160(a.re, part[(int64_t)p * M + k].re);
    q160_add160(a.im, part[(int64_t)p * M + k].im);
  }
  double h, l;
  q160_to_dd(a.re, &h, &l);
  C_hi[k] = h;
  C_lo[k] = l;
  q160_to_dd(a.im, &h, &l);
  S_hi[k] = h;
  S_lo[k] = l;
}

}  // namespace

extern "C" ssh_status ssh_ntilde_noalloc(int d, int64_t N, int64_t M, const double* s_hi, const double* s_lo,
                                         const int32_t* n, double* C_hi, double* C_lo, double* S_hi, double* S_lo,
                                         void* stream) {
  if (d < 1 || d > ssh::kMaxDim || N < 1 || M < 0 || !s_hi || (M > 0 && (!n || !C_hi || !C_lo || !S_hi || !S_lo))) {
    ssh::set_error("ssh_ntilde_noalloc: bad arguments");
    return SSH_EINVAL;
  }
  if (N > ((int64_t)1 << 31) || M > ((int64_t)1 << 31)) {
    ssh::set_error("ssh_ntilde_noalloc: N or M too large");
    return SSH_EINVAL;
  }
  const size_t pos_bytes = ((size_t)N * d * sizeof(q128) + 255) / 256 * 256;
  const size_t acc_bytes = (size_t)M * sizeof(NaAcc);
  if (pos_bytes + acc_bytes > kNoAllocScratchBytes) {
    ssh::set_error("ssh_ntilde_noalloc: N*d*16 + M*40 bytes exceeds the fixed 8 MiB device scratch "
                   "(use ssh_create / ssh_eval for larger problems)");
    return SSH_EINVAL;
  }
  if (M == 0) return SSH_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    ssh::set_error(std::string("ssh_ntilde_noalloc: no usable current device: ") + cudaGetErrorString(e));
    return SSH_ECUDA;
  }
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    ssh::set_error("ssh_ntilde_noalloc: device index " + std::to_string(dev) + " is not supported (at most " +
                   std::to_string(kNoAllocMaxDevices - 1) + ")");
    return SSH_ECUDA;
  }
  void* base = nullptr;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_ptr[dev]) {
      // first call on this device: the host-side name is not a device address, ask the runtime for it
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        ssh::set_error(std::string("ssh_ntilde_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        return SSH_ECUDA;
      }
      int n_sm = 0;
      e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess || n_sm < 1) {
        ssh::set_error(std::string("ssh_ntilde_noalloc: SM count query failed: ") + cudaGetErrorString(e));
        return SSH_ECUDA;
      }
      g_na_sms[dev] = n_sm;
      g_na_ptr[dev] = p;
    }
    base = g_na_ptr[dev];
    sms = g_na_sms[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  q128* u = reinterpret_cast<q128*>(base);
  NaAcc* part = reinterpret_cast<NaAcc*>(reinterpret_cast<unsigned char*>(base) + pos_bytes);
  const size_t avail = kNoAllocScratchBytes - pos_bytes;  // >= acc_bytes, checked above
  // particle splits: enough blocks for two per SM, as many as the scratch holds
  const int64_t kblocks = (M + kNoAllocThreads - 1) / kNoAllocThreads;
  int64_t psplit = (2 * (int64_t)sms + kblocks - 1) / kblocks;
  psplit = std::min<int64_t>(psplit, (int64_t)(avail / acc_bytes));
  psplit = std::max<int64_t>(1, std::min<int64_t>(psplit, N));
  const int64_t plen = (N + psplit - 1) / psplit;
  psplit = (N + plen - 1) / plen;
  const int64_t nd = N * d;
  k_na_turns<<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(nd, s_hi, s_lo, u);
  dim3 grid((unsigned)kblocks, (unsigned)psplit);
  k_na_ntilde<<<grid, kNoAllocThreads, 0, st>>>(d, N, M, u, n, plen, part);
  k_na_reduce<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(M, (int)psplit, part, C_hi, C_lo, S_hi, S_lo);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    ssh::set_error(std::string("ssh_ntilde_noalloc: launch failed: ") + cudaGetErrorString(e));
    return SSH_ECUDA;
  }
  return SSH_OK;
}
