// post.cu -- post-processing of a configuration on the GPU: the histogram of pair distances behind the pair
// correlation function g_2(r) (the supplement's Fig. S1b shows g_2(r) of the quenched states).
//
// Distances are decided in exact integer arithmetic, so the counts are reproducible bit for bit:
//   * each fractional coordinate becomes u = floor(s_hi 2^32) (uint32; the low word of the dd position is not used),
//   * a coordinate difference is the uint32 difference read as int32, which is the minimum image in units of
//     L 2^-32, and r2 = sum_a dx_a^2 is an exact integer,
//   * with q = floor(r_max / L 2^32) (one correctly rounded division), bin b holds the pairs with
//     E_b <= r2 < E_(b+1), E_b = ceil(b^2 q^2 / nbins^2) (exact, in 128-bit integers): bins of width r_max / nbins
//     up to one unit L 2^-32.
// Pairs are ordered: (i, j) with i < n_ref (the reference particles) and j != i any particle.  Each thread owns
// one reference particle; a block stages chunks of partners in shared memory and counts into a block histogram
// in shared memory, added into the output with one 64-bit atomic per bin and block.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include "ssh_internal.h"

namespace ssh {

namespace {

constexpr int kPhThreads = 256;        // reference particles per block
constexpr int kPhTile = 256;           // partners staged per round
constexpr int64_t kPhChunk = 16384;    // partners per block
constexpr int kPhMaxBins = 4096;

__device__ __forceinline__ uint32_t quant(double s) { return __double2uint_rz(s * 4294967296.0); }

// grid (partner chunks, reference tiles); dynamic shared memory: E[nb + 1] (uint64), hist[nb] (uint32),
// partner tile [d][kPhTile] (uint32)
__global__ void __launch_bounds__(kPhThreads) k_pair_hist(const double* __restrict__ s_hi, int64_t N, int d,
                                                          int64_t nref, uint32_t q, const unsigned long long* __restrict__ E,
                                                          int nb, unsigned long long* __restrict__ counts) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* sE = reinterpret_cast<unsigned long long*>(smem);
  uint32_t* hist = reinterpret_cast<uint32_t*>(sE + nb + 1);
  uint32_t* tile = hist + nb;
  const int tid = threadIdx.x;
  for (int b = tid; b <= nb; b += kPhThreads) sE[b] = E[b];
  for (int b = tid; b < nb; b += kPhThreads) hist[b] = 0;
  const int64_t i = (int64_t)blockIdx.y * kPhThreads + tid;
  uint32_t qi[4] = {0, 0, 0, 0};
  if (i < nref)
    for (int a = 0; a < d; a++) qi[a] = quant(s_hi[(int64_t)a * N + i]);
  const float inv_w = (float)nb / (float)q;
  const int64_t j_begin = (int64_t)blockIdx.x * kPhChunk;
  const int64_t j_end = j_begin + kPhChunk < N ? j_begin + kPhChunk : N;
  for (int64_t j0 = j_begin; j0 < j_end; j0 += kPhTile) {
    __syncthreads();  // the previous tile is consumed (and, first time, E and hist are set)
    const int64_t jt = j0 + tid;
    if (jt < j_end)
      for (int a = 0; a < d; a++) tile[a * kPhTile + tid] = quant(s_hi[(int64_t)a * N + jt]);
    __syncthreads();
    if (i >= nref) continue;
    const int cnt = (int)(j_end - j0 < kPhTile ? j_end - j0 : kPhTile);
    for (int t = 0; t < cnt; t++) {
      if (j0 + t == i) continue;
      unsigned long long r2 = 0;
      bool in = true;
      for (int a = 0; a < d; a++) {
        const int32_t dx = (int32_t)(qi[a] - tile[a * kPhTile + t]);  // minimum image, exact
        const uint32_t ax = dx < 0 ? (uint32_t)(-(int64_t)dx) : (uint32_t)dx;
        in = in && ax < q;                         // |dx| < q < 2^31: the sum below cannot overflow
        r2 += (unsigned long long)ax * ax;
      }
      if (!in || r2 >= sE[nb]) continue;
      int b = (int)(sqrtf((float)r2) * inv_w);    // a guess, corrected exactly against the integer edges
      b = b < 0 ? 0 : (b >= nb ? nb - 1 : b);
      while (b > 0 && r2 < sE[b]) b--;
      while (b + 1 < nb && r2 >= sE[b + 1]) b++;
      atomicAdd(&hist[b], 1u);
    }
  }
  __syncthreads();
  for (int b = tid; b < nb; b += kPhThreads)
    if (hist[b]) atomicAdd(&counts[b], (unsigned long long)hist[b]);
}

}  // namespace

}  // namespace ssh

extern "C" ssh_status ssh_pair_histogram(ssh_ctx* h, int64_t n_ref, double r_max, int nbins, uint64_t* counts) {
  using namespace ssh;
  if (!h || !counts) { set_error("ssh_pair_histogram: NULL argument"); return SSH_EINVAL; }
  Ctx& c = h->c;
  if (n_ref < 1 || n_ref > c.N) { set_error("ssh_pair_histogram: n_ref must be in [1, N]"); return SSH_EINVAL; }
  if (nbins < 1 || nbins > kPhMaxBins) { set_error("ssh_pair_histogram: nbins must be in [1, 4096]"); return SSH_EINVAL; }
  if (!(r_max > 0) || !(r_max < 0.5 * c.L)) { set_error("ssh_pair_histogram: need 0 < r_max < L / 2"); return SSH_EINVAL; }
  const double qd = std::floor(r_max / c.L * 4294967296.0);
  if (qd < 1.0) { set_error("ssh_pair_histogram: r_max below the position resolution L 2^-32"); return SSH_EINVAL; }
  const uint32_t q = (uint32_t)qd;
  std::vector<unsigned long long> E((size_t)nbins + 1);
  const unsigned __int128 den = (unsigned __int128)nbins * (unsigned __int128)nbins;
  for (int b = 0; b <= nbins; b++) {
    const unsigned __int128 num = (unsigned __int128)b * b * (unsigned __int128)q * q;
    E[b] = (unsigned long long)((num + den - 1) / den);
  }
  cudaSetDevice(c.device);
  void* dE = nullptr;
  void* dC = nullptr;
  cudaError_t e = cudaMalloc(&dE, sizeof(unsigned long long) * E.size());
  if (e == cudaSuccess) e = cudaMalloc(&dC, sizeof(unsigned long long) * nbins);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dE, E.data(), sizeof(unsigned long long) * E.size(), cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(dC, 0, sizeof(unsigned long long) * nbins, c.stream);
  if (e == cudaSuccess) {
    const dim3 grid((unsigned)((c.N + kPhChunk - 1) / kPhChunk), (unsigned)((n_ref + kPhThreads - 1) / kPhThreads));
    const size_t smem = sizeof(unsigned long long) * (nbins + 1) + sizeof(uint32_t) * nbins + sizeof(uint32_t) * 4 * kPhTile;
    if (smem > 48 * 1024) e = cudaFuncSetAttribute(k_pair_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      k_pair_hist<<<grid, kPhThreads, smem, c.stream>>>((const double*)c.s_hi.p, c.N, c.d, n_ref, q,
                                                        (const unsigned long long*)dE, nbins, (unsigned long long*)dC);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(counts, dC, sizeof(unsigned long long) * nbins, cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (dE) cudaFree(dE);
  if (dC) cudaFree(dC);
  if (e != cudaSuccess) {
    set_error(std::string("ssh_pair_histogram: ") + cudaGetErrorString(e));
    return SSH_ECUDA;
  }
  return SSH_OK;
}
