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
// in shared memory, added into the output with one 64-bit atomic per bin and block.  ssh_g2 turns the counts into
// g_2(r) (host arithmetic over the bins).
//
// Also: the shell averages of S(k) = |n~(k)|^2 / N (Eq. structurefactor; the supplement's Fig. S1a) and the
// truncated order metric of Eq. tau from the context's last evaluation, in double-double on the device.  Shell
// membership is an exact integer decision on |n|^2 (edges ceil(b^2 n2max / nbins^2)); every shell is summed by
// one block in a fixed order (a strided pass, then a shared-memory tree), so the results are reproducible.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
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

constexpr int kSkThreads = 256;
constexpr int kSkMaxBins = 65536;

// block b < nbins: shell b; block nbins: the wavevectors beyond n2max (they enter tau only).  out[b] = (sum S,
// sum (S - 1)^2) over the shell, each a dd pair.
__global__ void __launch_bounds__(kSkThreads) k_sk_shells(const double* __restrict__ C_hi, const double* __restrict__ C_lo,
                                                          const double* __restrict__ S_hi, const double* __restrict__ S_lo,
                                                          const int32_t* __restrict__ idx, const int64_t* __restrict__ off,
                                                          double N, double* __restrict__ out) {
  __shared__ dd sh_s[kSkThreads], sh_t[kSkThreads];
  const int b = blockIdx.x, tid = threadIdx.x;
  dd as = dd_make(0.0), at = dd_make(0.0);
  for (int64_t i = off[b] + tid; i < off[b + 1]; i += kSkThreads) {
    const int32_t k = idx[i];
    const dd c = dd_make(C_hi[k], C_lo[k]), sn = dd_make(S_hi[k], S_lo[k]);
    const dd sk = dd_div(dd_add(dd_sqr(c), dd_sqr(sn)), dd_make(N));
    const dd t = dd_add_d(sk, -1.0);
    as = dd_add(as, sk);
    at = dd_add(at, dd_sqr(t));
  }
  sh_s[tid] = as;
  sh_t[tid] = at;
  __syncthreads();
  for (int w = kSkThreads / 2; w > 0; w >>= 1) {
    if (tid < w) {
      sh_s[tid] = dd_add(sh_s[tid], sh_s[tid + w]);
      sh_t[tid] = dd_add(sh_t[tid], sh_t[tid + w]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    out[4 * b + 0] = sh_s[0].hi;
    out[4 * b + 1] = sh_s[0].lo;
    out[4 * b + 2] = sh_t[0].hi;
    out[4 * b + 3] = sh_t[0].lo;
  }
}

// one block: res[2b], res[2b + 1] the mean S of shell b (0 when empty), res[2 nbins], res[2 nbins + 1] tau = scale x
// the sum of every block's sum (S - 1)^2 (shells in order, then the beyond-n2max block)
__global__ void __launch_bounds__(kSkThreads) k_sk_final(const double* __restrict__ part, const int64_t* __restrict__ off,
                                                         int nbins, dd scale, double* __restrict__ res) {
  __shared__ dd sh[kSkThreads];
  const int tid = threadIdx.x;
  dd acc = dd_make(0.0);
  for (int b = tid; b <= nbins; b += kSkThreads) {
    acc = dd_add(acc, dd_make(part[4 * b + 2], part[4 * b + 3]));
    if (b < nbins) {
      const int64_t cnt = off[b + 1] - off[b];
      const dd m = cnt > 0 ? dd_div(dd_make(part[4 * b], part[4 * b + 1]), dd_make((double)cnt)) : dd_make(0.0);
      res[2 * b] = m.hi;
      res[2 * b + 1] = m.lo;
    }
  }
  sh[tid] = acc;
  __syncthreads();
  for (int w = kSkThreads / 2; w > 0; w >>= 1) {
    if (tid < w) sh[tid] = dd_add(sh[tid], sh[tid + w]);
    __syncthreads();
  }
  if (tid == 0) {
    const dd t = dd_mul(scale, sh[0]);
    res[2 * nbins] = t.hi;
    res[2 * nbins + 1] = t.lo;
  }
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

extern "C" ssh_status ssh_structure_factor(ssh_ctx* h, int nbins, int64_t n2max, double K, int64_t* counts,
                                           double* mean, double* tau, double* k_mid) {
  using namespace ssh;
  if (!h || !counts || !mean || !tau) { set_error("ssh_structure_factor: NULL argument"); return SSH_EINVAL; }
  Ctx& c = h->c;
  if (c.shard_n > 0) { set_error("ssh_structure_factor: a particle-shard context holds only its own share"); return SSH_EINVAL; }
  if (!c.have_result) { set_error("ssh_structure_factor: no evaluation yet"); return SSH_EINVAL; }
  if (nbins < 1 || nbins > kSkMaxBins) { set_error("ssh_structure_factor: nbins must be in [1, 65536]"); return SSH_EINVAL; }
  if (n2max < 0) { set_error("ssh_structure_factor: n2max must be >= 0"); return SSH_EINVAL; }
  if (!(K >= 0) || !std::isfinite(K)) { set_error("ssh_structure_factor: K must be >= 0 and finite"); return SSH_EINVAL; }
  const int64_t M = c.M;
  const int d = c.d;
  if (n2max == 0 || K == 0) {
    // defaults: the largest |n|^2 of the set, and K = its largest |k|
    int64_t top = 0;
    for (int64_t k = 0; k < M; k++) {
      int64_t m = 0;
      for (int a = 0; a < d; a++) {
        const int64_t v = c.ks.n_int[(size_t)k * d + a];
        m += v * v;
      }
      top = std::max(top, m);
    }
    if (n2max == 0) n2max = std::max<int64_t>(top, 1);
    if (K == 0) K = 2.0 * M_PI / c.L * std::sqrt((double)std::max<int64_t>(top, 1));
  }
  // shell of every wavevector (internal order) from its exact |n|^2; bin nbins: beyond n2max
  std::vector<int64_t> E((size_t)nbins + 1);
  const unsigned __int128 den = (unsigned __int128)nbins * (unsigned __int128)nbins;
  for (int b = 0; b <= nbins; b++)
    E[b] = (int64_t)(((unsigned __int128)b * (unsigned __int128)b * (unsigned __int128)n2max + den - 1) / den);
  std::vector<int32_t> bin((size_t)M);
  std::vector<int64_t> off((size_t)nbins + 2, 0);
  for (int64_t k = 0; k < M; k++) {
    int64_t m = 0;
    for (int a = 0; a < d; a++) {
      const int64_t v = c.ks.n_int[(size_t)k * d + a];
      m += v * v;
    }
    int b = nbins;
    if (m <= n2max) {
      b = (int)(std::upper_bound(E.begin() + 1, E.begin() + nbins, m) - (E.begin() + 1));  // E_b <= m < E_(b+1)
    }
    bin[k] = b;
    off[b + 1]++;
  }
  for (int b = 0; b <= nbins; b++) off[b + 1] += off[b];
  std::vector<int32_t> idx((size_t)std::max<int64_t>(M, 1));
  {
    std::vector<int64_t> pos(off.begin(), off.end() - 1);
    for (int64_t k = 0; k < M; k++) idx[pos[bin[k]]++] = (int32_t)k;  // ascending k within a shell
  }
  // 2 (K L)^d / N^2 in dd
  dd kl = two_prod(K, c.L), scale = dd_make(2.0);
  for (int a = 0; a < d; a++) scale = dd_mul(scale, kl);
  scale = dd_div(scale, dd_mul(dd_make((double)c.N), dd_make((double)c.N)));
  cudaSetDevice(c.device);
  void *d_idx = nullptr, *d_off = nullptr, *d_part = nullptr, *d_res = nullptr;
  std::vector<double> res((size_t)2 * nbins + 2);
  cudaError_t e = cudaMalloc(&d_idx, sizeof(int32_t) * idx.size());
  if (e == cudaSuccess) e = cudaMalloc(&d_off, sizeof(int64_t) * off.size());
  if (e == cudaSuccess) e = cudaMalloc(&d_part, sizeof(double) * 4 * ((size_t)nbins + 1));
  if (e == cudaSuccess) e = cudaMalloc(&d_res, sizeof(double) * res.size());
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_idx, idx.data(), sizeof(int32_t) * idx.size(), cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess) {
    k_sk_shells<<<(unsigned)(nbins + 1), kSkThreads, 0, c.stream>>>(
        (const double*)c.C_hi.p, (const double*)c.C_lo.p, (const double*)c.S_hi.p, (const double*)c.S_lo.p,
        (const int32_t*)d_idx, (const int64_t*)d_off, (double)c.N, (double*)d_part);
    k_sk_final<<<1, kSkThreads, 0, c.stream>>>((const double*)d_part, (const int64_t*)d_off, nbins, scale, (double*)d_res);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(res.data(), d_res, sizeof(double) * res.size(), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  for (void* p : {d_idx, d_off, d_part, d_res})
    if (p) cudaFree(p);
  if (e != cudaSuccess) {
    set_error(std::string("ssh_structure_factor: ") + cudaGetErrorString(e));
    return SSH_ECUDA;
  }
  for (int b = 0; b < nbins; b++) {
    counts[b] = off[b + 1] - off[b];
    mean[2 * b] = res[2 * b];
    mean[2 * b + 1] = res[2 * b + 1];
    if (k_mid) k_mid[b] = 2.0 * M_PI / c.L * std::sqrt((double)n2max) * ((double)b + 0.5) / (double)nbins;
  }
  tau[0] = res[2 * nbins];
  tau[1] = res[2 * nbins + 1];
  return SSH_OK;
}

extern "C" ssh_status ssh_g2(int d, int64_t N, double L, int64_t n_ref, double r_max, int nbins, const uint64_t* counts,
                             double* r_mid, double* g2) {
  using namespace ssh;
  if (d < 1 || d > kMaxDim || N < 2 || !(L > 0) || n_ref < 1 || n_ref > N || !(r_max > 0) || nbins < 1 || !counts ||
      !g2) {
    set_error("ssh_g2: bad arguments");
    return SSH_EINVAL;
  }
  // volume of the unit ball in d = 1..4: pi^(d/2) / Gamma(d/2 + 1)
  const double vd[5] = {0.0, 2.0, M_PI, 4.0 * M_PI / 3.0, M_PI * M_PI / 2.0};
  const double w = r_max / nbins;
  const double dens = (double)n_ref * (double)(N - 1) / std::pow(L, d);
  for (int b = 0; b < nbins; b++) {
    const double shell = vd[d] * (std::pow((double)(b + 1), d) - std::pow((double)b, d)) * std::pow(w, d);
    g2[b] = (double)counts[b] / (dens * shell);
    if (r_mid) r_mid[b] = ((double)b + 0.5) * w;
  }
  return SSH_OK;
}
