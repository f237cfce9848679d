// ssh_internal.h -- library-private state shared by the C-ABI layer and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ssh.h"
#include "dd.cuh"
#include "kset.h"

namespace ssh {

// Byte sizes of the per-precision element types (the largest is allocated once).
constexpr size_t kTabBytes = 32;    // one complex table entry / phasor
constexpr size_t kAccBytes = 40;    // one complex partial sum
constexpr size_t kRAccBytes = 20;   // one real partial sum
constexpr int kForceThreads = 128;

struct FireBufs;  // fire.cu

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Launch {          // per-precision launch shape of the two hot kernels
  int nt_psplit = 1;     // particle splits of the collective-density kernel
  int nt_pchunk = 32;    // particles staged in shared memory per pass
  int nt_stride = 1;     // shared-memory row stride (entries), odd
  size_t nt_smem = 0;
  int f_ksplit = 1;      // column splits of the force kernel
};

// kernel ids for the event profiler (ssh_prof_*)
enum KernelId { kKTwiddle = 0, kKNtilde, kKNtReduce, kKFinalize, kKCoef, kKForce, kKFReduce, kKFire, kKCount = 16 };

struct ProfRec {
  int id;
  cudaEvent_t e0, e1;
};

struct Prof {
  bool on = false;
  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> pool;
  double ms[kKCount] = {0};
  int64_t launches[kKCount] = {0};
};

struct Ctx {
  int d = 0;
  int64_t N = 0, M = 0, Npad = 0;
  double L = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  KSet ks;
  TableLayout tl;
  NtPlan nt;
  FPlan fp;
  std::vector<int32_t> f_split;  // per precision? the same column split serves all precisions
  Launch launch[3];
  int sm_count = 148;
  // device memory
  DevBuf s_hi, s_lo;           // fractional positions, [d][N]
  DevBuf rows, slots, blocks, grows, cols, fsplit;
  DevBuf tab;                  // [nrows][Npad] table entries
  DevBuf part;                 // [psplit][M] partial sums
  DevBuf C_hi, C_lo, S_hi, S_lo;  // [M] internal order
  DevBuf coef;                 // [M]
  DevBuf blk;                  // per reduce block partials
  DevBuf scal;                 // scalars (see k_finalize)
  DevBuf fpart;                // [ksplit][d][N]
  DevBuf F_hi, F_lo;           // [d][N] physical force
  int n_red_blocks = 0;
  dd pref;                     // 4 pi / L
  bool have_positions = false;
  bool have_result = false;
  int last_prec = -1;
  bool last_force = false;
  Prof prof;
  const int* run_flag = nullptr;  // device status word: kernels return at once when it is non-zero
  dd inv_L;                       // 1 / L
  FireBufs* fire = nullptr;       // minimiser state, allocated on first ssh_minimize
};

// record an event pair around a launch when profiling is on
void prof_begin(Ctx* c, int id);
void prof_end(Ctx* c);
cudaError_t prof_collect(Ctx* c);

// device scalar block written by k_finalize (doubles)
enum { kScPhiHi = 0, kScPhiLo, kScSmaxHi, kScSmaxLo, kScCmax, kScScaleExp, kScA2MaxHi, kScA2MaxLo, kScCount = 16 };

// kernels.cu
cudaError_t plan_upload(Ctx* c);
cudaError_t eval_phi_grad(Ctx* c, int prec, bool want_force);
void setup_launch(Ctx* c);

void set_error(const std::string& msg);

// fire.cu
ssh_status minimize(Ctx* c, const ssh_min_params* p, ssh_min_result* res);
void fire_free(Ctx* c);
ssh_status fire_begin(Ctx* c, const ssh_min_params* p);
ssh_status fire_steps(Ctx* c, int prec, int64_t nsteps);
ssh_status fire_state(Ctx* c, ssh_min_result* r, int* dev_status);

}  // namespace ssh
