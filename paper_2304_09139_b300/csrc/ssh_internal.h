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

// work item of the tensor-core GEMM (tc.cu): one CTA
struct TcItem {
  int32_t cfg, kind;    // kind 0: density tile, 1: force tile
  int32_t a, b;         // row tile (density) / particle tile (force); column tile
  int32_t ks0, nks;     // K-step range
  int32_t slot, pad;    // density: partial slot (tile * ksplit + split)
};

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
enum KernelId {
  kKTwiddle = 0, kKNtilde, kKNtReduce, kKFinalize, kKCoef, kKForce, kKFReduce, kKFire,
  kKTcPrep, kKTcDens, kKTcFinish, kKTcCoef, kKTcForce, kKTcTables, kKCount = 16
};

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

// ---- device-side view of one configuration: every pointer and size a kernel needs.  A single context is
// a batch of one; a batch concatenates the descriptors of its members.
struct CfgDev {
  int d, nrows, lo_base, hi_base, qmin, ksplit, nblk, nb_fire;
  int psplit[3], pchunk[3];
  int64_t N, M, Npad;
  int64_t plen[3];
  double* s_hi;
  double* s_lo;
  const TabRow* rows;
  const NtSlot* slots;
  const NtBlock* blocks;
  const int32_t* g_rows;
  const FCol* cols;
  const int32_t* fsplit;
  void* tab;
  void* part;
  double *C_hi, *C_lo, *S_hi, *S_lo;
  const double* wk;  // [M] internal order: the weight v~(k) of each wavevector in Phi and F (1 by default)
  void* coef;
  void* blk;
  double* scal;
  void* fpart;
  double *F_hi, *F_lo;
  dd pref, inv_L;
  // tensor-core fixed-point path (tc.cu); tc = 0 when the configuration uses the integer-pipe kernels
  int tc, tc_R1, tc_nP, tc_RT, tc_CTd, tc_PT, tc_KSf, tc_CTf, tc_bexp, tc_nblk, tc_gs, tc_ts, tc_ntab;
  int tc_d, tc_lift;   // the path's number of axes (2, 3 or 4); d = 1 on two lifted axes: n = 2^tc_lift n1 + n2
  // two-axis path: the last row tile's canonical p (those >= tc_trP0) run as one transposed density tile, rows
  // (n1, cos / sin) of a_j(n1) for n1 < tc_trN1 from local row tc_trRow0 of that row tile, columns (p, cos / sin)
  int tc_tr, tc_trP0, tc_trRow0, tc_trN1;
  int tc_Rax[4];       // per axis: powers 0..tc_Rax[a] in the tables
  int64_t tc_KS, tc_NJ, tc_NPg;  // density K-steps; particle groups and row groups of the digit tensor (a chunk)
  int64_t tc_j0, tc_n, tc_nbuf;  // this chunk: first particle, particles, particle stride of the chunk buffers
  uint8_t *tc_wT, *tc_aB, *tc_fB;  // digit tensor of w_j(p); density B (a_j(n1)); force B (coefficients)
  void* tc_a1;         // a_j(n1) as signed Q2.126, [n1][j]
  void* tc_tab;        // per (axis, particle): first-quadrant tables e^{2 pi i k s} (k < 8), e^{2 pi i 8 b s}
  long long* tc_acc;   // density level groups per tile [tile][3][32][128], summed by integer atomics
  long long* tc_facc;  // force limbs [axis][3][N], summed by integer atomics
  const int32_t* tc_em;       // [p][n1][2]: internal k index of (n1, +-p), or -1
  const int32_t* tc_pvec;     // [p]: (n2 & 0xffff) | (n3 << 16); four axes: 10-bit fields n2 | n3 << 10 | n4 << 20
  const int32_t* tc_tilemap;  // [RT][CTd] -> tile slot, or -1
  const void* tc_tmap;        // two 128-byte tensor maps of the digit tensor: density box, force box
  int* tc_err;
  // minimiser state (null when the context has not minimised yet)
  double L;  // box length
  double *lb_S, *lb_Y, *lb_G, *lb_P, *lb_part;  // L-BFGS: history [pair][d N], gradient, direction, partials
  void* lb_mat;
  void* fs;
  double *v_hi, *v_lo, *bs_hi, *bs_lo, *bF_hi, *bF_lo, *fdots;  // fdots: [3][n_dchunk] FIRE dot partials
  int n_dchunk;    // chunks of the FIRE dot products: d ceil(N / kDotChunk)
  const int* run;  // status word that turns this configuration's kernels into no-ops when non-zero, or null
};

// compact launch grid over several configurations: block b of a launch works on block blk of configuration cfg
// (only the blocks each configuration needs are launched)
struct BlockMap {
  int32_t cfg, blk;
};

// work items of the persistent kernels and of the twiddle kernel
struct TwItem {
  int32_t cfg, pad;
  int64_t start;  // first table entry of a 128-entry block
};
struct NtItem {
  int32_t cfg, blk, ps, pad;  // k-block, particle split
};
struct FItem {
  int32_t cfg, pb, ks, pad;   // particle block, column split
};
constexpr int kTwThreads = 128;

// launch view of an engine (device pointers, counts, grid extents) for one precision
constexpr int kMaxTcPhases = 64;  // particle chunks of a tensor-core member, at most
struct TcPhase {
  int tab_off = 0, tab_n = 0, prep_off = 0, prep_n = 0, dens_off = 0, dens_n = 0, force_off = 0, force_n = 0;
  int rtab_off = 0, rtab_n = 0, rprep_off = 0, rprep_n = 0;  // the preparation again, before the force items
  int prep4 = 0, rprep4 = 0;  // the last items of each preparation range: those of four-axis members
};

struct EngineView {
  const CfgDev* cfgs = nullptr;
  const int* list = nullptr;  // configurations evaluated in this precision
  int nlist = 0;
  const TwItem* tw = nullptr;
  int ntw = 0;
  const NtItem* nt = nullptr;
  int nnt = 0;
  const FItem* fi = nullptr;
  int nfi = 0;
  size_t nt_smem = 0;
  int64_t maxM = 0, maxND = 0;
  int maxblk = 0;
  int* counters = nullptr;  // two ints: density queue, force queue
  int sm_count = 148;
  // tensor-core members (fixed point only)
  const int* tc_list = nullptr;
  int ntc_list = 0;
  const TwItem* tc_prep = nullptr;
  int ntc_prep = 0;
  const TcItem* tc_dens = nullptr;
  int ntc_dens = 0;
  const TcItem* tc_force = nullptr;
  int ntc_force = 0;
  // particle chunks: phase c runs chunk c of every member that has one (its tables, preparation and density
  // items), and, in reverse order, its force items, preceded by the preparation again where the member's
  // buffers no longer hold that chunk.  Offsets index the arrays above (items) and the block maps (tables).
  int ntc_phase = 0;
  TcPhase tc_ph[kMaxTcPhases];
  int64_t tc_max_grid = 0;  // largest (R1 + 1) nP of the members
  size_t tc_prep_smem = 0;  // largest preparation shared memory of the members
  int64_t tc_maxND = 0;     // largest (the path's axes) x N of the members (d = 1 runs on two lifted axes)
  // block maps of the tensor-core members' light kernels: tables (128 threads over the path's axes x N),
  // density finish (64 threads), coefficients (128 threads over (R1 + 1) nP), force finish (64 threads over d N)
  const BlockMap *tc_bm_tab = nullptr, *tc_bm_fin = nullptr, *tc_bm_coef = nullptr, *tc_bm_ff = nullptr;
  int ntc_bm_tab = 0, ntc_bm_fin = 0, ntc_bm_coef = 0, ntc_bm_ff = 0;
};

struct Ctx;

// minimiser state of one configuration (device memory)
// kFsDevErr: a bounded wait of a tensor-core kernel gave up during the step's evaluation (the step is undone)
enum { kFsRunning = 0, kFsConverged = 1, kFsNan = 2, kFsStageDone = 3, kFsMaxSteps = 4, kFsDevErr = 5 };
struct FireState {
  int status;
  int rejected_now;
  int zero_v;
  int stage;
  double dt, alpha, cv, cf;
  long long n_pos, step, stage_step, rejected;
  double phi_hi, phi_lo, smax_hi, smax_lo;
  double best_smax;
  long long best_step;
  // parameters
  double dt_max, alpha_start, f_alpha, f_inc, f_dec;
  long long n_min, stall_window, max_steps;
  double target, stage_floor;
  double phi_tol;  // the guard rejects a step only when Phi rises by more than phi_tol sqrt(Phi_accepted)
  // minimiser: kMethodFire or kMethodLbfgs (lbfgs.cu), and the L-BFGS state
  int method;
  int lb_count, lb_head;      // history pairs kept; ring slot of the newest
  int lb_need_dir, lb_accepted, lb_sd, lb_backtracks;
  double lb_alpha, lb_gp, lb_gamma, lb_dmax;  // step length, G.p, scale of H0, largest fractional move
  int dots_ticket, pad_ticket;                 // last-block counter of the FIRE dot products
};
enum { kMethodFire = 0, kMethodLbfgs = 1 };
constexpr int kLbMaxPairs = 8;
constexpr int kLbPartStride = 48;  // doubles per block partial of the L-BFGS passes (>= 5 kLbMaxPairs + 1)
struct LbMat {                     // per member: S^T Y and Y^T Y by ring slot, the direction's coefficients
  double StY[kLbMaxPairs][kLbMaxPairs], YtY[kLbMaxPairs][kLbMaxPairs];
  double t[kLbMaxPairs], w1[kLbMaxPairs];
  int ticket_dir, ticket_pairs;    // last-block counters of the two passes
  int pad[2];
};

// A set of configurations evaluated together.  Members keep their own buffers (Ctx); the engine holds their
// descriptors, the per-precision member lists and the work lists, all in device memory.
// Work decomposition of the tensor-core GEMMs, chosen by the batch autotuner (ssh_batch_autotune): density
// K-range pieces per member as a percentage of its share of the SMs, and whether force items run in
// particle-tile bundles (largest bundle first) or one by one (largest first).
struct EngineTune {
  int dens_pct = 100;
  int force_bundle = 1;
};

struct Engine {
  int device = 0;
  EngineTune tune;  // set by the caller before engine_build
  int sm_count = 148;
  std::vector<Ctx*> members;
  std::vector<int> prec_of;  // current precision per member; -1 = listed under every precision
  bool fire_mode = false;
  std::vector<CfgDev> host_cfgs;
  DevBuf d_cfgs, d_lists, d_all, d_tw, d_nt, d_f, d_counters, d_tclist, d_tcprep, d_tcdens, d_tcforce, d_bm;
  EngineView view[3];
  std::vector<int> h_lists;
  std::vector<TwItem> h_tw;
  std::vector<NtItem> h_nt;
  std::vector<FItem> h_f;
  const int* all = nullptr;  // every member, for the minimiser kernels
  int nall = 0;
  int64_t maxND_all = 0;
  int max_nb_fire = 0;
  // block maps of the minimiser's kernels: dot products (nb_fire blocks of 256 per member), element-wise
  // updates (64 threads over d N)
  const BlockMap *bm_dots = nullptr, *bm_nd = nullptr;
  int nbm_dots = 0, nbm_nd = 0;
  int methods = 1;  // minimisers present among the members: bit kMethodFire, bit kMethodLbfgs (set by the caller)
};

// tile plan and buffers of the tensor-core path of one configuration (tc.cu)
struct TcPlan {
  bool on = false;
  int d = 0;                     // the path's number of axes: 2, 3 or 4 (d = 1 runs on two lifted axes)
  int lift = 0;                  // d = 1: n = 2^lift n1 + n2, n2 in [-2^(lift - 1), 2^(lift - 1))
  int R1 = 0;                    // n1 in [0, R1]
  int Rax[4] = {0, 0, 0, 0};     // largest |n_a| per axis (powers held in the tables)
  int nP = 0;                    // canonical sub-vectors p = (n2[, n3[, n4]]) of the half set, sorted by |p|^2
  int64_t Nc = 0;                // particles per chunk (the buffers below hold one chunk), a multiple of 128
  int nchunk = 1;                // chunks of N, evaluated one after another
  int64_t KS = 0;                // density K-steps (16 particles each) of a full chunk
  int RT = 0, CTd = 0;           // density row tiles (128 rows (p, cos/sin)), column tiles (32 columns (n1, cos/sin);
                                 // with tr, one more: the transposed tile's B operand, w_j(p) of the last row tile)
  // transposed remainder tile (two-axis path): the last row tile holds at most 16 canonical p, whose members have
  // n1 < trN1; their density is one tile with rows (n1, cos / sin) of a_j(n1), written into that row tile of the digit
  // tensor from local row trRow0 (past every K row the force reads), and columns (p, cos / sin) of w_j(p)
  int tr = 0, trP0 = 0, trRow0 = 0, trN1 = 0;
  int PT = 0, KSf = 0, CTf = 0;  // force particle tiles (of a chunk), K-steps (16 rows (p, cos/sin)), column tiles (16/d n1, all axes)
  int64_t NJ = 0, NPg = 0;       // digit tensor: particle groups (of a chunk) and row groups of 8
  int bexp = 0;                  // 2^bexp > |n_a| (a >= 2): scale of the weighted force coefficients
  int gs = 0, ts = 0;            // force epilogue scales
  std::vector<int32_t> tiles;    // density tiles in use: rt * CTd + ct
  std::vector<int32_t> tilemap;  // [RT * CTd] -> index into tiles, or -1
  std::vector<int32_t> em;       // [nP][R1 + 1][2] internal index of (n1, p) / (n1, -p), or -1
  std::vector<int32_t> pvec;     // [nP] packed (n2, n3) or (n2, n3, n4), as tc_pvec
  std::vector<int32_t> ks_ct;    // force K-steps per column tile
  int fsplit = 1;                // force K ranges per (particle tile, column tile), at most (see tc_setup)
  int ntab = 0;                  // table entries per (axis, particle)
  size_t prep_smem = 0;          // dynamic shared memory of the preparation kernel
  alignas(64) unsigned char tmap_h[256];  // host copy of the two tensor maps (source of the upload)
  DevBuf wT, aB, fB, a1, tab, acc, facc, em_d, pvec_d, tilemap_d, tmap, err;
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
  DevBuf wk;                   // [M] internal order: weights v~(k) (ssh_set_weights), 1 by default
  double wmax = 1.0;           // the largest weight (the energy guard's error bound scales with it)
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
  dd inv_L;                       // 1 / L
  FireBufs* fire = nullptr;       // minimiser state, allocated on first ssh_minimize
  Engine* eng = nullptr;          // this context alone (plain evaluations)
  cudaGraphExec_t eval_graph[3][2] = {};  // one evaluation per (precision, with force), replayed; reset with eng
  bool tc_requested = false;      // fixed point on the tensor cores (d = 1, 2, 3)
  int64_t tc_chunk_req = 0;        // particles per chunk on that path (0: as device memory allows)
  TcPlan tc;
  // particle shard: evaluations sum and force only particles [shard_p0, shard_p0 + shard_n) of the N (shard_n = 0:
  // every particle, the ordinary context); the exchange with the other shards goes through the caller (shard.cu)
  int64_t shard_p0 = 0, shard_n = 0;
};

// first particle and particle count a context's evaluations cover (its shard, or all N)
inline int64_t part_p0(const Ctx* c) { return c->shard_n > 0 ? c->shard_p0 : 0; }
inline int64_t part_n(const Ctx* c) { return c->shard_n > 0 ? c->shard_n : c->N; }
// FIRE dot products are summed per chunk of kDotChunk particles of one axis, so that a shard boundary on a multiple
// of it leaves every chunk's partial sum to one shard (the totals then agree bit for bit with the unsharded sums)
constexpr int64_t kDotChunk = 2048;
inline int64_t dot_chunks(int d, int64_t N) { return (int64_t)d * ((N + kDotChunk - 1) / kDotChunk); }

// Launch with programmatic dependent launch: the kernel's CTAs may be made resident while the previous kernel on
// the stream is still finishing, and each waits (grid_dep_wait, its first statement) until that kernel has
// completed and its memory is visible.  This hides the launch gap between the short kernels of a step.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}
#ifdef __CUDACC__
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// A bounded wait of the tensor-core GEMM gave up during this configuration's last evaluation, so its sums are
// incomplete (the error word stays set until the host reports it).
__device__ __forceinline__ bool tc_failed(const CfgDev& c) {
  return c.tc && c.tc_err && *reinterpret_cast<volatile const int*>(c.tc_err) != 0;
}
#endif

// record an event pair around a launch when profiling is on
void prof_begin(Prof* p, cudaStream_t st, int id);
void prof_end(Prof* p, cudaStream_t st);
cudaError_t prof_collect(Prof* p, cudaStream_t st);

// engine.cu
CfgDev make_cfgdev(const Ctx* c, bool fire_mode);
cudaError_t engine_build(Engine* e, const std::vector<Ctx*>& members, const std::vector<int>& prec_of, bool fire_mode,
                         cudaStream_t st);
void engine_free(Engine* e);
cudaError_t engine_eval(const Engine* e, int prec, bool want_force, cudaStream_t st, Prof* prof);
void kernels_set_attributes(size_t smem_max);

// fire.cu (minimiser kernels over the members of an engine)
void fire_fill_cfgdev(const Ctx* c, CfgDev* g);
cudaError_t fire_alloc(Ctx* c);
cudaError_t fire_step_engine(const Engine* e, cudaStream_t st, Prof* prof);
FireState fire_params(const ssh_min_params* p);
// the public status of a minimiser run that ended with device status word `status`
ssh_status fs_status_code(int status);
// error bound coefficient of Phi in arithmetic prec for configuration c: |dPhi| <= coef sqrt(Phi)
double fire_phi_tol(const Ctx* c, int prec);
// (re)start the members idx of e: v = 0 when first, accepted Phi / S_max from their scal, stage parameters
cudaError_t fire_stage_init_engine(const Engine* e, const std::vector<int>& idx, const std::vector<FireState>& params,
                                   const std::vector<int>& first, cudaStream_t st);

// device scalar block written by k_finalize (doubles)
enum { kScPhiHi = 0, kScPhiLo, kScSmaxHi, kScSmaxLo, kScCmax, kScScaleExp, kScA2MaxHi, kScA2MaxLo, kScCount = 16 };
constexpr int kPackTail = kScCount + 1;  // packed results: the scalars, then int {non-finite force, tc status}

// lbfgs.cu (the L-BFGS minimiser's step kernels)
cudaError_t lbfgs_pre(const Engine* e, cudaStream_t st);
cudaError_t lbfgs_post_accept(const Engine* e, cudaStream_t st);
cudaError_t lbfgs_post_pairs(const Engine* e, cudaStream_t st);
cudaError_t lbfgs_stage_g(const CfgDev* cfgs, int64_t maxND, const int* d_idx, int n, cudaStream_t st);

// tc.cu (tensor-core fixed-point path, d = 1, 2, 3)
int64_t tc_coef_blocks(const Ctx& c);  // blocks (128 threads) of the coefficient kernel
bool tc_eligible(const Ctx& c);
int tc_finish_blocks(const Ctx& c);  // blocks of the density finish kernel (its reduction partials)
cudaError_t tc_setup(Ctx* c);
void tc_free(Ctx* c);
size_t tc_footprint(const Ctx& c);
void tc_fill_cfgdev(const Ctx* c, CfgDev* g);
// particle chunks of a tensor-core member: their number, the descriptor of chunk ch (from the member's), and the
// work of one chunk: density K-steps (tiles x K-steps), tables blocks, preparation items, GEMM items
int tc_chunks(const Ctx* c);
void tc_chunk_cfgdev(const Ctx* c, int ch, CfgDev* g);
int64_t tc_density_steps(const Ctx* c, int ch);
int64_t tc_table_blocks(const Ctx* c, int ch);
void tc_prep_items(const Ctx* c, int cfg, int ch, std::vector<TwItem>& prep);
void tc_gemm_items(const Ctx* c, int cfg, int ch, int64_t pieces, std::vector<TcItem>& dens, std::vector<TcItem>& force);
cudaError_t tc_launch_density(const EngineView& v, cudaStream_t st, Prof* prof);
// the two halves of tc_launch_density: the GEMM phases (into the exact tile accumulators), then the finish
cudaError_t tc_launch_density_gemms(const EngineView& v, cudaStream_t st, Prof* prof);
cudaError_t tc_launch_dens_finish(const EngineView& v, cudaStream_t st, Prof* prof);
// the exact density tile accumulators of a tensor-core context: device pointer and int64 words
long long* tc_acc_ptr(const Ctx* c);
int64_t tc_acc_words(const Ctx* c);
cudaError_t tc_launch_force(const EngineView& v, cudaStream_t st, Prof* prof);
cudaError_t tc_launch_force_finish(const EngineView& v, cudaStream_t st, Prof* prof);
// the counting instance of the GEMM is in use (ssh_gemm_counters): evaluations launch directly, not from graphs
bool tc_counters_on();

// kernels.cu
cudaError_t plan_upload(Ctx* c);
void eval_graphs_reset(Ctx* c);  // drop the cached evaluation graphs (the engine changed)
cudaError_t eval_phi_grad(Ctx* c, int prec, bool want_force);
void setup_launch(Ctx* c);

void set_error(const std::string& msg);

// fire.cu
ssh_status minimize(Ctx* c, const ssh_min_params* p, ssh_min_result* res);
void fire_free(Ctx* c);
ssh_status fire_begin(Ctx* c, const ssh_min_params* p);
ssh_status fire_steps(Ctx* c, int prec, int64_t nsteps);
ssh_status fire_state(Ctx* c, ssh_min_result* r, int* dev_status);
// the pieces of one FIRE step that a sharded run interleaves with its exchanges (shard.cu): the minimiser's
// engine for prec; the dot-product partials of every chunk into out ([3][n_dchunk]); the FIRE controls from summed
// partials, then the move; the acceptance and the undo; a stage start from the results already in place
cudaError_t fire_engine_for(Ctx* c, int prec, Engine** out);
cudaError_t fire_dots_partials(const Engine* e, double* out, cudaStream_t st);
cudaError_t fire_control_move(const Engine* e, const double* tot, cudaStream_t st);
cudaError_t fire_accept_restore(const Engine* e, cudaStream_t st);
ssh_status fire_begin_from_results(Ctx* c, const ssh_min_params* p);
bool fire_begun(const Ctx* c);  // a FIRE run has begun on this context

// zero fields of pin take the context's defaults; validates the result
ssh_status complete_params(const ssh_ctx* h, const ssh_min_params* pin, ssh_min_params* out);

// device bytes a configuration occupies once created and minimised (plans, tables, partial sums, state)
size_t device_footprint(const Ctx& c);

}  // namespace ssh

// the public handle: one configuration plus its pinned host staging
struct ssh_ctx {
  ssh::Ctx c;
  // pinned staging for positions and results: 2 d N doubles, then the packed results' tail (the scalars and two
  // status words, kPackTail doubles)
  double* h_stage = nullptr;
  cudaEvent_t stage_done = nullptr;  // recorded after the last upload from h_stage
  ssh::DevBuf d_pack;               // the packed results on the device, laid out as h_stage (allocated on first use)
};
