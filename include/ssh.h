/*
 * ssh.h -- C ABI of the stealthy-hyperuniform collective-coordinate library (arXiv:2304.09139) for B300.
 *
 * The library evaluates, for N points in a periodic box of side L in d dimensions,
 *   n~(k) = C(k) + i S(k) = sum_j exp(i k.r_j)                       (Eq. ntilde; sign +, see below)
 *   Phi   = sum over the M independent k (half-space, 0 < |k| <= K) of |n~(k)|^2
 *                                                                     (Eq. energy with eps0 = 1, constant dropped)
 *   S(k)  = |n~(k)|^2 / N,  S_max = max_k S(k)                       (Eqs. structurefactor, smax)
 *   F_j   = -grad_j Phi = 2 sum_k k [C(k) sin(k.r_j) - S(k) cos(k.r_j)] (Eq. force)
 * on the GPU, and minimises Phi with FIRE (Simulations).  k = 2 pi n / L for integer n in the half-space
 * {first non-zero component of n > 0}; chi = M / (d (N - 1)) (Definitions).  The paper writes exp(-i k.r);
 * |n~|, Phi, S and F do not depend on that sign, only the sign of S(k) does.
 *
 * Conventions for every entry point:
 *   * Return value: SSH_OK or an error code; no C++ exception crosses this boundary.  On error,
 *     ssh_last_error() returns a thread-local message describing it.
 *   * Host arrays are owned by the caller.  The library copies inputs in and writes outputs into caller
 *     buffers before returning; it never keeps a caller pointer.
 *   * Device memory and CUDA streams are owned by the library (one stream per context unless the caller
 *     installs its own with ssh_set_stream).  Calls on one context are not thread-safe.
 *   * Double-double (dd) values are passed as a (hi, lo) pair of doubles whose exact sum is the value.
 *   * Positions and forces are row-major [N][d].
 */
#ifndef SSH_H_
#define SSH_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ssh_ctx ssh_ctx; /* opaque, library-owned */

typedef enum {
  SSH_OK = 0,
  SSH_EINVAL = 1,    /* an argument is out of range or inconsistent */
  SSH_ENOMEM = 2,    /* device or host allocation failed */
  SSH_ECUDA = 3,     /* a CUDA call failed (no device, launch error, ...) */
  SSH_ENAN = 4,      /* non-finite value in positions or results */
  SSH_ENOTCONV = 5,  /* the minimiser hit its step cap or stalled above the target */
  SSH_ETIMEOUT = 6,  /* a bounded device or host wait gave up */
  SSH_EBUSY = 7,     /* result not ready yet / no capacity now */
  SSH_ENOTFOUND = 8  /* unknown ticket or handle */
} ssh_status;

/* Arithmetic of an evaluation.
 *   SSH_FP64 -- plain binary64 phases, sums and products (the paper's cheap first stage).
 *   SSH_DD   -- double-double on the FP64 pipe, as the paper describes (~106-bit significands).
 *   SSH_FX   -- 128-bit fixed point on the integer pipes (Q0.128 positions, exact phase reduction, exact
 *               sums, 2^-126 resolution): dd-or-better accuracy on the units B300 has most of.
 */
typedef enum { SSH_FP64 = 0, SSH_DD = 1, SSH_FX = 2 } ssh_prec;

/* Implementation of SSH_FX evaluations (same arithmetic class, results agree to the 1e-28 normwise bound):
 *   SSH_FX_AUTO    -- the library's choice: the tensor cores where the set is within their limits, else the
 *                     integer pipes
 *   SSH_FX_INTEGER -- 128-bit fixed point on the integer pipes, any d
 *   SSH_FX_TENSOR  -- both sums as exact-digit GEMMs on the tensor cores (15 balanced 7-bit digits per 2^-104
 *                     fixed-point value in bf16, fp32 accumulation kept exact by bounded read-outs; d = 1 runs on
 *                     two lifted axes, n = 2^b n_1 + n_2).  A wavevector set beyond the path's limits (d = 3 with
 *                     max |n_2| + max |n_3| above 211; d = 4 with some |n_a| above 64, a >= 2, or with
 *                     768 (max |n_2| + max |n_3| + max |n_4| + 3) + 4 P above 200 KiB, P the number of
 *                     distinct canonical (n_2, n_3, n_4); more than 16384 distinct (n_2, .., n_d)), or
 *                     N above 2^22, runs on the integer pipes; ssh_get_fx_impl reports which implementation a
 *                     context uses. */
enum { SSH_FX_AUTO = 0, SSH_FX_INTEGER = 1, SSH_FX_TENSOR = 2 };
#define SSH_FX_AUTO_TENSOR 1

typedef struct {
  int device;       /* CUDA device ordinal (default 0) */
  int fx_impl;      /* SSH_FX_AUTO (0, default), SSH_FX_INTEGER or SSH_FX_TENSOR */
  int tc_chunk;     /* tensor-core path: particles per chunk (0, default: every particle at once when the chunk
                     * buffers fit in about 70% of the free device memory, else as many equal chunks as needed).
                     * Chunks run one after another through the same buffers; results do not depend on the
                     * chunking (the sums are exact integers).  Rounded up to a multiple of 128 and to at most
                     * 64 chunks. */
  int shard_first;  /* particle shard (ssh_shard_*): the context's evaluations sum and force only the particles */
  int shard_count;  /* [shard_first, shard_first + shard_count) of the N; both 0 (default): every particle.  Needs the
                     * tensor-core path; shard_first a multiple of 2048, shard_count too unless the shard ends at N */
  int reserved[3];  /* zero */
} ssh_opts;

/* Library version string, e.g. "ssh 0.1 sm_103a". Never NULL. */
const char* ssh_version(void);

/* Thread-local message for the most recent non-OK status returned on this thread ("" if none). */
const char* ssh_last_error(void);

/*
 * Create a context for N points in d dimensions in a periodic box of side L (Definitions).
 * Exactly one of chi > 0 (M = round-half-even(chi d (N-1)) smallest |k| of the half-space, ties broken
 * lexicographically) or K > 0 (every half-space k with |k| <= K, complete shells) must be given.
 * 1 <= d <= 4, N >= 1, L > 0 finite, chi < 1 (the paper's disordered regime is chi < 1/2).
 * opts may be NULL.  On success *out owns device memory sized for this (d, N, M); free with ssh_destroy.
 * Errors: SSH_EINVAL (arguments), SSH_ECUDA (no device), SSH_ENOMEM.
 */
ssh_status ssh_create(int d, int64_t N, double L, double chi, double K, const ssh_opts* opts, ssh_ctx** out);

/* Release everything a context owns.  NULL is a no-op. */
void ssh_destroy(ssh_ctx* ctx);

/* Sizes: any pointer may be NULL. */
ssh_status ssh_get_dims(const ssh_ctx* ctx, int* d, int64_t* N, int64_t* M, double* L);

/* The implementation SSH_FX evaluations of this context use: SSH_FX_INTEGER or SSH_FX_TENSOR. */
ssh_status ssh_get_fx_impl(const ssh_ctx* ctx, int* impl);

/* Weights v~(k) of the wavevectors (Eq. energy's v~(k); the paper notes that a general positive v~(k) funnels the
 * minimiser to chosen ground states): Phi = sum_k v~(k) |n~(k)|^2 and F = -grad Phi; S(k) and S_max do not change.  w holds M values
 * in the order of ssh_get_kset, each finite and in [0, 1024]; NULL restores 1 for every wavevector (the
 * default).  Weight 1 keeps the exact integer force coefficients of the fixed-point paths; other weights enter
 * them through a double-double product (relative error 2^-105).  Stream-ordered; takes effect at the next
 * evaluation.  Errors: SSH_EINVAL. */
ssh_status ssh_set_weights(ssh_ctx* ctx, const double* w);

/* Post-processing (the supplement's Fig. S1b, g_2(r) of a state): counts of ordered particle pairs (i, j), i < n_ref,
 * j != i, by minimum-image distance, nbins bins of width r_max / nbins on [0, r_max), 0 < r_max < L / 2.  Decided
 * in exact integers: coordinates floor(s 2^32) of the high words of the current positions, squared distances in
 * units (L 2^-32)^2, bin edges ceil(b^2 q^2 / nbins^2) with q = floor(r_max / L 2^32) (bins exact to one unit).
 * g_2 of bin b is counts[b] / (n_ref (N - 1) / L^d) / (volume of the shell b).  1 <= n_ref <= N, 1 <= nbins <= 4096;
 * counts: nbins host uint64.  Synchronous.  Errors: SSH_EINVAL, SSH_ECUDA. */
ssh_status ssh_pair_histogram(ssh_ctx* ctx, int64_t n_ref, double r_max, int nbins, uint64_t* counts);

/* g_2(r) from pair counts (the supplement's Fig. S1b), host arithmetic only (no context, no GPU): g2[b] =
 * counts[b] / (n_ref (N - 1) / L^d x v_d ((b + 1)^d - b^d) w^d), w = r_max / nbins, v_d the volume of the unit
 * ball: each shell's count over the count an ideal gas of the same density gives there.  r_mid[b] = (b + 1/2) w
 * (may be NULL).  counts, r_mid, g2: nbins host values.  Errors: SSH_EINVAL. */
ssh_status ssh_g2(int d, int64_t N, double L, int64_t n_ref, double r_max, int nbins, const uint64_t* counts,
                  double* r_mid, double* g2);

/* Shell averages of S(k) = |n~(k)|^2 / N (Eq. structurefactor; the supplement's Fig. S1a shows S(k) on a linear
 * scale) and the order metric tau of Eq. tau, from the context's last evaluation, in double-double on the GPU.
 * Shells: edges E_b = ceil(b^2 n2max / nbins^2) (exact integers); shell b < nbins - 1 holds the wavevectors with
 * E_b <= |n|^2 < E_(b+1), the last E_(nbins-1) <= |n|^2 <= n2max, i.e. |k| = 2 pi |n| / L in
 * [b, b + 1) x 2 pi sqrt(n2max) / (L nbins).  counts[b] (int64) is the shell's population, mean[2b], mean[2b+1] the
 * dd mean of S over it (0 when empty), k_mid[b] (may be NULL) the shell's middle |k|.  tau (dd, 2 doubles): the
 * integral of [S(k) - 1]^2 over k, divided by (2 pi D)^d rho^2 with D = 1 / K and rho = N / L^d, taken as the
 * lattice sum over every wavevector of the context and its mirror -k (cells (2 pi / L)^d):
 * tau = 2 (K L)^d / N^2 sum_k [S(k) - 1]^2.  The paper's tau is an ensemble integral in the thermodynamic limit;
 * over one configuration's wavevectors this is a finite-size estimate (a K-mode context with a cutoff beyond the
 * exclusion region carries more of the integral).  Each shell and tau are summed in a fixed order, so repeated
 * calls return the same bits.  1 <= nbins <= 65536; n2max = 0 takes the largest |n|^2 of the set and K = 0 its
 * largest |k|.  Synchronous.  Errors: SSH_EINVAL (no
 * evaluation yet, a particle-shard context, arguments), SSH_ECUDA. */
ssh_status ssh_structure_factor(ssh_ctx* ctx, int nbins, int64_t n2max, double K, int64_t* counts, double* mean,
                                double* tau, double* k_mid);

/* Particle chunks of the tensor-core path (ssh_opts.tc_chunk): their number and the particles per chunk; both 0
 * when the context uses the integer pipes.  Either pointer may be NULL. */
ssh_status ssh_get_tc_chunks(const ssh_ctx* ctx, int* nchunk, int64_t* chunk);

/* The tensor-core path's density tile plan (a diagnostic of this library; no counterpart in the paper): row tiles
 * (128 rows (p, cos / sin)), column tiles (32 columns), density
 * tiles in use, and whether the last row tile's wavevectors run as one transposed tile (two-axis sets whose last
 * row tile holds at most 16 canonical p: rows (n1, cos / sin), columns (p, cos / sin); column tiles then counts its
 * B operand).  All 0 on the integer pipes.  Any pointer may be NULL. */
ssh_status ssh_get_tc_plan(const ssh_ctx* ctx, int* row_tiles, int* col_tiles, int* tiles, int* transposed);

/* The M wavevector indices n (k = 2 pi n / L) in public order: by |n|^2, then lexicographic (a context of
 * ssh_create_kset: the order of its list).  n: caller buffer of M*d int32 (row-major), or NULL to query M only. */
ssh_status ssh_get_kset(const ssh_ctx* ctx, int64_t* M, int32_t* n);

/* A context over a given wavevector set instead of the ball (the paper's other exclusion regions, e.g. the
 * anisotropic ones of ssh_kset_build_region): M distinct vectors n (row-major [M][d] int32), each in the half
 * space (first non-zero component positive) with |n_a| <= 32767.  Public order is the list's.  Otherwise as
 * ssh_create (d, N, L, opts).  Errors: SSH_EINVAL (a vector out of the half space, repeated or out of range),
 * SSH_ECUDA, SSH_ENOMEM. */
ssh_status ssh_create_kset(int d, int64_t N, double L, int64_t M, const int32_t* n, const ssh_opts* opts,
                           ssh_ctx** out);

/* Host only: the wavevectors of an anisotropic exclusion region sum_a w_a n_a^2 <= R^2 (w: d integers in
 * [1, 2^20]; NULL: the ball, as ssh_kset_build).  K mode: every half-space n with that norm at most
 * (K L / 2 pi)^2 (1 + 1e-12); chi mode: the first M = round-half-even(chi d (N - 1)) in the order (norm, then
 * lexicographic on the signed components), which is also the list's order.  n: cap rows of d int32 or NULL
 * to query M.  Errors: SSH_EINVAL (bad arguments, cap < M with M still written). */
ssh_status ssh_kset_build_region(int d, int64_t N, double L, double chi, double K, const int32_t* w, int64_t cap,
                                 int32_t* n, int64_t* M);

/* Host only (no GPU needed): the wavevector set that ssh_create would build for these arguments, in public
 * order.  n: caller buffer of cap rows of d int32, or NULL to query M.  Errors: SSH_EINVAL for bad
 * arguments or cap < M (M is still written). */
ssh_status ssh_kset_build(int d, int64_t N, double L, double chi, double K, int64_t cap, int32_t* n, int64_t* M);

/* Install a caller-owned cudaStream_t (passed as void*) for all later work on ctx; NULL restores the
 * context's own stream.  The caller keeps ownership and must keep the stream alive. */
ssh_status ssh_set_stream(ssh_ctx* ctx, void* cuda_stream);

/* Block the host until all work queued on the context's stream has finished. */
ssh_status ssh_sync(ssh_ctx* ctx);

/* Positions in physical units r (N*d row-major, dd as hi + lo; lo may be NULL for zero).  Values are
 * wrapped into [0, L) (periodic box).  The caller's arrays are read before the call returns, so they may be
 * reused at once; the upload itself is queued on the context's stream, ahead of any later work there.
 * Errors: SSH_ENAN for a non-finite coordinate (the previous positions are kept). */
ssh_status ssh_set_positions(ssh_ctx* ctx, const double* r_hi, const double* r_lo);

/* Positions as fractional coordinates s = r / L (N*d row-major, dd, lo may be NULL); exact, no division.
 * Each value is reduced into [0, 1) by its exact fraction; one already in [0, 1) with a zero low word is kept
 * as it is (-0 becomes +0).  Same ownership, ordering and errors as ssh_set_positions. */
ssh_status ssh_set_positions_frac(ssh_ctx* ctx, const double* s_hi, const double* s_lo);

/* Current fractional positions s in [0, 1) as dd (N*d row-major); either pointer may be NULL. */
ssh_status ssh_get_positions_frac(ssh_ctx* ctx, double* s_hi, double* s_lo);

/* Current positions in physical units, r = L s in [0, L) as dd (N*d row-major; the dd product of the stored s
 * with L); either pointer may be NULL.  Errors: SSH_EINVAL (no positions), SSH_ECUDA. */
ssh_status ssh_get_positions(ssh_ctx* ctx, double* r_hi, double* r_lo);

/*
 * One evaluation of Phi, S_max and F at the current positions in arithmetic `prec` (Eqs. energy, smax,
 * force), results copied to the caller: phi[2] and smax[2] as dd (either may be NULL), F_hi / F_lo the
 * force in physical units (N*d row-major; either may be NULL).  Blocks until the copies are done.
 * Errors: SSH_EINVAL (no positions set / bad prec), SSH_ECUDA, SSH_ENAN (non-finite result).
 */
ssh_status ssh_energy_grad(ssh_ctx* ctx, int prec, double phi[2], double smax[2], double* F_hi, double* F_lo);

/*
 * The same evaluation with inputs already resident on the device and results left there: it only
 * enqueues kernels on the context's stream and returns (no host synchronisation).  want_force = 0 skips
 * the force sum (energy and S_max only).  Read results later with ssh_get_results / ssh_get_ntilde.
 */
ssh_status ssh_eval(ssh_ctx* ctx, int prec, int want_force);

/* Copy the results of the last evaluation to the host (synchronises the stream).  Any pointer may be NULL.
 * The force is present only if the last evaluation computed it. */
ssh_status ssh_get_results(ssh_ctx* ctx, double phi[2], double smax[2], double* F_hi, double* F_lo);

/* n~(k) = C + i S of the last evaluation, M entries each as dd, in public k order; any pointer may be NULL. */
ssh_status ssh_get_ntilde(ssh_ctx* ctx, double* C_hi, double* C_lo, double* S_hi, double* S_lo);

/*
 * Minimisation (Simulations: FIRE of Bitzek et al. 2006 on Phi, with the paper's stopping rule read as
 * "S_max at or below a target").  Parameters; zero fields take the defaults that ssh_min_defaults writes.
 *   dt0, dt_max            time steps in physical units (defaults dt_max = 1/sqrt(2 N max|k|^2), dt0 = dt_max/10)
 *   alpha_start, f_alpha, f_inc, f_dec, n_min   FIRE constants (defaults 0.1, 0.99, 1.1, 0.5, 5)
 *   n_stages, stage_prec   precision ladder, e.g. {SSH_FP64, SSH_DD} (default {SSH_FX} when the context's
 *                          fixed point runs on the tensor cores, else {SSH_FP64, SSH_FX}); a stage
 *                          ends when S_max <= stage_floor[s] or S_max has not halved in stall_window[s]
 *                          steps (0, the default: 200 for an FP64 stage, 5000 for dd or fixed point); the
 *                          last stage ends only at the target, the step cap or a stall
 *   max_steps, smax_target step cap (default 200000) and convergence target (default 1e-36)
 *   chunk                  steps between host checks of the device status word (default 64)
 *   max_seconds            wall-time limit, 0 = none
 *   method                 SSH_MIN_FIRE (the paper's minimiser) or SSH_MIN_LBFGS: limited-memory BFGS (8 pairs,
 *                          compact representation of Byrd, Nocedal and Schnabel 1994) with a backtracking Armijo
 *                          line search on the same energy and force, the same stop rules and precision ladder;
 *                          no particle moves more than a tenth of the mean spacing in one step
 */
enum { SSH_MIN_FIRE = 0, SSH_MIN_LBFGS = 1 };
typedef struct {
  double dt0, dt_max, alpha_start, f_alpha, f_inc, f_dec;
  int n_min;
  int n_stages;
  int stage_prec[3];
  int method;                /* SSH_MIN_FIRE (0, default) or SSH_MIN_LBFGS */
  double stage_floor[3];
  int64_t stall_window[3];
  int64_t max_steps;
  double smax_target;
  int64_t chunk;
  double max_seconds;
} ssh_min_params;

typedef struct {
  int status;              /* SSH_OK (converged), SSH_ENOTCONV, SSH_ENAN, SSH_ETIMEOUT */
  int final_prec;          /* precision of the last stage run */
  int stages_used;
  int pad0;
  int64_t steps;           /* FIRE steps including rejected ones */
  int64_t stage_steps[3];
  int64_t rejected;        /* steps undone by the energy guard */
  double smax[2], phi[2];  /* accepted S_max and Phi (dd) in the final precision */
  double dt;               /* final time step */
  double wall_s, stage_wall_s[3];
} ssh_min_result;

/* Fill p with the defaults for this context (see ssh_min_params). */
ssh_status ssh_min_defaults(const ssh_ctx* ctx, ssh_min_params* p);

/*
 * Minimise Phi from the current positions with FIRE on the device (velocity update, step acceptance,
 * convergence test and precision switch all run in kernels; the host only replays a CUDA graph of steps
 * and reads a status word between chunks).  An energy guard undoes any step that raises Phi (dt halves,
 * v = 0).  On return the context holds the accepted positions (ssh_get_positions_frac).  p may be NULL
 * (defaults); res may be NULL.  Returns SSH_OK when S_max <= smax_target, SSH_ENOTCONV on the step cap or
 * a stall of the last stage, SSH_ENAN, SSH_ETIMEOUT (max_seconds), SSH_EINVAL, SSH_ECUDA.
 */
ssh_status ssh_minimize(ssh_ctx* ctx, const ssh_min_params* p, ssh_min_result* res);

/*
 * Stepper: the same device FIRE step as ssh_minimize, driven one step at a time.
 *   ssh_fire_begin  v = 0, and Phi, S_max and F at the current positions in p->stage_prec[0] (p as for
 *                   ssh_minimize; stage floors are ignored, the step cap and target still stop the run)
 *   ssh_fire_steps  enqueue exactly nsteps steps in precision prec on the context's stream and return
 *                   without synchronising; steps after the run has stopped do nothing.  Steps replay a
 *                   captured CUDA graph, except while the profiler is on: then each kernel is launched
 *                   directly so that it carries its own event pair
 *   ssh_fire_state  synchronise and report steps, rejected steps, S_max, Phi and dt of the accepted state;
 *                   *running = 1 while the device status word says the run continues
 */
ssh_status ssh_fire_begin(ssh_ctx* ctx, const ssh_min_params* p);
ssh_status ssh_fire_steps(ssh_ctx* ctx, int prec, int64_t nsteps);
ssh_status ssh_fire_state(ssh_ctx* ctx, ssh_min_result* res, int* running);

/*
 * Batch: many independent configurations of any sizes resident on one GPU, evaluated and minimised through the
 * same persistent launches (work queues of (configuration, tile) items, largest first) and graph-captured steps.
 * Every member keeps its own launch shape, so its arithmetic -- and its result -- is the same alone and in any
 * batch.  Members are numbered 0, 1, ... in the order they were added.
 */
typedef struct ssh_batch ssh_batch;
ssh_status ssh_batch_create(const ssh_opts* opts, ssh_batch** out);
void ssh_batch_destroy(ssh_batch* batch);
/* Add a configuration (as ssh_create) with fractional positions s (N*d row-major dd, s_lo may be NULL). */
ssh_status ssh_batch_add(ssh_batch* batch, int d, int64_t N, double L, double chi, double K, const double* s_hi,
                         const double* s_lo, int* slot);
/* Number of members and the total (k, particle) pairs sum_i M_i N_i of one evaluation. */
ssh_status ssh_batch_size(const ssh_batch* batch, int* n, int64_t* pairs);
/* The context of member `slot` (owned by the batch; valid until ssh_batch_destroy), for ssh_get_results,
 * ssh_get_ntilde, ssh_get_positions_frac. */
ssh_status ssh_batch_member(ssh_batch* batch, int slot, ssh_ctx** ctx);
/* The batch autotuner (no counterpart in the paper; it tunes this library's work decomposition of the tensor-core
 * GEMMs for this mix of members): each candidate is
 * timed over reps evaluations of prec, with one untimed evaluation first.  The candidates are density K-range pieces
 * per member at 50, 100, 200 or 400% of its share of the SMs, and force items in particle-tile bundles or one by
 * one.  The fastest becomes the batch's decomposition for ssh_batch_eval and its steps.  It is remembered for the
 * process per device, set of member shapes (d, N, M, chunks) and precision; a repeated call times only the default and the
 * remembered choice (candidates = 0).  Results do not change: only the order of exact integer sums does.
 * Synchronous.  Errors: SSH_EINVAL (bad arguments, empty batch, a member without positions), SSH_ECUDA. */
typedef struct {
  int dens_pieces_pct; /* chosen density pieces, % of each member's SM share (default 100) */
  int force_bundles;   /* chosen force order: 1 bundles (default), 0 one by one */
  double ms_default;   /* mean evaluation time with the defaults */
  double ms_tuned;     /* with the chosen decomposition */
  int candidates;      /* decompositions timed (0: the process's remembered choice) */
  int reserved[3];
} ssh_tune;
ssh_status ssh_batch_autotune(ssh_batch* b, int prec, int reps, ssh_tune* out);

/* Phi, S_max and F (want_force) of every member in one batched evaluation; synchronises. */
ssh_status ssh_batch_eval(ssh_batch* batch, int prec, int want_force);
/* Minimise every member to completion (p as for ssh_minimize; zero fields take each member's defaults).  Steps
 * are replayed in chunks of chunk_steps (0 = 32) between host checks; max_seconds 0 = no limit.  results: array
 * of n, may be NULL.  Returns SSH_OK if every member converged, else the first failing status. */
ssh_status ssh_batch_minimize(ssh_batch* batch, const ssh_min_params* p, int64_t chunk_steps, double max_seconds,
                              ssh_min_result* results);
/* Stepper for timing: begin every member's run (as ssh_fire_begin), then enqueue exactly nsteps batched steps
 * without synchronising (members whose run ended are skipped; stages do not advance). */
ssh_status ssh_batch_begin(ssh_batch* batch, const ssh_min_params* p);
ssh_status ssh_batch_steps(ssh_batch* batch, int64_t nsteps);
/* Event profiler of the batch's launches (see ssh_prof_enable); while on, steps are launched directly. */
ssh_status ssh_batch_prof_enable(ssh_batch* batch, int on);
ssh_status ssh_batch_prof_read(ssh_batch* batch, int n, double* ms, int64_t* launches);

/*
 * Server: ensemble requests minimised with continuous batching.  A worker thread keeps a batch of running
 * configurations resident in HBM; queued requests are admitted (smallest M N first, or first come first served)
 * while a slot is free, the request's device footprint (plans, tables, partial sums, positions, forces,
 * minimiser state) fits the HBM budget and the batch's pairs per step stay under a cap, so requests that arrive
 * while others run join the running batch and their steps share the same launches.  Every running member
 * advances one step per batched step, so the cap bounds the step time that small requests share with large
 * ones.  Finished members are retired between chunks and their memory is released.  Thread-safe.
 */
typedef struct ssh_server ssh_server;
typedef struct {
  int device;                  /* CUDA device */
  int max_slots;               /* members running at once (default 256) */
  int64_t hbm_budget_bytes;    /* device bytes for running members (default 64 GiB) */
  int64_t chunk_steps;         /* at most this many steps between admissions / retirements (default 32); fewer
                                  when steps are long, so that the host checks about every 0.1 s */
  int64_t max_pairs_per_step;  /* admission stops while the running members' sum of M N would exceed it
                                  (default 2^28, about 10 ms per step); bounds the step time that every
                                  running request shares; a larger request runs only in an empty batch */
  int policy;                  /* 0: smallest M N first (default), 1: first come first served */
  int fx_impl;                 /* fixed-point implementation of the members (ssh_opts.fx_impl) */
} ssh_server_opts;
typedef struct {
  int d;
  int want_positions;       /* 1: keep the final positions for ssh_result_positions */
  int64_t N;
  double L, chi, K;         /* as ssh_create */
  const double* s_hi;       /* initial fractional positions, N*d row-major (copied at submission) */
  const double* s_lo;       /* may be NULL */
  const ssh_min_params* params;  /* NULL = defaults */
} ssh_request;
typedef struct {
  int status;               /* SSH_OK converged, SSH_ENOTCONV, SSH_ENAN, or the admission error */
  int final_prec;
  int has_positions;
  int pad0;
  int64_t steps, rejected;
  double smax[2], phi[2];
  double t_submit, t_admit, t_done;  /* seconds since the server started */
} ssh_result;
typedef struct {
  int64_t submitted, completed, converged, running, queued, hbm_used_bytes;
} ssh_server_stats;
ssh_status ssh_server_create(const ssh_server_opts* opts, ssh_server** out);
/* Stops the worker (running members are abandoned) and frees everything. */
void ssh_server_destroy(ssh_server* server);
/* Queue a request; *ticket identifies it.  Errors: SSH_EINVAL (bad request, larger than the budget). */
ssh_status ssh_submit(ssh_server* server, const ssh_request* req, uint64_t* ticket);
/* SSH_OK with the result when finished, SSH_EBUSY while queued or running, SSH_ENOTFOUND for unknown or
 * cancelled tickets, SSH_ECUDA if the worker stopped on a device error. */
ssh_status ssh_poll(ssh_server* server, uint64_t ticket, ssh_result* out);
/* Final fractional positions (N*d row-major dd) of a finished request submitted with want_positions. */
ssh_status ssh_result_positions(ssh_server* server, uint64_t ticket, double* s_hi, double* s_lo);
/* Forget a finished request's result. */
ssh_status ssh_release(ssh_server* server, uint64_t ticket);
/* Cancel a request that is still queued (SSH_EBUSY once admitted). */
ssh_status ssh_cancel(ssh_server* server, uint64_t ticket);
ssh_status ssh_server_get_stats(ssh_server* server, ssh_server_stats* out);

/*
 * Event profiler (tracing).  When enabled, every kernel the context launches is bracketed by a CUDA event
 * pair on the context's stream; ssh_prof_read synchronises the stream and returns, per kernel id, the
 * summed device time in milliseconds and the launch count since the last ssh_prof_enable call.
 * Kernel ids: 0 twiddle tables, 1 collective density n~, 2 density reduction, 3 Phi/S_max finalise,
 * 4 force coefficients, 5 force, 6 force reduction, 7 minimiser kernels of a FIRE step (two event pairs
 * per step: update, acceptance); tensor-core fixed point (SSH_FX_TENSOR): 8 digit preparation, 9 density
 * GEMM, 10 density and force finish, 11 force coefficient digits, 12 force GEMM, 13 per-particle power
 * tables.  n entries are written (at most 16).
 */
ssh_status ssh_prof_enable(ssh_ctx* ctx, int on);

/*
 * Measured operation rate of one pipe of the current part, for roofline denominators (the paper has no
 * counterpart: it names no GPU and reports no timing).  A kernel keeps every SM busy (8 CTAs of 256 threads per
 * SM) with independent chains of one operation for about 100 ms, timed with CUDA events, best of three:
 *   SSH_PIPE_FP64_FMA  fma.rn.f64 (the pipe of the SSH_DD and SSH_FP64 kernels), per instruction
 *   SSH_PIPE_FP32_FMA  fma.rn.f32, per instruction
 *   SSH_PIPE_IMAD      mad.lo.u32 (the pipe of the integer SSH_FX kernels), per instruction
 *   SSH_PIPE_IMAD_HI   mad.hi.u32, per instruction
 *   SSH_PIPE_DD_CMAC   one complex double-double multiply plus one complex double-double add (the dd density
 *                      kernel's work per pair), per pair of operations
 *   SSH_PIPE_FX_CMUL   one product of first-quadrant 128-bit fixed-point phasors (three truncated 128 x 128-bit
 *                      products), per product
 * *ops_per_s receives the rate; *ms (may be NULL) the duration of the timed launch.  Synchronous; runs on
 * device `device` and restores the current device.  Errors: SSH_EINVAL, SSH_ECUDA.
 */
enum { SSH_PIPE_FP64_FMA = 0, SSH_PIPE_FP32_FMA = 1, SSH_PIPE_IMAD = 2, SSH_PIPE_IMAD_HI = 3, SSH_PIPE_DD_CMAC = 4,
       SSH_PIPE_FX_CMUL = 5 };
ssh_status ssh_pipe_rate(int device, int kind, double* ops_per_s, double* ms);

/*
 * Limit, in clock cycles, of every wait of the tensor-core GEMM on its pipeline (operand stages, work items, the
 * accumulator) on CUDA device `device`; 0 restores the default of 2e9 cycles (about one second at the maximum SM
 * clock).  The paper has no counterpart: it is this library's failure detection.  A wait that runs out does not
 * trap: the kernel skips its remaining work, lets its copies and MMAs in flight land (those drains always use the
 * default limit), records the failure in the error word of every configuration of that launch and returns.  The
 * host then reports SSH_ETIMEOUT: ssh_get_results / ssh_energy_grad for that evaluation, ssh_minimize,
 * ssh_fire_state, batches and the server for a run, whose failing step is undone first.  Reporting clears the
 * word, so the context stays usable.  A limit shorter than a real wait makes evaluations fail; it exists so that
 * this path can be tested.  Synchronises the device; applies to launches that start after it returns.
 * Errors: SSH_EINVAL (negative), SSH_ECUDA.
 */
ssh_status ssh_set_wait_limit(int device, int64_t cycles);

/* Cycle counters of the tensor-core GEMM, for measuring where its time goes (no counterpart in the paper; a
 * diagnostic of this library).  While enabled (for the whole process), every tensor-core GEMM launch uses a
 * second instance of the kernel that records, per CTA, clock64() cycles spent in each of its waits and phases;
 * the production instance has none of that code.  Evaluations and FIRE steps then launch their kernels directly
 * instead of replaying captured graphs, and a batch stepper rebuilt meanwhile captures none.  Enabling clears the records.  ssh_gemm_counters_read copies them out: uint64
 * out[2][256][16], [0] = the last density launch, [1] = the last force launch, one row per CTA (CTA index mod
 * 256), fields: 0 CTA cycles, 1 producer waiting for a free stage, 2 MMA thread waiting for operands, 3 MMA thread
 * waiting for the accumulator, 4 MMA thread waiting for an item, 5 epilogue waiting for the accumulator,
 * 6 epilogue read-out, 7 epilogue arithmetic and atomics, 8 items, 9 K-steps, 10 MMA thread cycles, 11 / 12 start
 * and end (global timer, ns).  Switch it while no other thread of the process launches evaluations (a server's
 * worker included): the switch is a plain process-wide flag.  Errors: SSH_EINVAL, SSH_ECUDA. */
ssh_status ssh_gemm_counters(int device, int enable);
ssh_status ssh_gemm_counters_read(int device, uint64_t* out);
ssh_status ssh_prof_read(ssh_ctx* ctx, int n, double* ms, int64_t* launches);

/*
 * Particle shards of one configuration (Simulations: both sums of a step are independent reductions over the
 * particles, so the particles can be split across GPUs with one exchange per sum).  A shard context is created
 * with ssh_opts.shard_first / shard_count over the whole configuration (N, the wavevector set and every
 * normalisation are the whole configuration's); it holds all N positions but its evaluations sum n~ over, and
 * compute F and FIRE moves for, its own particles only.  The caller owns the exchange: two device buffers that it
 * sums element-wise over every shard (an all-reduce; integer addition for the density, which is exact in any
 * order, and binary64 addition for the dot products, where each element is non-zero on one shard at most), on
 * the context's stream or after ssh_sync.  Every shard then holds the whole configuration's Phi, S_max and n~,
 * bit for bit the values of one unsharded context, and the same force and FIRE trajectory for its particles.
 * Only FIRE (the paper's minimiser) in fixed point runs sharded.  The positions of other shards' particles in a
 * shard context are never moved: read each shard's own range.  ssh_eval, ssh_energy_grad, ssh_minimize,
 * ssh_fire_begin and ssh_fire_steps return SSH_EINVAL on a shard context.
 *
 *   ssh_shard_words       int64 words of the density exchange, binary64 words of the dot-product exchange
 *   ssh_shard_density     enqueue this shard's part of the density sum (Eq. ntilde) into dens_out, a device buffer
 *                         of dens_words int64: exact level groups of the tensor-core GEMM's tiles, to be summed
 *   ssh_shard_finish      from dens_total (the sum over every shard): Phi, S_max, n~ and, with want_force, F of this
 *                         shard's particles (Eqs. energy, smax, force); read with ssh_get_results / ssh_get_ntilde
 *   ssh_shard_fire_begin  a FIRE run from the results of the last ssh_shard_finish (with force): p as for
 *                         ssh_fire_begin (method FIRE, one fixed-point stage)
 *   ssh_shard_step_dots   one FIRE step, first part: the dot products F.v, F.F, v.v of this shard's particles as
 *                         partial sums per chunk of 2048 particles into dots_out (dots_words binary64)
 *   ssh_shard_step_move   second part, from dots_total (the sum over every shard): the FIRE controls, the move of
 *                         this shard's particles and their density sum into dens_out
 *   ssh_shard_step_finish third part, from dens_total: Phi, S_max, F, the energy guard's acceptance or undo, the
 *                         stop rules; ssh_fire_state then reports the step (the same on every shard)
 * All enqueue work on the context's stream and return without synchronising.  Errors: SSH_EINVAL (not a shard
 * context, no positions, no FIRE run begun, a NULL buffer), SSH_ECUDA.
 */
ssh_status ssh_shard_words(const ssh_ctx* ctx, int64_t* dens_words, int64_t* dots_words);
ssh_status ssh_shard_density(ssh_ctx* ctx, int64_t* dens_out);
ssh_status ssh_shard_finish(ssh_ctx* ctx, const int64_t* dens_total, int want_force);
ssh_status ssh_shard_fire_begin(ssh_ctx* ctx, const ssh_min_params* p);
ssh_status ssh_shard_step_dots(ssh_ctx* ctx, double* dots_out);
ssh_status ssh_shard_step_move(ssh_ctx* ctx, const double* dots_total, int64_t* dens_out);
ssh_status ssh_shard_step_finish(ssh_ctx* ctx, const int64_t* dens_total);

/*
 * Allocation-free collective density, for callers that cannot allocate device memory: a program that hands a
 * GPU's memory to another framework's pool or arena at start-up (a cudaMalloc of its own would fail, or fragment
 * that pool behind its accounting), or a real-time loop that must not allocate after start-up (cudaMalloc and
 * cudaFree can synchronise the device and take unbounded time).  The paper has no counterpart; it is a service
 * of this library.
 *
 * Computes C_k + i S_k = sum_j exp(2 pi i n_k.s_j) for k = 0..M-1 in 128-bit fixed point, like SSH_FX,
 * with every pointer a DEVICE pointer owned by the caller: s_hi, s_lo fractional positions [N][d]
 * row-major (s_lo may be NULL), n the wavevector indices [M][d] int32, outputs C_hi, C_lo, S_hi, S_lo [M]
 * (dd), all in the order of n.  Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 * stream) and the call returns without synchronising.
 *
 * Memory: it calls no cudaMalloc / cudaFree.  Its working memory is one fixed 8 MiB device array per
 * device, present for the life of the process; calls need N*d*16 (rounded up to 256) + M*40 bytes of it
 * and larger ones are rejected with SSH_EINVAL.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) and the device's SM count; make that first call before any stream capture.  Every call on a device
 * shares the array: calls whose kernels may overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller.
 * Errors: SSH_EINVAL (arguments, size), SSH_ECUDA (no current device, launch failure).
 */
ssh_status ssh_ntilde_noalloc(int d, int64_t N, int64_t M, const double* s_hi, const double* s_lo, const int32_t* n,
                              double* C_hi, double* C_lo, double* S_hi, double* S_lo, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SSH_H_ */
