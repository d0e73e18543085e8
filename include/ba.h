/*
 * libmmba -- majorization-minimization LiDAR bundle adjustment on one GPU.
 *
 * C ABI.  Every entry point returns a ba_status (no exception crosses the
 * boundary); the message of the last failure on a handle is available from
 * ba_last_error().  A handle is not thread-safe: all its work is ordered on
 * the CUDA stream given in its configuration.  Pointers marked "host or
 * device" are read according to the mem_kind argument (BA_MEM_HOST: ordinary
 * or pinned host memory; BA_MEM_DEVICE: memory of the handle's device); the
 * library copies what it keeps, so callers keep ownership of their buffers.
 *
 * Problem (Sec. III of the paper, Eq. 1-3): N_T scans with poses
 * T_j = (R_j, t_j) in SE(3) mapping scan to world coordinates (q = R p + t)
 * observe N_f planar voxels; observation o = (voxel i, scan j) is the point
 * cluster (P_f, v_f, N) of the N points of voxel i seen by scan j, in scan
 * coordinates (Eq. 2).  The cost is c(T) = sum_i lambda_min(cov_i(T)), the
 * smallest eigenvalue of each voxel's world-point covariance (Eq. 1).  The
 * optimiser is Levenberg-Marquardt on the MM surrogate of Eq. 3, which
 * decouples the poses, so each iteration solves one damped 6x6 system per
 * scan (Algorithm 2: CalRes, CalJH, Solver).
 *
 * Data formats
 *  - pose: 12 doubles, R row-major then t (scan -> world).
 *  - cluster ("aggregate"), 10 doubles, in one of two forms:
 *      BA_AGG_RAW_SUMS: P_f = sum p p^T as (xx, xy, xz, yy, yz, zz),
 *                       v_f = sum p (x, y, z), N;
 *      BA_AGG_CENTRED:  S = sum (p - m)(p - m)^T as (xx, .., zz),
 *                       m = v_f / N (x, y, z), N.
 *    Raw sums are converted once at load: m = v / N and
 *    S_ab = fma(-v_a, m_b, P_ab).  Raw sums lose digits to cancellation when
 *    points are far from the scan origin; prefer the centred form.
 *  - observations are voxel-major CSR: voxel i owns observations
 *    voxel_offsets[i] .. voxel_offsets[i+1]-1; obs_scan[o] is the scan of o.
 *  - plane record (9 doubles per voxel): lambda0 <= lambda1 <= lambda2 of the
 *    voxel covariance, its unit eigenvector u for lambda0, the voxel
 *    centroid c.  d = u^T c.
 *  - increment per scan: (dphi, dt); the update is R' = Exp(dphi) R,
 *    t' = t + dt.
 */
#ifndef BA_H
#define BA_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ba_handle ba_handle;

typedef enum {
  BA_OK = 0,
  BA_ERR_INVALID_ARG = 1, /* malformed input; nothing was changed */
  BA_ERR_OOM = 2,         /* device allocation failed */
  BA_ERR_CUDA = 3,        /* a CUDA call failed; the handle should be destroyed */
  BA_ERR_STATE = 4,       /* call not valid in the handle's state (e.g. no data loaded) */
  BA_ERR_NUMERIC = 5,     /* the cost became NaN or infinite */
  BA_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
  BA_ERR_CAPACITY = 7     /* request exceeds a fixed capacity */
} ba_status;

enum { BA_FP64 = 0, BA_MIXED = 1 };
enum { BA_HESS_EXACT = 0, BA_HESS_GAUSS_NEWTON = 1 };
enum { BA_MEM_HOST = 0, BA_MEM_DEVICE = 1 };
enum { BA_AGG_RAW_SUMS = 0, BA_AGG_CENTRED = 1 };

typedef void* (*ba_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*ba_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

typedef struct {
  int32_t precision;         /* BA_FP64 (default) or BA_MIXED */
  int32_t max_iters;         /* ba_solve limit (default 200) */
  double rel_tol;            /* ba_solve stops after an accepted step with
                                c - c' <= rel_tol * c + abs_tol (default 1e-8) */
  double abs_tol;            /* default 0 */
  double mu0;                /* initial Marquardt damping (default 1e-4) */
  int32_t fixed_scan;        /* scan held fixed to remove the gauge freedom
                                (default 0; -1 = none) */
  int32_t hessian_mode;      /* BA_HESS_EXACT (default) or BA_HESS_GAUSS_NEWTON */
  int32_t max_consec_reject; /* ba_solve stops after this many rejected steps in a row (default 10) */
  int32_t device;            /* CUDA device ordinal (default 0) */
  void* cuda_stream;         /* cudaStream_t for all work; NULL = the legacy default stream */
  ba_alloc_fn alloc;         /* optional device allocator; NULL = cudaMallocAsync on the stream */
  ba_free_fn free;
  void* alloc_ctx;
} ba_config;

typedef struct {
  double cost;            /* cost at the current (accepted) poses */
  double cost_before;     /* cost when the call started */
  double mu;              /* current damping */
  double nu;              /* current damping growth factor */
  double last_rho;        /* gain ratio of the last step (NaN if undefined) */
  double last_pred;       /* predicted reduction of the last step */
  double last_trial_cost; /* cost at the last trial poses */
  int32_t iters;          /* LM iterations run since load (accepted or not) */
  int32_t accepted;       /* accepted steps since load */
  int32_t consec_reject;  /* rejected steps in a row */
  int32_t last_accepted;
  int32_t converged;      /* the last accepted step met the tolerance */
  int32_t solve_failed;   /* a 6x6 factorisation failed in the last step */
  int32_t iters_this_call;
  int32_t reserved;
} ba_stats;

/* Fill *cfg with the defaults listed above. */
void ba_config_default(ba_config* cfg);

/* Create a handle on cfg->device.  Allocates nothing on the device yet.
 * Errors: BA_ERR_INVALID_ARG (bad config), BA_ERR_CUDA. */
ba_status ba_create(const ba_config* cfg, ba_handle** out);

/* Load a problem given as point clusters (Eq. 2), voxel-major CSR.
 *   n_scans >= 1, n_voxels >= 1, n_obs >= n_voxels (else BA_ERR_INVALID_ARG);
 *   n_scans < 2^29, n_obs < 2^31 (else BA_ERR_CAPACITY).
 *   voxel_offsets: n_voxels + 1 int64, voxel_offsets[0] = 0, strictly
 *     increasing (every voxel has at least one observation), last = n_obs.
 *   obs_scan: n_obs int32 in [0, n_scans).
 *   agg: n_obs x 10 doubles (row per observation) in form agg_form; every N
 *     must be >= 1 and every value finite.
 *   poses: n_scans x 12 doubles, initial poses; each R orthonormal to 1e-6.
 * All four arrays live in host or device memory per mem_kind.  The library
 * validates everything (BA_ERR_INVALID_ARG names the first violation), builds
 * its device layout (voxel-sorted slices and a scan-major copy, Algorithm 1's
 * mappers; the voxels in a spatial order taken from the initial positions of
 * the scans observing them, whatever their input order), and evaluates
 * planes, cost, gradient and Hessian at the initial poses.  Replaces any previously loaded problem.  The LM state (mu, nu,
 * counters) is reset.  A mixed-precision load of host arrays copies the
 * clusters in chunks (halving in size towards the end) on a stream of the
 * handle and sets each chunk up while the next one crosses the host link;
 * the call returns when the whole load is done (or has failed, with every
 * copy drained). */
ba_status ba_load_observations(ba_handle* h, int32_t n_scans, int64_t n_voxels, int64_t n_obs,
                               const int64_t* voxel_offsets, const int32_t* obs_scan, const double* agg,
                               int32_t agg_form, const double* poses, int32_t mem_kind);

/* Same, from raw scan-frame points: observation o owns points
 * point_offsets[o] .. point_offsets[o+1]-1 (n_obs + 1 int64, at least one
 * point each), points is n_points x 3 doubles.  Clusters are formed on the
 * device in centred form (mean, then scatter about the mean). */
ba_status ba_load_points(ba_handle* h, int32_t n_scans, int64_t n_voxels, int64_t n_obs, const int64_t* voxel_offsets,
                         const int32_t* obs_scan, const int64_t* point_offsets, const double* points,
                         const double* poses, int32_t mem_kind);

/* Run exactly n_iters LM iterations (Algorithm 2 and Sec. IV-C-1: per-scan
 * damped solve A = H + mu diag(H), A delta = -g by LDL^T ("Solver"),
 * retraction, trial cost evaluation of Eq. 1 ("CalRes"), accept/reject by
 * the gain ratio and damping update ("PredResReduction", "Adjust"; the
 * Levenberg-Marquardt rule of Fig. 1, read as Nielsen's update), and on
 * acceptance the new planes, gradient and Hessian of Eq. 3 ("CalJH")).
 * The predicted reduction is L = sum_j -(g_j^T D_j + D_j^T H_j D_j / 2); a
 * step is accepted iff every factorisation succeeded, L > 0 and
 * c(T') < c(T); then mu *= max(1/3, 1 - (2 rho - 1)^3), nu = 2 with
 * rho = (c(T) - c(T')) / L, else mu *= nu, nu *= 2.  out may be NULL.  Synchronises the
 * stream only when out is given.  BA_ERR_NUMERIC if the cost became
 * non-finite.  Iterations after the solve has stopped (see ba_solve) are
 * still run. */
ba_status ba_iterate(ba_handle* h, int32_t n_iters, ba_stats* out);

/* Iterate (Algorithm 2's outer loop, Sec. IV-C-1) until an accepted step
 * meets the tolerance, max_iters iterations have run since load, or
 * max_consec_reject steps in a row were rejected.  The paper gives no stop
 * rule beyond its iteration; this one is the relative cost change of an
 * accepted step.  Synchronises the stream. */
ba_status ba_solve(ba_handle* h, ba_stats* out);

/* Current poses, n_scans x 12 doubles (R row-major, then t; scan -> world),
 * to host (synchronises) or device memory (stream-ordered).  They are the
 * accepted iterates of the update T <- T + Delta T of Sec. IV-C-1, read as
 * the retraction R' = Exp(dphi) R, t' = t + dt (Exp by Rodrigues' formula,
 * its second-order series below 1e-6 rad). */
ba_status ba_poses(ba_handle* h, double* out, int32_t mem_kind);

/* Cost c(T) = sum_i lambda_min(cov_i) of Eq. 1 at the current poses: the
 * smallest eigenvalue of each voxel's world-point covariance (1/N_i
 * normalisation), summed over voxels (synchronises). */
ba_status ba_cost(ba_handle* h, double* out);

/* LM state and counters of Algorithm 2's loop: damping mu (Sec. IV-C-1),
 * its growth factor nu, the last gain ratio and predicted reduction
 * (synchronises). */
ba_status ba_get_stats(ba_handle* h, ba_stats* out);

/* Replace the current poses (host or device, n_scans x 12) and the damping
 * state (mu, nu of Sec. IV-C-1), then re-evaluate planes, cost, gradient and
 * Hessian there (Eq. 1, Eq. 3).  With
 * this a solve can be resumed from saved poses.  mu <= 0 keeps the current
 * mu; nu <= 0 keeps the current nu.  The device layout (the voxel order,
 * and with it the order of every floating-point sum) is a function of the
 * loaded inputs, the poses passed to the load included: a resume reproduces
 * an uninterrupted solve bit for bit when it loads the same inputs and then
 * sets the saved state. */
ba_status ba_set_state(ba_handle* h, const double* poses, double mu, double nu, int32_t mem_kind);

/* Plane records (n_voxels x 9 doubles, input voxel order) at the current
 * poses: the eigen-decomposition of each voxel's covariance that Eq. 1 and
 * Eq. 3 use (lambda0..2, the normal u of lambda0, the centroid c). */
ba_status ba_planes(ba_handle* h, double* out, int32_t mem_kind);

/* Gradient (n_scans x 6) and Hessian (n_scans x 36, row-major, world frame,
 * rotation block first) of the MM surrogate of Eq. 3 at the current poses
 * (Algorithm 2, "CalJH"), with respect to the increment (dphi, dt) of the
 * retraction above.  The paper defers these derivatives to earlier work;
 * they are derived here from Eq. 3 in its fixed-plane form
 * c_M = (1/N_i) sum_k (u^T (R p_k + t) - d)^2: per observation, with
 * w = R^T u, e = u^T t - d, s = w^T v_f + N e, m = R (P_f w + e v_f),
 * g = (2/N_i) [m x u; s u] and the exact second-order H (the term
 * (u m^T + m u^T)/2 - (u^T m) I of its rotation block is dropped under
 * BA_HESS_GAUSS_NEWTON).  Either output may be NULL. */
ba_status ba_gradient(ba_handle* h, double* g, double* H, int32_t mem_kind);

/* ---- Voxel-sharded solve -------------------------------------------------
 * One problem's voxels split over several handles (e.g. one per GPU, each
 * holding whole voxels with all their observations and every scan's pose):
 * the cost (Eq. 1) and the surrogate's g and H (Eq. 3) are sums over voxels,
 * so each shard computes its part and the parts are added (an all-reduce of
 * n_scans x 27 values and a scalar per exchange); every shard then runs the
 * same deterministic per-scan solves and LM decision on the totals, and the
 * shards' poses stay bit-identical.  One iteration, on every shard:
 *   ba_shard_partials -> sum over shards -> ba_shard_set_totals
 *   ba_shard_trial    -> sum of the trial costs over shards -> ba_shard_decide
 * ba_shard_decide computes, on acceptance, the shard's g and H at the new
 * poses: read them with ba_shard_partials (their cost partial is then the
 * accepted trial cost's share; install the summed trial cost as the total).
 * After a load or ba_set_state exchange the partials again before a trial.
 *
 * ba_shard_partials: the handle's g, H (n_scans x 27 doubles: g (6), then
 * H's upper triangle row by row (21); world frame, rotation first) and cost
 * over its own voxels at the current poses, to host (synchronises) or device
 * memory (stream-ordered); either pointer may be NULL.  Call it before
 * ba_shard_set_totals, which overwrites them. */
ba_status ba_shard_partials(ba_handle* h, double* gH, double* cost, int32_t mem_kind);
/* Install the totals over all shards (gH_total in the layout above, host or
 * device; cost_total >= 0) as this handle's g, H and current cost.  From now
 * on a scan counts as unobserved only if its total Hessian diagonal is zero.
 * Synchronises. */
ba_status ba_shard_set_totals(ba_handle* h, const double* gH_total, double cost_total, int32_t mem_kind);
/* Per-scan damped solves from the totals and retraction (Algorithm 2,
 * Solver), then the trial voxel pass over this shard's voxels (CalRes);
 * *trial_cost receives this shard's part of the trial cost.  No decision.
 * Synchronises. */
ba_status ba_shard_trial(ba_handle* h, double* trial_cost);
/* The LM decision (gain ratio, Nielsen's update; as ba_iterate) with the
 * trial cost summed over every shard; on acceptance the trial poses become
 * current and the shard's g, H are computed there (CalJH).  *accepted (may be
 * NULL) receives the decision.  BA_ERR_NUMERIC if the cost is not finite.
 * Synchronises. */
ba_status ba_shard_decide(ba_handle* h, double trial_cost_total, int32_t* accepted);

/* Number of kernel launches the handle has issued since creation. */
int64_t ba_kernel_launches(const ba_handle* h);

/* Device bytes the handle holds for its loaded problem (0 if none). */
int64_t ba_device_bytes(const ba_handle* h);

/* Without a user allocator, device memory comes from a library-owned
 * stream-ordered pool per device that keeps freed memory for the next problem
 * (no unmapping and remapping between jobs).  This call waits for the device
 * to go idle and returns the pool's unused memory to the driver. */
ba_status ba_release_cached_memory(int32_t device);

/* Upper estimate of the device bytes a handle of this precision holds for a
 * problem of these sizes once loaded, and of the extra bytes its load needs
 * transiently (*peak_extra, may be NULL), for admission control. */
int64_t ba_estimate_bytes(int32_t precision, int32_t n_scans, int64_t n_voxels, int64_t n_obs, int64_t* peak_extra);

/* Per-kernel timing.  While enabled, each iteration kernel the handle
 * launches is bracketed by a pair of CUDA events recorded on the handle's
 * stream (enabling clears earlier records).  ba_profile_read synchronises
 * the stream and returns, for one kernel kind, the summed event time in
 * milliseconds and the number of launches recorded.  A scan pass launched
 * after a rejected step returns at once and is still counted.  The LM
 * decision runs in the last block of each iteration's voxel pass, so its time
 * is part of BA_KERNEL_VOXEL_PASS and BA_KERNEL_DECIDE records no launch (the
 * kind is kept for callers that read it). */
enum { BA_KERNEL_VOXEL_PASS = 0, BA_KERNEL_SCAN_PASS = 1, BA_KERNEL_SOLVE = 2, BA_KERNEL_DECIDE = 3 };
ba_status ba_profile_enable(ba_handle* h, int32_t enable);
ba_status ba_profile_read(ba_handle* h, int32_t kind, double* total_ms, int64_t* launches);

/* Release the handle and all its device memory.  NULL is ignored. */
void ba_destroy(ba_handle* h);

/* Message of the last failure on h (empty if none); for h == NULL, the last
 * failure of ba_create on this thread. */
const char* ba_last_error(const ba_handle* h);

const char* ba_status_string(ba_status s);

/* ---- Batched execution --------------------------------------------------
 * A batch steps many independent problems (jobs) together: every iteration
 * launches each kernel kind once over a device-side table of the jobs, so
 * hundreds of small jobs cost three launches per iteration instead of three
 * each.  Jobs are ordinary handles, loaded and read with the calls
 * above; each keeps its own LM state (damping, acceptance, stopping rule of
 * its own configuration) and its results are bit-identical to running it
 * alone, because every kernel block belongs to exactly one job and runs the
 * same work it would run in the job's own launch.  Jobs in one batch must be
 * on the same device and of the same precision.  The batch's iterations are
 * captured once into a CUDA graph per (membership, iteration count) and
 * replayed.  A handle may be in one batch at a time; while it is, its own
 * iterate/solve calls must not overlap the batch's work (the batch calls
 * return only after the GPU has finished). */
typedef struct ba_batch ba_batch;

/* stream: cudaStream_t for the batch's work (NULL = legacy default). */
ba_status ba_batch_create(void* stream, ba_batch** out);
/* Add a loaded handle (BA_ERR_STATE if not loaded, BA_ERR_INVALID_ARG on a
 * device or precision mismatch or if already present).  The batch does not
 * own the handle: remove it before destroying it. */
ba_status ba_batch_add(ba_batch* b, ba_handle* job);
ba_status ba_batch_remove(ba_batch* b, ba_handle* job);
int32_t ba_batch_size(const ba_batch* b);
/* Exactly n_iters LM iterations of every job (ba_iterate semantics). */
ba_status ba_batch_iterate(ba_batch* b, int32_t n_iters);
/* Iterate every job until it stops by its own configuration (ba_solve
 * semantics), in rounds of `chunk` iterations; a stopped job's blocks exit
 * at once.  *n_active_out (may be NULL) receives the number of jobs still
 * running when the call returns (0 unless max_rounds ran out;
 * max_rounds <= 0 means no limit). */
ba_status ba_batch_solve(ba_batch* b, int32_t chunk, int32_t max_rounds, int32_t* n_active_out);
/* Per-job stop flags after ba_batch_solve rounds: done_out[k] = 1 if the
 * k-th added job has stopped (n = ba_batch_size entries, host memory). */
ba_status ba_batch_done(ba_batch* b, int32_t* done_out);
void ba_batch_destroy(ba_batch* b);
const char* ba_batch_last_error(const ba_batch* b);
/* Kernel launches issued by the batch's iterations (3 per iteration). */
int64_t ba_batch_kernel_launches(const ba_batch* b);

/* Autotuner of the batch's launch settings (mixed precision only): times
 * every candidate of (register cap of the voxel pass: 4, 6 or 8 resident
 * blocks of 128 threads per SM) x (L2 prefetch distance of its slot rows: 0,
 * 2 or 4) over iters_per_trial solve iterations of the batch's own jobs, the
 * candidates interleaved over `passes` passes, and keeps the fastest for the
 * batch's later iterations.  Only settings that change no arithmetic are
 * candidates, so results are bit-identical whatever it picks; the tuning
 * iterations are real iterations of the jobs' solves (ba_batch_solve
 * semantics).  A pass during which a job stops is not counted; with no
 * complete pass the settings stay as they were (chosen = -1).  FP64 batches
 * have nothing to tune (n_candidates = 0). */
typedef struct {
  int32_t n_candidates;
  int32_t chosen;           /* index of the kept candidate, -1 if none */
  int32_t passes;           /* complete passes measured */
  int32_t min_blocks[16];
  int32_t prefetch[16];
  double ms_per_iter[16];   /* mean over the complete passes */
} ba_tune_report;
ba_status ba_batch_autotune(ba_batch* b, int32_t iters_per_trial, int32_t passes, ba_tune_report* out);
/* Per-kernel timing of the batch's iterations.  While enabled, iterations
 * are launched directly instead of through the CUDA graph (groups one after
 * another on the batch's stream), each kernel launch bracketed by a pair of
 * CUDA events; enabling clears earlier records.  ba_batch_profile_read
 * synchronises and returns, for one kernel kind (BA_KERNEL_VOXEL_PASS,
 * BA_KERNEL_SCAN_PASS, BA_KERNEL_SOLVE), the summed event time in
 * milliseconds and the number of launches (one per group and iteration). */
ba_status ba_batch_profile_enable(ba_batch* b, int32_t enable);
ba_status ba_batch_profile_read(ba_batch* b, int32_t kind, double* total_ms, int64_t* launches);
/* Apply launch settings chosen earlier (e.g. a cached ba_batch_autotune
 * result): min_blocks in {4, 6, 8}, prefetch in [0, 16].  Results do not
 * depend on them.  BA_ERR_INVALID_ARG outside those ranges. */
ba_status ba_batch_set_launch(ba_batch* b, int32_t min_blocks, int32_t prefetch);

/* ---- Served execution (continuous batching) -----------------------------
 * The paper solves one problem at a time; a server keeps many independent
 * jobs (submaps, sessions) resident on one GPU and steps them together
 * through one batch (above).  Admission is by device memory: a job is
 * accepted only if the bytes held by the resident jobs plus this job's
 * upper estimate (ba_estimate_bytes, including the load's temporaries) fit
 * in mem_budget.  A job whose own stopping rule fires leaves at the end of
 * the step: its poses and statistics are copied to host memory kept by the
 * server and its device memory is released, so later submissions fit.  A
 * job's results are bit-identical to solving it alone in a batch of one
 * with the same iterations per step.  Not thread-safe; every call runs on
 * the configuration's stream. */
typedef struct ba_server ba_server;

/* One job's problem, as for ba_load_observations (host or device per
 * mem_kind; the server copies what it keeps during ba_server_submit). */
typedef struct {
  int32_t n_scans;
  int64_t n_voxels;
  int64_t n_obs;
  const int64_t* voxel_offsets; /* n_voxels + 1 */
  const int32_t* obs_scan;      /* n_obs */
  const double* agg;            /* n_obs x 10 */
  int32_t agg_form;             /* BA_AGG_RAW_SUMS | BA_AGG_CENTRED */
  const double* poses;          /* n_scans x 12, initial */
  int32_t mem_kind;             /* BA_MEM_HOST | BA_MEM_DEVICE */
} ba_job_desc;

/* cfg configures every job (precision, stopping rule, device, stream,
 * allocator); mem_budget > 0 bytes.  Errors: BA_ERR_INVALID_ARG. */
ba_status ba_server_create(const ba_config* cfg, int64_t mem_budget, ba_server** out);
/* Load a job now if it fits next to the resident jobs; *job_id receives its
 * id (ids start at 1 and are never reused).  BA_ERR_CAPACITY: it does not
 * fit now; nothing was loaded and the caller may submit it again after a
 * step has retired jobs.  BA_ERR_INVALID_ARG: malformed job (as
 * ba_load_observations) or a job larger than the whole budget. */
ba_status ba_server_submit(ba_server* s, const ba_job_desc* job, uint64_t* job_id);
/* One round: first the asynchronously submitted jobs whose load has finished
 * join the batch (when nothing is resident but loads are in flight, the call
 * waits up to 100 ms for one); then n_iters LM iterations (ba_solve
 * semantics) of every resident job that has not stopped, then retirement of
 * the jobs that stopped.  *n_resident_out and *n_retired_out (either may be
 * NULL) receive the jobs still resident and the jobs retired by this step. */
ba_status ba_server_step(ba_server* s, int32_t n_iters, int32_t* n_resident_out, int32_t* n_retired_out);
/* *done = 0: the job is resident or still being admitted.  *done = 1: it has
 * finished; its poses (n_scans x 12 doubles, host) and statistics are copied
 * to poses_out and stats_out (either may be NULL) and the server forgets the
 * job, so a later poll of the same id is BA_ERR_INVALID_ARG (as is an
 * unknown id).  A job whose asynchronous admission failed polls once with
 * *done = 1 and the failure's status (its message in
 * ba_server_last_error); the server then forgets it. */
ba_status ba_server_poll(ba_server* s, uint64_t job_id, int32_t* done, double* poses_out, ba_stats* stats_out);
/* Cancel a job: a resident job leaves the batch at once (its device memory
 * is released; the other jobs' results do not change), a finished job's
 * unpolled results are dropped, a job still being admitted is dropped when
 * its load returns (at once if the load has not started).
 * BA_ERR_INVALID_ARG for an unknown id. */
ba_status ba_server_cancel(ba_server* s, uint64_t job_id);
/* Asynchronous admission.  Charges the job's estimate plus its load's
 * transient peak against the budget now (BA_ERR_CAPACITY / BA_ERR_INVALID_ARG
 * as ba_server_submit) and returns its id at once; a library loader thread then
 * creates the job's handle on a CUDA stream of its own, makes that stream
 * wait for the work already queued on input_stream (a cudaStream_t the
 * caller produced the inputs on, e.g. a side stream generating them; NULL =
 * the inputs are ready now), loads the job (validation, layout build,
 * set-up) and synchronises that stream, while the caller's thread goes on
 * stepping the resident jobs.  The job joins the batch at the first
 * ba_server_step after its load finished, and from then on is charged like
 * a synchronously admitted job.  The inputs described by job (host or device
 * memory) must stay valid and unchanged until ba_server_job_state leaves
 * BA_JOB_LOADING.  A failed load is reported by ba_server_poll.  A user
 * allocator in the configuration is then called from the loader threads.
 * The other ba_server_* calls stay single-threaded: make them from one
 * thread. */
enum { BA_JOB_UNKNOWN = -1, BA_JOB_LOADING = 0, BA_JOB_RESIDENT = 1, BA_JOB_FINISHED = 2, BA_JOB_FAILED = 3 };
ba_status ba_server_submit_async(ba_server* s, const ba_job_desc* job, void* input_stream, uint64_t* job_id);
/* Where a job is: BA_JOB_LOADING (its inputs are still read), BA_JOB_RESIDENT
 * (loaded; joined or about to join the batch), BA_JOB_FINISHED (results
 * waiting for ba_server_poll), BA_JOB_FAILED (admission failed; poll it for
 * the reason), BA_JOB_UNKNOWN. */
int32_t ba_server_job_state(ba_server* s, uint64_t job_id);
/* Jobs submitted asynchronously that have not joined the batch yet. */
int32_t ba_server_loading(const ba_server* s);
/* Number of loader threads (1 .. 16, default 3), each loading one job at a
 * time; only before the first ba_server_submit_async (BA_ERR_STATE after). */
ba_status ba_server_set_loaders(ba_server* s, int32_t n);
/* 1 if a job of these sizes would be admitted now, else 0 (lets a caller
 * prepare a job's inputs only when they can be taken). */
int32_t ba_server_fits(const ba_server* s, int32_t n_scans, int64_t n_voxels, int64_t n_obs);
/* Device bytes held by the resident jobs (what admission charges). */
int64_t ba_server_bytes_in_use(const ba_server* s);
int32_t ba_server_resident(const ba_server* s);
/* Kernel launches of the server's batch. */
int64_t ba_server_kernel_launches(const ba_server* s);
const char* ba_server_last_error(const ba_server* s);
/* Releases every resident job and the finished results not yet polled. */
void ba_server_destroy(ba_server* s);

/* Stateless point-cluster formation (Eq. 2) on the device: for each of n_obs
 * observations with points point_offsets[o] .. point_offsets[o+1]-1 of
 * points (n x 3 doubles), write the centred cluster (S, m, N) to
 * agg_out[10 * o ..].  The sums of the points' deviations from the
 * observation's first point are exact (fixed-point integers at half the last
 * bit of that point's largest coordinate; smaller coordinates rounded to
 * it); m and S are formed from them in FP64.  Observations outside that
 * range (see layout.cu) take the same sums in FP64.  All pointers are device
 * memory; stream is a cudaStream_t (NULL = legacy default).  Observations
 * with no point get N = 0 and zeros.  Errors: BA_ERR_INVALID_ARG (n_obs < 0
 * or NULL pointers), BA_ERR_CUDA. */
ba_status ba_aggregate_points(int64_t n_obs, const int64_t* point_offsets, const double* points, double* agg_out,
                              void* stream);

/* ---- Preprocessing: raw scans -> observations (Sec. IV-B, Algorithm 1) -----
 * L1 voxelisation (Eq. 4): every point p of scan j goes to world coordinates
 * w = R_j p + t_j (each axis fma(R_a0, p0, fma(R_a1, p1, fma(R_a2, p2,
 * t_a))), the index floor(w / d) per axis, the floor of the correctly
 * rounded quotient; the points of one scan in one voxel form one centred
 * cluster (Eq. 2), summed in point order as shifted sums (deviations from
 * the run's first point) in fixed chunks, so results are deterministic and
 * agree with the mean-then-scatter definition to rounding.  Bottom-up levels
 * (Eq. 5): the level-k index of a level-(k-1) cluster is floor(index / 2)
 * per axis, and the clusters with the same (level-k index, scan) are merged
 * in scan-then-child order; level k has voxel size 2^(k-1) d.
 * Selection (Algorithm 1, Selection): a voxel is kept if it has at least
 * min_obs observations and, for tau > 0, the smallest eigenvalue of the
 * covariance of its points at the given poses is below tau times the second
 * smallest (tau <= 0 keeps every voxel).
 * Output: voxels of all levels (level 1 first, each level by index x, y, z),
 * the observations of a voxel by scan; voxel_off / obs_scan / agg (centred,
 * scan coordinates) load directly with ba_load_observations(BA_AGG_CENTRED).
 * Indices must lie in [-2^20, 2^20) (BA_ERR_CAPACITY otherwise); at most
 * 2^32 - 1 points per call.
 * Adaptive asynchronous loader (Sec. IV-B): points in host memory, or more
 * points than one batch holds, are processed in batches of whole scans (a
 * scan longer than a batch is split) of batch_points points, or of the share
 * alpha of the free device memory.  Host batches are copied on a separate
 * stream, by a library thread, into two device buffers while the previous
 * batch is clustered, so only two batches of points are ever on the device;
 * the batches' level-1 clusters are then ordered by one sort and the pieces
 * of split scans merged.  Pinned host memory lets the copies run at full
 * speed; pageable memory works too.  The result does not depend on the
 * batching beyond the rounding of clusters of split scans. */
typedef struct {
  double voxel_size;  /* d, the level-1 voxel edge (default 1.0) */
  int32_t levels;     /* L >= 1 (default 1) */
  double tau;         /* planarity threshold (default 0: keep all) */
  int32_t min_obs;    /* observations a voxel needs to be kept (default 1) */
  int32_t device;     /* CUDA device (default 0) */
  void* cuda_stream;  /* cudaStream_t (NULL = legacy default) */
  int32_t profile;    /* nonzero: time the stages with CUDA events (default 0) */
  int64_t batch_points; /* points per batch of the loader (0 = from alpha) */
  double alpha;         /* share of free device memory for point batches (default 0.25) */
} ba_voxelize_config;

/* Stages timed when profile is set (ba_voxels_stage_ms): world points and
 * level-1 keys; the level-1 sort (with the key packing); the (voxel, scan)
 * runs of the sorted points (includes one host synchronisation); the
 * clusters' chunked sums; their per-run finish; all higher levels (includes
 * host synchronisations); the selection's per-observation terms and
 * per-voxel test; the output writes; the ordering of the batches' level-1
 * clusters (batched calls only). */
enum {
  BA_VOX_KEYS = 0,
  BA_VOX_SORT = 1,
  BA_VOX_RUNS = 2,
  BA_VOX_CLUSTER_PASS = 3,
  BA_VOX_CLUSTER_FINISH = 4,
  BA_VOX_LEVELS = 5,
  BA_VOX_SELECT = 6,
  BA_VOX_EMIT = 7,
  BA_VOX_MERGE = 8,
  BA_VOX_STAGES = 9
};

typedef struct ba_voxels ba_voxels;

void ba_voxelize_config_default(ba_voxelize_config* cfg);
/* Points of scan j are points[scan_point_off[j] .. scan_point_off[j+1]-1]
 * (n x 3 doubles, scan frame); poses n_scans x 12 (scan -> world).  All three
 * arrays in host or device memory per mem_kind (the library copies them).
 * On success *out owns the result on the device (free with
 * ba_voxels_destroy).  Errors: BA_ERR_INVALID_ARG (malformed offsets,
 * non-finite poses, bad config), BA_ERR_CAPACITY, BA_ERR_OOM, BA_ERR_CUDA;
 * the message is in ba_voxelize_last_error() of the calling thread. */
ba_status ba_voxelize(const ba_voxelize_config* cfg, int32_t n_scans, const int64_t* scan_point_off,
                      const double* points, const double* poses, int32_t mem_kind, ba_voxels** out);
ba_status ba_voxels_size(const ba_voxels* v, int64_t* n_voxels, int64_t* n_obs);
/* Copy the result out (any pointer may be NULL): voxel_off (n_voxels + 1),
 * obs_scan (n_obs), agg (n_obs x 10), level (n_voxels), index (n_voxels x 3). */
ba_status ba_voxels_read(const ba_voxels* v, int64_t* voxel_off, int32_t* obs_scan, double* agg, int32_t* level,
                         int32_t* index, int32_t mem_kind);
int64_t ba_voxels_kernel_launches(const ba_voxels* v);
/* Number of loader batches the call used (0 when there were no points). */
int64_t ba_voxels_batches(const ba_voxels* v);
/* Device milliseconds of one stage (summed over levels) of the call that made
 * v; 0 when it was not profiled.  BA_ERR_INVALID_ARG for a bad stage. */
ba_status ba_voxels_stage_ms(const ba_voxels* v, int32_t stage, double* ms);
const char* ba_voxelize_last_error(void);
void ba_voxels_destroy(ba_voxels* v);

/* Check of the device-side wait bound (the paper has no counterpart).  The
 * staged scan pass of the mixed path waits on mbarriers for its bulk copies,
 * and every such wait gives up after a bounded number of polls, sets a flag
 * and lets the host return BA_ERR_TIMEOUT instead of hanging.  This call runs
 * one warp on `device` that waits on an mbarrier nothing arrives on, with a
 * limit of `polls` polls (1 .. 1e6), and then a follow-up launch.  Returns
 * BA_OK if the wait gave up and the context still works, BA_ERR_TIMEOUT if
 * the wait did not give up, BA_ERR_INVALID_ARG / BA_ERR_CUDA otherwise. */
ba_status ba_check_bounded_wait(int32_t device, int32_t polls);

/* Check of the set-up's integer-arithmetic conversions between binary64 and
 * binary32 (the paper has no counterpart): n pseudo-random and special values
 * (seeded) are converted both ways by them and by the hardware on `device`;
 * mismatches[0] / [1] receive the number of differing binary64 -> binary32 /
 * binary32 -> binary64 results (0 expected).  Errors: BA_ERR_INVALID_ARG,
 * BA_ERR_CUDA. */
ba_status ba_check_conversions(int32_t device, int64_t n, uint64_t seed, uint64_t* mismatches);

/* Allocation-free cost evaluation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they need
 * a cost -- a mapping loop on a vehicle under a fixed memory budget, where
 * cudaMalloc/cudaFree may synchronise the device and stall the loop, or an
 * application whose own allocator already holds the GPU's memory.
 *
 * Computes the cost -- the sum over voxels of the smallest eigenvalue of the
 * covariance of the voxel's points placed by the poses -- for the caller's
 * voxel-major CSR clusters in centred form (n_obs x 10 doubles), poses
 * (n_scans x 12) and offsets/scan indices, all device memory of the calling
 * thread's current device, and writes the cost to *cost_out (device) and,
 * if lambda0_out is not NULL, each voxel's smallest eigenvalue (device,
 * n_voxels doubles).  Work is ordered on `stream` (a cudaStream_t, NULL =
 * legacy default); the call does not synchronise.
 *
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Its
 * scratch (block partials and an error word) is one file-scope device array
 * of (BA_NOALLOC_MAX_VOXELS / 128 + 32) doubles (512 KB plus 256 bytes)
 * that every GPU loading the library holds until the process exits.  The
 * first call on a device looks up that array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the array and it keeps the last call's contents; each
 * call overwrites the partials it sums and re-arms the error word itself, so
 * nothing has to be cleared by the caller -- but calls whose work overlaps
 * on the GPU (different streams, or several host threads) race on it and
 * must be serialised by the caller.
 *
 * The looked-up address is cached per device for the life of the process;
 * it does not survive cudaDeviceReset or any other teardown of the device's
 * primary context, so do not call this entry point across such a reset.
 *
 * Errors: BA_ERR_INVALID_ARG (sizes below 1, n_obs < n_voxels, NULL
 * pointers), BA_ERR_CAPACITY (n_voxels > BA_NOALLOC_MAX_VOXELS),
 * BA_ERR_CUDA (no current device or one of its launches failed; an error
 * left pending by earlier, unrelated work on the calling thread is cleared
 * on entry and not reported by this call).  Offsets or scan
 * indices found out of range on the device leave the cost NaN (and the
 * voxel's lambda0 NaN); inputs are otherwise not validated. */
#define BA_NOALLOC_MAX_VOXELS 8388608
ba_status ba_eval_cost_noalloc(int32_t n_scans, int64_t n_voxels, int64_t n_obs, const int64_t* voxel_offsets,
                               const int32_t* obs_scan, const double* agg_centred, const double* poses,
                               double* cost_out, double* lambda0_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
