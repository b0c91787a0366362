/*
 * vrps.h -- C ABI of the GB300 (sm_103a) variance-reduced ProxSkip tomography library.
 *
 * Method: Papoutsellis, Kereta, Papafitsoros, "Split, Skip and Play: Variance-Reduced
 * ProxSkip for Tomography Reconstruction is Extremely Fast" (arXiv 2602.09527).
 * The library solves Eq. (tomography_problem), Section 2.1,
 *     min_x  1/2 ||A x - b||^2 + alpha TV(x) + I_{x >= 0}(x),
 * with A a Joseph (linear-interpolation) discretisation of the Radon transform, split into
 * N staggered subsets of projection angles (Section 1.2; Fig. 1 caption), and the
 * algorithms of Algorithm 1 (ISTA, FISTA, ProxSGD/SAGA/SVRG/L-SVRG and their Skip variants).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every array argument named x, y, r, v, b, dual, out is a DEVICE pointer on the current
 *    CUDA device unless the comment says "host".  Arrays are float32, densely packed,
 *    caller-owned; the library never frees or retains them past the call.
 *  - Image layout: 2D row-major [ny][nx]; 3D [nz][ny][nx] (x fastest).
 *    Sinogram layout: 2D [rows][n_bins]; 3D [rows][nv][nu]; for a subset, row r is the
 *    r-th angle (view) of the subset in increasing angle index.
 *  - Subset i (0 <= i < N) holds angles {i, i+N, i+2N, ...}; subset -1 means all angles
 *    in natural order.
 *  - Calls are asynchronous on `stream` (cudaStream_t; NULL = the legacy default stream)
 *    unless documented otherwise.  Two calls that share one geometry handle must not run
 *    concurrently: the handle owns scratch buffers used by proj_fwd, prox_tv and solve.
 *  - Every call returns an int status: VRPS_OK (0) or a negative VRPS_ERR_* code; the
 *    message of the last failure on the calling thread is vrps_last_error().  No C++
 *    exception crosses this boundary.  Invalid arguments are rejected before any launch.
 */
#ifndef VRPS_H
#define VRPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* vrps_stream_t;   /* identical to cudaStream_t */
typedef struct vrps_geom vrps_geom;         /* opaque, library-owned */

enum vrps_status {
  VRPS_OK = 0,
  VRPS_ERR_INVALID_ARG = -1,   /* bad size, pointer, enum value or geometry */
  VRPS_ERR_OUT_OF_MEMORY = -2, /* a library-owned allocation failed */
  VRPS_ERR_CUDA = -3,          /* a CUDA runtime call or kernel launch failed */
  VRPS_ERR_TIMEOUT = -4,       /* a bounded device-side wait expired */
  VRPS_ERR_DIVERGED = -5,      /* the objective became non-finite */
  VRPS_ERR_UNSUPPORTED = -6,   /* valid request outside what this build implements */
  VRPS_ERR_INTERNAL = -7       /* a self-test found the library misbehaving */
};

enum vrps_algo {               /* Algorithm 1 and its estimator table */
  VRPS_ALGO_ISTA = 0,          /* full gradient, prox every iteration */
  VRPS_ALGO_FISTA = 1,         /* ISTA + Beck-Teboulle momentum */
  VRPS_ALGO_SVRG = 2,          /* ProxSVRG (p = 1) */
  VRPS_ALGO_SAGA = 3,          /* ProxSAGA (p = 1) */
  VRPS_ALGO_PROXSKIP = 4,      /* full gradient, prox with probability p */
  VRPS_ALGO_VR_PROXSKIP = 5    /* estimator from opts, prox with probability p */
};

enum vrps_estimator {
  VRPS_EST_SVRG = 0,           /* snapshot every N iterations */
  VRPS_EST_SAGA = 1,           /* table of subset gradients (stored as subset residuals) */
  VRPS_EST_LSVRG = 2,          /* snapshot refreshed with probability 1/N */
  VRPS_EST_SGD = 3             /* plain subset gradient, no variance reduction */
};

/* Message of the last failed call on this thread ("" if none).  Valid until the next call. */
const char* vrps_last_error(void);
/* ABI version (major*10000 + minor*100 + patch). */
int vrps_version(void);

/* ---------------------------------------------------------------- geometry
 * 2D parallel beam (Section 2.1, "discrete Radon transform"; projector choice: Joseph).
 * Pixel (ix,iy) centre ((ix-(nx-1)/2) pixel, (iy-(ny-1)/2) pixel); bin j at
 * s_j = (j-(n_bins-1)/2) bin_spacing; ray {x cos t + y sin t = s_j}.
 * angles_rad: HOST array of n_angles float64 angles, copied.  n_subsets: N >= 1 (<= n_angles).
 * On success *out receives a handle bound to the current device; free with vrps_geom_free.
 * Errors: INVALID_ARG (sizes <= 0, spacings <= 0, NULL pointers), OUT_OF_MEMORY, CUDA. */
int vrps_geom_par2d(int nx, int ny, double pixel, int n_angles, const double* angles_rad,
                    int n_bins, double bin_spacing, int n_subsets, vrps_geom** out);

/* 3D circular cone beam.  Source S = sod (cos b, sin b, 0); detector centre
 * -(sdd-sod)(cos b, sin b, 0); detector axes e_u = (-sin b, cos b, 0), e_v = (0,0,1);
 * pixel (iu,iv) centre (iu-(nu-1)/2) du, (iv-(nv-1)/2) dv.  Voxel (ix,iy,iz) centre
 * ((i-(n-1)/2) voxel).  betas_rad: HOST array of n_views float64 source angles, copied.
 * Errors: INVALID_ARG as above, more than 65535 views or 65536 detector columns or rows, or
 * when the source lies inside the volume's bounding circle; UNSUPPORTED when a ray would be
 * marched along z (cone angle above 45 degrees). */
int vrps_geom_cone3d(int nx, int ny, int nz, double voxel, int n_views, const double* betas_rad,
                     int nu, int nv, double du, double dv, double sod, double sdd,
                     int n_subsets, vrps_geom** out);

/* Releases the handle and every library-owned device buffer it holds.  NULL is accepted.
 * Synchronises the device before freeing. */
int vrps_geom_free(vrps_geom* g);

/* Sizes: n = image elements, m = sinogram elements (all angles), rows of subset `subset`
 * (-1: all) and elements per row (n_bins or nu*nv).  Any output pointer may be NULL. */
int vrps_geom_sizes(const vrps_geom* g, int subset, int64_t* n, int64_t* m, int* rows,
                    int* row_len, int* dims);

/* Number of Joseph samples of subset `subset` (-1: all angles): pairs (ray, dominant-axis
 * line or plane) at which at least one interpolation tap lies inside the image, counted on
 * the host in float64.  One sample is one "ray-voxel" of the projector throughput metric. */
int vrps_geom_samples(const vrps_geom* g, int subset, int64_t* samples);

/* Launch-shape autotuner (no counterpart in the paper).  For a 2D geometry, times subset 0's
 * forward for shared-memory bands of 16 ... 96 KB walked one or 2, 4, 8 bands per CTA
 * (double-buffered copies), and its adjoint with one and two pixels per thread (CUDA events,
 * best of `reps` after one warm-up), and keeps the fastest of each in the handle; later
 * projections, solves and batched jobs on the handle use them.  Results change only the
 * grouping of floating-point sums (outputs agree to rounding).  out4 (HOST, nullable, 4
 * doubles): chosen band bytes, pixels per thread, tuned forward + adjoint time in
 * microseconds, bands per CTA; the adjoint's angle shares per pixel tile (1, 2, 4: partial sums
 * added in share order by the last share) are timed with the pixels per thread, and the 2D FGP
 * output tile (32 wide with a balanced height, 32 x 16 or 16 x 16) on a 32-iteration prox call
 * (see vrps_launch_shape);
 * with more than one subset the all-angle forward and adjoint get their own band / bands per
 * CTA and angle shares, timed on the full sinogram (see vrps_launch_shape_full).
 * 3D geometries: times three iterations of the streaming FGP prox for chunks of 4 ... 128 z
 * planes, and subset 0's adjoint with 16 and 32 voxels per thread along z, and keeps the
 * fastest of each (out4: FGP chunk, adjoint voxels per thread, FGP time and adjoint time in
 * microseconds); untuned, the FGP chunk is the longest of 64, 32, 16, 8 planes giving at least
 * 8 CTAs per SM, else 4, and the adjoint takes 16 voxels.  Neither changes the results.
 * Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA. */
int vrps_autotune(vrps_geom* g, int reps, double* out4, vrps_stream_t stream);

/* Sets the launch shapes by hand (0 = built-in default for each): forward band bytes, forward
 * bands per CTA, adjoint pixels per thread (2D: 1 or 2; 3D: voxels per thread along z, 16 or
 * 32), 3D FGP planes per chunk, 2D FGP output tile (0: 32 columns by 32 or 27 rows, whichever
 * gives the busiest SM less work when the tiles are spread over the SMs -- 27 at 512^2 and
 * 1024^2 on 152 SMs; 1: 32 x 16; 2: 16 x 16; 3: 32 x 32; 4: 32 x 27; all give the same bits),
 * adjoint angle shares per tile.  Errors: INVALID_ARG. */
int vrps_set_launch_shape(vrps_geom* g, int fwd_band_bytes, int fwd_group, int adj_pixels_per_thread,
                          int fgp3_chunk, int fgp_tile, int adj_split);
/* Current launch shapes of the handle in the same order (HOST int[6]; 0 = default; the 3D FGP
 * chunk is reported as the effective one for 3D geometries). */
int vrps_launch_shape(const vrps_geom* g, int* out6);
/* 2D geometries: launch shapes of the all-angle passes (SVRG snapshots, full gradients,
 * full-sinogram projections), which vrps_autotune times separately on the full sinogram
 * (HOST int[3]: forward band bytes, forward bands per CTA, adjoint angle shares; 0 = as for
 * subsets; vrps_set_launch_shape resets them to 0).  Errors: INVALID_ARG. */
int vrps_launch_shape_full(const vrps_geom* g, int* out3);

/* ---------------------------------------------------------------- operators
 * y = A_i x  (Section 1.2: the forward operator of subset i; i = -1 for A).
 * x: [n] image.  y: [rows(i) * row_len] sinogram rows of subset i, overwritten.
 * Ray-driven gather; no atomics.  Errors: INVALID_ARG (NULL, subset out of range). */
int vrps_proj_fwd(const vrps_geom* g, int subset, const float* x, float* y, vrps_stream_t stream);

/* Synchronises `stream`, then reads and clears the handle's device error word: returns
 * VRPS_ERR_TIMEOUT when a bounded device-side wait of an earlier call on this handle expired
 * since the last check (the 2D forward projector waits, with an iteration limit, for its
 * bulk copies, and the CTAs of the 2D prox's cooperative launch wait, with a poll limit, at a
 * grid barrier between blocks of iterations; an expired wait leaves that projection or prox
 * incomplete), VRPS_OK otherwise.
 * vrps_solve, vrps_power_iteration and vrps_objective check the word themselves; callers of
 * the asynchronous vrps_proj_fwd / vrps_proj_adj / vrps_prox_tv check it with this call.
 * No counterpart in the paper.  Errors: INVALID_ARG, CUDA, TIMEOUT. */
int vrps_check_error(const vrps_geom* g, vrps_stream_t stream);

/* Self-test of the device-side bounded waits (no counterpart in the paper): one CTA arrives at
 * the 2D prox's grid barrier on a fresh counter that needs two arrivals, so its wait can only
 * end by its poll limit (`polls`, 1 ... 2^24); checks on the host that the wait gave up, set
 * the error word and let the kernel return, and that the device still runs work afterwards.
 * Synchronises `stream`.  Returns VRPS_OK when all of that held.  Errors: INVALID_ARG (polls
 * outside the range), OUT_OF_MEMORY, CUDA, INTERNAL (the wait did not report its expiry). */
int vrps_selftest_bounded_wait(unsigned polls, vrps_stream_t stream);

/* x = A_i^T r, the exact transpose of vrps_proj_fwd for the same subset, computed
 * pixel (voxel) by pixel as a gather over the rays that touch it; no atomics.
 * r: [rows(i) * row_len]; x: [n], overwritten.  Errors as vrps_proj_fwd. */
int vrps_proj_adj(const vrps_geom* g, int subset, const float* r, float* x, vrps_stream_t stream);

/* x = prox_{tau g}(v), g = TV (+ I_{x>=0} when nonneg != 0): Eq. (proximal_definition)
 * solved by `iters` iterations of FGP on the dual (Section 2.1; Beck & Teboulle 2009).
 * dual: NULL for a cold start (zero dual), or a [dims * n] float32 buffer holding the
 * warm-start dual on entry and the final dual on exit (component-major: d/dx, d/dy[, d/dz]).
 * v and x may not alias; iters >= 0 (0 returns the projection with the given dual);
 * tau > 0.  Uses library-owned scratch of 2 * dims * n floats held by the handle.
 * Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA. */
int vrps_prox_tv(const vrps_geom* g, const float* v, float* x, float tau, int iters, int nonneg,
                 float* dual, vrps_stream_t stream);

/* Allocation-free variant of vrps_prox_tv for 2D images (the paper has no counterpart; it
 * exists for callers that cannot let a library allocate device memory -- for example an
 * application that owns the whole device-memory budget through its own pool, or a
 * latency-critical loop where the implicit synchronisation of cudaMalloc is not acceptable).
 * Same operation and arguments as vrps_prox_tv on an nx x ny image (v, x: [nx*ny], dual:
 * NULL or [2*nx*ny], caller-owned device buffers), but no geometry handle and no
 * allocation: the scratch lives in a fixed array in device global memory of
 * VRPS_NOALLOC_MAX_PIXELS x 10 floats (about 10 MB).  With CUDA's default lazy module loading
 * a GPU reserves that array when this entry point first runs on it (with
 * CUDA_MODULE_LOADING=EAGER, every GPU that loads the library reserves it) and keeps it until
 * the process exits.  nx*ny above VRPS_NOALLOC_MAX_PIXELS is rejected with INVALID_ARG.
 * The first call on each device looks up the array's device address (with that device
 * current) and caches it for the process; make that first call before any stream capture,
 * and do not use the entry point on a device after cudaDeviceReset (the cached address would
 * be stale).  All calls share the array, which keeps the last call's contents (a cold start
 * clears its dual): calls that overlap on the GPU -- on different streams, or from different
 * host threads -- race with each other and must be serialised by the caller. */
#define VRPS_NOALLOC_MAX_PIXELS (512 * 512)
int vrps_prox_tv2d_noalloc(int nx, int ny, const float* v, float* x, float tau, int iters, int nonneg,
                           float* dual, vrps_stream_t stream);

/* L = lambda_max(A^T A) by `iters` power iterations from a Philox4x32-10 start vector
 * (key = seed, counter = (e/4, 0, 0, 1), element e takes word e%4, value (u+0.5)/2^32),
 * with float64 inner products.  *L_out is a HOST double; the call synchronises `stream`.
 * Sets the step sizes of Section 3 (gamma = factor / L). */
int vrps_power_iteration(const vrps_geom* g, int iters, uint64_t seed, double* L_out,
                         vrps_stream_t stream);

/* Objective of Eq. (tomography_problem) at x (the indicator is not evaluated):
 * out3 (HOST, 3 doubles) = { F, 1/2||Ax-b||^2, TV(x) } with float64 reductions.
 * b: [m] sinogram, all angles, natural order.  Synchronises `stream`. */
int vrps_objective(const vrps_geom* g, const float* x, const float* b, double alpha,
                   double* out3, vrps_stream_t stream);

/* Draws of Algorithm 1 for iterations k0 .. k0+count-1 (device int32 [count][3]):
 * Philox4x32-10 with key (seed mod 2^32, seed >> 32), counter (k mod 2^32, k >> 32, job, 0);
 * [0] = subset i_k = floor(u0 N / 2^32), [1] = skip coin theta_k = (u1 < floor(p 2^32)),
 * 1 when p >= 1, [2] = L-SVRG refresh coin (u2 < floor(2^32 / N)). */
int vrps_philox_schedule(uint64_t seed, uint32_t job, int64_t k0, int count, int n_subsets,
                         double p, int32_t* out, vrps_stream_t stream);

/* ---------------------------------------------------------------- instrumentation
 * Launch accounting and kernel timing (no counterpart in the paper; used to measure the
 * kernels against their roofline).  vrps_kernel_launches(): cumulative number of CUDA
 * kernels this library has launched in the process.  While profiling is enabled every
 * launch is bracketed by CUDA events recorded on the launching stream; vrps_profile_read
 * synchronises the device, folds the elapsed times into per-kernel totals and copies up to
 * `cap` entries (HOST array) with *count set to the number of kernel families seen.  `bytes`
 * sums the launches' algorithmic DRAM traffic: each float32 array the launch must read or
 * write, counted once (0 for kernels that state none).
 * vrps_profile_enable(0) stops recording and clears the totals. */
typedef struct vrps_kernel_stat {
  char name[32];
  uint64_t launches;
  double total_ms;
  double bytes;
} vrps_kernel_stat;

uint64_t vrps_kernel_launches(void);
int vrps_profile_enable(int on);
int vrps_profile_read(vrps_kernel_stat* out, int cap, int* count);

/* ---------------------------------------------------------------- solver */
typedef struct vrps_solve_opts {
  int estimator;      /* vrps_estimator, used by VRPS_ALGO_VR_PROXSKIP */
  int fgp_iters;      /* FGP inner iterations per prox call (>= 0) */
  int max_iters;      /* outer iterations K (> 0) */
  int nonneg;         /* 1: include I_{x>=0} in the prox */
  int power_iters;    /* iterations of the Lipschitz estimate when gamma <= 0 */
  int eval_every;     /* evaluate F every this many iterations (0: never) */
  double f_star;      /* reference optimum for the relative gap (used when target_gap > 0) */
  double target_gap;  /* stop at the first evaluation with (F - f_star)/|f_star| <= this */
  const float* x0;    /* optional initial image [n] (NULL: zeros) */
  double* history;    /* optional HOST [history_cap][4]: iteration, F, seconds, data passes */
  int history_cap;
  int host_io;        /* 1: b and x_out are HOST pointers (copied inside the call) */
  int n_subsets;      /* 0: the geometry's N; otherwise the number of subsets for this solve */
  uint32_t job;       /* Philox counter word 2 (independent streams for batched jobs) */
  int storage;        /* vrps_storage of the solver's copy of b and of the estimator table
                       * (SVRG: A x~; SAGA: residual rows); arithmetic is float32 either way */
  int correction_epochs; /* with BF16 storage: the last correction_epochs * N iterations switch
                       * to float32 storage, starting from an exact float32 full gradient
                       * (SVRG: a snapshot; SAGA: the table rebuilt at the current point;
                       * 0: no switch; the whole run must then be longer than the switch) */
} vrps_solve_opts;

/* Storage of sinogram-sized solver state (not in the paper: a precision/footprint choice). */
typedef enum vrps_storage {
  VRPS_STORAGE_FP32 = 0,
  VRPS_STORAGE_BF16 = 1,
  VRPS_STORAGE_FP16 = 2   /* holds value * 2^s, s chosen from the data's RMS (|stored| <= 65504) */
} vrps_storage;

typedef struct vrps_report {
  int iterations;     /* outer iterations performed */
  int prox_calls;     /* FGP prox evaluations */
  int snapshots;      /* full-gradient refreshes (SVRG / L-SVRG) */
  int evaluations;    /* objective evaluations written to history */
  double passes;      /* data passes: subset gradients / N + full gradients */
  double gamma;       /* step size used */
  double lipschitz;   /* L estimate (0 when gamma was given) */
  double objective;   /* last evaluated F (NaN if none) */
  double seconds;     /* device time of the iteration loop (CUDA events) */
  int reached;        /* 1 when target_gap was reached */
} vrps_report;

/* Defaults: SVRG estimator, 50 FGP iterations, 100 iterations, nonneg, 100 power
 * iterations, no evaluation, N from the geometry. */
void vrps_solve_opts_default(vrps_solve_opts* opts);

/* Runs Algorithm 1's family on Eq. (tomography_problem).
 * b: [m] sinogram, all angles in natural order (device, or host with opts->host_io).
 * alpha > 0: TV weight.  algo: vrps_algo.  p in (0,1] for the Skip variants (ignored
 * otherwise).  gamma > 0: step; gamma <= 0: factor/L with L from the power iteration and
 * factor 1.99 (ISTA, ProxSkip), 1 (FISTA, SVRG, L-SVRG, SGD), 1/3 (SAGA) (Section 3).
 * seed: Philox key for i_k, theta_k and the L-SVRG coin.  x_out: [n] final iterate x_K.
 * Synchronous: returns after the last kernel finished (the report needs the results).
 * Library-owned workspace (about 12 n + 3 m floats) is kept by the handle between calls.
 * Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA, DIVERGED (non-finite F at an evaluation). */
int vrps_solve(const float* b, const vrps_geom* g, double alpha, int algo, double p, double gamma,
               uint64_t seed, const vrps_solve_opts* opts, float* x_out, vrps_report* report,
               vrps_stream_t stream);

/* Reference minimiser of Eq. (tomography_problem) by preconditioned PDHG (the paper's long-run
 * solver for x* and F*, Section 2.1 and Section 3): Chambolle-Pock on K = [A; D] with the
 * diagonal steps of Pock and Chambolle (2011): tau_j = 1 / (column sum of A + column sum of
 * |D|), sigma = 1 / ray sum of A for the data rows and 1/2 for the difference rows; x0 = 0.
 * b: [m] device sinogram in natural angle order.  nonneg: include I_{x>=0}.  Every
 * eval_every iterations (0: never) F(x) is evaluated into the HOST array history
 * [history_cap][2] (iteration, F).  x_out: [n] device.  The call allocates its own
 * 3n + (dims) n + 3m floats and frees them before returning (synchronous).  Errors:
 * INVALID_ARG, OUT_OF_MEMORY, CUDA, DIVERGED. */
int vrps_pdhg(const float* b, const vrps_geom* g, double alpha, int iters, int nonneg, int eval_every,
              double* history, int history_cap, float* x_out, vrps_report* report, vrps_stream_t stream);

/* ---------------------------------------------------------------- batched / served jobs
 * Many independent VR-ProxSkip reconstructions (Algorithm 1 with a variance-reduced
 * estimator, x0 = 0) advancing together; no counterpart in the paper, which runs one problem.
 * A batch holds 2D jobs or 3D jobs, fixed by its first job.  One tick performs one iteration
 * of every running job, each phase of the tick being one persistent launch over all jobs'
 * tiles (optionally replayed from a CUDA graph; a 3D tick replays its prox phase only when a
 * job takes a prox step).  A job's
 * result is bit-identical to vrps_solve(b, geom, alpha, VRPS_ALGO_VR_PROXSKIP, p, gamma,
 * seed, {estimator, fgp_iters, max_iters, nonneg, n_subsets, job, storage,
 * correction_epochs}) whatever other jobs share its ticks.
 * The batch owns one CUDA stream; device inputs must be ready when vrps_batch_submit is
 * called (it synchronises that stream once to read the draws).  A geometry handle serves one
 * running job at a time (its workspace holds the job's state) and may be reused once the job
 * has finished. */
typedef struct vrps_batch vrps_batch;

typedef struct vrps_job {
  const vrps_geom* geom;  /* geometry (caller-owned, kept alive until the job finished) */
  const float* b;         /* device [m] sinogram in natural angle order (read during submit) */
  float* x_out;           /* device [n]: the final iterate, written when the job finishes */
  double alpha;           /* TV weight >= 0 */
  double p;               /* skip probability in (0, 1] */
  double gamma;           /* step > 0 */
  uint64_t seed;          /* Philox key */
  uint32_t job;           /* Philox counter word 2 */
  int estimator;          /* vrps_estimator */
  int fgp_iters;          /* 0 .. 128 (2D and 3D) */
  int max_iters;          /* iterations of this job (> 0) */
  int n_subsets;          /* 0: the geometry's N */
  int nonneg;
  int storage;            /* vrps_storage */
  int correction_epochs;  /* see vrps_solve_opts */
} vrps_job;

/* Creates an empty batch on the current device.  Errors: CUDA, OUT_OF_MEMORY. */
int vrps_batch_create(vrps_batch** out);
/* Waits for the batch's work, releases its buffers, graphs and events. */
int vrps_batch_free(vrps_batch* batch);
/* on = 0: launch each tick's kernels directly instead of replaying captured graphs. */
int vrps_batch_set_graphs(vrps_batch* batch, int on);
/* Scheduling of a batch that shares the GPU with other work (no counterpart in the paper).
 * set_stream_priority: recreates the batch's stream with this CUDA stream priority (clamped
 * to the device's range; lower numbers run first when thread blocks of several streams
 * wait for the same SMs).  set_grid_share: the persistent launches take this fraction (0, 1]
 * of the resident thread-block slots (default 1), leaving the rest of the GPU to other
 * streams.  Neither changes any result.  Both only before the batch's first job.
 * Errors: INVALID_ARG (NULL batch, share out of range, jobs already submitted), CUDA. */
int vrps_batch_set_stream_priority(vrps_batch* batch, int priority);
int vrps_batch_set_grid_share(vrps_batch* batch, double share);
/* Admits a job before the next tick: allocates its state in the geometry's workspace,
 * reorders b subset-major, draws its Philox schedule and (SAGA) builds its table.  *id is
 * the job's handle.  Errors: INVALID_ARG (bad field, geometry busy, 2D job in a 3D batch or
 * the reverse), UNSUPPORTED (more than 256 running jobs), OUT_OF_MEMORY, CUDA. */
int vrps_batch_submit(vrps_batch* batch, const vrps_job* job, int* id);
/* Enqueues up to `ticks` ticks (fewer when every job finishes); *active = jobs still
 * running.  Returns once the work is enqueued (the host may block on a work-list slot that
 * the device still reads).  Errors: INVALID_ARG (NULL batch, or a running job's geometry was
 * given a launch shape after admission that the batch's launches were not sized for), CUDA. */
int vrps_batch_step(vrps_batch* batch, int ticks, int* active);
/* *done = 1 once job `id` has finished on the device, with its report (seconds = device
 * time from admission to completion).  Errors: INVALID_ARG, TIMEOUT (a bounded device wait
 * of the job expired), CUDA. */
int vrps_batch_poll(vrps_batch* batch, int id, int* done, vrps_report* report);
/* Runs ticks until job `id` finished, waits for it and reports it. */
int vrps_batch_wait(vrps_batch* batch, int id, vrps_report* report);
/* Waits until every enqueued tick has completed. */
int vrps_batch_sync(vrps_batch* batch);
/* Ticks enqueued so far and running jobs. */
int vrps_batch_ticks(const vrps_batch* batch, long long* ticks, int* active);
/* Device bytes a job's state occupies on top of its geometry's tables (for admission by
 * HBM footprint). */
int vrps_job_footprint(const vrps_geom* g, const vrps_job* job, size_t* bytes);

#ifdef __cplusplus
}
#endif

#endif /* VRPS_H */
