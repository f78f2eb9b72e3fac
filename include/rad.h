/*
 * rad.h - C ABI of a GB300 (sm_103a) library for the far-field, spectrally
 * resolved Lienard-Wiechert radiation of PIC macro-particles with the general
 * form-factor formalism of Pausch et al., "Quantitatively consistent
 * computation of coherent and incoherent radiation in particle-in-cell codes -
 * a general form factor formalism for macro-particles" (NIM A, 2018).
 *
 * What the library computes.  For a grid of observation directions n (unit
 * vectors) and frequencies omega, and for every call (one PIC time step t with
 * step dt), every macro-particle k (position r, normalised velocity beta, its
 * time derivative beta_dot, weighting w = electrons per macro-particle):
 *
 *   A_k = n x [(n - beta_k) x beta_dot_k] / (1 - beta_k . n)^2       (Eq. 1)
 *   chi_k = exp(i omega (t - n . r_k / c))                         (Eq. 1)
 *   U(n, omega) += w_k dt A_k chi_k          (coherent amplitude)
 *   V(n, omega) += sqrt(w_k) dt A_k chi_k    (incoherent amplitude)
 *
 * summed over particles and calls on the device (the in-situ evaluation of the
 * inner sum of Eq. 13 per time step, Sec. 3.3).  The spectra are read out as
 *
 *   coherent   = K0 f(omega)^2 |U|^2
 *   incoherent = K0 (1 - f(omega)^2) |V|^2
 *   total      = coherent + incoherent          [J s / sr per rad/s]
 *
 * with K0 = q_e^2 / (16 pi^3 eps0 c) (Eq. 1, 2) and f the amplitude form
 * factor of the macro-particle shape, Table 1 normalised to f(0) = 1.  Per
 * macro-particle this is Eq. 12: w + (w^2 - w) f^2 times one electron.
 *
 * Conventions.
 *  - SI units throughout.  Particle arrays are structure-of-arrays: r, beta and
 *    beta_dot are [3][N] (all x, then all y, then all z), w is [N], all double.
 *  - Spectra are row-major [n_dir][n_omega] doubles.
 *  - Every entry point returns a rad_status; nothing else crosses the ABI
 *    (no exceptions, no exit).  A CUDA error leaves the object failed: every
 *    later call on it returns RAD_ESTATE.
 *  - Invalid particle data (non-finite values, |beta| >= 1, w <= 0) is
 *    detected on the device; the offending particles contribute nothing and
 *    the next synchronising call (rad_spectrum, rad_sync, rad_job_result)
 *    returns RAD_EDATA once.
 *  - Objects are not thread-safe: one thread at a time per object.  Distinct
 *    objects are independent.  Work runs on the CUDA stream given at creation
 *    (NULL = the legacy default stream), in stream order.
 *  - Diagnostics: with the environment variable RAD_LOG=1 the library prints
 *    CUDA errors, calls refused for the wrong device and the tuner's choices
 *    to stderr; RAD_LOG=2 adds the server's admissions and completions.
 *  - An object belongs to the CUDA device that is current when it is created:
 *    calls on a context (and rad_job_feed on a server) made with another
 *    device current return RAD_EINVAL, and a batch takes contexts of one
 *    device.  A server's worker thread runs on the server's device.
 */
#ifndef RAD_H
#define RAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RAD_OK = 0,
  RAD_EINVAL = 1,   /* bad argument: size, pointer, grid value, unknown enum */
  RAD_ENOMEM = 2,   /* device or pinned-host allocation failed */
  RAD_ECUDA = 3,    /* a CUDA call failed; the object is now failed */
  RAD_EDATA = 4,    /* invalid particle data was seen (reported once) */
  RAD_ETIMEOUT = 5, /* a bounded wait ran out */
  RAD_EBUSY = 6,    /* no capacity right now (queue full, slots or memory) */
  RAD_ESTATE = 7    /* object failed earlier, or call not valid in this state */
} rad_status;

/* Macro-particle shapes of Table 1 (Sec. 3.3). */
typedef enum {
  RAD_FF_POINT = 0, /* delta distribution: f = 1 (fully coherent, Sec. 3.2) */
  RAD_FF_CIC = 1,   /* box of width Delta: f = sinc(omega Delta / 2c) */
  RAD_FF_TSC = 2,   /* box * box: f = sinc^2 */
  RAD_FF_QSC = 3,   /* box * box * box: f = sinc^3 */
  RAD_FF_GAUSS = 4  /* Gaussian of std sigma: f = exp(-omega^2 sigma^2 / 2c^2) */
} rad_ff_kind;

/* Form-factor choice. width is Delta (CIC/TSC/QSC) or sigma (GAUSS) in metres,
 * ignored for POINT.  The shape enters only at readout, so one accumulation can
 * be read out with several shapes (rad_spectrum_ff).
 * flags = RAD_FF_3D takes the box shapes as axis-aligned 3-D products
 * rho(x) rho(y) rho(z) of the 1-D shape (Sec. 3.1-3.2), so the form factor
 * depends on the direction: f(n, omega) = prod_d f_1(omega n_d).  Without it f
 * depends on omega only (Table 1 with n along one axis, as printed).  The
 * Gaussian is isotropic and ignores the flag. */
#define RAD_FF_3D 1
/* RAD_FF_LITERAL (at rad_create only): also accumulate the paper's literal
 * in-situ sum P = sum_t sum_k F_k(omega) dt A_k chi_k with the per-particle
 * weight F_k = sqrt(w_k + (w_k^2 - w_k) f(omega)^2) (Eq. 13 with Eq. 12), read
 * out by rad_spectrum_literal as K0 |P|^2.  For equal weights, or one
 * macro-particle, it equals the split total; otherwise it differs by the
 * cross-particle terms the split estimate treats as incoherent.  Costs one more
 * sqrt per amplitude update; such contexts run on their own (not in
 * rad_batch or the server). */
#define RAD_FF_LITERAL 2
typedef struct {
  int32_t kind;  /* rad_ff_kind */
  int32_t flags; /* 0, RAD_FF_3D, RAD_FF_LITERAL or both */
  double width;
} rad_ff;

typedef enum {
  RAD_PREC_MIXED = 0, /* float-float retarded time and phase, FP32 sin/cos; the
                         sum over particles runs in FP32 (default kernel: on the
                         tensor cores, mma.sync TF32 with both operands split
                         into hi and lo parts, FP32 accumulation); compensated
                         FP32 accumulation over calls (default) */
  RAD_PREC_FP64 = 1   /* plain kernel: everything in FP64, one thread per bin */
} rad_prec;

typedef struct rad_ctx rad_ctx;

/* rad_create - set up one spectrum job.
 *  omega   host [n_omega] angular frequencies, rad/s, finite and > 0.
 *  dirs    host [n_dir][3] observation directions; each is normalised here
 *          (must be finite and non-zero).
 *  ff      default shape for rad_spectrum.
 *  prec    rad_prec.
 *  stream  cudaStream_t to run on (NULL = legacy default stream).
 *  out     receives the context; the caller owns it (rad_destroy).
 * Copies the grids to the device and allocates the resident accumulators
 * (64 B per (direction, frequency) bin in MIXED mode, 96 B in FP64 mode).
 * Errors: RAD_EINVAL (sizes < 1, n_omega * n_dir > 2^31 - 1, bad values),
 * RAD_ENOMEM, RAD_ECUDA. */
rad_status rad_create(const double* omega, int32_t n_omega, const double* dirs, int32_t n_dir,
                      rad_ff ff, int32_t prec, void* stream, rad_ctx** out);

/* rad_accumulate - add one time step (Eq. 13, inner sum over macro-particles,
 * evaluated in-situ, Sec. 3.3).
 *  n        number of macro-particles (0 is a no-op).
 *  r        [3][n] positions, m.           | device pointers are read in stream
 *  beta     [3][n] velocities / c.         | order: keep them unchanged until the
 *  beta_dot [3][n] d(beta)/dt, 1/s.        | work has run (rad_sync or an event).
 *  w        [n] electrons per macro-particle (> 0; need not be integer).
 *  t, dt    time of the step and its length, s (dt > 0).
 * Host pointers are accepted too: they are copied to library staging buffers
 * inside the call (pinned memory makes the copy asynchronous).
 * The phase is computed in FP32 about one reference point per call (the first
 * particle), which covers particles within 2^21 turns of the highest frequency
 * from it (40 um at 1e20 rad/s, seen from any direction of the grid).  A call
 * spread wider (all macro-particles of a simulation domain, Sec. 3.3) is sorted
 * on the device along the grid's mean direction and given one reference point
 * per 256 particles; its results are as deterministic as any other call's.
 * The context keeps ~92 bytes of device memory per macro-particle of the
 * largest call (records and sort buffers).
 * Errors: RAD_EINVAL, RAD_ENOMEM, RAD_ECUDA, RAD_ESTATE. */
rad_status rad_accumulate(rad_ctx* ctx, int64_t n, const double* r, const double* beta,
                          const double* beta_dot, const double* w, double t, double dt);

/* rad_spectrum - read out coherent, incoherent and total spectra with the
 * context's shape.  Each output is [n_dir][n_omega] doubles, host or device
 * memory, or NULL to skip.  Synchronises the context's stream.
 * Errors: RAD_EDATA (once, after invalid particles), RAD_ECUDA, RAD_ESTATE. */
rad_status rad_spectrum(rad_ctx* ctx, double* coherent, double* incoherent, double* total);

/* rad_spectrum_ff - as rad_spectrum with another shape (e.g. CIC vs TSC read
 * out of the same accumulation). */
rad_status rad_spectrum_ff(rad_ctx* ctx, rad_ff ff, double* coherent, double* incoherent,
                           double* total);

/* In-situ coupling to a particle pusher that provides positions and velocities
 * each PIC step but not beta_dot (the inner sum of Eq. 13 is evaluated in situ
 * at every step, Sec. 3.3).  rad_push_step hands over step j: r_j, beta_j, w_j
 * at time t_j with step length dt_j (host or device arrays, copied).  The
 * context keeps the last two steps on the device; when step j+1 arrives it
 * accumulates step j with the central difference
 *   beta_dot_j = (beta_{j+1} - beta_{j-1}) / (t_{j+1} - t_{j-1}),
 * second-order accurate (the first step uses the forward difference
 * (beta_1 - beta_0) / (t_1 - t_0)).  rad_push_flush accumulates the last held
 * step with the backward difference and clears the history.  Macro-particle k
 * must be the same in every step (same count and order); RAD_EINVAL otherwise.
 * Needs 192 bytes of device memory per macro-particle. */
rad_status rad_push_step(rad_ctx* ctx, int64_t n, const double* r, const double* beta,
                         const double* w, double t, double dt);
rad_status rad_push_flush(rad_ctx* ctx);

/* rad_spectrum_literal - the paper's literal spectrum K0 |P|^2 ([n_dir][n_omega]
 * doubles, host or device) of a context created with RAD_FF_LITERAL, with the
 * creation shape.  RAD_ESTATE for other contexts.  Synchronises the stream. */
rad_status rad_spectrum_literal(rad_ctx* ctx, double* literal);

/* rad_spectrum_species - spectra of a particle population made of several
 * species (particle classes), each accumulated in its own context with its own
 * macro-particle shape ffs[s] (Sec. 3.2 per species, optionally RAD_FF_3D):
 *   coherent   = K0 |sum_s f_s U_s|^2   (amplitudes of all species add first),
 *   incoherent = K0 sum_s (1 - f_s^2) |V_s|^2,   total = their sum.
 * ctxs: n_species distinct contexts (1 <= n_species <= 16) created with the
 * same frequencies, directions and precision; ffs: their shapes.  Outputs as in
 * rad_spectrum ([n_dir][n_omega] doubles, host or device, NULL to skip), written
 * on the first context's stream.  Synchronises every context.  Errors:
 * RAD_EINVAL (grids or precisions differ, a context repeated, a bad shape),
 * RAD_ESTATE, RAD_ECUDA; RAD_EDATA once, after writing the spectra, when a
 * species saw invalid particles. */
rad_status rad_spectrum_species(rad_ctx* const* ctxs, const rad_ff* ffs, int32_t n_species,
                                double* coherent, double* incoherent, double* total);

/* rad_sync - wait for the context's queued work; report RAD_EDATA / errors. */
rad_status rad_sync(rad_ctx* ctx);

/* rad_reset - zero the accumulators (keeps grids and buffers). */
rad_status rad_reset(rad_ctx* ctx);

/* rad_destroy - free everything (synchronises the stream first). NULL is ok. */
void rad_destroy(rad_ctx* ctx);

/* Checkpoint / multi-rank merge.  The state blob is a versioned, self-
 * describing copy of the accumulators and the grids' shape; it is valid on any
 * context created with the same grids and precision.
 * rad_state_size   bytes needed for the blob (0 if ctx is NULL).
 * rad_state_export copy the state into host_buf (n >= rad_state_size).
 * rad_state_import replace the state by the blob.
 * rad_state_merge  add the blob's amplitudes to the state: contexts fed
 *                  disjoint particle subsets (e.g. one per rank) merge into the
 *                  amplitudes of all particles (amplitudes add before |.|^2,
 *                  Eq. 2).  Errors: RAD_EINVAL on size / shape / version mismatch. */
size_t rad_state_size(const rad_ctx* ctx);
rad_status rad_state_export(rad_ctx* ctx, void* host_buf, size_t n);
rad_status rad_state_import(rad_ctx* ctx, const void* host_buf, size_t n);
rad_status rad_state_merge(rad_ctx* ctx, const void* host_buf, size_t n);

/* Tile configuration of the mixed-precision kernel (see rad_tune).
 *  variant   kernel build.  FP32 accumulation: 0 = 256 threads x 2 frequencies
 *            per thread (3 blocks per SM), 1 = 256 x 4, 2 = 128 x 2, 5 = 256 x 2
 *            (4 blocks per SM).  Tensor-core accumulation (TF32 hi/lo), a warp per
 *            32 frequencies: 3 (3 blocks per SM), 4 (4 blocks per SM), 7 = 3 with
 *            each staged particle tile swept in two frequency passes; a warp per
 *            64 frequencies (2 frequencies per thread): 8 (2 blocks per SM) and 9
 *            (as 8, with the phases' float-float cross terms formed by one more
 *            MMA per block; the default of a new context).  6 = FP32 with the
 *            literal sum, used by, and only by, RAD_FF_LITERAL contexts.
 *  omega_tile frequencies per tile: a multiple of 32 x frequencies per thread x
 *            passes, at most 256 x frequencies per thread x passes; directions
 *            per tile follow from the block's bin count.  RAD_EINVAL otherwise.
 *  chunk     macro-particles per work item (multiple of 256), 0 = automatic. */
typedef struct {
  int32_t variant;
  int32_t omega_tile;
  int32_t chunk;
  int32_t reserved;
} rad_tile;

rad_status rad_get_tile(const rad_ctx* ctx, rad_tile* tile);
rad_status rad_set_tile(rad_ctx* ctx, const rad_tile* tile);

/* rad_tune - time candidate tiles on synthetic particles (n of them, or fewer
 * when n x bins is large; the chunk size is then left automatic) and keep the
 * fastest for this context's grid shape.  Results are cached per shape
 * bucket in memory and, when the environment variable RAD_TUNE_CACHE names a
 * file, on disk.  Leaves the accumulators unchanged. */
rad_status rad_tune(rad_ctx* ctx, int64_t n);

/* Batched accumulation: one step of many independent jobs in one persistent
 * launch.  Each job keeps its own tile shape, so its result is bitwise the
 * same alone or in a batch.  A batch with identical particle counts and
 * pointers on consecutive calls is replayed from a captured CUDA graph. */
typedef struct {
  int64_t n;
  const double* r;        /* device [3][n] */
  const double* beta;     /* device [3][n] */
  const double* beta_dot; /* device [3][n] */
  const double* w;        /* device [n] */
  double t;
  double dt;
} rad_step;

typedef struct rad_batch rad_batch;

/* rad_batch_create - group n_jobs MIXED-precision contexts (distinct) for
 * batched launches on `stream`.  The contexts stay owned by the caller and
 * must outlive the batch; they must not be used on their own while the batch
 * has queued work (rad_batch_sync). */
rad_status rad_batch_create(rad_ctx* const* ctxs, int32_t n_jobs, void* stream, rad_batch** out);
/* rad_batch_accumulate - steps[i] goes to ctxs[i] (n = 0 skips that job). */
rad_status rad_batch_accumulate(rad_batch* b, const rad_step* steps);
rad_status rad_batch_sync(rad_batch* b);
void rad_batch_destroy(rad_batch* b);

/* Serving: a continuous-batching request loop.  Jobs arrive at any time
 * (rad_job_submit); a background scheduler admits them while a slot is free
 * and their device footprint fits the budget, keeps their amplitudes resident
 * on the device, and runs every pending step of all admitted jobs in batched
 * persistent launches, so work of newly arrived jobs overlaps with the others.
 * Steps are fed incrementally (rad_job_feed copies the particles into the
 * server's device staging, so the caller may reuse its buffers on return). */
typedef struct rad_server rad_server;
typedef int64_t rad_job_id;

typedef struct {
  const double* omega; /* host [n_omega] */
  int32_t n_omega;
  int32_t n_dir;
  const double* dirs;  /* host [n_dir][3] */
  rad_ff ff;
  int64_t max_particles; /* largest n any step of this job will have */
  int32_t max_queued;    /* steps that may wait in device staging (>= 1) */
  int32_t reserved;
} rad_job_desc;

typedef struct {
  int64_t submitted, admitted, completed, rounds;
  int64_t updates;           /* amplitude updates done (particle x omega x n x step) */
  int64_t footprint_bytes;   /* device bytes held by admitted jobs now */
  int64_t peak_footprint_bytes;
  int32_t active, waiting;
} rad_server_stats;

/* hbm_budget: device bytes the admitted jobs may hold in total; max_slots:
 * jobs admitted at once. */
rad_status rad_server_create(size_t hbm_budget, int32_t max_slots, void* stream,
                             rad_server** out);
/* Round policy of the scheduler.  Each round runs one pending step from each
 * of a set of admitted jobs in one batched launch:
 *   RAD_SERVE_ALL: every admitted job with a step ready (equal shares);
 *   RAD_SERVE_OLDEST: jobs in arrival order until the round holds round_updates
 *     amplitude updates (particles x bins), at least one job;
 *   RAD_SERVE_LEAST_SERVED: the same in order of
 *     the updates each job has had so far (new and small jobs first; ties in
 *     arrival order);
 *   RAD_SERVE_LEAST_SERVED_AGED: as least served, with each job's updates reduced
 *     by its time since submission times one round's updates per 12 ms, so that
 *     large jobs that have waited long are not passed over indefinitely;
 *   RAD_SERVE_OLDEST_BACKFILL (default, round_updates = 2e9): the oldest job
 *     with a step ready always; the others, least served first, each only if
 *     the round's updates stay within max(round_updates, 17/16 of the oldest
 *     job's step), so the oldest job runs at >= 16/17 of its own pace (the tail
 *     latency of a FIFO queue) while small jobs progress in the margin.
 * round_updates >= 1 for all but RAD_SERVE_ALL, which ignores it.  Takes effect
 * from the next round.  RAD_EINVAL for an unknown policy or round_updates < 1. */
enum { RAD_SERVE_ALL = 0, RAD_SERVE_OLDEST = 1, RAD_SERVE_LEAST_SERVED = 2, RAD_SERVE_LEAST_SERVED_AGED = 3,
       RAD_SERVE_OLDEST_BACKFILL = 4 };
rad_status rad_server_set_policy(rad_server* s, int32_t policy, int64_t round_updates);
/* Copies the grids; the job waits until it can be admitted. RAD_EINVAL if it
 * could never fit the budget. */
rad_status rad_job_submit(rad_server* s, const rad_job_desc* desc, rad_job_id* id);
/* Queue one step (host or device arrays). RAD_EBUSY if max_queued steps are
 * already waiting (try again later). */
rad_status rad_job_feed(rad_server* s, rad_job_id id, const rad_step* step);
/* No more steps for this job; its spectrum is read out after the last one. */
rad_status rad_job_finish(rad_server* s, rad_job_id id);
/* done = 1 once the spectrum is ready. */
rad_status rad_job_poll(rad_server* s, rad_job_id id, int32_t* done);
/* Wait (up to timeout_s seconds, < 0 = forever) for the spectrum and copy it
 * out ([n_dir][n_omega] host doubles, NULL to skip); releases the job.
 * Reports the job's arrival-to-ready latency in *latency_s when non-NULL. */
rad_status rad_job_result(rad_server* s, rad_job_id id, double timeout_s, double* coherent,
                          double* incoherent, double* total, double* latency_s);
rad_status rad_server_stats_get(rad_server* s, rad_server_stats* st);
void rad_server_destroy(rad_server* s);

/* Kernel timing.  While enabled, every rad_accumulate of this context records
 * CUDA events around its pre-pass and accumulate kernels on the context's
 * stream.  rad_profile_read synchronises the stream, returns the summed kernel
 * times (ms) and the number of timed calls since the last read, and resets the
 * sums.  Disabled by default. */
rad_status rad_profile_enable(rad_ctx* ctx, int32_t on);
rad_status rad_profile_read(rad_ctx* ctx, double* prepass_ms, double* accumulate_ms,
                            int64_t* calls);

/* Effective SM clock of the accumulate kernels timed since the last call (or
 * since profiling was enabled): the SM cycle counter divided by elapsed
 * nanoseconds, each summed over the kernels' CTA lifetimes, in MHz; 0 when none
 * ran.  sm_mhz: host double (out).  Synchronises the context's stream and
 * resets the sums.  RAD_EINVAL for a NULL argument. */
rad_status rad_profile_clock(rad_ctx* ctx, double* sm_mhz);

/* Accumulation without any allocation.
 *
 * Some callers cannot allocate device memory: code running inside a host
 * application that owns the GPU's memory pool, a plug-in called from a
 * time-step loop that forbids cudaMalloc (it would synchronise the device and
 * stall the simulation), or a process that must keep its footprint fixed.
 * rad_accumulate_static serves them.  It adds one time step into accumulators
 * the caller owns and calls no cudaMalloc, cudaFree or allocating library
 * routine.  Its working memory (grid tables, per-particle records, per-chunk
 * partial sums, counters) is one file-scope device array of
 * RAD_STATIC_SCRATCH_BYTES (about 14 MB).  Every GPU that loads the library
 * holds that array until the process exits.  It is not a counterpart of
 * anything in the paper.
 *
 *  omega   device [n_omega] angular frequencies, rad/s (> 0).
 *  dirs    device [n_dir][3] observation directions (normalised here).
 *  n, r, beta, beta_dot, w, t, dt   as rad_accumulate; device arrays only.
 *  state   device float [16][n_omega * n_dir], read and updated: the same
 *          layout as a context's accumulators (U.e1, U.e2, V.e1, V.e2 re/im
 *          compensated sums, then their compensations; the same bytes as the
 *          payload of rad_state_export for a MIXED context with these grids).
 *          Zero it to start a new accumulation.
 *  stream  cudaStream_t (NULL = legacy default stream).
 * Limits: n_omega <= RAD_STATIC_MAX_OMEGA, n_dir <= RAD_STATIC_MAX_DIRS,
 * n_omega * n_dir <= RAD_STATIC_MAX_BINS, n <= RAD_STATIC_MAX_PARTICLES.
 * Larger sizes return RAD_EINVAL before anything is enqueued.
 *
 * The first call on a device looks up the array's device address on that
 * device (cudaGetSymbolAddress), so make that first call before any stream
 * capture.  Every call shares the one array and clears what must start at zero.
 * Calls whose work overlaps on the GPU (other streams or threads) race on it,
 * so serialise them.  Returns RAD_OK once the work is enqueued, RAD_EINVAL for
 * bad host-side arguments, or RAD_ECUDA if the set-up or a launch failed.
 * What the device finds is reported by rad_static_status: particles with
 * invalid data contribute nothing; a frequency or direction that is not finite
 * and positive (non-zero) makes the whole step a no-op, leaving `state` as it
 * was; a bounded wait that gave up leaves the step partly added. */
#define RAD_STATIC_MAX_OMEGA 4096
#define RAD_STATIC_MAX_DIRS 4096
#define RAD_STATIC_MAX_BINS 65536
#define RAD_STATIC_MAX_PARTICLES 65536
#define RAD_STATIC_SCRATCH_BYTES (14u << 20)
rad_status rad_accumulate_static(const double* omega, int32_t n_omega, const double* dirs,
                                 int32_t n_dir, int64_t n, const double* r, const double* beta,
                                 const double* beta_dot, const double* w, double t, double dt,
                                 float* state, void* stream);
/* rad_static_status - what the device reported for the latest
 * rad_accumulate_static call with particles on the current device: RAD_OK,
 * RAD_EDATA (some particles were invalid and skipped), RAD_EINVAL (a frequency
 * or direction was invalid: the step was skipped), RAD_ETIMEOUT (a bounded
 * wait gave up: the step is incomplete), RAD_ECUDA (a debug build's index
 * check failed, or the read failed).  Reads 4 bytes of the scratch array on
 * `stream` (NULL = legacy default stream) and synchronises that stream; it
 * allocates nothing.  The word belongs to the shared array, so the answer is
 * about whichever call ran last on this device. */
rad_status rad_static_status(void* stream);

/* Diagnostics. */
const char* rad_status_str(rad_status s);
/* rad_last_error - last non-OK status of this context (sticky until reset). */
rad_status rad_last_error(const rad_ctx* ctx);
/* Number of kernels this library has launched in this process (all objects),
 * counted on the host at launch time; graph replays count their kernels. */
int64_t rad_kernel_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* RAD_H */
