/*
 * dpstokes.h - C ABI of the GB300 doubly-periodic FCM mobility library.
 *
 * The library computes the mobility product [U; Omega] = M [F; T] (Eq. 58 of Hashemi et al.,
 * "Computing hydrodynamic interactions in confined doubly-periodic geometries in linear time")
 * for N particles in a box that is periodic in x and y, with one of three conditions in z:
 * open (free space), a no-slip wall at zmin (bottom wall), or no-slip walls at zmin and zmax
 * (slit channel).  The product follows the eight steps of Sec. III.D: ES-kernel spreading
 * (Eqs. 7, 9, 53-54), xy FFT + Chebyshev transform in z, the doubly-periodic pressure and
 * velocity boundary-value problems per wavenumber (Eqs. 15-24), the wall correction
 * (Eqs. 41-44; Appendix A, Eqs. A4-A10 with zero slip lengths), the k = 0 mode (Sec. III.C,
 * Eq. A12), inverse transforms with the curl for angular velocities, and ES interpolation
 * (Eqs. 10-11).
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * - The xy box is [0, Lx) x [0, Ly); Lx, Ly are full periods, h = Lx/nx = Ly/ny (must agree),
 *   wavenumbers are k = 2 pi n / L.  x and y are wrapped modulo the periods.
 * - z nodes are the nz Chebyshev extrema nodes on [zmin, zmax], both ends included (Sec. III.D).
 * - The ES support of the monopole (M) and dipole (D) kernels is alpha = m h / 2 (Sec. III.E).
 * - Particle arrays are row-major [n][3] double (x, y, z / Fx, Fy, Fz / ...).
 * - Every function returns a dps_status; nothing traps or aborts.  Errors that can be seen on
 *   the host return at once.  Errors that depend on the data (a height outside [zmin, zmax], an
 *   envelope crossing an open boundary, a non-finite input) set a device status word that
 *   dpstokes_status() reads; the outputs of that apply are then undefined.
 * - Buffers passed to the library stay owned by the caller.  The plan owns all grids, spectra,
 *   tables and workspaces and frees them in dpstokes_destroy().
 */
#ifndef DPSTOKES_H
#define DPSTOKES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dps_plan_s* dps_plan_t;

/* z boundary condition (Sec. II; Appendix A) */
typedef enum {
  DPS_FREE = 0,         /* open in z: no wall, kernels must stay inside [zmin, zmax]          */
  DPS_BOTTOM_WALL = 1,  /* no-slip wall at zmin, open above; kernels must stay below zmax     */
  DPS_SLIT = 2          /* no-slip walls at zmin and zmax                                      */
} dps_wall_mode;

/* arithmetic of the hot path */
typedef enum {
  DPS_FP64 = 0,   /* every stage in double precision                                           */
  DPS_MIXED = 1   /* spreading, FFTs, Chebyshev transforms, interpolation in float (float
                     accumulation); the banded BVP solves and the wall-correction boundary rows
                     in double                                                                   */
} dps_precision;

/* how torques enter (the two routes of Sec. III.D, the paragraph after the algorithm) */
typedef enum {
  DPS_TORQUE_NONE = 0,              /* forces only                                                */
  DPS_TORQUE_SPECTRAL_CURL = 1,     /* spread the torque field tau Delta^W_D, add its half-curl in
                                       Fourier-Chebyshev space, and transform the half-curl of the
                                       velocity back for the angular velocities: 6 fields are
                                       spread and transformed each way (the paper's GPU route)     */
  DPS_TORQUE_KERNEL_DERIVATIVE = 2  /* spread (1/2) grad Delta^W_D x tau with the force density and
                                       interpolate Omega_j = (1/2) h^2 sum w_c u x grad Delta^W_D:
                                       3 fields each way.  The kernel derivative is zero beyond the
                                       point where |phi'| is smallest before the support edge
                                       (beta v sqrt(1 - v) = 1, v = (t/alpha)^2, larger root); the z
                                       derivative is the exact one of the imaged envelope.  Needs
                                       beta_D > 3 sqrt(3) / 2.  Both routes approximate the same
                                       operator; they differ by the kernel sampling error          */
} dps_torque_route;

typedef enum {
  DPS_OK = 0,
  DPS_ERR_INVALID_ARG = -1,   /* bad sizes or parameters, inconsistent pointer combination      */
  DPS_ERR_OUT_OF_DOMAIN = -2, /* a height outside [zmin, zmax] or an envelope through an open
                                 boundary (footnote to step 1 of Sec. III.D)                     */
  DPS_ERR_OOM = -3,           /* device allocation failed in dpstokes_plan_create               */
  DPS_ERR_CUDA = -4,          /* a CUDA runtime call failed                                      */
  DPS_ERR_TIMEOUT = -5,       /* a bounded wait gave up: a device copy did not complete in about a
                                 second (TMA column pass), or a server ticket within its timeout */
  DPS_ERR_NONFINITE = -6,     /* a non-finite position, force or torque                          */
  DPS_ERR_BUSY = -7           /* a server's queue is at its limit: the request was not accepted   */
} dps_status;

typedef struct {
  int32_t nx, ny;  /* xy grid; 8 <= nx, ny <= 6144, 2,3,5,7-smooth                              */
  int32_t nz;      /* Chebyshev nodes on [zmin, zmax] including both ends, 5 <= nz <= 257      */
} dps_grid;

typedef struct {
  int32_t m_M;     /* monopole ES support in cells, 2 <= m <= 12; alpha_M = m_M h / 2          */
  double beta_M;   /* monopole ES shape parameter beta (Eq. 54), > 0                            */
  int32_t m_D;     /* dipole support (used only with torques)                                  */
  double beta_D;   /* dipole shape parameter                                                    */
  double eta;      /* viscosity (Eq. 4), > 0                                                    */
  int32_t with_torque;  /* dps_torque_route: 0 forces only; 1 or 2: applies take torques and
                           return angular velocities, by the spectral curl (1) or by kernel
                           derivatives (2)                                                     */
  int32_t precision;    /* dps_precision                                                       */
  int64_t max_n;        /* largest particle count an apply may pass                           */
} dps_kernel_params;

/* Build a plan: validates the box, grid and kernels, builds the Chebyshev/quadrature/transform
 * tables and allocates every device buffer an apply needs (no allocation happens in apply).
 * Host-detectable errors: non-positive sizes, h_x != h_y, nz out of range, a non-smooth xy size,
 * m out of range or its envelope wider than half the box, a slit narrower than 2 alpha, an
 * unknown torque route, beta_D <= 3 sqrt(3) / 2 with the kernel-derivative route.
 * The current CUDA device at the call is the plan's device.  *out is NULL on error. */
dps_status dpstokes_plan_create(dps_plan_t* out, double Lx, double Ly, double zmin, double zmax,
                                int32_t wall_mode, const dps_grid* grid,
                                const dps_kernel_params* kp);

/* Wall conditions beyond no-slip stationary walls (Appendix A, Eqs. A1-A12): slip lengths and
 * uniform tangential wall velocities.  The tangential velocity obeys u - l0 du/dz = u^W_0 at zmin
 * and u + lH du/dz = u^W_H at zmax (the normal velocity vanishes at a wall).  Slip enters the
 * wall data of the correction (minus the DP velocity plus or minus l times its z derivative there),
 * the correction's boundary rows and the k = 0 rows; a wall velocity enters the k = 0 rows only,
 * which makes the product affine in the forces.  For the bottom-wall geometry the paper prints slip
 * for the slit only; the bottom-wall rows here are the slit's restricted to the decaying family.
 * A very large l0 above one wall under an open top makes the k = 0 response grow with l0 (a net
 * force has no steady state over a shear-free wall); l0 must be finite. */
typedef struct {
  double slip_bottom;   /* l0 >= 0 at zmin (bottom wall and slit)                                 */
  double slip_top;      /* lH >= 0 at zmax (slit only; 0 otherwise)                                */
  double uw_bottom[2];  /* (u, v) of the wall at zmin (bottom wall and slit)                       */
  double uw_top[2];     /* (u, v) of the wall at zmax (slit only; 0 otherwise)                     */
} dps_wall_params;

/* dpstokes_plan_create with wall conditions; wp = NULL means no-slip stationary walls (what
 * dpstokes_plan_create builds).  DPS_ERR_INVALID_ARG also for a negative or non-finite slip length
 * or wall velocity, and for slip or a wall velocity on a wall the geometry does not have. */
dps_status dpstokes_plan_create_ex(dps_plan_t* out, double Lx, double Ly, double zmin, double zmax,
                                   int32_t wall_mode, const dps_grid* grid, const dps_kernel_params* kp,
                                   const dps_wall_params* wp);

/* One mobility product, enqueued on `stream` (a cudaStream_t, NULL for the legacy stream).  All of
 * an apply's work is ordered after earlier work on `stream` and before later work on it (when the
 * wavenumber-space stages run in several column chunks, DPS_CHUNKS in the environment at plan
 * creation, they fork onto two plan-owned streams and join back before the apply's last kernels).
 * positions, forces: device [n][3]; torques: device [n][3] or NULL; out_vel: device [n][3];
 * out_angvel: device [n][3] or NULL.  torques and out_angvel must both be NULL for a plan built
 * without torques and both non-NULL for one built with torques.  0 <= n <= max_n.  Outputs are
 * fully overwritten.  Asynchronous: no host synchronisation, no allocation.  Two applies on the
 * same plan must not run concurrently (they share the plan's buffers). */
dps_status dpstokes_apply(dps_plan_t plan, int64_t n, const double* positions, const double* forces,
                          const double* torques, double* out_vel, double* out_angvel, void* stream);

/* Same product from HOST arrays: copies the inputs to plan-owned device staging buffers, runs
 * dpstokes_apply on `stream`, copies the outputs back and synchronises the stream.  Pinned host
 * memory gives the fastest copies.  Returns the device status of the apply. */
dps_status dpstokes_apply_host(dps_plan_t plan, int64_t n, const double* positions,
                               const double* forces, const double* torques, double* out_vel,
                               double* out_angvel, void* stream);

/* Synchronises `stream`, reads and clears the device status word of the plan's last apply. */
dps_status dpstokes_status(dps_plan_t plan, void* stream);

/* Frees every buffer of the plan (synchronises the device first).  NULL is ignored. */
void dpstokes_destroy(dps_plan_t plan);

/* Static description of the error code (never NULL). */
const char* dpstokes_error_string(dps_status status);

/* Plan facts for callers and diagnostics. */
typedef struct {
  int64_t device_bytes;     /* device memory owned by the plan                                  */
  int32_t nkx;              /* nx/2 + 1 stored wavenumbers in x                                 */
  int32_t pitch;            /* complex elements per stored grid row                             */
  int32_t nfields;          /* fields spread and transformed: 6 for the spectral-curl torque
                               route, else 3                                                   */
  int32_t record_words;     /* 32-bit words per particle kernel record                          */
  double h;                 /* grid spacing                                                     */
  double alpha_M, alpha_D;  /* kernel supports                                                  */
  int32_t launches_per_apply; /* kernels one apply launches                                       */
  int32_t nchunks;          /* column chunks of the wavenumber-space pipeline                     */
  int32_t fft_col_width;    /* x-wavenumber columns per block of the y-FFT pass                   */
  int32_t solve_blocks;     /* persistent blocks of the FP64 per-wavenumber solve                 */
  int32_t fft_register_rows; /* 1: the x-FFT passes run register-staged (one butterfly per thread
                               and stage, one shared buffer), 0: shared-memory-staged           */
  int32_t fft_register_cols; /* the y-FFT passes: 0 shared-memory-staged, 1 register-staged,
                               2 register-staged with cp.async prefetch, 3 with TMA prefetch   */
  int32_t interp_variant;   /* interpolation (step 8): 0 a warp per particle, 1 tile gather,
                               2 staged gather (see dpstokes_plan_set_interp)                    */
  int32_t cheb_tensor_cores; /* Chebyshev transforms on the tensor cores (tcgen05, tf32
                               three-product split; mixed precision, nz <= 128): bit 0 the
                               forward transform, bit 1 the backward transform (spectral-curl
                               torques; beyond 96 nodes in two launches of half the planes)    */
} dps_plan_info;
dps_status dpstokes_plan_info(dps_plan_t plan, dps_plan_info* out);

/* Interpolation variant by hand (no counterpart in the paper): 0 a warp per particle gathering its
 * support rows from global memory; 1 the tile gather, the transpose of the spread (a block per
 * 32 x 8 tile of node columns reads each column once and adds its share of every covering
 * particle's sums to a per-tile slot; a second kernel adds a particle's slots in a fixed order);
 * 2 the staged gather (a block per particle bin copies the grid region its particles' supports
 * cover into shared memory, four planes at a time, and its warps gather their particles from
 * there).  All compute the sums of Eqs. 10-11 up to summation order.  DPS_ERR_INVALID_ARG for 1
 * or 2 where the variant does not apply: both need forces only or spectral-curl torques with
 * m_M = m_D; 2 needs mixed precision and supports of at most 6 nodes (m <= 5).  The staged gather
 * is the default where it applies, else the warp per particle; the autotuner tries the others. */
dps_status dpstokes_plan_set_interp(dps_plan_t plan, int32_t variant);

/* Autotuner (no counterpart in the paper).  Times the plan's applies on the given particles (same
 * arguments and rules as dpstokes_apply) over a small set of launch shapes, one knob at a time:
 * the column width (1, 2, 4, 8) and variant (register- or shared-memory-staged) of the y-FFT pass
 * within the shared-memory and thread limits, the
 * persistent grid of the FP64 solve (1-4 blocks per SM within the allocated workspace) and the
 * column chunks of the wavenumber-space pipeline (1, 2, 4); a candidate replaces the current shape
 * when it is at least 2 % faster.  The plan keeps the chosen shapes (dpstokes_plan_info reports
 * them); results do not depend on them beyond summation order.  Synchronises `stream`; on return the
 * outputs hold the product computed with the chosen shapes and *best_ms (if not NULL) its time.
 * Returns the device status of the applies. */
dps_status dpstokes_plan_autotune(dps_plan_t plan, int64_t n, const double* positions, const double* forces,
                                  const double* torques, double* out_vel, double* out_angvel, void* stream,
                                  double* best_ms);

/* Sets the xy-FFT launch shapes by hand (no counterpart in the paper): `row_register` chooses the
 * register-staged (1) or shared-memory-staged (0) variant of the x-FFT passes, `col_register` that
 * of the y-FFT passes (0 shared-memory-staged, 1 register-staged, 2 register-staged with the next
 * block's columns prefetched by cp.async, 3 the same prefetched by TMA box loads), `col_width` (1, 2,
 * 4 or 8) the x-wavenumber columns per block of the
 * y pass.  Results do not depend on the shapes beyond summation order.  DPS_ERR_INVALID_ARG (plan
 * unchanged) when plan is NULL, a variant is out of range, or the shape does not fit this plan's
 * sizes within the thread and shared-memory limits; dpstokes_plan_info reports the shapes in use. */
dps_status dpstokes_plan_set_fft(dps_plan_t plan, int32_t row_register, int32_t col_register, int32_t col_width);

/* Sets the wavenumber-space pipeline shape by hand (no counterpart in the paper): `solve_blocks`
 * persistent blocks of the FP64 solve (1 .. the number the plan's workspace was sized for, which
 * dpstokes_plan_info reports as solve_blocks right after creation) and `nchunks` column chunks
 * (1, 2, 4 or 8, at least 64 x-wavenumbers each) whose FP64 solves run on a plan-owned stream
 * beside the float transforms of the neighbouring chunks.  Results do not depend on the shape
 * beyond summation order.  DPS_ERR_INVALID_ARG (plan unchanged) when plan is NULL or a value is
 * out of range. */
dps_status dpstokes_plan_set_pipeline(dps_plan_t plan, int32_t solve_blocks, int32_t nchunks);

/* Per-stage timing.  With timing enabled, every apply brackets each kernel launch with a pair of
 * CUDA events on the stream that launch runs on (the wavenumber-space stages run in column chunks
 * on two internal streams forked from and joined back to the caller's stream, so their kernels
 * overlap); dpstokes_stage_times() waits for the last apply to finish and writes, per stage, the sum
 * of its launch durations in milliseconds, in this order (DPS_NUM_STAGES values):
 *   0 init, 1 particle records, 2 binning, 3 spread, 4 x-FFT forward, 5 y-FFT forward,
 *   6 Chebyshev forward transform, 7 FP64 per-wavenumber solves, 8 correction + curl + inverse
 *   Chebyshev transform, 9 y-FFT inverse, 10 x-FFT inverse, 11 interpolation.
 * *count receives the number written (min(capacity, DPS_NUM_STAGES)); DPS_ERR_INVALID_ARG if no
 * timed apply has been enqueued since timing was enabled. */
#define DPS_NUM_STAGES 12
dps_status dpstokes_enable_timing(dps_plan_t plan, int32_t enable);
dps_status dpstokes_stage_times(dps_plan_t plan, double* ms_out, int32_t capacity, int32_t* count);

/* Spreading without device allocation (no counterpart in the paper: this is a deployment aid).
 * Some callers cannot call cudaMalloc: a host application whose memory manager owns every byte of
 * device memory and hands out nothing outside its own pool, or a latency-critical loop that cannot
 * afford the implicit device synchronisation of an allocation.  This entry point runs the library's
 * spreading stage (particle envelope records, binning and the tile-gather spread, in double
 * precision, on the same node heights as a plan) using only a scratch array of fixed size, 64 MiB, compiled into
 * the library as device memory; every GPU that loads the library holds that array until the
 * process exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *   - out_grid: caller-owned device buffer of nfields * nz * ny * ldx doubles (nfields = 6 with
 *     the spectral-curl torque route: force fields, then torque fields; else 3: the force
 *     density, plus the half-curl of the torque envelopes with the kernel-derivative route), laid
 *     out [field][c][y][x] with row stride ldx (even, >= nx); it is zeroed and then receives the
 *     spread node values.
 *   - The other arguments mean what they mean in dpstokes_plan_create / dpstokes_apply;
 *     kp->precision, kp->eta and kp->max_n are ignored.
 *   - Returns DPS_ERR_INVALID_ARG when the problem needs more scratch than the fixed array holds
 *     (roughly 80k particles with torques at m = 5, 33 Chebyshev nodes) or when an argument is
 *     invalid.  Particles outside the domain contribute nothing; their errors are not reported.
 *   - The first call on a device looks up the array's device address (once per device, with that
 *     device current); make that first call before any stream capture.
 *   - Every call shares the one array and keeps the previous call's contents in it (everything the
 *     stage needs zeroed is cleared on each call); calls that overlap on the GPU, on any streams,
 *     race with each other. */
dps_status dpstokes_spread_noalloc(double Lx, double Ly, double zmin, double zmax, int32_t wall_mode,
                                   const dps_grid* grid, const dps_kernel_params* kp, int64_t n,
                                   const double* positions, const double* forces,
                                   const double* torques, double* out_grid, int64_t ldx,
                                   void* stream);

/* ---- Batched applies ----------------------------------------------------------------------
 * No counterpart in the paper: independent products (different plans, sizes and wall modes) run
 * concurrently, each exactly as dpstokes_apply would compute it. */
typedef struct {
  dps_plan_t plan;
  int64_t n;
  const double* positions;  /* device [n][3], as in dpstokes_apply                               */
  const double* forces;     /* device [n][3]                                                      */
  const double* torques;    /* device [n][3] or NULL (must match the plan)                        */
  double* out_vel;          /* device [n][3]                                                      */
  double* out_angvel;       /* device [n][3] or NULL (must match the plan)                        */
  int32_t* status;          /* device int32 or NULL: receives the request's dps_status from the
                               device checks (what dpstokes_status would return), and the plan's
                               status word is cleared                                            */
} dps_request;

/* Enqueue `count` requests after the work already on `stream` and before later work on it.  The
 * requests run concurrently on a pool of 8 library-owned streams (created on the device's first
 * batch, or by dpstokes_batch_prepare); requests that name the same plan run in the order given.
 * Every argument check of dpstokes_apply is made for every request before anything is enqueued
 * (DPS_ERR_INVALID_ARG, nothing enqueued).  Asynchronous, no allocation, no host
 * synchronisation: a batch may be captured into a CUDA graph (call dpstokes_batch_prepare before
 * the capture) and the graph replayed; the plans then must stay alive while it is in use.  Calls
 * from several host threads are serialised while they enqueue (a per-device lock); a plan must
 * still be used by one product at a time. */
dps_status dpstokes_apply_batch(const dps_request* reqs, int32_t count, void* stream);

/* Create the current device's batch stream pool now (idempotent). */
dps_status dpstokes_batch_prepare(void);

/* ---- Serving ------------------------------------------------------------------------------
 * No counterpart in the paper.  A server owns a worker thread, `slots` streams and a cache of
 * plans keyed by every plan parameter (one plan per key).  Whenever a slot is free the worker
 * looks at the 64 oldest queued requests and admits the oldest whose plan is cached and idle,
 * else the oldest whose key has no plan yet, creating that plan if the memory budget allows after
 * evicting least-recently-used idle plans (an eviction frees device memory, which synchronises
 * the device); requests whose plan is busy wait without holding up the others.  A request that can
 * never fit the budget completes with DPS_ERR_OOM.  Each admitted request copies its inputs from
 * host memory, runs the product and copies the outputs back on its slot's stream, so requests
 * overlap on the device.  Outputs in page-locked memory receive the device-to-host copy
 * directly; pageable outputs are copied through a pinned staging buffer of the slot and then into
 * the caller's arrays by the worker when the request retires (a direct copy into pageable memory
 * would hold the worker until that product finished).  Results are those of dpstokes_apply_host
 * on a plan with the same parameters.  Submissions may come from any number of host threads. */
typedef struct dps_server_s* dps_server_t;

typedef struct {
  double Lx, Ly, zmin, zmax;  /* plan parameters, as in dpstokes_plan_create                      */
  int32_t wall_mode;
  dps_grid grid;
  dps_kernel_params kp;       /* kp.max_n is part of the plan key; 0 <= n <= kp.max_n             */
  int64_t n;
  const double* positions;    /* HOST [n][3] (pinned memory copies fastest); read after admission */
  const double* forces;       /* HOST [n][3]                                                      */
  const double* torques;      /* HOST [n][3] or NULL (must match kp.with_torque)                  */
  double* out_vel;            /* HOST [n][3], written before the request completes                */
  double* out_angvel;         /* HOST [n][3] or NULL                                              */
  dps_wall_params walls;      /* wall conditions (all zero: no-slip stationary walls); part of the
                                 plan key                                                        */
} dps_serve_request;

typedef struct {
  int32_t status;             /* dps_status of the request                                         */
  double t_submit;            /* steady-clock seconds: submission, admission, completion seen by  */
  double t_start;             /* the worker (completion is polled every ~20 microseconds)        */
  double t_done;
} dps_serve_result;

typedef struct {
  int64_t queued, running;    /* requests waiting / on a slot                                      */
  int64_t plans_resident, plans_created, plans_evicted;
  int64_t bytes_resident;     /* device bytes held by cached plans                                 */
  int64_t rejected;           /* submissions refused with DPS_ERR_BUSY (queue at its limit)        */
} dps_server_stats;

/* memory_budget_bytes > 0 bounds the plans' device memory; 1 <= slots <= 64.  The server works on
 * the device current at creation. */
dps_status dpstokes_server_create(dps_server_t* out, int64_t memory_budget_bytes, int32_t slots);

/* Load shedding: at most max_queued requests wait for admission (0, the default: no limit).  A
 * submission that finds the queue full is refused at once with DPS_ERR_BUSY (no ticket), so under
 * an offered load above the server's capacity the accepted requests keep a bounded latency. */
dps_status dpstokes_server_set_queue_limit(dps_server_t server, int64_t max_queued);

/* Queue a request (the descriptor is copied; the host buffers must stay valid until the request's
 * dpstokes_server_wait returns).  *ticket identifies it.  DPS_ERR_INVALID_ARG for n outside
 * [0, kp.max_n] or after destroy has begun; DPS_ERR_BUSY when the queue is at its limit;
 * parameter errors are reported by the result. */
dps_status dpstokes_server_submit(dps_server_t server, const dps_serve_request* req, int64_t* ticket);

/* Wait up to timeout_s seconds for a ticket; DPS_ERR_TIMEOUT if it has not completed (it keeps
 * running), DPS_ERR_INVALID_ARG for an unknown or already collected ticket. */
dps_status dpstokes_server_wait(dps_server_t server, int64_t ticket, double timeout_s,
                                dps_serve_result* result);

dps_status dpstokes_server_stats(dps_server_t server, dps_server_stats* out);

/* Finish every queued and running request, then free the slots and all cached plans. */
void dpstokes_server_destroy(dps_server_t server);

/* ---- Brownian increments ------------------------------------------------------------------
 * g = M^{1/2} w by the Lanczos process in the Krylov subspace of the mobility (Sec. IV.C), with the
 * plan's product as the operator.  Vectors have dimension d = 3n for a plan without torques
 * (layout [n][3]) and d = 6n with torques ([n][3] force part, then [n][3] torque part; the result
 * likewise: velocities, then angular velocities).  Each iteration applies the product once and
 * re-orthogonalises against the whole basis (two classical Gram-Schmidt passes); the host forms
 * T_j^{1/2} e_1 of the tridiagonal Lanczos matrix (Jacobi eigendecomposition; eigenvalues below
 * zero take a zero root) and eps_j = ||g_j - g_{j-1}|| / ||g_{j-1}||.  The process stops at the
 * first j >= 2 with eps_j <= tol, when the Krylov space is exhausted (beta_j = 0), or after
 * max_iter products. */
typedef struct dps_lanczos_s* dps_lanczos_t;

/* Basis storage for up to max_iter vectors of dimension 6 max_n (or 3 max_n) of `plan` on the
 * plan's device; 2 <= max_iter <= 128.  The plan must outlive the handle. */
dps_status dpstokes_lanczos_create(dps_lanczos_t* out, dps_plan_t plan, int32_t max_iter);

/* positions: device [n][3]; w, g: device [d] (w is the caller's i.i.d. standard normal vector and
 * is not modified; g receives the increment); 0 <= n <= max_n; tol >= 0.  iters, eps (NULL or host
 * scalars): products applied and the last eps_j (0 before the second iteration); eps_hist (NULL or
 * host array of max_iter doubles): eps_2, eps_3, ... .  Runs on `stream` and synchronises it once
 * per iteration (not graph-capturable); returns the device status of the products (as
 * dpstokes_status) or a host error.  The handle's buffers serve one call at a time. */
dps_status dpstokes_lanczos_sample(dps_lanczos_t lz, int64_t n, const double* positions, const double* w,
                                   double* g, double tol, int32_t* iters, double* eps, double* eps_hist,
                                   void* stream);

void dpstokes_lanczos_destroy(dps_lanczos_t lz);

/* Stochastic drift by random finite differences (Sec. IV.C, footnote: two extra solves per step):
 * out = (1/delta) [M(q + delta/2 W) - M(q - delta/2 W)] [W; 0], whose average over a standard
 * normal W is the divergence of the mobility with respect to the positions q (for spheres the
 * configuration is the positions only, so the torque part of the vector multiplied is zero).
 * positions, W: device [n][3]; out: device [n][3] (velocity part), followed by [n][3] (angular
 * part) for a plan with torques; delta > 0 (a length; the displaced heights must stay legal, else
 * the device status reports DPS_ERR_OUT_OF_DOMAIN).  Two products on `stream` through the plan's
 * staging buffers (not concurrently with dpstokes_apply_host on the same plan); no host
 * synchronisation, graph-capturable. */
dps_status dpstokes_rfd_drift(dps_plan_t plan, int64_t n, const double* positions, const double* W,
                              double delta, double* out, void* stream);

/* Host utility (no GPU): y = T^{1/2} e_1 for the symmetric tridiagonal T with diagonal alpha[j] and
 * off-diagonal beta[j-1] (beta may be NULL for j = 1), 1 <= j <= 128; the step the sampler takes on
 * the host each iteration. */
dps_status dpstokes_tridiag_sqrt_e1(int32_t j, const double* alpha, const double* beta, double* y);

/* Diagnostics for tests: run the apply pipeline on `stream` up to and including stage
 * `last_stage` (1 = particle records, 2 = spread, 3 = forward xy FFT, 4 = per-k solve,
 * 5 = inverse xy FFT, 6 = interpolation; the outputs may be NULL below stage 6) and copy plan buffer `which` (0 = grid/spectrum,
 * 1 = particle records, 2 = occupied plane range [2 x int32]) to the device pointer dst
 * (at most dst_bytes).  Returns DPS_ERR_INVALID_ARG for unknown stages or buffers. */
dps_status dpstokes_debug_run(dps_plan_t plan, int64_t n, const double* positions,
                              const double* forces, const double* torques, double* out_vel,
                              double* out_angvel, void* stream, int32_t last_stage);
dps_status dpstokes_debug_copy(dps_plan_t plan, int32_t which, void* dst, int64_t dst_bytes,
                               void* stream);

/* Failure injection and path forcing for tests (no counterpart in the paper).  code 1: in the next
 * apply the forward tensor-core transform withholds its matrix multiplies and their completion
 * signals, so the producers' bounded waits for a free operand stage run out (about a second): the
 * kernel records DPS_ERR_TIMEOUT in the status word (read by dpstokes_status), its blocks free
 * their tensor memory and leave, and the plan stays usable for the next apply.  code 2: in the
 * next apply every bin of the staged interpolation takes its global-memory gather (the path a bin
 * whose region does not fit in shared memory takes).  code 3: in the next apply the forward
 * TMA-staged y-FFT column pass arms its buffers' barriers but issues no box load, so its bounded
 * waits run out (about a second, then a second bounded wait for copies in flight, of which there
 * are none): the kernel records DPS_ERR_TIMEOUT and its blocks leave.  An injection applies to one
 * apply and then clears itself.  code 0 clears it.  DPS_ERR_INVALID_ARG for other codes, for code
 * 1 on a plan that does not use the tensor-core forward transform, for code 2 on a plan whose
 * interpolation variant is not 2, or for code 3 on a plan whose column pass is not the TMA-staged
 * one (plan_info.fft_register_cols != 3). */
dps_status dpstokes_debug_inject(dps_plan_t plan, int32_t code);

#ifdef __cplusplus
}
#endif

#endif /* DPSTOKES_H */
