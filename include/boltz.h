/*
 * boltz.h -- C ABI of libboltz: fast spectral evaluation of the Boltzmann collision
 * operator Q(f, f) for the variable-hard-sphere kernel on an N^3 periodised velocity
 * grid, computed independently in every spatial cell, on one NVIDIA GB300 (sm_103a).
 *
 * The method is the fast spectral scheme of Dimarco, Loubere, Narski and Rey,
 * "An efficient numerical method for solving the Boltzmann equation in
 * multidimensions" (arxiv 1608.08009), Sec. 3.3 (Carleman representation, separated
 * angular quadrature), Sec. 3.2 (L2 conservation projection, Eq. minim1) and Sec. 3.1
 * (collision step f <- f + dt Q, Eq. f_coll), organised per cell as in Sec. 4.2: one
 * forward transform of f, then for every quadrature direction the kernel coefficients
 * and inverse transforms, then the gather into Q.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Layout.     A batch of cells is stored cell after cell; one cell is f[x][y][z] with
 *              z fastest, N^3 values, value (i, j, k) taken at velocity
 *              (-L + i dv, -L + j dv, -L + k dv), dv = 2L/N.  Q has the layout and the
 *              element type of f.  Moments are U[c] = (rho, rho u_x, rho u_y, rho u_z, E)
 *              = sum_v (1, v_x, v_y, v_z, |v|^2/2) f(v) dv^3, float64.
 *  Memory.     Every f / Q / U pointer is a device pointer the caller allocated and
 *              owns; the library never frees it.  The grid object owns its tables
 *              (host and device copies) until boltz_destroy_grid.
 *  Streams.    `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *              stream).  Every compute call is asynchronous on that stream.
 *  Errors.     Argument errors are returned synchronously and leave the stream
 *              untouched.  Conditions found on the device (non-finite results, cell
 *              indices outside their pool, a bounded wait that gave up) are OR-ed
 *              into a device status word that boltz_stream_status() reads.  No call
 *              aborts, traps or waits without bound.  boltz_last_error() gives a
 *              thread-local message for the last failing call of the calling thread.
 *  Devices.    A grid is bound to the device that was current when it was created;
 *              calls must be made with that device current.
 */
#ifndef BOLTZ_H
#define BOLTZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BOLTZ_OK = 0,
  BOLTZ_EINVAL = 1,        /* bad argument (null pointer, size, unsupported value)      */
  BOLTZ_ENOMEM = 2,        /* host or device allocation failed                          */
  BOLTZ_ECUDA = 3,         /* a CUDA runtime call failed (message in boltz_last_error)  */
  BOLTZ_EUNSUPPORTED = 4,  /* valid request the library has no kernel for (e.g. N, prec) */
  BOLTZ_ENONFINITE = 5,    /* device status: a NaN or Inf was produced                  */
  BOLTZ_ETIMEOUT = 6       /* device status: a bounded mbarrier wait in a kernel gave up  */
} boltz_status;

/* Arithmetic of the transforms and angular products (the hot loop).  Moments, the
 * conservation projection and the f <- f + dt Q update are float64 in every mode. */
typedef enum {
  BOLTZ_FP64 = 0,          /* float64 register FFTs on CUDA cores (the plain form)      */
  BOLTZ_FP32_FFT = 1,      /* float32 register FFTs on CUDA cores, float32 tables       */
  BOLTZ_TF32_DFT = 2,      /* every inverse 1D pass of the term loop as a dense DFT
                              contraction on the tensor cores (tcgen05, kind::tf32, f32
                              accumulate in TMEM); inputs rounded to tf32 (~1e-3 relative
                              per pass).  N = 16, 32; reduced-precision comparison mode  */
  BOLTZ_3XBF16_DFT = 3,    /* as BOLTZ_TF32_DFT on kind::f16 with bf16 operands split into
                              high and low parts (Ah Wh + Ah Wl + Al Wh): ~16 significant
                              bits per product, ~1e-4 relative per pass                 */
  BOLTZ_3XTF32_DFT = 4     /* as BOLTZ_TF32_DFT with operands split into tf32 high and
                              low parts, Ah Wh + Ah Wl + Al Wh: float32-class accuracy  */
} boltz_precision;

/* Options of boltz_create_grid.  Pass NULL for all defaults; boltz_default_opts()
 * fills the defaults so that single fields can be changed. */
typedef struct {
  int dirs_kind;     /* half-sphere direction set (Sec. 3.3 quadrature), default 0:
                        0 = product grid, midpoints in theta and varphi, weights
                            (pi/A1)(pi/A2) sin(theta)  (the paper's uniform grids)
                        1 = spherical Fibonacci points, weights 2 pi / M
                        2 = Gauss-Legendre in cos(theta) x midpoints in varphi       */
  int dirs_a1;       /* A1 of the product grids (must divide M); <= 0: smallest divisor
                        of M that is >= sqrt(M) (M = 64 -> 8 x 8)                     */
  double R_trunc;    /* Carleman ball radius R; <= 0: R = 2 S with S = 2L/(3+sqrt 2)
                        the support radius of the periodisation rule (Sec. 3.3)       */
  double C_gamma;    /* VHS constant, B = C_gamma |q|^gamma; default 1                */
  int radial_rank;   /* terms of the radial expansion of Btilde when gamma != 1;
                        <= 0: 1 for gamma == 1 (exact decoupling), 16 otherwise       */
  int inner_nodes;   /* Gauss-Legendre nodes of the inner radial integral, default 128 */
  int project;       /* 1 (default): apply the conservation projection to Q          */
  int term_groups;   /* split each cell's separated terms over this many thread-block
                        clusters (1 = default: one cluster per cell).  G > 1 lowers the
                        latency of batches too small to fill the GPU at the cost of G - 1
                        extra forward transforms per cell; the cluster that finishes a
                        cell's last group (a per-cell arrival counter, no waiting) sums
                        the partial gains in group order and runs the epilogue.  Needs
                        device scratch of (G + 1) N^3 values per cell (grown on demand,
                        kept with the grid).  Clamped to [1, M_eff].  Results depend on G (rounding
                        order of the gain sum) but not on the batch size.               */
  int cluster_size;  /* thread-block cluster size (CTAs per cell) of the float32 path;
                        0 = default (N 8: 1, 16: 1, 24: 3, 32: 1, 48: 12, 64: 16).  Also
                        built: 16: 2, 4; 24: 2, 6; 32: 8, 4, 16; 48: 8.  Larger clusters give
                        each CTA a thinner slab (fewer threads, more CTAs per SM).  At N = 32
                        size 1 is one 512-thread CTA per cell that holds half the spectrum
                        and the gain in tensor memory and runs each inverse transform in two
                        halves of x; it takes no term groups (with term_groups > 1 the
                        default becomes 8, an explicit 1 returns BOLTZ_EUNSUPPORTED) and, by
                        default, is not used for f stored in float64 (clusters of 8 there).
                        The float64 path always uses its own size (8: 1, 16: 2, 24: 3,
                        32: 8).  Results agree across sizes up to float32 rounding (transform
                        order) and the rounding of the moment sums.  Other values:
                        BOLTZ_EUNSUPPORTED. */
} boltz_grid_opts;

typedef struct boltz_grid_s* boltz_grid;

/* A batch of cells that share one grid. */
typedef struct {
  boltz_grid grid;
  int64_t n_cells;   /* number of cells, >= 0 (0 is a no-op)                          */
  int prec;          /* a boltz_precision                                             */
  int f_is_fp64;     /* 1: f and Q are float64; 0: float32                            */
} boltz_batch;

void boltz_default_opts(boltz_grid_opts* opts);

/* Build a grid: velocity grid, direction set {e_j, w_j}, the separated kernel tables
 * alpha_j(k) = Btilde phi(xi_k . e_j), alpha'_j(k) = psi(|Pi_{e_j-perp} xi_k|) on the
 * full mode set (Sec. 3.3, 3D decoupling formula; psi is the disk transform
 * 2 pi R J1(R s)/s), the loss multiplier D(k) = sum_j w_j alpha_j alpha'_j and the 5x5
 * matrix of the projection (Sec. 3.2, Eq. minim1).  For gamma != 1 the kernel is not
 * separable in 3D and a rank-r radial expansion is tabulated instead (r terms per
 * direction).  Builds the tables on the host in float64 and copies them to the
 * current device.
 *   N_v     points per axis: 8, 16, 24, 32 (float64 and float32 paths) and 48, 64
 *           (float32 path only: a float64 pencil of 48 or 64 values does not fit one
 *           thread's registers; float64 batches on these grids return
 *           BOLTZ_EUNSUPPORTED).  Other even sizes: BOLTZ_EUNSUPPORTED.
 *   L       half-width of the velocity box [-L, L)^3, > 0.
 *   gamma   VHS exponent in [-3, 1] (1 = hard spheres, 0 = Maxwell molecules).
 *   M_dirs  number of directions, 1..4096.
 *   out     receives the handle; unchanged on error.
 * Errors: EINVAL, EUNSUPPORTED (N_v), ENOMEM, ECUDA.  Blocking (host work + copies). */
boltz_status boltz_create_grid(int N_v, double L, double gamma, int M_dirs,
                               const boltz_grid_opts* opts, boltz_grid* out);

/* Two-dimensional grid for Maxwell molecules (Sec. 3.3, dimension two; Eq. dfor0): the
 * Carleman kernel is the constant Btilde = 2 C_gamma (opts->C_gamma, default 1;
 * C_gamma = 1/(2 pi) is the normalisation of the 2D BKW solution of Test 1.1), A = M_dirs
 * equally spaced angles theta_p = pi p / A with weight pi / A, alpha_p(k) =
 * Btilde 2R Sinc(R xi_k . e_p), alpha'_p(k) = 2R Sinc(R xi_k . e_p-perp); S, R as in 3D
 * (opts->R_trunc).  Cells are N_v x N_v arrays [x][y] (y fastest); boltz_collide,
 * boltz_relax (and _indexed, _host, _noalloc) and boltz_moments accept batches on it;
 * moments are (rho, rho u_x, rho u_y, 0, E).  Term groups and cluster sizes do not apply.
 *   N_v     8, 16, 32 (float64 and float32), 64 (float32 only).
 *   M_dirs  number of angles A, 1..4096.
 * Errors: EINVAL, EUNSUPPORTED (N_v), ENOMEM, ECUDA. */
boltz_status boltz_create_grid2d(int N_v, double L, int M_dirs, const boltz_grid_opts* opts, boltz_grid* out);

/* Free the grid and its tables.  Synchronises the device first.  NULL is a no-op. */
boltz_status boltz_destroy_grid(boltz_grid g);

/* Q = Q(f, f) for every cell of the batch (Sec. 3.3), projected so that the moments
 * of Q vanish (Sec. 3.2) unless the grid was built with project = 0.  f and Q are
 * device arrays of n_cells * N^3 elements (float32 or float64 per f_is_fp64); they must
 * not overlap.  One kernel launch on `stream`; HBM sees one read of f and one write of
 * Q per cell.  Errors: EINVAL, EUNSUPPORTED (prec for this N), ECUDA. */
boltz_status boltz_collide(const boltz_batch* b, const void* f, void* Q, void* stream);

/* Advance the homogeneous relaxation df/dt = Q(f) (Sec. 3.1, Eq. relax) in place by
 * `steps` steps of size dt.  rk_order 1: forward Euler f <- Pi(f + dt Q(f))
 * (Eq. f_coll); rk_order 2: Heun, f1 = Pi(f + dt Q(f)), f <- Pi(f/2 + (f1 + dt Q(f1))/2).
 * Pi projects onto the moments the cells had when the call started (Eq. minim1 with U
 * fixed), so rounding does not accumulate in rho, rho u, E.  Uses library-owned scratch
 * (one float64 moment row per cell, and one copy of f for rk_order 2), grown on demand
 * and kept with the grid.  Errors: EINVAL (dt <= 0, steps < 0, rk_order), EUNSUPPORTED,
 * ENOMEM, ECUDA. */
boltz_status boltz_relax(const boltz_batch* b, void* f, double dt, int steps, int rk_order,
                         void* stream);

/* Forward-Euler relaxation as boltz_relax with rk_order 1, allocating no memory.  The
 * paper has no counterpart; this exists for callers that cannot let the library call
 * cudaMalloc / cudaFree (a framework whose caching allocator holds the device memory, a
 * stepping loop that must not stall on the device-wide synchronisation a free implies,
 * an embedding that forbids library-owned device memory).  The per-cell moment targets
 * live in a fixed array inside the library's device image, 65536 cells * 5 doubles
 * (2.5 MiB), held on every device that loads the library until process exit.
 * n_cells above 65536 returns BOLTZ_EINVAL.  It runs boltz_relax's launches with one
 * term group: on a grid with term_groups = 1 the result equals boltz_relax (rk_order 1)
 * bit for bit; with term_groups > 1 it equals it up to the rounding of the gain sum.
 * All calls on a device share the array and it keeps the last call's contents; each
 * call's first launch rewrites the targets of all its cells before they are read, but
 * calls that overlap on the GPU race on the array, so serialise them.  Each call made
 * while its stream is not capturing looks the array's device address up
 * (cudaGetSymbolAddress) and caches it per device; a call during stream capture uses
 * the cached address, so make the first call on a device before any stream capture.
 * f: device array of n_cells * N^3 elements, updated in place.  Errors: EINVAL,
 * EUNSUPPORTED, ECUDA. */
boltz_status boltz_relax_noalloc(const boltz_batch* b, void* f, double dt, int steps, void* stream);

/* boltz_relax for distributions in HOST memory (Sec. 3.1, Eq. relax; the steps are those
 * of boltz_relax).  f_in, f_out: host arrays of n_cells * N^3 elements (float32 or
 * float64 per f_is_fp64), owned by the caller; they may be the same array.  Page-locked
 * memory (cudaHostAlloc / cudaHostRegister) lets the copies overlap the compute; pageable
 * memory is accepted and serialises.  The batch runs in chunks (boltz_host_chunks gives
 * them): chunk_cells > 0 gives equal chunks of that many cells; 0 gives the default, small
 * chunks at both ends growing by 3/2 towards an eighth of the batch in the middle, so
 * only a small first upload and a small last download stay exposed.  The upload of a
 * chunk, the collision steps of the previous one and the download of the one before run
 * concurrently on two library streams and `stream`.  Returns once the work
 * is enqueued; `stream` is ordered after the last download, so synchronise it (or call
 * boltz_stream_status) before reading f_out or reusing f_in.  The result equals
 * boltz_relax on the same cells bit for bit.  Staging buffers (three chunks, a Heun
 * stage and the chunk's moment targets) are owned by the grid and grown on demand; calls
 * on one grid must not overlap.  Errors: EINVAL, EUNSUPPORTED, ENOMEM, ECUDA. */
boltz_status boltz_relax_host(const boltz_batch* b, const void* f_in, void* f_out, double dt, int steps,
                              int rk_order, int64_t chunk_cells, void* stream);

/* The chunks boltz_relax_host runs a batch in, for n_cells cells of cell_bytes bytes of f
 * each (N^3 or N^2 values of 4 or 8 bytes) and its chunk_cells argument.  chunk_cells > 0:
 * equal chunks of that many cells, the last one shorter.  0: a ramp of chunks from 32 MiB
 * of f growing by 3/2 up to the middle size (an eighth of the batch, at least 64 MiB, at
 * most 1 GiB of f), equal middle chunks, and the same ramp reversed, when the batch holds
 * both ramps and one middle chunk; smaller batches get about eight equal chunks of at
 * least 64 MiB (or the whole batch).  Host only, no device work.  Writes the first
 * min(count, cap) chunk sizes to sizes (host array owned by the caller) and returns the
 * number of chunks, or -1 on invalid arguments (n_cells, chunk_cells or cap negative,
 * cell_bytes not positive, sizes null with cap > 0). */
int64_t boltz_host_chunks(int64_t n_cells, int64_t cell_bytes, int64_t chunk_cells, int64_t* sizes, int64_t cap);

/* ---- Ragged batches ------------------------------------------------------------------
 * A plan advances several groups of cells, each group on its own grid (any mix of N_v,
 * M_dirs, gamma, precision), by `steps` Euler (rk_order 1) or Heun (rk_order 2) steps of
 * the relaxation of Sec. 3.1 (Eq. relax, Eq. f_coll) per boltz_plan_run, projecting onto
 * the moments each cell had when the run started (as boltz_relax).  The kernels are
 * specialised per N, so a step is one launch per group; the plan captures the whole step
 * loop as one CUDA graph in which every group is a concurrent branch, and
 * boltz_plan_run launches that graph on `stream`.
 * Autotuning (BOLTZ_PLAN_AUTOTUNE) chooses each group's (term groups, cluster size) at
 * plan creation on copies of the groups' cells: every candidate of a group is timed alone
 * and the three fastest are kept; then, starting from the grids' own settings, the groups
 * are visited slowest first and a kept candidate is adopted only if the whole concurrent
 * step (all groups at once, as the graph runs them) gets faster by more than 1 %.  With
 * BOLTZ_PLAN_TUNE_PRECISION as well, a float32 register-FFT group whose N has tensor-core
 * transforms (16, 32) may also be switched to BOLTZ_3XTF32_DFT when that is faster (a
 * float32-class precision with a different rounding).  Without autotuning a group uses
 * its grid's term_groups and the default cluster size, and the results equal
 * boltz_relax's bit for bit.  BOLTZ_PLAN_SERIAL puts the groups one after another on one
 * branch (for comparison).
 * Ownership: the caller owns the grids and the device arrays f, which must stay valid and
 * in place for the plan's life; each group's grid must be distinct and must not be used
 * by other calls while the plan runs (its scratch is shared).  The plan owns its
 * streams, scratch (targets, Heun stage) and graph.  boltz_plan_create synchronises
 * `stream` and the device.  Errors: EINVAL, EUNSUPPORTED, ENOMEM, ECUDA. */
typedef struct boltz_plan_s* boltz_plan;

typedef struct {
  boltz_grid grid;
  int64_t n_cells;   /* cells of this group, >= 0                                       */
  int prec;          /* a boltz_precision                                               */
  int f_is_fp64;     /* 1: f is float64; 0: float32                                     */
  void* f;           /* device array [n_cells][N^3], advanced in place by each run      */
} boltz_group;

enum { BOLTZ_PLAN_AUTOTUNE = 1, BOLTZ_PLAN_SERIAL = 2, BOLTZ_PLAN_TUNE_PRECISION = 4 };

boltz_status boltz_plan_create(const boltz_group* groups, int n_groups, double dt, int steps, int rk_order,
                               int flags, void* stream, boltz_plan* out);
/* One graph launch: every group advances by the plan's steps.  Asynchronous on stream. */
boltz_status boltz_plan_run(boltz_plan p, void* stream);
/* The launch configuration chosen for group `group`: term groups, cluster size and the
 * tuned duration of one launch in microseconds (0 when not tuned).  Outputs nullable. */
boltz_status boltz_plan_group_info(boltz_plan p, int group, int* term_groups, int* cluster, double* tuned_us);
/* The precision a group's launches use (its own, or BOLTZ_3XTF32_DFT when autotuning with
 * BOLTZ_PLAN_TUNE_PRECISION chose the tensor-core transforms).  Errors: EINVAL. */
boltz_status boltz_plan_group_precision(boltz_plan p, int group, int* prec);
/* Synchronises the device, frees the plan.  NULL is a no-op. */
boltz_status boltz_plan_destroy(boltz_plan p);

/* Cells addressed through an index array (ragged batches, resident pools): cell c of the
 * call is slot cell_idx[c] of f (and of Q), with slot s at offset s * N^3.  cell_idx is a
 * device array of n_cells int64 values; slots must be distinct and lie in
 * [0, pool_cells).  An index outside the pool is not dereferenced: that cell writes
 * nothing and boltz_stream_status() later returns BOLTZ_EINVAL.
 * boltz_collide_indexed: Q(f) of the listed slots (as boltz_collide).
 * boltz_relax_indexed:   forward-Euler steps of the listed slots in place (as
 *   boltz_relax with rk_order 1; targets per slot in library scratch sized for the pool).
 * Errors: EINVAL, EUNSUPPORTED, ENOMEM, ECUDA. */
boltz_status boltz_collide_indexed(const boltz_batch* b, const void* f, void* Q, const int64_t* cell_idx,
                                   int64_t pool_cells, void* stream);
boltz_status boltz_relax_indexed(const boltz_batch* b, void* f, const int64_t* cell_idx, int64_t pool_cells,
                                 double dt, int steps, void* stream);

/* ---- Serving: continuous batching of relaxation jobs ------------------------------------
 * A job is a batch of n_cells cells of one grid (one cell for boltz_server_submit), each
 * relaxing under df/dt = Q(f) (Sec. 3.1, Eq. relax) for `steps` forward Euler steps of
 * size dt with the projection after each step (each step projects onto the moments the
 * cell has at that step).  The server makes ONE device allocation of hbm_budget_bytes
 * and carves everything it uses on the device out of it: the grids' index lists and,
 * per admitted job, its float32 distributions plus, on grids with term_groups G > 1, its
 * term-group scratch ((G + 1) N^3 floats per cell).  A job is admitted when those regions
 * fit, so the device memory the server holds never exceeds the budget.  Queues are per
 * grid, first come first served within a grid: a job that does not fit yet waits without
 * holding back the other grids.  All resident cells of a grid advance by one indexed
 * launch per iteration; each finished job is copied back to its host buffer
 * asynchronously and its regions return to the arena when that copy completes.  A job's
 * result does not depend on which other jobs are resident.  Every grid has its own
 * stream (ordered after the work queued on `stream` at creation) and at most two
 * iterations in flight, so grids advance at their own pace.  Calls are not thread-safe.
 *   create: grids (one per grid shape a job may use, kept alive by the caller), prec,
 *           dt, budget.  EINVAL if the budget cannot hold one cell of every grid (with
 *           its scratch and the index lists); ENOMEM if the allocation fails.
 *   submit / submit_batch: f_host, out_host: n_cells * N^3 floats each (pinned memory
 *           recommended), owned by the caller until poll reports the job done; returns a
 *           job id.  EINVAL for a job larger than the budget can ever hold.
 *   step:   admission, then one iteration (one step of every resident job, retirement of
 *           the finished ones) for every grid with resident jobs, waiting where a grid
 *           already has two iterations in flight, and, when a queued job waits for memory,
 *           for the result copies of finished jobs (which return theirs); reports counts
 *           (jobs).
 *   pump:   as step, but never waits: a grid with two iterations in flight is skipped;
 *           n_launched = iterations issued (nullable).  For serving loops.
 *   poll:   done = 1 once out_host holds the result.
 *   stats:  reserved (= the budget), used and peak used bytes of the arena, resident
 *           cells and jobs, queued jobs. */
typedef struct boltz_server_s* boltz_server;
typedef struct {
  size_t reserved_bytes;   /* device bytes the server holds: the budget */
  size_t used_bytes;       /* of those, in index lists and admitted jobs' regions */
  size_t peak_used_bytes;  /* largest used_bytes so far */
  int64_t resident_cells;
  int64_t resident_jobs;
  int64_t queued_jobs;
} boltz_server_stats;
boltz_status boltz_server_create(const boltz_grid* grids, int n_grids, int prec, double dt,
                                 size_t hbm_budget_bytes, void* stream, boltz_server* out);
boltz_status boltz_server_submit(boltz_server s, int grid_index, const float* f_host, float* out_host,
                                 int steps, int64_t* job_id);
boltz_status boltz_server_submit_batch(boltz_server s, int grid_index, const float* f_host, float* out_host,
                                       int64_t n_cells, int steps, int64_t* job_id);
boltz_status boltz_server_step(boltz_server s, int* n_resident, int* n_queued);
boltz_status boltz_server_pump(boltz_server s, int* n_resident, int* n_queued, int* n_launched);
boltz_status boltz_server_poll(boltz_server s, int64_t job_id, int* done);
boltz_status boltz_server_stats_get(boltz_server s, boltz_server_stats* out);
/* Checkpoint of one job: f_host (n_cells * N^3 floats) receives the job's state after
 * every iteration issued for it so far, *remaining_steps the steps still to run (0 once
 * finished).  Synchronises the job's grid stream.  The state plus the remaining steps is
 * all a job needs: submitting them to any server with the same grid continues the job
 * and gives the same bits as an uninterrupted run. */
boltz_status boltz_server_checkpoint(boltz_server s, int64_t job_id, float* f_host, int* remaining_steps);
boltz_status boltz_server_destroy(boltz_server s);

/* ---- Fast Kinetic Scheme in one space dimension (Sec. 3.1) ------------------------------
 * Transport of the piecewise-constant distribution (Eq. transport, Eq. f_bar) coupled to
 * the collision step at the cell centres (Eq. relax and Eq. f_coll with the rescaled
 * operator Q / tau of the numerical tests, forward Euler, projected onto the moments of
 * the transported values, Sec. 3.2).  Cells form rows of n_x cells of width dx along x;
 * the velocity grid is the batch's grid.  Each x-velocity's intervals move exactly with
 * v_x; after a time t the centre of cell j lies in the interval that started as cell
 * j - ceil(v_x t / dx - 1/2), so a step moves each x-velocity's column of centre values
 * by 0 or +-1 cells, fused into the collision launch's loads: one launch per step, f
 * read once and the new f written once.  The state holds only the time t (t += dt per
 * step).
 *   create:  grid, n_x >= 1, dx > 0.  EUNSUPPORTED for N > 64.
 *   step:    f_in -> f_out (device, n_cells * N^3 each, n_cells a multiple of n_x,
 *            out of place: f_out != f_in); inflow_lo / inflow_hi: device [rows][N^3],
 *            the states left of each row's cell 0 and right of its cell n_x - 1 (fixed
 *            Dirichlet states, or a neighbouring sub-domain's edge cells at the start
 *            of the step for a split domain, Sec. 4.2, fig. mpi-decomp).  dt > 0 with
 *            dt |v_x| <= dx for every grid velocity (Eq. Time; EINVAL otherwise), tau > 0.
 *            Asynchronous on `stream`; device conditions as boltz_collide.
 *   time / set_time: the accumulated time (checkpoint and resume).
 *   shifts:  d[kx] (N ints), the column moves the next step of size dt would make. */
typedef struct boltz_fks_s* boltz_fks;
boltz_status boltz_fks_create(boltz_grid g, int64_t n_x, double dx, boltz_fks* out);
boltz_status boltz_fks_step(boltz_fks s, const boltz_batch* b, const void* f_in, void* f_out,
                            const void* inflow_lo, const void* inflow_hi, double dt, double tau,
                            void* stream);
boltz_status boltz_fks_time(boltz_fks s, double* t);
boltz_status boltz_fks_set_time(boltz_fks s, double t);
boltz_status boltz_fks_shifts(boltz_fks s, double dt, int* d);
boltz_status boltz_fks_destroy(boltz_fks s);

/* U[c] = (rho, rho u, E) of every cell (Eq. i5 on the grid, Eq. DM), float64,
 * U a device array of n_cells * 5 doubles.  Errors: EINVAL, ECUDA. */
boltz_status boltz_moments(const boltz_batch* b, const void* f, double* U, void* stream);

/* Synchronise `stream`, then read and clear the device status word of the current
 * device.  Returns BOLTZ_ECUDA if the stream itself reported an error, else the first
 * condition the word holds of: BOLTZ_ETIMEOUT (a bounded mbarrier wait gave up; that
 * launch's results are invalid), BOLTZ_EINVAL (a cell index outside its pool; that cell
 * was not written), BOLTZ_ENONFINITE (a NaN or Inf was produced); else BOLTZ_OK. */
boltz_status boltz_stream_status(void* stream);

/* Thread-local message of the last failing call of this thread ("" if none). */
const char* boltz_last_error(void);

/* Self-check of the library's own float <-> double conversions, which the 2D kernel
 * runs on the integer pipes because GB300 issues the hardware conversions to its narrow
 * FP64 pipe.  Compares them with the hardware conversions on the current device:
 * float -> double on all 2^32 float bit patterns, double -> float (round to nearest
 * even) on 2^32 pseudo-random doubles and on the ties and near-ties between neighbouring
 * floats.  mismatches: host array of 2 counts (float -> double, double -> float); both
 * 0 when the conversions are exact.  Synchronous; allocates 16 bytes of device memory.
 * Errors: EINVAL (null pointer), ENOMEM, ECUDA. */
boltz_status boltz_selftest_conversions(uint64_t* mismatches);

/* Grid description for callers and tests.  Any output pointer may be NULL.
 *   S, R       support radius and Carleman radius; M_eff = M_dirs * radial_rank. */
boltz_status boltz_grid_info(boltz_grid g, int* N_v, double* L, double* dv, double* S,
                             double* R, int* M_eff);

/* Copy the float64 host tables out (for parity checks of the table builder):
 * e [M_dirs * 3], w [M_eff], alpha [M_eff * N^3], alphap [M_eff * N^3], D [N^3], each in
 * the (kx, ky, kz) FFT storage order of the mode numbers (index i holds k = i for
 * i < N/2, else i - N).  Any pointer may be NULL; sizes are in elements. */
boltz_status boltz_grid_tables(boltz_grid g, double* e, double* w, double* alpha,
                               double* alphap, double* D);

/* Version string of the library. */
const char* boltz_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BOLTZ_H */
