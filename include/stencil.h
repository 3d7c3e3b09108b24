/* stencil.h - C ABI of the GB300 temporally-blocked Jacobi stencil engine.
 *
 * The engine advances first-order Jacobi stencils (Table 2 of Zohouri, Podobas, Matsuoka,
 * "Combined Spatial and Temporal Blocking for High-Performance Stencil Computation on FPGAs
 * Using OpenCL", arXiv 1802.00438):
 *   Diffusion 2D (5-point), Diffusion 3D (7-point), Hotspot 2D and Hotspot 3D (thermal, with a
 *   per-cell power input and an ambient temperature),
 * with the clamped boundary of Sec. 5.1 (an out-of-range neighbour is the boundary cell), using
 * the combined spatial and temporal blocking of Sec. 3.1-3.2: overlapped tiles with halos of
 * width rad * T (Eq. 2), T time steps fused per pass over device memory, redundant halo
 * computation and masked stores (Sec. 3.2).  A run of `steps` steps is ceil(steps / T) passes
 * (Eq. 8); when T does not divide `steps` the last pass fuses the remainder (Sec. 3.2).
 *
 * Layout: every grid is a dense row-major float array, x fastest:
 *   index(x, y, z) = x + nx * (y + ny * z)
 * Neighbours: w = x-1, e = x+1, n = y-1, s = y+1, b = z-1, a = z+1.
 *
 * Coefficients (host array, copied into the launch):
 *   Diffusion 2D  [cc, cw, ce, cs, cn]                     (Table 2 row 1)
 *   Diffusion 3D  [cc, cw, ce, cs, cn, cb, ca]             (Table 2 row 2)
 *   Hotspot 2D    [sdc, Rx, Ry, Rz, amb]                   (Table 2 row 3: sdc, Rx_1, Ry_1,
 *                                                          Rz_1, TEMP_AMB)
 *   Hotspot 3D    [cc, cw, ce, cs, cn, cb, ca, sdc, amb]   (Table 2 row 4)
 *
 * Arithmetic is float32 (Sec. 5.1: all benchmarks are single precision).  A plan made with
 * `exact = 1` evaluates every cell in the order Table 2 prints it, one rounding per operation,
 * and is bit-identical to a plain sequential Jacobi loop; with `exact = 0` it contracts the
 * same expression into fused multiply-adds.
 *
 * Errors: every entry point returns 0 (ST_OK) or a negative ST_ERR_* code and never throws.
 * Launches are asynchronous on the plan's stream; a device-side failure is reported by
 * stencil_plan_sync() or by the next call on the plan.  A plan is not thread-safe; distinct
 * plans are independent.
 */
#ifndef GB300_STENCIL_H
#define GB300_STENCIL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ST_ABI_VERSION 4

/* status codes */
#define ST_OK                    0
#define ST_ERR_INVALID_ARG      -1   /* null pointer, bad enum, overlapping buffers, steps < 0 */
#define ST_ERR_DIMS_MISMATCH    -2   /* nx, ny, nz differ from the plan's */
#define ST_ERR_UNSTABLE_COEFFS  -3   /* strict plan: coefficients break the stability bound */
#define ST_ERR_CUDA             -4   /* a CUDA runtime call or a launch failed */
#define ST_ERR_OOM              -5   /* device allocation failed */
#define ST_ERR_TIMEOUT          -6   /* a bounded device-side wait gave up */
#define ST_ERR_UNSUPPORTED      -7   /* valid request with no compiled kernel */
#define ST_ERR_TOO_LARGE        -8   /* grid exceeds the fixed buffer of stencil_run_noalloc */

/* stencil kinds (Table 2) */
#define ST_DIFFUSION 0
#define ST_THERMAL   1
/* Diffusion 2D with per-cell coefficients: Table 2 row 1 whose five coefficients are arrays
 * (Sec. 5.1 lets a kernel variable be a scalar argument or an array), each cell updated with its own
 * cc, cw, ce, cs, cn in the printed order.  The arrays are five dense planar grids
 * [cc | cw | ce | cs | cn] of nx*ny floats each, passed to stencil_run in place of the power
 * map (device pointer, 5*nx*ny floats, read only); stencil_run's host `coeffs` is unused and
 * may be NULL.  2D, float32 storage, not strict (the stability bound would need the planes on
 * the host). */
#define ST_DIFFUSION_VAR 2

/* storage types of the grids between passes */
#define ST_F32  0
#define ST_BF16 1
#define ST_F16  2
#define ST_F64  3   /* verification reductions only */

typedef struct stencil_plan_s *stencil_plan;

/* Problem and tuning description for stencil_plan_create. */
typedef struct {
    int kind;        /* ST_DIFFUSION, ST_THERMAL or ST_DIFFUSION_VAR */
    int ndim;        /* 2 or 3 */
    int nx, ny, nz;  /* grid size in cells, each >= 1; nz is ignored (taken as 1) for 2D */
    int storage;     /* grid storage between passes: ST_F32, or ST_BF16 / ST_F16 (2D contracted
                        plans of ST_DIFFUSION / ST_THERMAL, rad <= 1: 16-bit codes with a
                        float32 offset and scale per block; arithmetic stays float32.  Passes
                        store each cell as its difference from its block's first cell
                        (scale 1); fp16 differences saturate at +-65504) */
    int force_T;     /* fused steps per pass (par_time, Sec. 3.2); 0 = the plan chooses */
    int force_bx;    /* tile width in cells incl. halos (bsize_x, Sec. 3.1); 0 = choose */
    int force_by;    /* 3D: tile height in cells incl. halos (bsize_y); 0 = choose.  2D: must
                        be 0 */
    int force_vec;   /* 2D: cells per thread along x (par_vec, Sec. 3.1); 3D: cells per thread,
                        16 (2 x 8 rows, three-plane windows), 8 (2 x 4 rows) or 4 (2 x 2 rows;
                        8 and 4: partial sums along z, contracted only); 0 = choose */
    int exact;       /* 1: Table 2 order, no fused multiply-add; 0: contracted */
    int strict;      /* 1: reject coefficients that break the explicit stability bound */
    void *stream;    /* cudaStream_t the plan launches on; NULL = the legacy default stream */
    int rad;         /* stencil radius (rad of Eqs. 1-2): 0 or 1 = the Table 2 stencils; 2..4 =
                        star diffusion of that radius (4*rad+1 points; ST_DIFFUSION, 2D, float32
                        storage), coefficients [cc, then per distance d = 1..rad: cw_d, ce_d,
                        cs_d, cn_d], each neighbour clamped to the grid on its axis (Sec. 5.1) */
    int partial_rows; /* 2D contracted streaming kernels: 1 = partial sums updated in place,
                        2 = two alternating sets of partial rows, 0 = choose */
    int resident;    /* 2D float32 plans of ST_DIFFUSION / ST_THERMAL, rad <= 1: 1 = resident
                        tiles (the whole grid stays on chip for the whole run: ONE cooperative
                        launch per run, halos exchanged through L2 every T steps; ST_ERR_UNSUPPORTED
                        when the grid does not fit), -1 = never, 0 = the plan chooses (resident
                        when the grid fits and nothing else is forced; force_T then sets the
                        steps per exchange and force_vec the cells per thread along x, 2 or 4) */
} stencil_desc;

/* What a plan chose (for reports and tests). */
typedef struct {
    int T;              /* fused steps per pass */
    int bx, by;         /* tile size in cells incl. halos (by = 0 for 2D streaming) */
    int halo;           /* halo width per side in cells (>= rad * T, Eq. 2) */
    int vec;            /* cells per thread (along x in 2D; x times rows in 3D) */
    int warps;          /* warps per block */
    int ctas;           /* blocks per launch (a multiple of the SM count where possible) */
    int sms;            /* streaming multiprocessors on the plan's device */
    long long scratch_bytes;   /* device scratch the plan owns */
    int exact;          /* as requested */
    int kernel_id;      /* internal kernel family (diagnostics) */
    double model_gcells;   /* the GPU restatement of Eqs. 3-9 with the library's calibration,
                              for this plan at 1000 steps, in 10^9 cell updates/s; 0 where no
                              calibration exists (exact and 16-bit plans) */
    int resident;       /* 1: resident tiles (T = steps between halo exchanges, bx x by the
                           tile incl. halos, ctas the co-resident blocks); 0: passes */
    int partial_rows;   /* 2D contracted streaming kernels: 1 in place, 2 two-row; else 0 */
} stencil_plan_info;

/* Create a plan for one problem shape on the current CUDA device.  Allocates one grid-sized
 * ping-pong scratch buffer (Sec. 2.1's second buffer) and keeps it until destroy.
 * out: receives the plan (NULL on failure).
 * Errors: ST_ERR_INVALID_ARG (bad desc), ST_ERR_UNSUPPORTED (e.g. a storage type or forced
 * parameter set with no compiled kernel), ST_ERR_OOM, ST_ERR_CUDA. */
int stencil_plan_create(stencil_plan *out, const stencil_desc *desc);

/* Advance grid_in by `steps` Jacobi steps (Sec. 2.1) into grid_out.
 * grid_in  : device pointer, nx*ny*nz floats, read only (never modified).
 * grid_out : device pointer, nx*ny*nz floats; may equal grid_in (in place); any other
 *            overlap with grid_in or power is ST_ERR_INVALID_ARG.
 * power    : device pointer to the per-cell power map (same layout) for ST_THERMAL, to the
 *            five coefficient planes for ST_DIFFUSION_VAR (must not overlap grid_out), NULL
 *            for ST_DIFFUSION.
 * coeffs   : host pointer to the coefficient array of the plan's stencil (layouts above);
 *            NULL is accepted for ST_DIFFUSION_VAR, which does not read it.
 * nx,ny,nz : must equal the plan's (ST_ERR_DIMS_MISMATCH); nz = 1 for 2D.
 * steps    : >= 0; 0 copies grid_in to grid_out.
 * Runs ceil(steps/T) passes on the plan's stream and returns without waiting. */
int stencil_run(stencil_plan plan, const void *grid_in, void *grid_out, const void *power,
                const float *coeffs, int nx, int ny, int nz, int steps);

/* Advance grid_in by `steps` Jacobi steps and keep every intermediate state: state t+1 (t =
 * 0 .. steps-1) lands at states + t * stride (in floats).  The passes are the plan's temporally
 * blocked ones (Sec. 3.2) with T = 8 steps fused, each fused step's compute block also written
 * out, so a trajectory costs ceil(steps / 8) launches instead of `steps`.  Used for the
 * adjoint's recomputation of the forward states between checkpoints.
 * plan     : a contracted (exact = 0), float32, 2D plan of ST_DIFFUSION or ST_THERMAL, rad <= 1
 *            (else ST_ERR_UNSUPPORTED).
 * grid_in  : device, nx*ny floats, read only; may not overlap the states written.
 * states   : device, steps states of nx*ny floats each, stride >= nx*ny floats apart.
 * power, coeffs : as for stencil_run.
 * steps    : >= 1.  Asynchronous on the plan's stream. */
int stencil_run_trajectory(stencil_plan plan, const void *grid_in, void *states, long long stride,
                           const void *power, const float *coeffs, int steps);

/* Wait for the plan's stream; returns the first asynchronous error seen (ST_ERR_CUDA,
 * ST_ERR_TIMEOUT) or ST_OK. */
int stencil_plan_sync(stencil_plan plan);

/* Bounded waits of a resident-tile plan: a block waits at most wait_ns (> 0; default 1 s) for a
 * neighbour's halo cells, then sets the plan's error flag (stencil_plan_sync returns
 * ST_ERR_TIMEOUT) and every block leaves; the output is then undefined.  hold_block >= 0 makes
 * that block stop publishing its cells from exchange hold_epoch (0-based) on (a test of the
 * timeout path: its neighbours give up); -1 = none.  Errors: ST_ERR_INVALID_ARG (no plan, wait_ns <= 0),
 * ST_ERR_UNSUPPORTED (the plan does not run resident tiles). */
int stencil_plan_set_wait(stencil_plan plan, long long wait_ns, int hold_block, int hold_epoch);

/* Fill *info with the plan's chosen parameters. */
int stencil_plan_get_info(stencil_plan plan, stencil_plan_info *info);

/* Enable (1) or disable (0) per-launch timing: with it on, stencil_run brackets every kernel
 * launch with CUDA events on the plan's stream.  stencil_plan_kernel_time then returns the
 * summed device time in milliseconds and the number of launches since the last reset
 * (it synchronises the plan's stream). */
int stencil_plan_set_timing(stencil_plan plan, int enable);
int stencil_plan_kernel_time(stencil_plan plan, double *ms, long long *launches, int reset);

/* Free the plan and its scratch.  NULL is accepted. */
int stencil_plan_destroy(stencil_plan plan);

/* ---- measured parameter choice (Sec. 5.3 and 5.4.2) --------------------------------------
 * The plan's own choice comes from the model alone (Eqs. 3-9 restated for the GB300).  The
 * paper narrows the configurations with its model and then builds and measures the few it
 * rates best; stencil_tune does the same on the caller's data and remembers the winner for the
 * problem key (kind, ndim, nx, ny, nz, storage, exact, rad) in a process-wide cache, which
 * stencil_plan_create consults whenever its desc forces nothing. */
typedef struct {
    int force_T, force_bx, force_by, force_vec;   /* the fastest configuration, as desc forces */
    int partial_rows, resident;                   /* (with these two desc fields) */
    double gcells;        /* its measured rate, 10^9 cell updates/s */
    double model_gcells;  /* the model's rate for it (0 where the family has no calibration) */
    int candidates;       /* compiled configurations for the problem */
    int timed;            /* how many of them were run and timed */
} stencil_tune_result;

/* Rank every compiled configuration for *desc by the model, run the top_k of them
 * (top_k = 0: all) once untimed and once timed (CUDA events on desc->stream) on the caller's
 * grids, and cache the fastest.
 * desc     : as for stencil_plan_create, with every force_* field, partial_rows and resident
 *            0 (else ST_ERR_INVALID_ARG).
 * grid_in, power, coeffs : as for stencil_run (device, device or NULL, host); not modified.
 * grid_out : device scratch of the grid's size, distinct from grid_in; its contents afterwards
 *            are the result of a `steps`-step run of the last configuration timed.
 * steps    : >= 1 Jacobi steps per timed run (a short but representative count).
 * result   : receives the winner.  Synchronous: returns after the last timed run.
 * Errors: ST_ERR_INVALID_ARG, ST_ERR_UNSUPPORTED (no configuration for the problem),
 * ST_ERR_OOM, ST_ERR_CUDA, ST_ERR_TIMEOUT, and stencil_run's own checks. */
int stencil_tune(const stencil_desc *desc, const void *grid_in, void *grid_out, const void *power,
                 const float *coeffs, int steps, int top_k, stencil_tune_result *result);

/* 1 when the plan took its configuration from the tuning cache, 0 otherwise (or for NULL). */
int stencil_plan_tuned(stencil_plan plan);

/* The cache: clear it; count its entries; write it to a text file (one entry per line:
 * kind ndim nx ny nz storage exact rad T bx by vec gcells); merge a file written that way into
 * it (a malformed line rejects the whole file with ST_ERR_INVALID_ARG and changes nothing).
 * An entry whose configuration has no compiled kernel is ignored by stencil_plan_create.
 * Host-only calls; safe to call from several threads. */
int stencil_tune_cache_clear(void);
int stencil_tune_cache_size(void);
int stencil_tune_cache_save(const char *path);
int stencil_tune_cache_load(const char *path);

/* ---- many grids in one graph launch ----------------------------------------------------- */

typedef struct stencil_batch_s *stencil_batch;

/* One 2D grid of a batch (contracted arithmetic). */
typedef struct {
    int kind;              /* ST_DIFFUSION or ST_THERMAL */
    int nx, ny;            /* >= 1 */
    int steps;             /* >= 0 */
    const void *grid_in;   /* device, nx*ny floats */
    void *grid_out;        /* device, nx*ny floats; may equal grid_in, no other overlap */
    const void *power;     /* device power map (ST_THERMAL) or NULL */
    float coeffs[5];       /* Table 2 coefficients (layouts above) */
} stencil_batch_grid;

/* Prepare `count` grids for repeated batched runs.  Every grid advances by its own step count
 * in ceil(steps/T) temporally-blocked passes (Eq. 8; the last pass fuses the remainder,
 * Sec. 3.2) with its own ping-pong scratch (Sec. 2.1); one (T, cells per thread) for the whole
 * batch comes from the GPU restatement of the paper's model (Eqs. 3-9), the compiled choice with
 * the least predicted total time.  The passes of all grids are cut into items of one tile column
 * (Sec. 3.1's overlapped tile) by 192 rows and queued pass by pass; ONE persistent kernel launch,
 * one warp per block and as many blocks as the device holds at once, pops the items in order,
 * and an item waits for the neighbouring tiles of its grid's previous pass (the halo it reads and
 * the cells of the ping-pong buffer it overwrites) before it starts.  Each such wait is bounded
 * (1 s by default, stencil_batch_set_wait): when one gives up, every block of the launch leaves
 * and stencil_batch_sync reports ST_ERR_TIMEOUT.  The launch, a reset of the queue's counters
 * before it and a copy of its status word after it are captured into one CUDA graph on `stream`
 * (NULL: an owned stream that synchronises with the legacy default stream).  Buffers and
 * coefficients are fixed at creation; the power maps' contents are read at every replay.
 * Errors: ST_ERR_INVALID_ARG, ST_ERR_UNSUPPORTED, ST_ERR_OOM, ST_ERR_CUDA. */
int stencil_batch_create(stencil_batch *out, const stencil_batch_grid *grids, int count,
                         void *stream);

/* stencil_batch_create with the queue's parameters chosen by the caller (0 = the library's
 * choice): rows_per_item, the rows of one tile column an item covers (>= T); force_T and
 * force_vec, the fused steps per pass and cells per thread of the launch's kernel (ST_ERR_
 * UNSUPPORTED when no compiled kernel matches). */
int stencil_batch_create_ex(stencil_batch *out, const stencil_batch_grid *grids, int count,
                            void *stream, int rows_per_item, int force_T, int force_vec);

/* Replay the batch's graph (asynchronous): every grid advances by its step count into its
 * grid_out. */
int stencil_batch_run(stencil_batch b);

/* Wait for the batch's stream.  Returns ST_ERR_TIMEOUT when a bounded wait of the last replay
 * gave up (its grids' results are then invalid; the batch and the CUDA context stay usable and
 * the next replay starts afresh), ST_ERR_CUDA on a CUDA error, else ST_OK. */
int stencil_batch_sync(stencil_batch b);

/* Set how long (wait_ns > 0 nanoseconds) an item of later replays may wait for the tiles it
 * depends on before the launch gives up.  hold_pass >= 0 is a test hook that makes the items of
 * that pass never report themselves finished, so the items of the next pass wait until the
 * limit runs out (a dependency that is never satisfied, without any fault); -1 turns it off.
 * Synchronises the batch's stream.  Errors: ST_ERR_INVALID_ARG, ST_ERR_CUDA. */
int stencil_batch_set_wait(stencil_batch b, long long wait_ns, int hold_pass);

/* Grid g's chosen fused steps T, cells per thread and pass count. */
int stencil_batch_get_grid(stencil_batch b, int g, int *T, int *vec, int *passes);

/* Kernel launches in the batch's graph: 1 (0 when no grid has work), or ST_ERR_INVALID_ARG. */
int stencil_batch_launch_count(stencil_batch b);

/* Wait for the batch's stream, free its graph and scratch.  NULL is accepted. */
int stencil_batch_destroy(stencil_batch b);

/* ---- adjoint (reverse-mode gradient) of a 2D run -------------------------------------------
 *
 * One step is affine in the field, u_{t+1} = A u_t + b(coeffs, power) (Sec. 2.1, Table 2,
 * clamped boundary), so for a scalar loss L with upstream gradient w = dL/du_steps:
 *   lambda_steps = w,  lambda_t = A^T lambda_{t+1},  dL/du_0 = lambda_0,
 *   dL/dcoeff_m = sum_{t<steps} sum_i lambda_{t+1}[i] dF_i/dcoeff_m (u_t),
 *   dL/dpower_i = k_dt * sum_{t=1..steps} lambda_t[i]           (Hotspot 2D only).
 * The transposed sweep is temporally blocked like the forward one (Sec. 3.2); forward states
 * are recomputed from checkpoints kept every `ckpt` steps. */
typedef struct stencil_adjoint_s *stencil_adjoint;

/* Prepare the gradient of a `steps`-step 2D run (kind ST_DIFFUSION or ST_THERMAL, nx x ny
 * cells).  Allocates ceil(steps/ckpt) checkpoint grids, ckpt state grids, two adjoint grids
 * and two forward plans on `stream` (cudaStream_t; NULL = legacy default stream).
 * Errors: ST_ERR_INVALID_ARG (kind, sizes, steps < 0, ckpt < 1), ST_ERR_OOM, ST_ERR_CUDA. */
int stencil_adjoint_create(stencil_adjoint *out, int kind, int nx, int ny, int steps, int ckpt,
                           void *stream);

/* Forward run u_out = u_steps (device pointers, nx*ny floats; u_out may equal u0), keeping
 * the checkpoints and a copy of the 5 host coefficients for stencil_adjoint_backward.
 * power: device power map for ST_THERMAL (NULL for ST_DIFFUSION); it must be passed unchanged
 * to the backward call.  Asynchronous on the object's stream. */
int stencil_adjoint_forward(stencil_adjoint a, const float *u0, const float *power,
                            const float *coeffs, float *u_out);

/* Gradients of the last forward run (device pointers, all on the object's stream):
 *   grad_out        : dL/du_steps, nx*ny floats (read only)
 *   grad_u0         : dL/du_0, nx*ny floats (may not overlap grad_out)
 *   grad_coeffs     : 5 floats, dL/dcoeffs in the coefficient layout of the kind
 *   grad_coeffs_abs : 5 floats or NULL: sum over (t, i) of |lambda_{t+1}[i] dF_i/dcoeff_m|,
 *                     the scale the rounding error of grad_coeffs[m] is relative to; with NULL
 *                     the sweep does not accumulate it (fewer operations per cell, the other
 *                     results bit-identical)
 *   grad_power      : dL/dpower, nx*ny floats (ST_THERMAL; NULL for ST_DIFFUSION)
 * Coefficient gradients are float32 sums in a fixed order (per thread at most 64 terms, then
 * error-free pairwise combination): deterministic for a given size.  Errors: ST_ERR_INVALID_ARG (no forward run yet, missing or
 * unexpected pointers), ST_ERR_CUDA. */
int stencil_adjoint_backward(stencil_adjoint a, const float *grad_out, const float *power,
                             float *grad_u0, float *grad_coeffs, float *grad_coeffs_abs,
                             float *grad_power);

/* Wait for the object's stream; returns ST_ERR_TIMEOUT if a kernel's bounded wait for staged
 * data gave up since the last call (the gradients of that backward run are invalid), ST_ERR_CUDA
 * on an asynchronous CUDA error, else ST_OK. */
int stencil_adjoint_sync(stencil_adjoint a);

/* Wait for the object's stream and free everything it owns.  NULL is accepted. */
int stencil_adjoint_destroy(stencil_adjoint a);

/* ---- float64 verification reductions ----------------------------------------------------- */

/* Bytes of device workspace stencil_reduce needs (caller-allocated, 8-byte aligned). */
size_t stencil_reduce_workspace_bytes(void);

/* Float64 statistics of a grid a (and of b and a - b when b is not NULL), for verification:
 * global sum / energy (sum of squares) to check conservation, and the L2 / L-infinity norms of
 * a difference against a reference.  Writes 8 doubles to the DEVICE pointer out, in order:
 *   sum(a), sum(a^2), max|a|, sum(b), sum(b^2), max|b|, sum((a-b)^2), max|a-b|
 * (entries 3..7 are 0 when b is NULL).  a_type / b_type: ST_F32 or ST_F64; n: elements (>= 1);
 * workspace: stencil_reduce_workspace_bytes() of device memory.  Deterministic: the summation
 * order depends on n only.  Asynchronous on `stream`.  Errors: ST_ERR_INVALID_ARG, ST_ERR_CUDA. */
int stencil_reduce(const void *a, int a_type, const void *b, int b_type, long long n,
                   double *out, void *workspace, void *stream);

/* ---- performance models (host only, no device work) ------------------------------------ */

/* Inputs of the paper's FPGA performance model (Sec. 4, Table 1 parameters). */
typedef struct {
    int ndim;                      /* 2 or 3 */
    long long dim_x, dim_y, dim_z; /* input size per dimension (dim_z ignored for 2D) */
    int bsize_x, bsize_y;          /* spatial block size (bsize_y: 3D only) */
    int rad, par_vec, par_time;    /* stencil radius, vector width, parallel time steps */
    int size_cell;                 /* bytes per cell */
    int num_read, num_write;       /* external memory accesses per cell update */
    long long iter;                /* iterations */
    double fmax_hz;                /* kernel operating frequency */
    double th_max_gbs;             /* maximum memory throughput, GB/s (10^9 B/s) */
} stencil_fpga_model_in;

typedef struct {
    double th_mem_gbs;             /* Eq. 3 */
    long long csize_x, csize_y;    /* Eq. 4 (csize_y: 3D) */
    long long bnum_x, bnum_y;      /* Eq. 5 */
    double t_cell;                 /* Eq. 6 */
    double t_read, t_write;        /* Eq. 7 and the write count (input size x num_write) */
    double run_time_s;             /* Eq. 8 */
    double throughput_gbs;         /* Eq. 9 */
} stencil_fpga_model_out;

/* The paper's performance model, Eqs. 3-9 (Sec. 4).  For 3D, where the paper gives Eq. 7 for
 * 2D only, the out-of-bound traversal is subtracted along x and along y.  Returns ST_OK or
 * ST_ERR_INVALID_ARG (missing pointer, non-positive sizes, a block no wider than its halos). */
int stencil_model_fpga(const stencil_fpga_model_in *in, stencil_fpga_model_out *out);

/* Inputs of the GPU restatement of the model (one fused pass = one launch). */
typedef struct {
    int ndim;                      /* 2 or 3 */
    long long nx, ny, nz;          /* grid */
    int steps;                     /* time steps of the run */
    int T;                         /* fused steps per pass (par_time) */
    int bx, by;                    /* tile incl. halos (by: 3D) */
    int halo_x, halo_y;            /* halo per side */
    int sms;                       /* streaming multiprocessors */
    double sm_hz;                  /* SM clock */
    double hbm_gbs;                /* device memory bandwidth, GB/s */
    double bytes_per_cell;         /* algorithmic bytes per cell per pass (8 or 12 for float32) */
    double ops_per_cell;           /* issued thread instructions per computed cell update */
    double issue_eff, hbm_eff;     /* calibration factors (fraction of peak reached) */
    double stream_overhead;        /* extra computed rows/planes of the streamed axis, fraction */
    double launch_s;               /* fixed cost per pass */
} stencil_gpu_model_in;

typedef struct {
    double passes;                 /* ceil(steps / T) */
    double bytes_per_pass;         /* algorithmic HBM bytes */
    double cells_computed_per_pass;/* halos included, times T */
    double t_hbm_s, t_alu_s;       /* HBM time and issue time of one pass */
    double t_pass_s;               /* max of the two, plus the launch cost */
    double run_time_s;             /* passes x t_pass_s */
    double gcells;                 /* nx*ny*nz*steps / run_time, in 10^9 cell updates/s */
} stencil_gpu_model_out;

/* GPU restatement of Eqs. 3-9: per pass, time = max(algorithmic bytes / (HBM bandwidth x
 * hbm_eff), computed cells x ops_per_cell / (SMs x 128 lanes x clock x issue_eff)) + launch
 * cost; run time over ceil(steps/T) passes (Eq. 8).  Returns ST_OK or ST_ERR_INVALID_ARG. */
int stencil_model_gpu(const stencil_gpu_model_in *in, stencil_gpu_model_out *out);

/* Allocation-free run of a 2D stencil (Diffusion 2D or Hotspot 2D); the paper has no
 * counterpart: it exists for callers that may not allocate device memory at the call site
 * (inside a memory pool or arena they do not own, on latency-bound paths that cannot absorb
 * cudaMalloc's synchronisation, or under a locked-down allocator).
 * Same arguments and result as stencil_run on a default plan, without a plan:
 *   kind            : ST_DIFFUSION or ST_THERMAL (2D only)
 *   grid_in/out     : device pointers, nx*ny floats, dense rows; grid_out may equal grid_in
 *   power           : device power map for ST_THERMAL, NULL for ST_DIFFUSION
 *   coeffs          : host array of 5 coefficients (layouts above)
 *   steps           : >= 0
 *   exact           : 1 = Table 2 order without fused multiply-adds, 0 = contracted
 *   T               : fused steps per pass, 0 = 8 (the default plan's)
 *   stream          : cudaStream_t, NULL = legacy default stream
 * Instead of a plan-owned ping-pong grid it uses one buffer the library reserves on every
 * device where it is loaded (16 MiB, held until the process exits): grids of more than
 * 4,194,304 cells return ST_ERR_TOO_LARGE.  It calls no cudaMalloc, cudaFree or allocating
 * routine.  All calls on a device share that buffer: calls whose work overlaps on the GPU
 * (different streams, unordered host threads) race on it.  The first call on each device looks
 * up the buffer's device address (cudaGetSymbolAddress) and caches it with the context it was
 * found in; make that first call before any stream capture.  After cudaDeviceReset (or any
 * re-creation of the device's primary context) the next call looks the address up again, so
 * it too should come before any capture.  Returns ST_OK or an ST_ERR_* code; launches are
 * asynchronous. */
int stencil_run_noalloc(int kind, const void *grid_in, void *grid_out, const void *power,
                        const float *coeffs, int nx, int ny, int steps, int exact, int T,
                        void *stream);

/* Measured FP32 arithmetic peak of the current device, for the arithmetic side of the roofline
 * R(T) = min(P_FP32 / flops per cell, HBM bandwidth x T / bytes per cell) that the paper's model
 * (Sec. 4, Eq. 6: compute-bound cell rate) sets against memory throughput.  Runs a kernel of
 * independent float32 fused multiply-add chains on every SM (a warm-up launch, then the best of
 * three timed launches, CUDA events on `stream`, NULL = legacy default stream) and writes the
 * rate in 10^12 flops/s (a multiply-add counted as 2) to *tflops.  Synchronous; allocates
 * nothing.  Errors: ST_ERR_INVALID_ARG (NULL tflops), ST_ERR_CUDA. */
int stencil_fp32_peak(double *tflops, void *stream);

/* Allocation-failure injection and allocation accounting (test hooks; no paper counterpart).
 * Every device allocation the library makes (plans, batches, adjoints, tuning) and its pinned
 * host allocations go through one allocator.  stencil_debug_fail_alloc(n), n > 0: the n-th such
 * allocation from now on fails as if the device were out of memory, without touching the
 * device; the call that makes it releases what it had allocated and returns ST_ERR_OOM.  The
 * hook then disarms itself; n = 0 disarms it at once.  Process-wide, not synchronised with
 * calls running on other threads.  Errors: ST_ERR_INVALID_ARG (n < 0).
 * stencil_debug_live_allocs(): the allocations the library holds now (a leak shows as a count
 * that does not return to its earlier value once the objects are destroyed). */
int stencil_debug_fail_alloc(int n);
long long stencil_debug_live_allocs(void);

/* Static description of a status code. */
const char *stencil_strerror(int code);

/* ABI version of the loaded library (ST_ABI_VERSION it was built with). */
int stencil_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GB300_STENCIL_H */
