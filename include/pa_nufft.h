/*
 * pa_nufft.h -- C ABI of the GB300 NEDNER-NUFFT library for planar-sensor
 * photoacoustic reconstruction (Schmid, Glatz, Zabihian, Liu, Drexler,
 * Scherzer, "Computational Realization of a Non-Equidistant Grid Sampling in
 * Photoacoustics with a Non-Uniform FFT").
 *
 * What the library computes (Sec. 2, eq:exact discretised as eq:disc_rec,
 * evaluated by the three NUFFT steps of Sec. 3), in physical units with sound
 * speed c.  Sensors m = 0..M-1 sit at (x_m, y_m) on the plane z = 0 with
 * detector areas h_m; data g[m][n] is sampled at t_n = n*dt, n = 0..n_t-1.
 * For the output grid nx x ny x nz with spacings dx, dy, dz
 * (X = nx dx, Y = ny dy, Z = nz dz), frequency indices j in
 * {-floor(N/2) .. ceil(N/2)-1} per axis and k = 2 pi j / X:
 *
 *   G1(j,n)  = sum_m (h_m/(dx dy)) g[m][n] exp(-i (kx x_m + ky y_m))   eq:NUDFT2
 *   w(j,l)   = c sign(l) sqrt(kx^2 + ky^2 + kz^2)     (sign(0) = +1)
 *   F(j,l)   = (dt/dz) W(j,l) sum_n G1(j,n) exp(-i w(j,l) t_n)         eq:NUDFT1
 *   W(j,l)   = 2 c |kz| / |K|,  W(0,0) = 2c            (factor 2 K_y / kappa, eq:exact)
 *   f[p][q][k] = Re( 1/(nx ny nz) sum_{j,l} F(j,l) exp(i(kx x_p + ky y_q + kz z_k)) )
 *
 * with voxel centres x_p = (p - floor(nx/2)) dx, y_q = (q - floor(ny/2)) dy,
 * z_k = k dz.  The sums over m and over n are evaluated approximately by the
 * NED-NUFFT (eq:NED_NUFFT) and the NER-NUFFT (eq:NER_NUFFT) with a
 * Kaiser-Bessel window of `width` taps on a grid oversampled by `sigma`; the
 * rest is exact.  All device arithmetic is FP32 (frequency arguments formed
 * in double-float precision).
 *
 * Conventions shared by every entry point:
 *  - Return value: PA_OK (0) or one of the PA_ERR_* codes below; on error
 *    pa_last_error() returns a message (thread-local, valid until the next
 *    call from the same thread).
 *  - Device buffers ("*_dev") are owned by the caller, live on the device the
 *    plan was created on, are not aliased with each other, and are dense
 *    C-order FP32 arrays.  Calls are asynchronous and ordered on `stream`
 *    (a cudaStream_t; NULL means the legacy default stream).  A call's
 *    kernels may be scheduled while the previous kernel of the stream
 *    drains (programmatic dependent launch), but none touches memory before
 *    that kernel has completed, so work queued before a call, the caller's
 *    own kernels included, is seen by it as with ordinary launches.
 *  - A plan owns its device workspace and tables; it is not safe to run one
 *    plan on two streams at the same time.
 */
#ifndef PA_NUFFT_H
#define PA_NUFFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PA_OK 0
#define PA_ERR_INVALID_ARG 1      /* NULL pointer, non-finite or out-of-range value */
#define PA_ERR_UNSUPPORTED_SIZE 2 /* a transform length is not 2^a 3^b 5^c 7^d or too large */
#define PA_ERR_CUDA 3             /* a CUDA runtime call failed (message has the CUDA error) */
#define PA_ERR_OOM 4              /* device allocation failed */
#define PA_ERR_TIMEOUT 5          /* a bounded device wait gave up (batched persistent path) */
#define PA_ERR_DEVICE 6           /* a kernel recorded an error in the plan's status word */

#define PA_FLAG_DEFAULT 0
/* Keep the general (windowed) spatial step even for sensors on the output
 * lattice; by default such plans take the lattice path (pa_plan_is_lattice). */
#define PA_FLAG_NO_LATTICE 1
/* Run the NER stage (Sec. 3) with the block kernels, which hold CB columns
 * per block, even where the warp-per-column kernels apply (sigma = 2, width
 * 8, n_t and nz powers of two in [256, 1024]).  Both compute the same
 * operator; the flag exists to compare them. */
#define PA_FLAG_BLOCK_NER 2

typedef struct pa_plan pa_plan;
typedef struct pa_batch pa_batch;

/* Output grid: nx x ny x nz voxels with spacings dx, dy, dz in metres. */
typedef struct {
  int32_t nx, ny, nz;
  double dx, dy, dz;
} pa_grid;

/* Output grid of the d = 2 operator: nx x nz pixels (x along the sensor line,
 * z the depth) with spacings dx, dz in metres. */
typedef struct {
  int32_t nx, nz;
  double dx, dz;
} pa_grid2;

/*
 * Create a reconstruction plan (Sec. 3: the set-up of both NUFFTs).
 *   out        receives the plan (set to NULL on failure).
 *   n_sensors  M >= 1.
 *   sensor_xy  host, [M][2] doubles (x_m, y_m) in metres; copied.  Any finite
 *              value is accepted: positions are reduced modulo X and Y, which
 *              is exact because the sums are X- and Y-periodic.
 *   weights    host, [M] detector areas h_m in m^2 (> 0), copied; NULL means
 *              h_m = X*Y/M (Sec. 2 requires sum h_m = X^(d-1)).
 *   n_t        number of time samples (>= 2); dt > 0 sampling step in s;
 *   c          sound speed in m/s (> 0).
 *   grid       output grid (sizes >= 2, spacings > 0).
 *   sigma      oversampling factor c of Sec. 3, integer in [2, 4].
 *   width      window taps 2K of Sec. 3, even, in {6, 8, 12, 16}.
 *   flags      PA_FLAG_DEFAULT or a bitwise or of PA_FLAG_NO_LATTICE and
 *              PA_FLAG_BLOCK_NER.
 *   stream     stream used for the initial uploads (a cudaStream_t or NULL).
 * Supported sizes: nx, ny, nz, n_t and sigma*nx, sigma*ny, sigma*n_t must be
 * products of 2, 3, 5, 7, with sigma*nx, sigma*ny, nz, nx, ny <= 4096,
 * sigma*n_t <= 4096 and sigma*nx, sigma*ny >= 2*width; else
 * PA_ERR_UNSUPPORTED_SIZE.  The plan is created on the current CUDA device.
 */
int pa_plan_create(pa_plan **out, int64_t n_sensors, const double *sensor_xy,
                   const double *weights, int64_t n_t, double dt, double c,
                   const pa_grid *grid, int sigma, int width, int flags,
                   void *stream);

/*
 * Create a plan for the d = 2 operator (Sec. 2 with d - 1 = 1; the paper's
 * 2-D setting of Sec. 6): sensors on the line z = 0 at x_m, images
 *   f[p][k] = Re( 1/(nx nz) sum_{jx,l} F(jx,l) e^{i(kx x_p + kz z_k)} ),
 *   F = (dt/dz) W G-hat,  G1(jx,n) = sum_m (h_m/dx) g[m][n] e^{-i kx x_m},
 * with omega, W and the NER step exactly as in 3-D (ky = 0).
 *   sensor_x   host, [M] doubles in metres; copied; reduced modulo X.
 *   weights    host, [M] detector lengths h_m in m (> 0), or NULL for X/M
 *              (Sec. 2 requires sum h_m = X).
 *   grid       output grid; sigma, width, n_t, dt, c as in pa_plan_create;
 *              flags: PA_FLAG_DEFAULT or PA_FLAG_BLOCK_NER.
 * The plan works with pa_reconstruct (f: device [nx][nz] float),
 * pa_reconstruct_adjoint, pa_reconstruct_cubic, pa_position_grad (grad_xy
 * [M][2]: d/dx_m, and 0 in the second column), pa_status, pa_plan_info,
 * pa_plan_buffer (G1 [nX1][1][n_t], image spectrum [nx][1][nz]), the
 * profiling calls and pa_plan_destroy.  pa_plan_update_positions[_device],
 * pa_plan_autotune, pa_position_grad_noalloc and batches return
 * PA_ERR_INVALID_ARG for it.  Sizes as in pa_plan_create for nx, nz, n_t.
 */
int pa_plan_create_2d(pa_plan **out, int64_t n_sensors, const double *sensor_x,
                      const double *weights, int64_t n_t, double dt, double c,
                      const pa_grid2 *grid, int sigma, int width, int flags,
                      void *stream);

/* *d = 2 for a plan of pa_plan_create_2d, 3 otherwise. */
int pa_plan_dims(const pa_plan *plan, int *d);

/*
 * Image quality measures of the paper's appendix, on device images (FP64
 * accumulation, deterministic block-ordered sums; synchronise `stream`;
 * scratch from the stream-ordered allocator).
 * pa_correlation: *rho = Cov(a, b) / sqrt(Var(a) Var(b)) over the n >= 2
 *   floats at a_dev and b_dev (eq:corrcoeff, population moments).
 * pa_tenenbaum: *value = (1/N) sum over the images of the stack
 *   u[n0][n1][n2] (images over the first two axes, N = n0 n1 n2) of
 *   (g * U)^2 + (g^T * U)^2 at the pixels where the 3x3 Sobel operator g lies
 *   inside the image; n0, n1 >= 3.  A 3-D reconstruction f[nx][ny][nz] is the
 *   stack of its nz depth images; a 2-D image f[nx][nz] is n2 = 1.
 */
/*
 * Gradient of L = <grad_f, A(h) g> with respect to the detector weights h_m
 * of eq:disc_rec (A is linear in h): grad_h[m] = (1/h_m) sum_n g[m][n]
 * (A^T grad_f)[m][n], the caller's sensor order.  Runs the adjoint into
 * scratch from the stream-ordered allocator; asynchronous on `stream`.
 * With weights that depend on the positions (Voronoi areas, say) the chain
 * rule adds sum_k grad_h[k] dh_k/dx_m to pa_position_grad's result.
 * 2-D and 3-D plans.  g_dev [M][n_t], grad_f_dev as pa_reconstruct's
 * output, grad_h_dev [M] float.
 */
int pa_weight_grad(pa_plan *plan, const float *g_dev, const float *grad_f_dev, float *grad_h_dev,
                   void *stream);

/*
 * Detector weights from the sensor positions: the Voronoi cells of the plan's
 * sensors in the periodic domain of eq:disc_rec (the X x Y torus for 3-D
 * plans, the circle X for 2-D plans), whose sizes sum to X Y (X):
 * pa_voronoi_weights writes the cell areas (lengths) to h_dev [M] float in
 * the caller's order.  pa_voronoi_grad adds the chain-rule term
 * sum_k grad_h[k] dh_k/dx_m to grad_xy_dev [M][2] (2-D plans: column 0),
 * so that pa_position_grad followed by pa_weight_grad and pa_voronoi_grad
 * gives dL/dx for weights that follow the positions.  Both use the plan's
 * current positions and binning; asynchronous on `stream`.  A cell with more
 * vertices than the kernel's buffer leaves its entries unwritten and sets a
 * status bit (pa_status).
 */
int pa_voronoi_weights(pa_plan *plan, float *h_dev, void *stream);
/*
 * Replace the plan's detector weights by h_dev [M] float (device, caller's
 * order, finite and > 0; say the output of pa_voronoi_weights): the tables
 * that carry h_m are rescaled on the device.  Synchronises `stream` (the
 * weights are also kept on the host for later position updates).
 */
int pa_plan_set_weights_device(pa_plan *plan, const float *h_dev, void *stream);
int pa_voronoi_grad(pa_plan *plan, const float *grad_h_dev, float *grad_xy_dev, void *stream);

int pa_correlation(const float *a_dev, const float *b_dev, int64_t n, double *rho, void *stream);
int pa_tenenbaum(const float *u_dev, int64_t n0, int64_t n1, int64_t n2, double *value, void *stream);

/*
 * Forward reconstruction f = A g (eq:disc_rec via NEDNER-NUFFT, Sec. 3).
 *   g_dev  device [M][n_t] float, sensor order as given to pa_plan_create.
 *   f_dev  device [nx][ny][nz] float (written entirely).
 */
int pa_reconstruct(pa_plan *plan, const float *g_dev, float *f_dev, void *stream);

/*
 * Adjoint g = A^T f: the exact transpose (real inner products) of the
 * approximate forward operator of this plan -- same windows, grids and
 * tables -- so that <A g, f> = <g, A^T f> up to FP32 rounding.
 *   f_dev  device [nx][ny][nz] float;  g_dev device [M][n_t] float (written).
 */
int pa_reconstruct_adjoint(pa_plan *plan, const float *f_dev, float *g_dev, void *stream);

/*
 * Sensor-position gradient of L = <grad_f, A(x) g> for fixed h_m, through the
 * window derivative of eq:NED_NUFFT:
 *   dL/dx_m = (h_m/(dx dy)) sum_n g[m][n] sum_{p,q} (sigma nx / X) phi'(Ux_m - p)
 *             phi(Uy_m - q) R[p][q][n],  likewise for y,
 * where R is the oversampled-grid cotangent of the transposed chain.
 *   g_dev        device [M][n_t] data the forward was applied to.
 *   grad_f_dev   device [nx][ny][nz] cotangent of the image.
 *   grad_g_dev   device [M][n_t] or NULL: also receives A^T grad_f.
 *   grad_xy_dev  device [M][2] float, receives (dL/dx_m, dL/dy_m).
 */
int pa_position_grad(pa_plan *plan, const float *g_dev, const float *grad_f_dev,
                     float *grad_g_dev, float *grad_xy_dev, void *stream);

/*
 * Position gradient without device allocation.  The paper has no counterpart;
 * this is a library convenience.  Same result as pa_position_grad (same
 * kernels), but the kernels' scratch -- the per-chunk partial sums of the
 * gradient, ceil(n_t/32) * n_sensors float2 values -- lives in a static device
 * array of the library (16 MiB, at most 2^21 partials; larger problems get
 * PA_ERR_UNSUPPORTED_SIZE) instead of the plan's workspace.  It is meant for
 * callers that cannot let a library allocate device memory while they run:
 * applications whose device memory is handed out by their own arena or
 * caching allocator (a cudaMalloc beside it can fail on a full device or
 * fragment the pool the application sized), and loops that take a gradient
 * step after step and must not stall on cudaMalloc/cudaFree, which may
 * synchronise the device and so hold up the work on every other stream.
 *   - The call allocates nothing: no cudaMalloc/cudaFree, no allocating
 *     library routine.  It launches one single-thread kernel that stores the
 *     plan's descriptor (passed as a kernel argument) into a static device
 *     descriptor, then the kernels of pa_position_grad.
 *   - The first call on a device looks up the static array's device address
 *     with that device current (cudaGetSymbolAddress), and again when the
 *     device's context has changed (after cudaDeviceReset, which also
 *     invalidates every plan of that device).  The plan's device must be
 *     current.
 *   - All calls share the one array and descriptor, which keep the last
 *     call's contents; every partial a call reads is rewritten by that call
 *     first, so nothing needs clearing.  Calls that overlap on the GPU
 *     (different streams, or host threads) race and must not be issued.
 * Arguments as in pa_position_grad.
 */
int pa_position_grad_noalloc(pa_plan *plan, const float *g_dev, const float *grad_f_dev,
                             float *grad_g_dev, float *grad_xy_dev, void *stream);

/*
 * Replace the sensor positions (host [M][2] doubles, metres) of an existing
 * plan; the binning and window taps are rebuilt and uploaded on `stream`.
 * Weights stay as they were.
 */
int pa_plan_update_positions(pa_plan *plan, const double *sensor_xy, void *stream);

/*
 * The same with the new positions in device memory (float32 [M][2], metres):
 * the reduction modulo (X, Y) and the split into base cell and fraction (in
 * FP64), the sort of the sensors by cell, the window taps and the spread
 * entry lists are rebuilt on the device, in the order the host builds them.
 * Synchronises `stream` once (to size the entry lists).  Returns
 * PA_ERR_INVALID_ARG for a non-finite position (the plan then holds the
 * finite remainder with the bad positions at 0).  The first call allocates
 * the plan's re-binning scratch (about 32 bytes per sensor plus 4 bytes per
 * oversampled cell); later calls allocate only when the entry lists grow.
 */
int pa_plan_update_positions_device(pa_plan *plan, const float *xy_dev, void *stream);

/*
 * Same-GPU baseline of Sec. 2's polynomial interpolation: identical NED and
 * inverse FFT, but the time transform is a plain n_t-point FFT per column
 * followed by 4-tap cubic Lagrange interpolation at the non-integer
 * frequencies instead of the NER-NUFFT.  Benchmark comparison only.
 */
int pa_reconstruct_cubic(pa_plan *plan, const float *g_dev, float *f_dev, void *stream);

/* Destroy a plan and free its device memory (NULL-safe; synchronises the device). */
int pa_plan_destroy(pa_plan *plan);

/*
 * Batched forward reconstruction of many independent 3-D plans of uneven
 * sizes, replayed as one CUDA graph.
 *   pa_batch_create: plans[n] (not owned; must outlive the batch; same sigma
 *                    and width), n >= 1.
 *   pa_batch_run:    g_dev[i] / f_dev[i] host arrays of n device pointers.
 *                    The first call with a set of buffers runs the launches
 *                    directly and captures the graph; later calls with the
 *                    same buffers replay it (other buffers: a new capture).
 *   pa_batch_set_mode: 0 (default): each instance's own single-plan launches
 *                    (the fastest kernels its sizes have), as 4 concurrent
 *                    branches of the graph, largest instances first;
 *                    1: one launch per stage over all instances (work lists
 *                    of (instance, tile)).  Both compute the same results.
 */
int pa_batch_create(pa_batch **out, int n, pa_plan *const *plans, void *stream);
int pa_batch_run(pa_batch *batch, const float *const *g_dev, float *const *f_dev, void *stream);
int pa_batch_set_mode(pa_batch *batch, int mode);
int pa_batch_destroy(pa_batch *batch);

/*
 * Read and clear the plan's device status word (synchronises `stream`):
 * *device_status = 0 when no kernel recorded an error.
 */
int pa_status(pa_plan *plan, int *device_status, void *stream);

/*
 * Test hook for the bounded waits (off by default; not for production use).
 * With item >= 0, the plan's pipelined interpolation kernel (the last stage
 * of pa_reconstruct_adjoint and pa_position_grad on plans whose n_t is a
 * multiple of 4 and width <= 8) posts the byte count of its work item `item`
 * on that item's mbarrier but issues none of the item's copies, and every
 * wait of that kernel gives up after `polls` polls (polls <= 0: the default
 * limit of 2^20).  The block that owns the item then finds its wait run out,
 * waits (bounded) for the copies it did issue, records PA_STATUS_WAIT_TIMEOUT
 * in the plan's status word and returns; nothing is left in flight and no
 * fault is raised, but the call's output is incomplete.  pa_status reports
 * the bit.  item < 0 switches the hook off again.  Synchronises `stream`
 * (the plan's device descriptor is rewritten on it).  3-D plans only.
 */
#define PA_STATUS_WAIT_TIMEOUT 1
int pa_plan_test_wait_fault(pa_plan *plan, int item, int polls, void *stream);

/*
 * Measure the alternative launch shapes of the plan's three heaviest stages
 * on the device and keep the fastest of each: samples per lane of the spread
 * (4 or 8), columns per block and block size of the NER kernels (2 or 4
 * columns, 128 or 256 threads, as the shared memory and the transform plans
 * allow; only for plans on the block NER kernels, see PA_FLAG_BLOCK_NER)
 * and the tile height of the interpolation (8, 16 or 32 columns).  The
 * forward results do not change (every shape sums in the same order); the
 * adjoint's shared-memory accumulation order follows the NER block shape, so
 * the adjoint and the gradient may change in the last bits.  Allocates a
 * test input of the plan's sizes for the duration of the call and
 * synchronises `stream`.  choice (NULL or int[4]) receives the shapes kept,
 * in that order (samples per lane, columns, threads, tile height).
 */
int pa_plan_autotune(pa_plan *plan, void *stream, int *choice);

/*
 * *is_lattice = 1 when the plan's sensors sit exactly on the output lattice,
 * x_m = (i - floor(nx/2)) dx and y_m = (k - floor(ny/2)) dy (modulo X, Y),
 * one per node (M = nx ny), and PA_FLAG_NO_LATTICE was not given.  Such a
 * plan computes the spatial step as a plain DFT over the lattice (the
 * equispaced case of Sec. 2, which the NER-only reconstruction uses: no
 * window, no oversampling in x and y) in pa_reconstruct and
 * pa_reconstruct_adjoint; pa_position_grad keeps the windowed path, whose
 * window derivative the gradient needs.  Positions set later with
 * pa_plan_update_positions are tested again; pa_plan_update_positions_device
 * switches the lattice path off.
 */
int pa_plan_is_lattice(const pa_plan *plan, int *is_lattice);

/*
 * *warp = 1 when the plan's NER stage (Sec. 3) runs the warp-per-column
 * kernels (one warp transforms, interpolates and back-transforms a whole
 * column; sigma = 2, width 8, n_t and nz powers of two in [256, 1024], and
 * PA_FLAG_BLOCK_NER not given), 0 when it runs the block kernels.
 */
int pa_plan_uses_warp_ner(const pa_plan *plan, int *warp);

/* Plan properties: sizes of the workspace in bytes and of the problem. */
int pa_plan_info(const pa_plan *plan, int64_t *n_sensors, int64_t *n_t,
                 int64_t *workspace_bytes);

/*
 * Copy one of the plan's intermediate buffers, as left by the last call, into
 * a caller buffer (tests and diagnostics).
 * which: 0 = G1, the spatial spectrum after the NED step (Sec. 3 step 1),
 *            complex64 [2*floor(nx/2)+1][floor(ny/2)+1][n_t] holding
 *            jx = -floor(nx/2)..floor(nx/2) and jy = 0..floor(ny/2);
 *        1 = the image spectrum after the NER step and the inverse DFT over
 *            depth, complex64 [nx][floor(ny/2)+1][nz] (jx = ix - floor(nx/2)).
 * dst_dev: device buffer of capacity_bytes; *bytes receives the size.  With
 * dst_dev NULL only *bytes is set.  Asynchronous on `stream`.
 */
int pa_plan_buffer(const pa_plan *plan, int which, void *dst_dev, int64_t capacity_bytes,
                   int64_t *bytes, void *stream);

/*
 * Per-stage timing with CUDA events recorded on the call's stream around
 * every kernel launch (diagnostics, off by default).  pa_profile_read waits
 * for the recorded events, returns per stage the summed device time in ms
 * and the number of launches since the last read, and clears them.
 * Stages: see pa_profile_stage_name (0 .. PA_PROFILE_STAGES-1).
 */
#define PA_PROFILE_STAGES 17
int pa_profile_enable(pa_plan *plan, int enable);
/*
 * Events around the launches of the selected stages only (bit k = stage k;
 * 0 switches profiling off, as pa_profile_enable(plan, 0) does).  Each event
 * pair sits between two kernels of the stream, so a timing run that brackets
 * one stage disturbs the others' back-to-back launches least.
 */
int pa_profile_select(pa_plan *plan, uint32_t stage_mask);
int pa_profile_read(pa_plan *plan, double *ms_total, int64_t *launches);
const char *pa_profile_stage_name(int stage);

/* Message of the last error on this thread ("" if none). */
const char *pa_last_error(void);

/* Library version string. */
const char *pa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PA_NUFFT_H */
