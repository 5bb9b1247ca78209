/*
 * sdfg_jacobi.h -- C ABI of libsdfgjacobi.so: the iterated 5-point Jacobi-2D
 * stencil on one GB300 (sm_103a), single grids, batches of uneven grids, and
 * a continuous-batching server.
 *
 * The operation (paper Sec. 6.1, "Jacobi Stencil": a 5-point stencil applied
 * repeatedly for T iterations on a 2-D domain with constant boundary
 * conditions; Fig. 1: a state loop over a map that ping-pongs between two
 * copies of the array; Appendix A: one state (timestep) completes before the
 * next begins):
 *
 *   for t = 1..T:  B[i][j] = 0.2 * (A[i][j] + ((A[i-1][j] + A[i+1][j])
 *                                              + (A[i][j-1] + A[i][j+1])))
 *                  for 1 <= i <= rows-2, 1 <= j <= cols-2;  then A <- B.
 *
 * The boundary ring (row 0, row rows-1, column 0, column cols-1) keeps its
 * input values for ever (Dirichlet).  The result is the full grid after T
 * steps, boundary included; the ring is copied exactly.
 *
 * Numerics (IEEE round-to-nearest throughout):
 *   - FP64: every update is evaluated in the order shown, with no fused
 *     multiply-add; results equal a plain FP64 loop bit for bit, whatever
 *     the kernel, tiling, fused depth or batch.
 *   - FP32 arithmetic (FP32 and BF16 storage): work units that touch the
 *     boundary ring, the one-step (naive) kernel and the register-resident
 *     kernel keep the order shown.  Units away from the ring reassociate the
 *     sum -- they share horizontal pair sums between neighbouring columns,
 *     carry the unscaled 5-point sums through the k fused steps of a pass and
 *     multiply by 0.2^k once, at the pass's last step -- which saves about a
 *     quarter of the FP32 work and is more accurate against FP64, not less.
 *     FP32 results are therefore bit-identical for the same geometry (fused
 *     depth k and segment height, hence alone or in any batch or server mix),
 *     and agree with other geometries to within the FP32 tolerance (max-abs
 *     1e-4 on fields in [0, 1]) rather than bit for bit.
 *   - BF16 storage: the steps fused into one pass stay in FP32 registers and
 *     values are rounded to BF16 each time a pass writes the grid, so the
 *     result also depends on k.
 *
 * Storage types: FP32 (arithmetic FP32), BF16 (the grid is stored in BF16;
 * arithmetic is FP32, and the steps fused into one pass stay in FP32
 * registers, so values are rounded to BF16 (nearest-even) each time a pass
 * writes the grid -- every k steps, or every step for the naive kernel; the
 * result therefore depends on k), FP64 (arithmetic FP64).
 *
 * Layout: row-major, `ld` elements between the starts of consecutive rows
 * (ld >= cols).  All grid pointers are DEVICE pointers unless a function says
 * otherwise.  `in` and `out` must either be the same pointer (in place) or
 * not overlap.  The fastest path needs 16-byte aligned pointers and
 * ld * sizeof(element) a multiple of 16; other layouts are staged through an
 * aligned internal copy (correct, slower).
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Functions described as asynchronous only enqueue work and return.
 *
 * Ownership: the caller owns every grid and descriptor.  The library owns
 * only its scratch (stream-ordered allocations it frees itself) and the
 * server's internal copies of descriptors.
 *
 * Errors: every function returns an sdfg_status.  Argument errors are found
 * on the host before any work is enqueued.  Errors of the CUDA runtime are
 * returned as SDFG_ERR_CUDA.  A device-side wait that runs out (persistent
 * kernels) records SDFG_ERR_TIMEOUT in a per-device error word, which
 * sdfg_device_error() reads.  sdfg_last_error() returns a thread-local
 * message about the most recent failure on the calling thread.
 */
#ifndef SDFG_JACOBI_H
#define SDFG_JACOBI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { SDFG_F32 = 0, SDFG_BF16 = 1, SDFG_F64 = 2 } sdfg_dtype;

typedef enum {
    SDFG_OK = 0,
    SDFG_PENDING = 1,           /* server request not finished yet           */
    SDFG_PAUSED = 2,            /* server request paused by a snapshot       */
    SDFG_ERR_INVAL = -1,        /* bad argument                              */
    SDFG_ERR_NOMEM = -2,        /* device allocation failed / over budget    */
    SDFG_ERR_CUDA = -3,         /* CUDA runtime or driver error              */
    SDFG_ERR_TIMEOUT = -4,      /* a bounded wait ran out                    */
    SDFG_ERR_BUSY = -5,         /* object in use / shutting down             */
    SDFG_ERR_UNSUPPORTED = -6   /* no GPU of the required architecture       */
} sdfg_status;

/* Kernel families for sdfg_config.kernel. */
typedef enum {
    SDFG_KERNEL_AUTO = 0,       /* autotuned choice                          */
    SDFG_KERNEL_NAIVE = 1,      /* one timestep per launch, one thread/point */
    SDFG_KERNEL_TEMPORAL = 2,   /* k timesteps per launch (one pass)         */
    SDFG_KERNEL_PERSISTENT = 3, /* one launch for all passes, dependency-driven */
    SDFG_KERNEL_RESIDENT = 4,   /* k timesteps per launch, each CTA's 256 x 112
                                   tile held in registers (FP32/BF16 storage;
                                   FP64 runs the temporal kernel instead);
                                   for grids that fit in L2, where a pass is
                                   latency-bound                            */
    SDFG_KERNEL_SKEWED = 5      /* one launch for all passes; each warp streams
                                   a chain of seg_rows rows (0: 640, 512 for
                                   BF16 storage) of one
                                   column strip through the k fused steps,
                                   chains skewed down by k rows per pass so
                                   that no rows are recomputed between them;
                                   chunk-level dependencies (tiling in
                                   (row, time) without halo rows)           */
} sdfg_kernel;

/*
 * Execution configuration (all fields 0 = choose automatically).
 *   k          timesteps fused per pass: 1, 2, 4 or 8 (paper App. B,
 *              StateFusion/MapToForLoop applied to the timestep loop);
 *   seg_rows   output rows per work unit (MapTiling along rows); for
 *              SDFG_KERNEL_SKEWED the chain length;
 *   warps      warps per CTA.
 */
typedef struct {
    int kernel;
    int k;
    int seg_rows;
    int warps;
} sdfg_config;

/*
 * Single grid, FP32, asynchronous.  in/out: device pointers to rows x cols
 * floats, ld = cols.  T >= 0 timesteps (T = 0 copies).  rows, cols >= 0; a
 * grid with fewer than 3 rows or columns has no interior and is copied.
 */
int sdfg_jacobi2d(const float *in, float *out, int rows, int cols, int T, void *stream);

/* Same for any storage type (sdfg_dtype) and pitch ld (elements). */
int sdfg_jacobi2d_ex(const void *in, void *out, int rows, int cols, int ld, int T, int dtype,
                     void *stream);

/* Same with an explicit configuration (cfg may be NULL = automatic). */
int sdfg_jacobi2d_cfg(const void *in, void *out, int rows, int cols, int ld, int T, int dtype,
                      const sdfg_config *cfg, void *stream);

/*
 * Single grid, FP32, asynchronous, allocating no device memory.  Same
 * operation and result as sdfg_jacobi2d.  The paper has no counterpart: this
 * entry point exists for callers that may not call cudaMalloc -- for example
 * a plug-in inside a host application that owns the whole device memory
 * budget, or a latency-critical loop that cannot afford an allocation's
 * implicit synchronisation.  Its ping-pong scratch grid is a fixed 32 MiB
 * device array inside the library (8,388,608 floats), which every GPU that
 * loads the library keeps until the process exits.
 *   - rows * cols must not exceed 8,388,608 (SDFG_ERR_INVAL otherwise);
 *   - in/out must be 16-byte aligned and cols a multiple of 4 (ld = cols);
 *   - the first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *     Under CUDA's lazy module loading (the default) that first look-up also
 *     loads the library's device code, which reserves the array and may
 *     synchronise the device; a caller that cannot allow that at an
 *     arbitrary point makes one call with rows = 0 (or cols = 0) at
 *     initialisation, which does only this set-up;
 *   - every call shares the one array and it keeps the last call's contents:
 *     calls whose work overlaps on the GPU (other streams, other threads)
 *     race on it, so serialise them.  No element needs to start at zero:
 *     every pass writes each element before it is read;
 *   - it always runs one launch per pass (SDFG_KERNEL_TEMPORAL), with the
 *     fused depth and segment height the autotuner cached for the shape, or
 *     the defaults; it never uses the persistent or register-resident
 *     kernels, so large grids run somewhat slower than sdfg_jacobi2d;
 *   - a bounded device wait that runs out is recorded in this entry point's
 *     own error word; sdfg_device_error() reads (and clears) it.
 * Calls no cudaMalloc, cudaFree or other allocating routine.
 */
int sdfg_jacobi2d_noalloc(const float *in, float *out, int rows, int cols, int T, void *stream);

/*
 * End-to-end call on HOST buffers (contiguous, ld = cols): copies h_in to the
 * device, runs T steps, copies the result to h_out, and returns when h_out
 * holds it.  Pinned host memory gives the fastest copies.  Device buffers are
 * cached by the library between calls of the same size.
 */
int sdfg_jacobi2d_host(const void *h_in, void *h_out, int rows, int cols, int T, int dtype,
                       void *stream);

/*
 * n independent end-to-end solves of HOST grids of one shape (h_in[i] ->
 * T steps -> h_out[i]; contiguous, ld = cols), pipelined: solve i uses one
 * of two device slots (input and result buffers, cached by the library)
 * and one of two library streams, so the host<->device copies of one solve
 * overlap the computation of the next.  Each solve copies its own input in
 * and its own result out.  The work starts after what is already queued on
 * `stream`, and the call returns when every h_out[i] holds its result.
 * Results equal those of n calls of sdfg_jacobi2d_host.  h_in[i] and
 * h_out[j] may repeat, but a buffer must not be read by one solve while
 * another solve writes it (an output buffer reused by solves i and i+1, or
 * an output that is also an input).  Pinned host memory gives overlapped
 * copies; pageable memory serialises them.  SDFG_ERR_INVAL as for
 * sdfg_jacobi2d_host, or for n < 0 or null arrays.
 */
int sdfg_jacobi2d_host_many(const void *const *h_in, void *const *h_out, int n, int rows, int cols, int T,
                            int dtype, void *stream);

/*
 * One solve, as used by the batch and the server.  Inputs: in, out, rows,
 * cols, ld, T (the step cap), tol, dtype.  tol = 0 runs exactly T steps.
 * tol > 0 stops at the first step t that is a multiple of the check stride
 * with rel_t <= tol, where rel_t = ||A_t - A_{t-1}||_2 / ||A_1 - A_0||_2 over
 * the interior (paper Sec. 3 "State": a transition condition that depends on
 * data).  Squared differences are formed in the storage precision's
 * arithmetic (FP32 for FP32/BF16) and summed in groups of at most 48 terms
 * (one lane: 4 columns x at most 12 rows) in FP32; every further level of
 * the reduction is FP64 in a fixed order.
 * Outputs: status, steps_done, rel_residual (rel at the final step),
 * r_first2.
 *
 * Resuming (the state of a solve is exactly the grid, the step count and
 * ||A_1 - A_0||^2): a descriptor with t_start > 0 continues a solve whose
 * grid after t_start steps is `in`; T stays the total cap, checks stay on
 * multiples of the check stride counted from step 0, and r_first2 must hold
 * the original solve's ||A_1 - A_0||^2 (returned in r_first2 by every solve
 * with tol > 0).  With the same configuration, a paused-and-resumed solve
 * equals the uninterrupted one bit for bit.
 * priority: the server admits higher priorities first (FIFO within one).
 */
typedef struct {
    const void *in;
    void *out;
    int rows, cols, ld;
    int T;
    double tol;
    int dtype;
    int status;
    int steps_done;
    double rel_residual;
    int t_start;      /* input: steps already done (0 = fresh solve)        */
    int priority;     /* input: server admission priority (higher first)    */
    double r_first2;  /* input when resuming; output of every tol > 0 solve */
} sdfg_desc;

/* Single-grid solve with tolerance; blocks until the outputs are filled. */
int sdfg_jacobi2d_solve(sdfg_desc *desc, int check_stride, const sdfg_config *cfg, void *stream);

/*
 * Batch of n independent grids in ONE persistent launch (paper Sec. 3,
 * Consume scope: workers dequeue units from a shared work list with atomics).
 * Blocks until done and fills every descriptor's outputs.  All descriptors
 * must share one dtype.  check_stride applies to descriptors with tol > 0.
 */
int sdfg_jacobi2d_batch(sdfg_desc *desc, int n, int check_stride, void *stream);

/*
 * Batch plans: build once, replay many times.  The plan captures the
 * launches (and their staging/finalise steps) in a CUDA graph.  cfg->kernel:
 * SDFG_KERNEL_PERSISTENT: every grid on the persistent kernel (fused depth
 * cfg->k, segments of cfg->seg_rows rows); SDFG_KERNEL_SKEWED: fixed-step
 * grids (tol = 0) of at least 2^20 points run as skewed chains of 512 rows
 * at the library's depth (8 for FP32/BF16, 4 for FP64) in one launch, every
 * other grid on the persistent kernel as above in a second launch; NULL: the
 * batch autotuner's cached choice for this class of batch, else the
 * persistent kernel.  Chains pay off for grids whose own work is long
 * (measured on 16 grids of 2048^2, 496 steps: 5064 against 3321 GUpdates/s);
 * on the uneven 512-grid batch the persistent kernel is faster.
 * plan_run is asynchronous; plan_results waits for the last run and fills
 * the outputs of desc[0..n-1] (the same order as at creation).
 */
typedef struct sdfg_batch_plan sdfg_batch_plan;
int sdfg_batch_plan_create(sdfg_batch_plan **plan, const sdfg_desc *desc, int n, int check_stride,
                           const sdfg_config *cfg, void *stream);
int sdfg_batch_plan_run(sdfg_batch_plan *plan, void *stream);
int sdfg_batch_plan_results(sdfg_batch_plan *plan, sdfg_desc *desc, int n);
int sdfg_batch_plan_destroy(sdfg_batch_plan *plan);

/*
 * Continuous-batching server.  Requests (sdfg_desc, tol > 0 or a fixed T)
 * are admitted while the sum of their device footprints stays within
 * hbm_budget_bytes and fewer than max_slots are active; every wave advances
 * all active grids by quantum_steps steps (or to their stop) in one
 * persistent launch; finished grids retire between waves and queued requests
 * take their place.  quantum_steps must be a multiple of check_stride.
 * The caller keeps each request's in/out alive until poll reports it done.
 */
typedef struct sdfg_server sdfg_server;
int sdfg_server_create(sdfg_server **server, size_t hbm_budget_bytes, int max_slots, int quantum_steps,
                       int check_stride, int device);
/* Optional, before the first submit (SDFG_ERR_BUSY while requests are in
 * flight): fused depth k, segment height and warps per CTA of every grid. */
int sdfg_server_set_config(sdfg_server *server, const sdfg_config *cfg);
int sdfg_server_submit(sdfg_server *server, const sdfg_desc *desc, uint64_t *req_id);
/* SDFG_PENDING while running; SDFG_OK or an error once done (result filled);
 * SDFG_PAUSED after a snapshot (out holds the grid after steps_done steps;
 * steps_done and r_first2 are what a resumed submission needs). */
int sdfg_server_poll(sdfg_server *server, uint64_t req_id, sdfg_desc *result);
/* Pause a request at the next wave boundary (a queued request pauses at
 * once, with out = in and steps_done = t_start).  SDFG_ERR_INVAL if unknown
 * or already finished. */
int sdfg_server_snapshot(sdfg_server *server, uint64_t req_id);
/* Waits until every submitted request is done; SDFG_ERR_TIMEOUT on expiry. */
int sdfg_server_drain(sdfg_server *server, int timeout_ms);
int sdfg_server_destroy(sdfg_server *server);

/*
 * The 1-D Laplace program printed in the paper's Fig. 1, on a device
 * float64[2][N] array A (row-major, rows contiguous):
 *   for t in 0..T-1, 1 <= i <= N-2:
 *     A[(t+1)%2][i] = A[t%2][i-1]*1 + A[t%2][i]*(-2) + A[t%2][i+1]*1
 * in that order (FP64, round-to-nearest).  The end cells of each row are never
 * written.  A is updated in place, both rows, exactly as the program leaves
 * it; the result is bit-identical to a plain FP64 loop.  Asynchronous.
 */
int sdfg_laplace1d(double *A, int N, int T, void *stream);

/*
 * The Jacobi method one dimension up (paper Sec. 6.1's stencil benchmark and
 * Fig. 1's ping-pong state loop, in 3-D): a 7-point stencil on a device box of
 * depth x rows x cols elements of type dtype (sdfg_dtype), row pitch ld
 * elements (ld >= cols), plane pitch rows * ld, planes contiguous.  For T
 * timesteps every interior point becomes
 *   (1/7) * (c + (((n + s) + (w + e)) + (u + d)))
 * (n, s: rows i-1, i+1; w, e: columns j-1, j+1; u, d: planes z-1, z+1), in
 * that order, round to nearest, in FP32 (FP32 and BF16 storage; BF16 is
 * rounded when each step is stored) or FP64 (bit-identical to a plain FP64
 * loop).  The one-cell outer shell keeps its input values.  out receives the
 * whole box after T steps; in is read only; in == out is allowed; T = 0, or
 * an extent below 3, copies.  in/out should be 16-byte aligned with ld *
 * sizeof(element) a multiple of 16; otherwise the box is staged through an
 * aligned copy.  Scratch: one box (two when staged), stream-ordered.
 * Asynchronous on `stream`.  SDFG_ERR_INVAL for negative extents or T, ld <
 * cols, an unknown dtype or a null pointer with a non-empty box.
 */
int sdfg_jacobi3d(const void *in, void *out, int depth, int rows, int cols, int ld, int T, int dtype,
                  void *stream);

/*
 * Red-black successive over-relaxation of the same 2-D Laplace problem: the
 * in-place, ordered counterpart of the Jacobi stencil (paper Sec. 6.1's
 * stencil; each half-sweep is one Map of independent points).  One of T
 * iterations updates every interior point with i + j even, then every one
 * with i + j odd, each as
 *   c <- (1 - omega) * c + (omega / 4) * ((n + s) + (w + e))
 * in that order, round to nearest: FP32 arithmetic for FP32 and BF16
 * storage (BF16 is rounded after each half-sweep), FP64 for FP64
 * (bit-identical to a plain FP64 loop).  The coefficients (1 - omega) and
 * omega / 4 are evaluated once in double.  omega = 1 is Gauss-Seidel; the
 * iteration converges for 0 < omega < 2.  Grid: rows x cols, row pitch ld
 * elements, device memory.  out receives the whole grid after T iterations;
 * in is read only; in == out is allowed; T = 0, or an extent below 3,
 * copies.  The boundary ring keeps its input values.  Alignment and scratch
 * as for sdfg_jacobi3d.  Asynchronous on `stream`.  SDFG_ERR_INVAL for
 * negative extents or T, ld < cols, a non-finite omega, an unknown dtype or
 * a null pointer with a non-empty grid.
 */
int sdfg_sor2d(const void *in, void *out, int rows, int cols, int ld, int T, double omega, int dtype,
               void *stream);

/* Autotuner: times candidate configurations for this shape and dtype on the
 * calling stream (min(T, 64) steps each: the streamed and persistent kernels
 * at k = 2, 4, 8 and several segment heights, plus the register-resident
 * kernel at k = 2, 4, 8 for FP32/BF16 grids whose two buffers fit in
 * 96 MiB), caches the best by shape class, and returns it.  Allocates two
 * scratch grids for the trials and frees them. */
int sdfg_autotune(int rows, int cols, int T, int dtype, sdfg_config *best, void *stream);

/* Batch autotuner: times candidate plans on the caller's batch (the grids
 * are overwritten by the trial runs): the persistent kernel at k = 4, 8 and
 * several segment heights, and, when no grid has tol > 0, the chain kernel at
 * k = 4, 8 for the large grids and the persistent kernel at 128- or 256-row
 * segments for the others; caches the best for batches of this
 * class (dtype, grid count, mean area), and returns it.  Plans created
 * afterwards with cfg == NULL for a batch of the same class use it. */
int sdfg_autotune_batch(const sdfg_desc *desc, int n, int check_stride, sdfg_config *best, void *stream);

/* Per-kernel CUDA-event timing inside the library (off by default).  While
 * enabled, every launch is bracketed by events on its own stream. */
int sdfg_stats_enable(int on);
int sdfg_stats_reset(void);
/* Sums over launches of kernel family `name` ("naive", "temporal",
 * "persistent", "reduce", "copy", "stencil3d", "sor", "resident",
 * "skewed"), or over the host copies of sdfg_jacobi2d_host and
 * sdfg_jacobi2d_host_many ("h2d", "d2h"); waits for the recorded events. */
int sdfg_stats_get(const char *name, long long *launches, double *total_ms);

/* Reads (and with clear != 0 resets) the current device's error words: the
 * one shared by the allocating entry points and the one of
 * sdfg_jacobi2d_noalloc.  SDFG_ERR_TIMEOUT if a bounded device wait ran out
 * since the last clear.  Creates no device state and allocates nothing. */
int sdfg_device_error(int clear);

/* Thread-local description of the last failure on this thread. */
const char *sdfg_last_error(void);

/*
 * Test hooks for the failure paths (no GPU fault is involved):
 *   hook 1, value 0/1: persistent launches created afterwards make their first
 *           work item wait on a flag that nothing sets, so the bounded wait
 *           runs out and the launch reports SDFG_ERR_TIMEOUT;
 *   hook 2, value ns: limit of every bounded device wait in persistent
 *           launches created afterwards (0 = default, 2 s);
 *   hook 3, value n: batch plans created afterwards with SDFG_KERNEL_SKEWED
 *           put fixed-step grids of at least n points on chains (-1 =
 *           default, 2^20; 0 = every fixed-step grid);
 *   hook 4, value L: chain length of those batch chains (0 = default, 512).
 */
int sdfg_test_hook(int hook, long long value);

/* Library version (major*10000 + minor*100 + patch). */
int sdfg_version(void);

/*
 * Host-only planning query (no GPU needed): the work decomposition the
 * temporal and persistent kernels use for a grid.  info[0..7] receives
 * {halo_cols, warp_cols, out_cols_per_strip, n_strips, seg_rows, n_segs,
 *  chunk_rows, stages}.
 */
int sdfg_plan_geometry(int rows, int cols, int dtype, int k, int seg_rows, int *info);

#ifdef __cplusplus
}
#endif

#endif /* SDFG_JACOBI_H */
