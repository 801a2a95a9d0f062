/*
 * stokes.h -- C ABI of libstokes: the periodized 2-D Stokes layer-potential sum on one GPU.
 *
 * What is computed (Marple, Barnett, Gillman, Veerapaneni, "A fast algorithm for
 * simulating multiphase flows through periodic geometries of arbitrary shape"):
 *
 *   u(x_i) =  sum_{m=-1,0,1} sum_{j in vesicle nodes, not (same curve and m = 0)}
 *                 S(x_i, y_j + m d) w_j f_j                        [stokeslet, Eq. (S);
 *                                                                    near images, Eq. (utotrep)]
 *          +  sum_{m=-1,0,1} sum_{j in wall nodes, not (j = i and m = 0)}
 *                 D(x_i, y_j + m d) w_j tau_j                      [stresslet, Eq. (D);
 *                                                                    near images, Eq. (Dnr)]
 *          +  (wall node i)    -kappa_i/(2 pi) t_i t_i^T w_i tau_i + jump * tau_i
 *                                                                  [Nystrom diagonal, Sec. 2.3;
 *                                                                    jump relation, Eq. (JR)]
 *          +  (vesicle node i) Kress log-split product-quadrature self term of the
 *                              single layer on the target's own curve   [Sec. 3.2]
 *
 * with S_ij = (1/(4 pi mu)) (delta_ij log(1/r) + r_i r_j / r^2),
 *      D_ij = (1/pi) r_i r_j (r . n_y) / r^4,   r = x - y,  d = (period, 0).
 * The Kress term for node i of a closed curve with n (even) equispaced-parameter nodes,
 * speed s_k = w_k n / (2 pi) and unit tangent t = (-n_2, n_1) is
 *   (1/(4 pi mu)) sum_k [ -R_{(i-k) mod n}/2 I + (2 pi/n) ( -L_ik/2 I + M_ik ) ] s_k f_k,
 *   R_j  = -(4 pi/n) sum_{p=1}^{n/2-1} cos(2 pi p j/n)/p - (4 pi/n^2)(-1)^j,
 *   L_ik = log(|x_i - x_k|^2 / (4 sin^2(pi (i-k)/n))), L_ii = log(s_i^2),
 *   M_ik = r r^T / r^2, M_ii = t_i t_i^T.
 *
 * Conventions shared by every call:
 *  - Arrays of 2-vectors are row-major (count, 2) doubles: x0, y0, x1, y1, ...
 *  - Normals are unit vectors pointing out of the fluid domain (upper wall up, lower wall
 *    down, vesicle outward); curvature kappa = -(x'' . n)/|x'|^2 (+1 on the unit circle).
 *  - period = 0 switches the +-d images off (m = 0 only).
 *  - Device pointers must be CUDA device (or managed) memory of the context's device;
 *    `stream` is a cudaStream_t (NULL = legacy default stream).  The caller owns every
 *    buffer it passes; the library copies what it keeps at stokes_geom_set and keeps no
 *    density, target or output pointer after a call returns.
 *  - Calls are asynchronous on `stream` unless stated otherwise.  Errors found on the
 *    device (non-finite density, a pipeline wait that timed out) are recorded in a device
 *    status word and returned by the next stokes_sync call.
 *  - One context per host thread; a context is not thread-safe.
 *  - Every call returns a stokes_status; stokes_last_error gives the message.
 */
#ifndef STOKES_H
#define STOKES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STOKES_API __attribute__((visibility("default")))

typedef enum {
    STOKES_OK = 0,
    STOKES_ERR_ARG = -1,            /* bad argument (NULL, size, layout, kind)          */
    STOKES_ERR_CUDA = -2,           /* CUDA runtime error                               */
    STOKES_ERR_NO_GEOM = -3,        /* no geometry set                                  */
    STOKES_ERR_ODD_N = -4,          /* vesicle curve with odd or too few nodes (Kress)  */
    STOKES_ERR_NONFINITE = -5,      /* non-finite density or geometry value             */
    STOKES_ERR_TIMEOUT = -6,        /* a device pipeline wait exceeded its bound        */
    STOKES_ERR_NOT_CONVERGED = -7,  /* iterative solve hit its iteration cap            */
    STOKES_ERR_OOM = -8             /* device allocation failed                         */
} stokes_status;

typedef enum {
    STOKES_FP64 = 0,        /* pair sum in FP64                                              */
    STOKES_FP32_KAHAN = 1   /* pair sum in FP32 with hi/lo coordinates and Kahan-compensated
                               per-thread accumulation; FP64 cross-tile reduction and FP64
                               self terms                                                    */
} stokes_precision;

typedef enum {
    STOKES_KIND_WALL = 0,     /* double-layer (stresslet) source curve, open and periodic    */
    STOKES_KIND_VESICLE = 1   /* single-layer (stokeslet) source curve, closed                */
} stokes_kind;

typedef struct stokes_ctx stokes_ctx;

/* Create a context on CUDA device `device`.  *out receives the handle. */
STOKES_API int stokes_create(int device, stokes_ctx **out);

/* Destroy a context and free its device memory (synchronizes the device). NULL is a no-op. */
STOKES_API int stokes_destroy(stokes_ctx *ctx);

/* Copy the last error message (NUL-terminated, truncated to len) into buf. */
STOKES_API int stokes_last_error(const stokes_ctx *ctx, char *buf, size_t len);

/*
 * Set the geometry (Sec. 2.3 discretization; one unit cell).  Replaces any previous one.
 *   n_curves      number of curves (>= 1)
 *   curve_offset  HOST int32[n_curves + 1]: node range of curve c is [off[c], off[c+1]),
 *                 off[0] = 0, strictly increasing; N = off[n_curves]
 *   curve_kind    HOST int32[n_curves]: stokes_kind of each curve
 *   nodes         DEVICE double[N][2]    quadrature nodes (trapezoid rule in a smooth
 *                                         parameter; vesicles: n equispaced parameter values)
 *   weights       DEVICE double[N]       trapezoid weights w_j = |x'(t_j)| 2 pi / n
 *   normals       DEVICE double[N][2]    unit normals (see conventions)
 *   curvature     DEVICE double[N]       curvature; read at wall nodes only, may be NULL when
 *                                         there is no wall curve
 *   period        lattice period d >= 0 (0: images off)
 *   mu            viscosity > 0
 * Vesicle curves need an even node count n >= 4 and n <= 1024 (Kress rule), else
 * STOKES_ERR_ODD_N / STOKES_ERR_ARG.  Synchronizes `stream` before returning.
 */
STOKES_API int stokes_geom_set(stokes_ctx *ctx, int n_curves, const int32_t *curve_offset,
                               const int32_t *curve_kind, const double *nodes,
                               const double *weights, const double *normals,
                               const double *curvature, double period, double mu, void *stream);

/*
 * Velocity at every node of the geometry, self terms included (the Nystrom operator).
 *   precision     stokes_precision
 *   slp_density   DEVICE double[N_ves][2]  vesicle force density f, rows in node order of the
 *                                           vesicle curves (may be NULL when N_ves = 0)
 *   dlp_density   DEVICE double[N_wall][2] wall density tau, rows in node order of the wall
 *                                           curves (may be NULL when N_wall = 0)
 *   jump          multiple of tau added at wall nodes: 0 = principal value D_{Gamma,Gamma},
 *                 -0.5 = interior limit of Eq. (JR)
 *   out_velocity  DEVICE double[N][2], written in node order (fully overwritten)
 */
STOKES_API int stokes_sum_eval(stokes_ctx *ctx, int precision, const double *slp_density,
                               const double *dlp_density, double jump, double *out_velocity,
                               void *stream);

/*
 * Velocity at free points: the plain trapezoid rule over every source node and image,
 * no self terms and nothing skipped (off-curve evaluation, e.g. interior flow fields).
 * Targets must not coincide with a source node (the kernels are singular there).
 *   n_targets     >= 0 (0 is a no-op)
 *   targets       DEVICE double[n_targets][2]
 *   out_velocity  DEVICE double[n_targets][2]
 */
STOKES_API int stokes_sum_eval_targets(stokes_ctx *ctx, int precision, const double *slp_density,
                                       const double *dlp_density, int n_targets,
                                       const double *targets, double *out_velocity, void *stream);

/*
 * stokes_sum_eval with HOST buffers: copies the densities to the device, evaluates and
 * copies the velocities back, on the context's own stream; returns when `out_host` holds
 * the result (synchronous), with any device-side status folded in.
 *   slp_density_host  HOST double[N_ves][2], dlp_density_host HOST double[N_wall][2],
 *   out_host          HOST double[N][2].  Pinned host memory gives the fastest copies.
 */
STOKES_API int stokes_sum_eval_host(stokes_ctx *ctx, int precision, const double *slp_density_host,
                                    const double *dlp_density_host, double jump, double *out_host);

/* Synchronize `stream` and return (then clear) the device status word: STOKES_OK,
 * STOKES_ERR_NONFINITE or STOKES_ERR_TIMEOUT. */
STOKES_API int stokes_sync(stokes_ctx *ctx, void *stream);

/*
 * Phase timing with CUDA events recorded on the call's stream.  With profiling on (on != 0)
 * every stokes_sum_eval / stokes_sum_eval_targets records events around its three phases:
 * density pack, pair kernel, finishing pass (FP64 reduction + self terms).
 * stokes_last_timing waits for the last call's events and writes the phase durations in
 * milliseconds to ms[0..2] (pack, pair, finish).  STOKES_ERR_ARG when no timed call exists.
 */
STOKES_API int stokes_set_profiling(stokes_ctx *ctx, int on);
STOKES_API int stokes_last_timing(stokes_ctx *ctx, double *ms);

/*
 * stokes_sum_eval_targets without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc where they evaluate -- code that
 * records a CUDA graph by stream capture, hosts that own all device memory through their own
 * pool, real-time loops that must not block on the allocator.  (stokes_sum_eval_targets may
 * grow the context's scratch buffer, with a device synchronisation, when it sees more
 * targets than before.)
 *   Arguments, layout and results are those of stokes_sum_eval_targets; the context (created
 *   and given a geometry beforehand) supplies the geometry and its preallocated source buffers.
 *   The cross-split partial sums live in a fixed device array inside the library of
 *   262,144 x 16 B = 4 MiB, held by every device that loads the library until the process
 *   exits.  n_targets may be at most 262,144 (STOKES_ERR_ARG beyond, with a message); for
 *   large n_targets fewer source splits are used so that splits x n_targets fits.
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 *   make that first call before any stream capture.
 *   All calls, from every context on a device, share the one array: calls whose kernels can
 *   overlap on the GPU (different streams without ordering between them) race on it and
 *   must be serialised by the caller.  Nothing in the array needs clearing between calls.
 */
STOKES_API int stokes_sum_eval_targets_noalloc(stokes_ctx *ctx, int precision,
                                               const double *slp_density,
                                               const double *dlp_density, int n_targets,
                                               const double *targets, double *out_velocity,
                                               void *stream);

/* Number of nodes N of the current geometry (0 when none). */
STOKES_API int stokes_num_nodes(const stokes_ctx *ctx);

/*
 * Batched evaluation of many independent channel instances in one launch.
 *
 * stokes_batch_set: like stokes_geom_set for n_inst instances at once.  Instance k owns the
 *   curves [inst_curve_offset[k], inst_curve_offset[k+1]) of the flattened curve list
 *   (HOST int32[n_inst + 1], from 0 to n_curves) and has its own period periods[k] (HOST
 *   double[n_inst]; all > 0 or all 0); mu is shared.  Sources of one instance never act on
 *   targets of another.  The library plans (target block x source split) work items per
 *   instance, sized so that every item costs about the same, and sorts them largest first.
 *   Synchronizes `stream`.  With n_inst = 1 this is stokes_geom_set.
 * stokes_batch_eval: velocities at every node of every instance (node order of the flattened
 *   list), computed by one persistent pair-kernel launch whose blocks take items from a work
 *   counter.  use_graph != 0 replays a CUDA graph of the whole evaluation (captured on the
 *   first call per precision and jump; the densities are copied into and the result out of
 *   the graph's own buffers on `stream`); use_graph = 0 launches the same kernels directly.
 *   stokes_sum_eval on a batched context takes the direct route.
 * stokes_batch_set_shape: the tuner's knobs of the batched launch for `precision`:
 *   targets_per_thread (FP32: 1, 2, 4; 0 keeps) and items_per_slot (work items per resident
 *   block the planner aims for, 1..64; 0 keeps).  Rebuilds the item tables and drops graphs.
 * stokes_batch_info: number of items, resident blocks of the persistent launch, and the
 *   current shape.
 * Free-point evaluation and stokes_set_launch are not available on a batched context.
 */
STOKES_API int stokes_batch_set(stokes_ctx *ctx, int n_inst, const int32_t *inst_curve_offset,
                                int n_curves, const int32_t *curve_offset,
                                const int32_t *curve_kind, const double *nodes,
                                const double *weights, const double *normals,
                                const double *curvature, const double *periods, double mu,
                                void *stream);
STOKES_API int stokes_batch_eval(stokes_ctx *ctx, int precision, const double *slp_density,
                                 const double *dlp_density, double jump, double *out_velocity,
                                 int use_graph, void *stream);
STOKES_API int stokes_batch_set_shape(stokes_ctx *ctx, int precision, int targets_per_thread,
                                      int items_per_slot);
STOKES_API int stokes_batch_info(const stokes_ctx *ctx, int precision, int *n_items,
                                 int *blocks, int *targets_per_thread, int *items_per_slot);

/*
 * Kernel-shape knobs of the pair sum for `precision` (used by the tuner):
 *   source_splits       chunks of the source range summed by separate blocks and reduced in
 *                       FP64 in fixed order; 0 = the occupancy/wave model's default
 *   targets_per_thread  FP32 path only: 1, 2 or 4 (0 keeps the current value)
 *   kahan_group         FP32 path only: sources (all images) summed in FP32 before each Kahan
 *                       update, 1, 2 or 4 (0 keeps the current value)
 * Results depend on these only through FP32/FP64 rounding.  May grow the context's scratch
 * buffer (device synchronisation).
 */
STOKES_API int stokes_set_launch(stokes_ctx *ctx, int precision, int source_splits,
                                 int targets_per_thread, int kahan_group);
STOKES_API int stokes_get_launch(const stokes_ctx *ctx, int precision, int *source_splits,
                                 int *targets_per_thread, int *kahan_group);

/* Nominal pair-image evaluations of one stokes_sum_eval: 3 N_t N_s (1 N_t N_s when period
 * is 0), counting skipped and self pairs.  Written to *pairs. */
STOKES_API int stokes_pair_count(const stokes_ctx *ctx, int n_targets, double *pairs);

#ifdef __cplusplus
}
#endif
#endif /* STOKES_H */
