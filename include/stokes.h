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
    STOKES_ERR_OOM = -8,            /* device allocation failed                         */
    STOKES_ERR_BOUNDS = -9          /* debug build: a device bounds check failed        */
} stokes_status;

typedef enum {
    STOKES_FP64 = 0,        /* pair sum in FP64                                              */
    STOKES_FP32_KAHAN = 1,  /* pair sum in FP32 with hi/lo coordinates and Kahan-compensated
                               per-thread accumulation; FP64 cross-tile reduction and FP64
                               self terms                                                    */
    STOKES_DOUBLE_FLOAT = 2 /* pair sum in double-float arithmetic on the FP32 pipes
                               (unevaluated float pairs, ~48-bit significands): coordinates
                               split exactly into three floats on fixed grids so r = x - y
                               is exact, error-free sums and FMA products, a table-driven
                               double-float logarithm; accuracy of the FP64 path (relative
                               error <= 1e-12) at a multiple of its speed on GPUs whose FP64
                               rate is a small fraction of their FP32 rate; every source tile
                               is summed in double-float and the tile sums in FP64; FP64 self
                               terms and cross-split reduction as above                      */
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
 * Replace the node data of the current geometry (same curves, same node counts): nodes,
 * weights, normals (DEVICE, as in stokes_geom_set) and curvature (DEVICE, may be NULL when
 * there is no wall).  Asynchronous on `stream`; no allocation, no re-planning.  Used by the
 * time stepper after every position update.  A non-finite value is reported by the next
 * stokes_sync.
 */
STOKES_API int stokes_geom_update(stokes_ctx *ctx, const double *nodes, const double *weights,
                                  const double *normals, const double *curvature, void *stream);

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
 * Pressure and traction at free points (FP64): the plain trapezoid rule over every source
 * node and image, as stokes_sum_eval_targets, of
 *   pressure  Q w f (vesicle sources, Eq. (Q)) + P w tau (wall sources, Eq. (P));
 *   traction  K w f (Eq. (K)) + T w tau (Eq. (T)) at targets with unit normals n_x, taking
 *             the dipole functions of Eq. (T) as d_x = (r . n_x)/r^2 (target) and
 *             d_y = (r . n_y)/r^2 (source), the reading under which T is the traction
 *             -p n_x + mu (grad u + grad u^T) n_x of the (D, P) pair.
 * Targets must lie off the curves (the kernels are singular on them; no on-curve rule).
 *   n_targets       >= 0 (0 is a no-op)
 *   targets         DEVICE double[n_targets][2], 16-byte aligned
 *   target_normals  DEVICE double[n_targets][2], 16-byte aligned (traction only)
 *   out_pressure    DEVICE double[n_targets];  out_traction  DEVICE double[n_targets][2]
 * Single-instance geometries only (STOKES_ERR_ARG on a batched context).  May grow the
 * context's scratch buffer (device synchronisation).  Asynchronous on `stream`.
 */
STOKES_API int stokes_sum_eval_pressure(stokes_ctx *ctx, const double *slp_density,
                                        const double *dlp_density, int n_targets,
                                        const double *targets, double *out_pressure,
                                        void *stream);
STOKES_API int stokes_sum_eval_traction(stokes_ctx *ctx, const double *slp_density,
                                        const double *dlp_density, int n_targets,
                                        const double *targets, const double *target_normals,
                                        double *out_traction, void *stream);

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
 * STOKES_ERR_NONFINITE, STOKES_ERR_TIMEOUT or (debug build) STOKES_ERR_BOUNDS. */
STOKES_API int stokes_sync(stokes_ctx *ctx, void *stream);

/* Failure-handling check: launches one block on `stream` that waits, with the pair kernels'
 * bounded wait, on a barrier nothing arrives at.  After the bound (~0.5 s) it records a
 * timeout in the context's status word and exits; the next stokes_sync returns
 * STOKES_ERR_TIMEOUT (and clears it), and the context stays usable.  For tests. */
STOKES_API int stokes_check_wait_timeout(stokes_ctx *ctx, void *stream);

/* Self-check of the FP64 logarithm the FP64 pair kernel and the Kress self pass use
 * (Eq. (S)'s log r and the log-split weights of Sec. 3.2 both go through it): out[i] =
 * that kernel-side log of x[i] for i < n.  x, out: DEVICE double[n], caller-owned; x must be
 * positive, finite and normal (the pair kernels pass r^2 >= 1e-150).  Asynchronous on
 * `stream`.  STOKES_ERR_ARG for n < 0 or NULL pointers.  For tests. */
STOKES_API int stokes_check_log64(stokes_ctx *ctx, const double *x, int n, double *out,
                                  void *stream);

/* Debug build (libstokes_debug.so, compiled with -DSTOKES_DEBUG; no counterpart in the paper):
 * the pair, pack and finishing kernels check every source-tile, target, density-row and
 * partial-sum index against the buffer it addresses; a failed check records a bit in the
 * context's status word and skips (or redirects to element 0) that access -- nothing traps --
 * and the next stokes_sync returns STOKES_ERR_BOUNDS (-9).  The release build (libstokes.so)
 * compiles the checks away.  stokes_debug_build returns 1 in the debug build, else 0.
 * The partial-sum checks bound every launch by the elements it writes or reads itself.
 * stokes_debug_tighten (debug build only; STOKES_ERR_ARG in the release build or for
 * elements < 0) makes those checks treat the last `elements` of them as out of range while
 * the buffers keep their size, so a test can see a check fire without any access leaving its
 * allocation.  0 restores the real bounds.  For tests. */
STOKES_API int stokes_debug_build(void);
STOKES_API int stokes_debug_tighten(stokes_ctx *ctx, long long elements);

/* ---------------------------------------------------------------------------------------------
 * Fast multipole evaluation at the nodes (FP64).  The same discrete sum as stokes_sum_eval
 * (pair sum over m in {-1, 0, +1} with the own curve skipped at m = 0, Kress self terms, wall
 * curvature diagonal, jump), with the pair sum by the 2-D FMM in complex variables: the
 * stokeslet and stresslet are written through the log potentials sum_j c_j log(z - w_j) of six
 * charge sets (q1, q2, conj(w) q, 2 n.T, nu T, nu T conj(w)) and their first two derivatives,
 * expanded to `order` terms (multipole to local conversions of Greengard and Rokhlin) on a
 * forest quadtree of uniform depth over the nodes and their +-d images; the 3 x 3 neighbour
 * leaves are summed directly.  The truncation error falls like ~0.5^order (about 1e-9
 * relative at order 20).  This is the O(N) evaluation the paper's method relies on.
 *
 * stokes_fmm_create builds the plan (sorted image sources, cells, interaction and near lists)
 * for `ctx`'s current single-instance geometry on the host (synchronous), with the depth
 * chosen so that occupied leaves hold at most `leaf_size` sources on average; order in
 * [4, 40], leaf_size in [4, 4096] (STOKES_ERR_ARG outside; STOKES_ERR_NO_GEOM without a
 * geometry).  The plan stays valid until ctx's geometry is set or updated again
 * (stokes_geom_set, stokes_batch_set, stokes_geom_update): stokes_fmm_eval then returns
 * STOKES_ERR_NO_GEOM.  stokes_fmm_eval takes the arguments of stokes_sum_eval (device
 * densities, out_velocity 2 N doubles, 16-byte aligned) and runs asynchronously on `stream`;
 * it uses ctx's packing and finishing buffers, so one context runs one evaluation at a time.
 * The caller owns the plan and destroys it before the context.
 * ------------------------------------------------------------------------------------------- */
typedef struct stokes_fmm stokes_fmm;

typedef struct {
    int order;             /* expansion order p                                             */
    int levels;            /* depth L of the forest below its roots                          */
    int sources;           /* image sources (nodes x images)                                 */
    int source_cells;      /* cells holding sources, all levels                              */
    int target_cells;      /* cells holding targets, all levels                              */
    double m2l_pairs;      /* multipole-to-local conversions per evaluation                   */
    double near_pairs;     /* directly summed target-source pairs per evaluation              */
    double plan_ms;        /* stokes_fmm_create, wall clock                                   */
    double device_bytes;   /* device memory the plan holds                                    */
} stokes_fmm_info;

STOKES_API int stokes_fmm_create(stokes_ctx *ctx, int order, int leaf_size, stokes_fmm **out);
/* A plan that also evaluates at n_targets free points (DEVICE array, 2 n_targets doubles,
 * (x, y) pairs, read once at creation; 1 <= n_targets <= 2^26): stokes_fmm_eval_targets then
 * gives the velocity there -- the near-image pair sum of stokes_sum_eval_targets, no self
 * terms -- to the plan's accuracy; stokes_fmm_eval still gives the node sum.  The points are
 * part of the plan (its target tree), so a new set needs a new plan.  STOKES_ERR_NONFINITE for
 * a non-finite point; otherwise as stokes_fmm_create. */
STOKES_API int stokes_fmm_create_targets(stokes_ctx *ctx, int order, int leaf_size, int n_targets,
                                         const double *targets, stokes_fmm **out);
/* As stokes_fmm_create_targets, but the plan's target tree holds the free points alone: no
 * cell, conversion or near list is made for the nodes, so an evaluation costs what the free
 * targets need.  Only stokes_fmm_eval_targets evaluates it; stokes_fmm_eval returns
 * STOKES_ERR_ARG. */
STOKES_API int stokes_fmm_create_targets_only(stokes_ctx *ctx, int order, int leaf_size,
                                              int n_targets, const double *targets,
                                              stokes_fmm **out);
STOKES_API int stokes_fmm_eval(stokes_fmm *fmm, const double *slp_density,
                               const double *dlp_density, double jump, double *out_velocity,
                               void *stream);
/* The velocity at the plan's free targets (out_velocity: 2 n_targets doubles, DEVICE, 16-byte
 * aligned), densities as stokes_fmm_eval; the node targets are not evaluated.  Asynchronous on
 * `stream`.  STOKES_ERR_ARG for a plan without free targets. */
STOKES_API int stokes_fmm_eval_targets(stokes_fmm *fmm, const double *slp_density,
                                       const double *dlp_density, double *out_velocity,
                                       void *stream);
/* Order of the following evaluations of this plan: 4 <= order <= the plan's order, or 0 for
 * the plan's order (the default).  The expansions are truncated at that order (the plan's
 * tree, lists and buffers are unchanged), so one plan serves a cheaper, less accurate
 * evaluation beside its full-order one; the error falls by ~0.45 per order.  Takes effect
 * at the next stokes_fmm_eval (evaluations already queued keep their order).
 * STOKES_ERR_ARG outside that range. */
STOKES_API int stokes_fmm_set_eval_order(stokes_fmm *fmm, int order);
/* Arithmetic of the following evaluations: STOKES_FP64 (default) or STOKES_FP32_KAHAN -- the
 * expansions (P2M, M2M, M2L, L2L, L2P) in FP32 complex arithmetic, and each directly summed
 * pair (near field, removal of a vesicle's own far-field pairs) in FP32 from coordinate
 * differences taken in FP64 and rounded once, accumulated in FP64; coordinates, offsets and
 * the final assembly of the velocity stay FP64.  FP32 rounding adds ~1e-6 relative, so it is
 * meant for orders up to ~16, whose truncation error is of that size anyway.  STOKES_ERR_ARG
 * for any other precision. */
STOKES_API int stokes_fmm_set_precision(stokes_fmm *fmm, int precision);
STOKES_API int stokes_fmm_get_info(const stokes_fmm *fmm, stokes_fmm_info *info);
STOKES_API int stokes_fmm_last_error(const stokes_fmm *fmm, char *buf, size_t len);
STOKES_API int stokes_fmm_destroy(stokes_fmm *fmm);

/* ---------------------------------------------------------------------------------------------
 * Close evaluation of the vesicles' single layer at nearby nodes (FP64).  The plain n-point
 * sum over a vesicle loses accuracy like exp(-2 pi delta / h) at a target delta away from a
 * vesicle of node spacing h.  stokes_close_eval ADDS to out_velocity (the node result of
 * stokes_sum_eval, 2 N doubles, 16-byte aligned DEVICE array), for every node x and every
 * vesicle image m closer than factor h to x (own vesicle at m = 0 excluded: the Kress rule
 * carries it), S_K[f](x) - S_1[f](x): S_1 the plain single-layer sum over that vesicle image,
 * S_K the single layer of the trigonometric interpolants of the vesicle's nodes and density by
 * the trapezoid rule on K n resampled points (error ~ exp(-2 pi K delta / h)).  The pairs are
 * found on the host by stokes_close_create (synchronous) for ctx's current single-instance
 * geometry: factor in (0, 50], upsample K >= 1 with K n <= 4096 for the largest vesicle
 * (STOKES_ERR_ARG otherwise).  The plan stays valid until ctx's geometry is set or updated
 * again (stokes_close_eval then returns STOKES_ERR_NO_GEOM).  stokes_close_eval takes the DEVICE
 * vesicle density of stokes_sum_eval and runs asynchronously on `stream`.
 * ------------------------------------------------------------------------------------------- */
typedef struct stokes_close stokes_close;

typedef struct {
    int upsample;     /* K                                                        */
    int pairs;        /* close (node, vesicle image) pairs                        */
    int targets;      /* nodes with at least one close pair                       */
    int vesicles;     /* vesicle curves resampled per evaluation                  */
    double factor;    /* closeness threshold in node spacings                     */
    double plan_ms;   /* stokes_close_create, wall clock                          */
} stokes_close_info;

STOKES_API int stokes_close_create(stokes_ctx *ctx, double factor, int upsample,
                                   stokes_close **out);
STOKES_API int stokes_close_eval(stokes_close *close, const double *slp_density,
                                 double *out_velocity, void *stream);
STOKES_API int stokes_close_get_info(const stokes_close *close, stokes_close_info *info);
STOKES_API int stokes_close_last_error(const stokes_close *close, char *buf, size_t len);
STOKES_API int stokes_close_destroy(stokes_close *close);

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
 * entry point exists for callers that cannot call cudaMalloc where they evaluate -- hosts
 * that own all device memory through a pool of their own and forbid other allocations,
 * plug-ins that run inside such a host on a fixed memory budget, real-time loops that must
 * not block on the allocator.  (stokes_sum_eval_targets may grow the context's scratch
 * buffer, with a device synchronisation, when it sees more targets than before.)
 *   Arguments, layout and results are those of stokes_sum_eval_targets; the context (created
 *   and given a single-instance geometry beforehand; a batched context gives STOKES_ERR_ARG)
 *   supplies the geometry and its preallocated source buffers.
 *   The cross-split partial sums live in a fixed device array inside the library of
 *   262,144 x 16 B = 4 MiB, held by every device that loads the library until the process
 *   exits.  n_targets may be at most 262,144 (STOKES_ERR_ARG beyond, with a message); for
 *   large n_targets fewer source splits are used so that splits x n_targets fits.
 *   The array's device address is looked up (cudaGetSymbolAddress) when a context is created
 *   on the device, so contexts created after a cudaDeviceReset use the new address.  Should
 *   that lookup have failed, the first call on the device looks it up instead; make that
 *   first call before any stream capture.
 *   All calls, from every context on a device, share the one array: calls whose kernels can
 *   overlap on the GPU (different streams without ordering between them) race on it and
 *   must be serialised by the caller.  Nothing in the array needs clearing between calls.
 *   Like every call on a context, it must not run concurrently with another call on the same
 *   context from a second host thread.  With profiling on, the call records the same three
 *   phase events as stokes_sum_eval_targets (stokes_last_timing reports them).
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
 *                       update, 1, 2, 4, 8 or 16 (0 keeps the current value; the batched launch
 *                       uses 8)
 * Results depend on these only through FP32/FP64 rounding.  May grow the context's scratch
 * buffer (device synchronisation).
 */
STOKES_API int stokes_set_launch(stokes_ctx *ctx, int precision, int source_splits,
                                 int targets_per_thread, int kahan_group);
STOKES_API int stokes_get_launch(const stokes_ctx *ctx, int precision, int *source_splits,
                                 int *targets_per_thread, int *kahan_group);

/*
 * Local frame of the FP32-Kahan stokeslet tiles (on by default).  The pair kernel normally
 * forms each difference x - y from (hi, lo) float pairs (three float operations per
 * coordinate).  With the local frame on, a target block whose targets all lie within 1/8
 * of the geometry's extent (max norm) of the block's middle target evaluates its stokeslet
 * (vesicle-source) tiles with coordinates relative to that target: each staged source and
 * each of its images is translated once per block, exactly up to one final rounding, and a
 * difference costs one float subtraction.  The rounding of a local coordinate is at most
 * half an ulp of the block radius, so near pairs keep their accuracy; blocks that are not
 * compact, and all stresslet (wall-source) tiles, keep the (hi, lo) form.  Node evaluations
 * order their targets for compact blocks: per instance, the walls in node order, then the
 * vesicles along a Morton curve of their centroids.  on = 0 turns the local frame off (every
 * tile in the (hi, lo) form).  Results differ only by rounding.
 */
STOKES_API int stokes_set_local_frame(stokes_ctx *ctx, int on);

/*
 * Graph replay of node sums (stokes_sum_eval on a single-instance geometry; no counterpart in
 * the paper, a launch-overhead measure).  The five launches of a sum (density pack, the FP64
 * self pass on a side stream, the pair kernel, the finishing pass) are captured once into a
 * CUDA graph on the context's own stream and relaunched as one graph on the caller's stream
 * while precision, jump and the density and output pointers repeat; a change of any of them,
 * of the geometry, of the launch shape or of the partial buffer captures anew.  Results are
 * bit-identical to the direct launches.  Modes: STOKES_GRAPH_OFF (direct launches),
 * STOKES_GRAPH_SMALL (default: geometries of at most 65,536 nodes, where the launches' host
 * overhead is a visible share of a sum), STOKES_GRAPH_ALWAYS.  Profiling (stokes_set_profiling)
 * uses the direct launches.  STOKES_ERR_ARG for another mode.
 */
typedef enum {
    STOKES_GRAPH_OFF = 0,
    STOKES_GRAPH_SMALL = 1,
    STOKES_GRAPH_ALWAYS = 2
} stokes_graph_mode;
STOKES_API int stokes_set_graph_mode(stokes_ctx *ctx, int mode);
/* Node-sum graphs captured and graph launches made by the context so far (host counters). */
STOKES_API int stokes_graph_stats(const stokes_ctx *ctx, long long *captures, long long *launches);
/* GPU time of a node sum: `reps` calls of stokes_sum_eval's work issued back to back from the
 * library on `stream` between two CUDA events, so the time is the device's, not a caller's
 * per-call overhead; *ms_per_sum = elapsed / reps.  Same arguments and results as
 * stokes_sum_eval (out holds the last call's velocities); synchronizes `stream` and returns the
 * device status like stokes_sync.  STOKES_ERR_ARG for reps < 1 or NULL ms_per_sum. */
STOKES_API int stokes_time_sums(stokes_ctx *ctx, int precision, const double *slp_density,
                                const double *dlp_density, double jump, double *out_velocity,
                                int reps, void *stream, double *ms_per_sum);

/* Nominal pair-image evaluations of one stokes_sum_eval: 3 N_t N_s (1 N_t N_s when period
 * is 0), counting skipped and self pairs.  Written to *pairs. */
STOKES_API int stokes_pair_count(const stokes_ctx *ctx, int n_targets, double *pairs);

/*
 * Launch-shape autotuner.  The paper evaluates these sums with a CPU FMM and has no
 * counterpart; the direct GPU sum has the shape knobs above, whose best values depend on the
 * problem size and the device, so the library times them.
 *
 * stokes_autotune: for the context's current geometry and `precision`, times each candidate
 *   shape `repeats` times (1..50; 0 = 5) after one untimed call, with CUDA events on `stream`,
 *   and applies the one with the smallest median time.  Candidates -- single instance:
 *   targets_per_thread {1, 2, 4} x kahan_group {2, 4, 8, 16} (FP32-Kahan; one shape otherwise) x
 *   the three source-split counts the wave model ranks cheapest for that shape and two and four
 *   times its cheapest, plus the shape the context had on entry; batched: targets_per_thread {1, 2, 4} (FP32-Kahan) x
 *   items_per_slot {1, 2, 4, 8, 16}.  The timed calls evaluate unit densities held in device
 *   buffers the tuner allocates and frees.  The choice is also recorded in a process-wide table
 *   under the geometry's size class (below); every later stokes_geom_set / stokes_batch_set
 *   whose geometry falls in a recorded class starts from the recorded shape instead of the
 *   wave model's default.  Results depend on the shape only through rounding.  Synchronizes
 *   `stream`; not for use while a stream is being captured.  Writes the outcome to *out (may
 *   be NULL).  FP64 and double-float batched launches share one items_per_slot value.
 * Size class: (SM count of the device, precision, instance count, and for each of the node
 *   counts N, wall nodes and vesicle nodes, ceil(2 log2 count)), i.e. half-octave buckets.
 * stokes_tune_lookup: 1 and *out filled when the table holds the class of the given counts,
 *   0 when it does not, STOKES_ERR_ARG for bad arguments.  Host only.
 * stokes_tune_save / stokes_tune_load: write the table to / merge it from a text file, one
 *   class per line (STOKES_ERR_ARG on an I/O or format error; a failed load changes nothing).
 * stokes_tune_clear: empty the table.
 * The table is guarded by a mutex; the calls on a context are not thread-safe (as elsewhere).
 */
typedef struct {
    int precision;
    int source_splits;       /* single instance (0 for batched)                        */
    int targets_per_thread;  /* FP32-Kahan: 1, 2 or 4; the fixed value otherwise        */
    int kahan_group;         /* FP32-Kahan single instance: 1, 2, 4, 8 or 16; else 0    */
    int items_per_slot;      /* batched: 1..16; else 0                                  */
    int candidates;          /* shapes timed (0 for a table lookup)                     */
    double best_ms;          /* median time of one evaluation with the chosen shape     */
    double initial_ms;       /* the same for the shape in use on entry (0 for a lookup) */
} stokes_tune_result;

STOKES_API int stokes_autotune(stokes_ctx *ctx, int precision, int repeats,
                               stokes_tune_result *out, void *stream);
STOKES_API int stokes_tune_lookup(int num_sms, int precision, int n_inst, int n_nodes,
                                  int n_wall_nodes, int n_ves_nodes, stokes_tune_result *out);
STOKES_API int stokes_tune_save(const char *path);
STOKES_API int stokes_tune_load(const char *path);
STOKES_API int stokes_tune_clear(void);

/* ===========================================================================================
 * Channel response and semi-implicit vesicle time stepping (built on the sums above).
 *
 * A stokes_sim holds one periodic channel (walls U, D) and V vesicles of n nodes each.
 *
 * Channel response (Sec. 2.2-2.3 and the three-step procedure of Sec. 3.1): the response
 * u_resp = D^near tau + sum_m c_m S(., y_m) (Eq. (urep)) to vesicle forces f and the pressure
 * drop p_drive per period (flow towards +x for p_drive > 0; g_T = p_drive (1, 0)).  The blocks
 * of the extended linear system [A B; C Q] (Eq. (BIEU), (BIED), (BIEgu), (BIEgT)) are
 * assembled in FP64 at stokes_sim_set_walls (A only for the dense wall solvers); A is
 * factored by the wall solver below, S = Q - C A^-1 B is pseudo-inverted (SVD, singular values
 * below 1e-13 sigma_max dropped), and a solve is the block elimination
 * c = S^+ (g - C A^-1 v), tau = A^-1 v - A^-1 B c (Sec. 4.1).  Side points: K Gauss-Legendre
 * nodes across the inlet x = 0 and their copies at x = d; proxies: M >= 2K points on a circle
 * of radius R_p about (d/2, 0).
 *
 * Wall solver (stokes_sim_set_wall_solver, read at the next stokes_sim_set_walls):
 *   STOKES_WALLS_LU32_REFINE: A is kept in FP64; an FP32 copy is LU-factored
 *     (partial pivoting) and inverted once (A32^-1); every solve A x = b starts from x = 0,
 *     r = b and repeats x += A32^-1 r (FP32), r = b - A x (FP64) until ||r|| <= 1e-14 ||b||,
 *     the residual stops shrinking, or 12 sweeps.  A = -I/2 + D is of the second kind and well
 *     conditioned, so each sweep gains ~5 digits and the result is the FP64 solution.
 *     Storage 12 (4 N_w)^2 bytes (16 during set-up); the FP32 factorization is far faster
 *     than the FP64 one on this hardware, and a sweep streams the two matrices once.
 *   STOKES_WALLS_LU64: FP64 LU (8 (4 N_w)^2 bytes), one triangular solve per solve.
 *   STOKES_WALLS_FDS (default): the fast direct solver of Sec. 4.  A = A_0 + A_{-1} + A_{+1}
 *     (Eq. (formA)); A_0 (the cell's own walls) in HBS form by recursive skeletonisation
 *     (interpolative decompositions against proxy circles, per-box inverses by
 *     Eqs. (def_muhD)-(def_muG)); A_{-1}, A_{+1} = L R from dyadic sections toward each
 *     neighbour (Sec. 4.2: proxy circles, the neighbour's near nodes for the touching
 *     section), recompressed by column skeletons (stokes_sim_set_fds_recompress); A^-1 by
 *     Sherman-Morrison-Woodbury (Eq. (woodbury1)).  O(N_w) storage and set-up; a solve is
 *     two tree passes and three small products.  Accurate to about
 *     1e-10 relative (the decompositions' tolerance, stokes_sim_set_fds_params); the block
 *     refinement below takes the channel response to round-off.  The compression runs on
 *     host threads (FP64), everything else on the device.
 * stokes_sim_wall_stats: refinement sweeps and relative residual ||b - A x|| / ||b|| of the
 *   last wall solve (0 and 0 for STOKES_WALLS_LU64; 0 and -1, not computed, for
 *   STOKES_WALLS_FDS).
 * Block refinement (stokes_sim_set_block_refinement, 0..8, default 3): the block solve is
 *   followed by that many residual corrections on the whole extended system,
 *   r = [v; g] - [A B; C Q][tau; c], [tau; c] += block solve of r, with A tau evaluated as the
 *   walls' double-layer sum.  The truncated S^+ alone leaves ~1e-6 of the data in the
 *   side-point rows (Poiseuille errors ~1e-6).  With corrections the wall solves inside the
 *   block solves are the fast direct solver's (~1e-10) or, with STOKES_WALLS_LU32_REFINE,
 *   single FP32-inverse sweeps (~1e-5; the corrections make up for them), and three
 *   corrections bring the result to round-off.  With 0 corrections every
 *   wall solve is refined to FP64 accuracy on its own.  (The solve of W = A^-1 B at
 *   stokes_sim_set_walls is refined to FP64 accuracy by the LU solvers; the fast direct
 *   solver gives it to its own ~1e-10.)
 *
 * Time step (Algorithm 1 steps 2-9): forces f_b = -kappa_B x_ssss, f = f_b + (sigma x_s)_s;
 * u_resp of f; GMRES (FP64, right preconditioned by each vesicle's self interaction) on
 * Eq. (tsteplinsys) with the arc-length correction Eq. (ALC):
 *   [I + dt kappa_B S d_ssss, -S d_s(x_s .); x_s . d_s, 0] [u; sigma] = [S f_b + u_resp; (L0-Lk)/(dt Lk)]
 * where S is the single layer of all vesicles with +-d images and Kress self terms.  With
 * precision STOKES_FP64 every pair sum of the step (right-hand side, channel response, GMRES
 * matvecs) is FP64; with STOKES_DOUBLE_FLOAT they are double-float sums (FP64-accurate, on the
 * FP32 pipes); with STOKES_FP32_KAHAN the right-hand side and channel response are
 * double-float, and GMRES runs on FP32-Kahan sums (to 1e-3, at most 40 iterations a sweep)
 * inside iterative refinement with double-float residuals while each refinement cuts the
 * residual 10x, then double-float GMRES finishes from that iterate.  In every mode the
 * returned relative residual meets tol for an FP64-accurate operator.  Then x += dt u, area correction (App. B) and
 * reparameterization (App. C, Algorithm 2).  d/ds = |x_alpha|^-1 d/d alpha by Fourier
 * differentiation.  The unknown vector, guesses and solutions are laid out per vesicle as
 * [u_x (n), u_y (n), sigma (n)], vesicle after vesicle (3 n V doubles).
 * Host pointers are used for set-up and state transfer; f, u_resp, guesses are DEVICE
 * pointers.  Calls are synchronous.  Errors as in the rest of this header;
 * STOKES_ERR_NOT_CONVERGED when GMRES reaches max_iter above tol.
 * ===========================================================================================
 */
typedef struct stokes_sim stokes_sim;

typedef enum {
    STOKES_WALLS_LU64 = 0,         /* FP64 LU of the wall operator                          */
    STOKES_WALLS_LU32_REFINE = 1,  /* FP32 LU + FP64 iterative refinement                   */
    STOKES_WALLS_FDS = 2           /* HBS + low-rank neighbours + SMW (Sec. 4), the default */
} stokes_wall_solver;

/* The fast direct solver after stokes_sim_set_walls (zeros, but walls_setup_ms, for the LU
 * solvers). */
typedef struct {
    int levels;             /* HBS levels below the root (root: both walls; level 1: each wall) */
    int max_rank;           /* largest skeleton of any HBS box                                 */
    int root_size;          /* order of the dense root block                                   */
    int neighbour_rank;     /* columns of L, both neighbours and both walls                    */
    int sections;           /* neighbour sections, both neighbours and both walls              */
    double host_ms;         /* compression and per-box inverses on host threads                */
    double device_ms;       /* uploads, the neighbour factors, A_0^-1 L (set-up only) and the
                               Woodbury matrix on the device                                  */
    double device_bytes;    /* device memory the solver holds                                  */
    double solve_bytes;     /* matrices a one-right-hand-side solve reads: the HBS tables
                               twice, L's and C's blocks, K^-1 S (recompressed) or R and K^-1 */
    double walls_setup_ms;  /* the whole stokes_sim_set_walls call, any solver                 */
    int neighbour_col_rank; /* rows of C, the column skeletons of the recompressed neighbour
                               factors (0 without the recompression)                          */
} stokes_fds_info;
typedef struct stokes_mlp stokes_mlp;

/* Initial iterate of the step's GMRES. */
typedef enum {
    STOKES_GUESS_ZERO = 0,      /* zero (the paper's plain method)                             */
    STOKES_GUESS_PREVIOUS = 1,  /* the previous step's solution                                */
    STOKES_GUESS_MLP = 2,       /* base guess (stokes_sim_set_warm_base) + the network's
                                   predicted change                                          */
    STOKES_GUESS_USER = 3,      /* the caller's DEVICE vector `guess`                          */
    STOKES_GUESS_EXTRAPOLATE = 4 /* 2 z_prev - z_prev2, linear extrapolation of the last two
                                   solutions (the previous solution while only one exists)    */
} stokes_guess;

/* What the learned warm start's predicted change is added to (stokes_sim_set_warm_base). */
typedef enum {
    STOKES_WARM_BASE_PREVIOUS = 0,    /* z_prev (default): the network predicts z - z_prev     */
    STOKES_WARM_BASE_EXTRAPOLATE = 1  /* 2 z_prev - z_prev2: the network predicts the second
                                         difference z - 2 z_prev + z_prev2; until two solutions
                                         exist the MLP guess is the previous solution and the
                                         targets are first differences                        */
} stokes_warm_base;

typedef struct {
    int iterations;      /* GMRES iterations (matvecs inside the Krylov loop)            */
    double residual;     /* final relative residual |b - A z| / |b|                     */
    double setup_ms;     /* forces, channel response, right-hand side, preconditioner   */
    double gmres_ms;     /* Krylov solve                                                 */
    double total_ms;     /* whole step including the position update                    */
    int refinements;     /* FP32-Kahan refinement sweeps (STOKES_FP32_KAHAN steps), else 0 */
    int accurate_residuals; /* FP64-accurate residuals of those sweeps (double-float or FMM) */
    double fmm_plan_ms;  /* host time of this step's FMM plan (residual FMM on), else 0; it
                            runs on a host thread beside the GPU's work                  */
    int precond_refresh; /* Newton-Schulz products of the preconditioner refresh
                            (stokes_sim_set_precond_refresh); 0: the blocks were factorised */
    double response_plan_ms; /* host time of the slower of the channel response's two FMM
                                plans (residual FMM on, walls present), else 0          */
    double plan_wait_ms; /* host time the step spent waiting for its FMM plan threads after
                            queueing the work that does not need them                  */
} stokes_step_stats;

STOKES_API int stokes_sim_create(int device, stokes_sim **out);
STOKES_API int stokes_sim_destroy(stokes_sim *sim);
STOKES_API int stokes_sim_last_error(const stokes_sim *sim, char *buf, size_t len);
/* Walls: HOST arrays of 2 n_per_wall nodes (lower wall then upper wall, each starting on the
 * inlet x = 0), weights, normals (out of the fluid), curvature; period > 0, mu > 0. */
STOKES_API int stokes_sim_set_walls(stokes_sim *sim, int n_per_wall, const double *nodes,
                                    const double *weights, const double *normals,
                                    const double *curvature, double period, double mu, int K,
                                    int M, double proxy_radius);
/* Vesicles: HOST positions (V n x 2, counter-clockwise, equispaced parameter), n even in
 * [8, 256]; kappa_B, mu and period (0 = no images, else equal to the walls'). */
STOKES_API int stokes_sim_set_vesicles(stokes_sim *sim, int V, int n, const double *x,
                                       double kappa_b, double mu, double period);
/* Wall solver mode (stokes_wall_solver; read at the next set_walls) and the statistics of the
 * last wall solve (see above). */
STOKES_API int stokes_sim_set_wall_solver(stokes_sim *sim, int mode);
STOKES_API int stokes_sim_wall_stats(const stokes_sim *sim, int *refinements, double *residual);
/* X <- A^-1 X with the wall solver of the last set_walls (A = -I/2 + D^near, the wall
 * operator; X a DEVICE array of 4 n_per_wall x nrhs doubles, column-major, unknowns
 * (tau_1, tau_2) interleaved per node, lower wall then upper).  The LU32 solver refines to
 * FP64 accuracy; the fast direct solver gives its own ~1e-10.  Synchronous.
 * STOKES_ERR_NO_GEOM without walls, STOKES_ERR_ARG for a NULL X or nrhs < 1. */
STOKES_API int stokes_sim_wall_solve(stokes_sim *sim, double *X, int nrhs);
/* Fast direct solver parameters (read at the next set_walls): relative tolerance of every
 * interpolative decomposition (1e-15..1e-3, default 1e-12), nodes per HBS leaf box (8..512,
 * default 64), proxy points per HBS box (16..512, default 64).  STOKES_ERR_ARG outside. */
STOKES_API int stokes_sim_set_fds_params(stokes_sim *sim, double tol, int leaf_nodes, int n_proxy);
/* Recompression of the fast direct solver's neighbour factors (read at the next set_walls;
 * on = 1 by default, 0 off).  The remark closing Sec. 4.2 notes that L R does not have optimal
 * rank and may be recompressed by further low-rank factorisations.  On, R = A_m(J, :) is
 * factored once more by skeletonising A_m's columns: each wall cut dyadically toward the end
 * whose sources the shift m d carries next to the cell, each section's columns interpolated
 * from a column skeleton J_c (an interpolative decomposition against the velocity its
 * densities make on a proxy circle, and for the touching section at the cell's nodes inside
 * it), so that A_m ~ L A_m(J, J_c) C with C block diagonal.  The solver then stores
 * K^-1 A_m(J, J_c) (l x l_c) in place of R (l x 4 N_w) and K^-1, and a one-right-hand-side
 * solve reads the HBS tables twice plus O(N_w) more instead of the 8 l 4 N_w bytes of R.
 * Either way the solution is accurate to about the decompositions' tolerance.
 * STOKES_ERR_ARG for on outside {0, 1}. */
STOKES_API int stokes_sim_set_fds_recompress(stokes_sim *sim, int on);
/* Statistics of the last stokes_sim_set_walls (see stokes_fds_info). */
STOKES_API int stokes_sim_fds_info(const stokes_sim *sim, stokes_fds_info *info);
STOKES_API int stokes_sim_set_block_refinement(stokes_sim *sim, int sweeps);
/* Precision of the factorization of the block-diagonal self preconditioner: STOKES_FP32_KAHAN
 * (default: the blocks assembled in FP32, FP32 batched LU and inverse, applied with exact
 * products of the FP32 entries and double-float sums (~1e-14 relative), so it is still one
 * fixed linear operator and GMRES's FP64 tolerance is unaffected) or STOKES_FP64.  Only the
 * iteration counts can differ. */
STOKES_API int stokes_sim_set_precond_precision(stokes_sim *sim, int precision);
/* Refresh of the FP32 preconditioner inverse (on = 1; default 0 = factorise every step): the
 * blocks move little in one step, so the previous step's inverse X is kept when
 * ||I - P X||_F <= 1e-3 on every block, or updated by up to three Newton-Schulz iterations
 * X <- X (2I - P X) (a batched SGEMM each, plus one for the check; the error squaring) while
 * it starts at most 0.5 and is seen to square (the result within ~1e-2 at worst); otherwise the
 * blocks are factorised as usual.  The refreshed inverse is
 * a fixed operator within the step, so GMRES's tolerance is unaffected; iteration counts can
 * differ slightly.  The first step, a new dt, stokes_sim_set_state and a precision change
 * factorise.  Steps then depend on the previous steps' preconditioners, so a resumed run
 * (stokes_sim_set_state) matches an uninterrupted one to the step tolerance, not bit for bit.
 * STOKES_ERR_ARG for on outside {0, 1}. */
STOKES_API int stokes_sim_set_precond_refresh(stokes_sim *sim, int on);
/* FP32 preconditioner (the default STOKES_FP32_KAHAN precision of stokes_sim_set_precond_precision):
 * on = 1 runs its batched GEMMs -- the assembly products and the Newton-Schulz refresh -- through
 * cuBLAS's BF16x9 emulation of FP32 on the tensor cores (each FP32 operand split into three
 * BF16 parts, products accumulated in FP32), wherever cuBLAS can emulate them, without
 * cuBLAS's infinity/NaN handling (the blocks are finite for a finite geometry); the LU
 * factorisation and inversion keep the default math mode.  0 (default): plain SGEMMs.  The
 * preconditioner is a fixed operator inside the FP64-accurate refinement, so the setting moves
 * the iteration count, not what a step converges to.  STOKES_ERR_ARG for another value. */
STOKES_API int stokes_sim_set_precond_tensor(stokes_sim *sim, int on);
/* Relative tolerance of each inner FP32-Kahan GMRES solve of a STOKES_FP32_KAHAN step
 * (1e-8..0.5, default 1e-3); the outer FP64-accurate refinement still ends at `tol`. */
STOKES_API int stokes_sim_set_inner_tolerance(stokes_sim *sim, double tol);
/* STOKES_FP32_KAHAN steps: take the FP64-accurate vesicle sums -- the right-hand side S f_b
 * and every refinement residual -- from the fast multipole method (stokes_fmm_*, FP64
 * expansions of `order`) instead of double-float direct sums, the paper's use of the FMM
 * inside the step (Sec. 3.2).  order 0 turns it off (default); otherwise order in [4, 40] and
 * leaf_size in [4, 4096].  The FMM's relative error (~0.48^order: ~1e-12 at order 36) must stay
 * well below the step's tol, since it bounds how small a residual the refinement can certify.
 * The plan is rebuilt each step (the geometry moves) by a host thread while the GPU computes
 * the forces and the channel response.  The wall double-layer sums of the channel response's
 * block refinement then come from an FMM plan of the walls at the same order, made once after
 * stokes_sim_set_walls.  The channel response's vesicle-to-wall and wall-to-vesicle sums come
 * from two plans built each step on host threads while the block preconditioner is built: one
 * of the vesicles with the wall nodes as its only targets, one of the walls with the vesicle
 * nodes as its only targets (stokes_fmm_create_targets_only). */
STOKES_API int stokes_sim_set_residual_fmm(stokes_sim *sim, int order, int leaf_size);
/* STOKES_FP32_KAHAN steps: run the Krylov sweeps' vesicle sums (the operator of every inner
 * GMRES iteration, the paper's FMM-accelerated matvec) on the step's FMM plan evaluated at
 * `order` (stokes_fmm_set_eval_order) instead of the FP32-Kahan direct sum.  order 0 turns it
 * off (default); otherwise order in [4, 40].  Order 14 matches the FP32-Kahan sum's ~5e-7
 * relative error and order 20 gives ~5e-9; the sweeps only need to resolve the inner
 * tolerance, and every convergence decision still uses the FP64-accurate residuals, so the
 * step's result and tolerance are unchanged.  Up to order 16 the sweep evaluations run in FP32
 * (stokes_fmm_set_precision), above it in FP64.  The plan (leaf size as set by
 * stokes_sim_set_residual_fmm) is made at the larger of the two orders, once per step.
 * STOKES_ERR_ARG outside the range. */
STOKES_API int stokes_sim_set_sweep_fmm(stokes_sim *sim, int order);
/* Close evaluation inside the step (the near-pair rule the paper applies to close vesicles,
 * Sec. 3.2): with factor > 0, every vesicle-vesicle single-layer sum of a step (right-hand
 * side, Krylov and residual matvecs in every precision, FMM sums) adds stokes_close_eval's
 * correction for the (node, vesicle image) pairs closer than factor node spacings, found for
 * the step's positions (stokes_close_create, on the host, once per step); upsample K as there
 * (K n <= 4096).  The block preconditioner and the channel response (vesicle-to-wall sums)
 * are unchanged.  factor 0 turns it off (default); STOKES_ERR_ARG for factor outside {0} and
 * (0, 50] or K outside [1, 64]. */
STOKES_API int stokes_sim_set_close_eval(stokes_sim *sim, double factor, int upsample);
/* u_resp (DEVICE, V n x 2) of forces f (DEVICE, V n x 2) at the vesicle nodes. */
STOKES_API int stokes_sim_channel_response(stokes_sim *sim, const double *f, double p_drive,
                                           double *u_resp);
/* Flow of the channel alone with wall velocity data v_walls (DEVICE, 2 N_w x 2, or NULL = 0),
 * g_u = 0, g_T = p_drive n, at n_targets DEVICE points. */
STOKES_API int stokes_sim_empty_channel(stokes_sim *sim, double p_drive, const double *v_walls,
                                        int n_targets, const double *targets, double *u_out);
/* Pressure of the same flow, p = P^near tau + sum_m c_m . Q(., y_m) (Eq. (P), (Q)), at
 * n_targets DEVICE points (p_out DEVICE double[n_targets]).  The representation fixes the
 * pressure's additive constant; the exact Poiseuille pressure is matched up to a constant. */
STOKES_API int stokes_sim_empty_channel_pressure(stokes_sim *sim, double p_drive,
                                                 const double *v_walls, int n_targets,
                                                 const double *targets, double *p_out);
/* One time step.  guess_mode is a stokes_guess; model is required for STOKES_GUESS_MLP
 * (n >= the warm-start modes, dimensions as below) and guess (DEVICE, 3 n V, layout above) for
 * STOKES_GUESS_USER.  GMRES always runs
 * to tol, so every guess only changes the iteration count, not the answer's tolerance. */
STOKES_API int vesicle_step_warmstart(stokes_sim *sim, double dt, double p_drive, int guess_mode,
                                      stokes_mlp *model, const double *guess, double tol,
                                      int max_iter, int precision, stokes_step_stats *stats);
/* Warm-start features and targets of the last step (DEVICE FP32; either may be NULL).  The
 * network predicts the change of the solution since the previous step (the learned guess is
 * z_prev + predicted change; z_prev = 0 and b_prev = 0 after stokes_sim_set_vesicles or
 * stokes_sim_set_state).  With nm the warm-start modes (stokes_sim_set_warm_modes, default 16):
 * features (V x 4 nm): per vesicle, in its principal-axes frame (centre c, angle theta of the
 *   second moments, length l = sqrt(A0 / pi)), the Fourier modes k = -nm/2..nm/2-1 (re, im)
 *   of the complex shape (x' + i y') / l, then of the change of the step's explicit velocity
 *   (S f_b + u_resp) since the previous step, rotated to the frame, over U = kappa_B/(mu l^2);
 * targets (V x 3 nm): modes k = -nm/2..nm/2-1 of the change of the solved velocity (frame,
 *   / U), then k = 0..nm/2-1 of the change of the tension / (kappa_B / l^2). */
STOKES_API int stokes_sim_last_features(stokes_sim *sim, float *features, float *targets);
/* Fourier modes nm of the warm-start features and targets: even, in [4, 64], at most the
 * nodes per vesicle (STOKES_ERR_ARG otherwise).  Default 16 (features 64, targets 48); the
 * paper-scale warm-start workload uses 32 (features 128, targets 96).  A network made for
 * another nm is refused by STOKES_GUESS_MLP steps. */
STOKES_API int stokes_sim_set_warm_modes(stokes_sim *sim, int modes);
/* History features (on != 0; default off): the features also carry, after the 4 nm above, the
 * previous solution z_prev and its change over the previous step (z_prev - z_prev2), both in
 * this step's frame and in the target representation (3 nm each): 10 nm features in all.  The
 * solution two steps back is reset with z_prev (set_vesicles, set_state) and made equal to it by
 * stokes_sim_set_history, so the first step after either sees a zero previous change. */
STOKES_API int stokes_sim_set_warm_history(stokes_sim *sim, int on);
/* Base of the learned guess and of the targets (a stokes_warm_base; STOKES_ERR_ARG otherwise).
 * Targets and network predictions are relative to this base, so a network must be trained and
 * used with the same base. */
STOKES_API int stokes_sim_set_warm_base(stokes_sim *sim, int base);
STOKES_API int stokes_sim_get_warm_modes(const stokes_sim *sim, int *modes);

/* Warm-start network: n_in -> H -> H -> n_out (4 nm -> H -> H -> 3 nm in the step) with SiLU, BF16 weights, FP32 accumulation, FP32
 * master parameters updated by Adam (flattened W1, b1, W2, b2, W3, b3; W row-major (out, in)),
 * input/output standardisation (mu_in, sd_in, mu_out, sd_out).  Host pointers for parameters
 * and normalisation; DEVICE FP32 pointers for data.  Synchronous. */
STOKES_API int stokes_mlp_create(int device, int n_in, int n_hidden, int n_out, stokes_mlp **out);
STOKES_API int stokes_mlp_destroy(stokes_mlp *mlp);
STOKES_API int stokes_mlp_last_error(const stokes_mlp *mlp, char *buf, size_t len);
STOKES_API int stokes_mlp_num_params(const stokes_mlp *mlp);
/* The layer widths the network was created with (so callers can size the normalisation
 * buffer: 2 (n_in + n_out) floats). */
STOKES_API int stokes_mlp_get_dims(const stokes_mlp *mlp, int *n_in, int *n_hidden, int *n_out);
STOKES_API int stokes_mlp_set_params(stokes_mlp *mlp, const float *theta);
STOKES_API int stokes_mlp_get_params(stokes_mlp *mlp, float *theta);
/* Adam state of the network (HOST float[n_params] first and second moments, step count), for
 * checkpoints; stokes_mlp_set_params resets it to zero. */
STOKES_API int stokes_mlp_get_adam(stokes_mlp *mlp, float *m, float *v, int *t);
STOKES_API int stokes_mlp_set_adam(stokes_mlp *mlp, const float *m, const float *v, int t);
STOKES_API int stokes_mlp_set_normalization(stokes_mlp *mlp, const float *norm);
STOKES_API int stokes_mlp_get_normalization(stokes_mlp *mlp, float *norm);
/* Column means / standard deviations of X (rows x n_in) and T (rows x n_out) as normalisation. */
STOKES_API int stokes_mlp_fit_normalization(stokes_mlp *mlp, int rows, const float *X, const float *T);
/* Predictions Y (batch x n_out) of X (batch x n_in). */
STOKES_API int stokes_mlp_forward(stokes_mlp *mlp, int batch, const float *X, float *Y);
/* Loss (1/B) sum (1/2)|y_hat - t_hat|^2 of rows idx[0..batch) (DEVICE int32; NULL = the first
 * batch rows) of X, T and its gradient (n_params FP32, host or device; either may be NULL). */
STOKES_API int stokes_mlp_loss_grad(stokes_mlp *mlp, int rows, const float *X, const float *T,
                                    const int *idx, int batch, float *grad, float *loss);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on that loss with learning rate lr. */
STOKES_API int stokes_mlp_train_step(stokes_mlp *mlp, int rows, const float *X, const float *T,
                                     const int *idx, int batch, float lr, float *loss);
/* State transfer (HOST, any may be NULL): positions (V n x 2), tension (V n), and the last
 * step's solution [u_x, u_y, sigma] per vesicle (3 n V). */
STOKES_API int stokes_sim_get_state(stokes_sim *sim, double *x, double *sigma, double *solution);
STOKES_API int stokes_sim_set_state(stokes_sim *sim, const double *x, const double *sigma);
/* Krylov subspace length of the step's restarted GMRES (default 80; storage 3 n V (m + 1)). */
/* Checkpoint / resume of a time-stepping run (HOST buffers, any may be NULL): the initial
 * perimeters L0[V] and areas A0[V] that the arc-length and area corrections hold, and the
 * previous step's solution zprev[3 n V] and right-hand side bprev[3 n V] that the warm starts
 * use.  With stokes_sim_get_state / stokes_sim_set_state (positions, tension) they make a run
 * resumable: a new stokes_sim with the same walls and vesicle count, set_state, then
 * set_history (in that order: set_state clears the history) continues bit-identically in FP64.
 * set_history also makes zprev the current iterate of STOKES_GUESS_PREVIOUS. */
STOKES_API int stokes_sim_get_history(stokes_sim *sim, double *L0, double *A0, double *zprev,
                                      double *bprev);
STOKES_API int stokes_sim_set_history(stokes_sim *sim, const double *L0, const double *A0,
                                      const double *zprev, const double *bprev);
STOKES_API int stokes_sim_set_restart(stokes_sim *sim, int restart);
STOKES_API int stokes_sim_sizes(const stokes_sim *sim, int *n_vesicles, int *nodes_per_vesicle,
                                int *wall_nodes);

#ifdef __cplusplus
}
#endif
#endif /* STOKES_H */
