// stokes_internal.cuh -- shared device/host definitions of libstokes (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/stokes.h"
#include "flog64.cuh"

namespace stokes {

constexpr double kPi = 3.14159265358979323846;

// Device status word bits (set by kernels, read by stokes_sync).
constexpr unsigned kStatusNonfinite = 1u;
constexpr unsigned kStatusTimeout = 2u;
constexpr unsigned kStatusBounds = 4u;

// Device bounds checks of the debug build (-DSTOKES_DEBUG, libstokes_debug.so): dcheck(ok,
// status) records kStatusBounds in the context's status word when ok is false and returns ok,
// so the caller skips (or redirects to a valid element) the access it guards -- nothing traps.
// In the release build it is the constant true and the checks compile away.
#ifdef STOKES_DEBUG
__device__ __forceinline__ bool dcheck(bool ok, unsigned *status) {
  if (!ok && status) atomicOr(status, kStatusBounds);
  return ok;
}
#else
__device__ __forceinline__ constexpr bool dcheck(bool, unsigned *) { return true; }
#endif

// Source tile (one pipeline stage) lengths.
constexpr int kTileF32 = 128;   // FP32 path: 128 sources x 32 B
constexpr int kTileF64 = 64;    // FP64 path: 64 sources x 48 B
constexpr int kStages = 3;      // ring of shared-memory stages per block

// Pair-kernel block shape.
constexpr int kThreadsF32 = 128;
constexpr int kTptF32 = 4;      // default targets per thread
constexpr int kThreadsF64 = 128;
constexpr int kTptF64 = 1;
constexpr int kThreadsDF = 64;  // double-float path: 64 threads x 2 targets, FP64 tiles/slots
constexpr int kTptDF = 2;

constexpr int kMaxVesicleNodes = 1024;  // Kress self pass stages one curve in shared memory
// Largest stored Kress self matrix (all vesicles, 24 n^2 bytes each); beyond it the self term
// is recomputed from the geometry on every sum.
constexpr long long kSelfMatrixMaxBytes = 4LL << 30;

// Per-curve description used by the finishing kernel.
struct CurveDev {
  int node_begin;   // first node index
  int n;            // node count
  int kind;         // STOKES_KIND_*
  int dens_begin;   // first row in the kind's density array
  int kress_off;    // offset of the curve's Kress table (vesicles), -1 for walls
};

// One unit of pair-kernel work: a block of consecutive targets of one instance against a
// contiguous range of that instance's source tiles.  An instance lists its wall tiles, then
// its vesicle tiles ("virtual" tile index vt); vt < nw maps to global tile wb + vt (stresslet
// tiles), otherwise to vb + vt - nw (stokeslet tiles).
struct ItemDesc {
  int tgt_begin, tgt_count;
  int vt_begin, vt_end;
  int wb, nw, vb;
  int pad_;
  long long part_off;       // this split's partial of target i is partial[part_off + i]
  double period;
};

struct DFConst;

// Arguments of the pair kernels (all precisions).
struct PairArgs {
  // targets
  int n_targets;
  const double2 *tgt;       // FP64 target points
  const int2 *tgt_skip;     // per target: source-slot range [x, y) skipped at image 0 (or NULL)
  const int *tgt_perm;      // FP32 node evaluation: node of each kernel target (or NULL = same)
  float local_radius;       // FP32: stokeslet tiles of a target block whose targets all lie
                            //   within this distance (max norm) of its middle target are
                            //   evaluated in that block's local frame; 0 disables
  double period;
  // single-instance grid launch: blockIdx.x = target block, blockIdx.y = split
  int n_tiles;
  int n_wall_tiles;
  int tiles_per_split;
  // persistent launch over an item table (batched instances)
  const ItemDesc *items;
  int n_items;
  int *counter;             // zeroed before the launch; blocks take items in table order
  // sources (slot order: wall tiles of every instance, then vesicle tiles of every instance,
  // each instance's run padded to the tile length)
  const void *src_pos;      // FP32: 2 float4 per slot, (x_hi, x_hi, y_hi, y_hi), (x_lo, x_lo, y_lo,
                            //   y_lo); FP64: double2 (x, y)
  const void *src_val;      // FP32: 2 float4 per slot, (q1, q1, q2, q2), (p1|n1, p1|n1, p2|n2,
                            //   p2|n2); FP64: double4_32a
  // outputs
  double2 *partial;
  long long partial_cap;    // elements of partial (debug bounds checks)
  int src_tiles;            // tiles the source buffers hold (debug bounds checks)
  unsigned *status;
  const LogTab *logtab;     // FP64 logarithm table (flog64)
  const DFConst *dfc;       // double-float path: coordinate grids and logarithm tables
};

// Constants of the double-float path (device, one per context).  Coordinates are split as
// v = h + m + l with h on the grid g_h (a power of two chosen so every |coordinate| and every
// |target - source| fits 24 bits of it) and m on g_m = g_h 2^-24, which makes h_t - h_s and
// m_t - m_s exact float differences.  The logarithm tables: for k = 0..127,
// a_k = 1 + (k + 1/2)/128 and kt[k] = (1/a_k hi, lo, log a_k hi, lo); for every biased float
// exponent e, et[e] = ((e - 127) ln 2 hi, lo).
struct DFConst {
  float4 kt[128];
  float2 et[256];
  double g_h, g_m;
  unsigned maxabs_bits;      // float bits of an upper bound of |coordinate| + |period|
  unsigned pad_[3];
};

// Per instance of a batched geometry (host and device copies).
struct InstDev {
  int node_begin, N;
  int wb32, nw32, vb32, nv32;   // wall / vesicle tile runs, FP32 tiles
  int wb64, nw64, vb64, nv64;   // the same in FP64 tiles
  int splits32, splits64;
  long long part_off32, part_off64;  // first partial of the instance
  double period;
};

}  // namespace stokes

using InstHost = stokes::InstDev;

struct stokes_ctx {
  int device = 0;
  std::string err;
  cudaStream_t own_stream = nullptr;
  cudaStream_t side_stream = nullptr;   // runs the FP64 self pass beside the pair kernel
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  // geometry (host metadata)
  bool have_geom = false;
  int N = 0, n_curves = 0, n_ves_nodes = 0, n_wall_nodes = 0;
  int n_wall_curves = 0, n_ves_curves = 0;
  double period = 0.0, mu = 1.0;
  std::vector<int> off, kind;
  int wall_slots = 0, ves_slots_f32 = 0, ves_slots_f64 = 0;  // padded slot counts
  int wall_slots_f64 = 0;
  int max_ves_n = 0;
  int splits_f32 = 0, splits_f64 = 0, splits_df = 0;
  int tpt_f32 = stokes::kTptF32;       // targets per thread of the FP32 pair kernel: 1, 2 or 4
  int kgroup_f32 = 4;          // sources summed in FP32 before each Kahan update: 1, 2 or 4
  bool local_frame = true;     // FP32: evaluate stokeslet tiles of compact blocks in a local frame
  float local_radius = 0.f;    // block radius admitted to the local frame (1/8 of the extent)

  // device geometry
  double2 *d_x = nullptr;        // [N] nodes
  double2 *d_nrm = nullptr;      // [N] normals
  double *d_w = nullptr;         // [N] weights
  double *d_kap = nullptr;       // [N] curvature (walls)
  int2 *d_tgt_skip32 = nullptr;  // [N] skip range in FP32 slot space
  int2 *d_tgt_skip64 = nullptr;  // [N] skip range in FP64 slot space
  int *d_node_dens = nullptr;    // [N] row in the node kind's density array
  int *d_wall_nodes = nullptr;   // [n_wall_nodes] node indices of wall nodes
  int *d_ves_nodes = nullptr;    // [n_ves_nodes] node indices of vesicle nodes
  int *d_tgt_perm = nullptr;     // [N] FP32 node-evaluation target order: per instance, walls in
                                 //   node order, then vesicles by Morton code of their centroid
  double2 *d_self = nullptr;     // [n_ves_nodes] Kress self term, by vesicle density row
  // Kress self blocks assembled per geometry (when they fit kSelfMatrixMaxBytes): for vesicle
  // v (in d_ves_curve_ids order) three n x n arrays (11, 12, 22) at d_selfG + d_selfG_off[v],
  // element k n + a the 2 x 2 block that node k's density contributes at node a; each sum's
  // self term is then a batched matvec instead of an FP64 pass over all the logs
  double *d_selfG = nullptr;
  long long *d_selfG_off = nullptr;
  bool self_matrix = false;
  stokes::CurveDev *d_curves = nullptr;  // [n_curves]
  int *d_ves_curve_ids = nullptr;        // [n_ves_curves]
  double *d_kress = nullptr;             // concatenated Kress tables T_j per vesicle size
  // FP32 source slots
  int *d_slot_node32 = nullptr;  // [slots] node index or -1
  float4 *d_src_pos32 = nullptr;
  float4 *d_src_val32 = nullptr;
  // FP64 source slots
  int *d_slot_node64 = nullptr;
  double2 *d_src_pos64 = nullptr;
  double4_32a *d_src_val64 = nullptr;
  // double-float source slots (FP64 slot layout): 2 float4 each of position and value
  float4 *d_src_pos_df = nullptr;
  float4 *d_src_val_df = nullptr;
  stokes::DFConst *d_dfc = nullptr;

  // scratch
  double2 *d_partial = nullptr;
  size_t partial_cap = 0;        // in double2 elements
  long long debug_tighten = 0;   // debug build: elements the bounds checks take off the
                                 //   partial sums a launch writes or reads (stokes_debug_tighten)
  long long batch_part32 = 0, batch_part64 = 0;  // partial sums of one batched evaluation
  unsigned *d_status = nullptr;
  // host-API staging
  double *d_h_slp = nullptr, *d_h_dlp = nullptr, *d_h_out = nullptr;

  int num_sms = 0;
  stokes::LogTab *d_logtab = nullptr;

  // batched instances (stokes_batch_set); n_inst = 1 for stokes_geom_set
  int n_inst = 1;
  std::vector<InstHost> inst;
  stokes::InstDev *d_inst = nullptr;
  int *d_node_inst = nullptr;            // [N] instance of each node
  stokes::ItemDesc *d_items32 = nullptr, *d_items64 = nullptr;
  int n_items32 = 0, n_items64 = 0;
  int *d_counter = nullptr;              // work counter of the persistent launch
  int batch_ips32 = 4, batch_ips64 = 4;  // items per resident block the tables aim for
  // CUDA graphs of one batched evaluation, per precision (built on first use)
  cudaGraphExec_t graph_exec[3] = {nullptr, nullptr, nullptr};  // indexed by precision
  double graph_jump[3] = {0.0, 0.0, 0.0};
  double *d_b_slp = nullptr, *d_b_dlp = nullptr, *d_b_out = nullptr;  // graph staging

  // single-instance node sums replayed from a CUDA graph (stokes_set_graph_mode): the graph
  // is captured for one (precision, jump, density and output pointers) and relaunched while
  // those repeat; anything that changes what it captured drops it (invalidate_node_graph)
  int graph_mode = 1;                    // STOKES_GRAPH_OFF / _SMALL / _ALWAYS
  cudaGraphExec_t node_graph = nullptr;
  int ng_precision = -1;
  double ng_jump = 0.0;
  const void *ng_slp = nullptr, *ng_dlp = nullptr, *ng_out = nullptr;
  long long graph_captures = 0, graph_replays = 0;  // node-sum graphs captured / launched

  // phase timing (stokes_set_profiling)
  bool profiling = false;
  bool timed = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace stokes {
// Bound the debug build's checks put on a launch's partial-sum indices: the elements the
// launch writes or reads (`needed`, within the allocation of `allocated`), less the elements
// stokes_debug_tighten takes off.
inline long long partial_check_cap(const stokes_ctx *c, long long allocated, long long needed) {
  const long long cap = needed < allocated ? needed : allocated;
  return cap > c->debug_tighten ? cap - c->debug_tighten : 0;
}
// Drops the captured node-sum graph (its kernels hold the pointers and launch shape of the
// moment of capture).  Called whenever the partial buffer, the launch shape or the geometry
// changes.
void invalidate_node_graph(stokes_ctx *c);
int set_geometry(stokes_ctx *c, int n_inst, const int *inst_curve_off, const double *periods,
                 int n_curves, const int32_t *curve_offset, const int32_t *curve_kind,
                 const double *nodes, const double *weights, const double *normals,
                 const double *curvature, double mu, cudaStream_t s);
}  // namespace stokes

// Launchers implemented in the .cu files.
namespace stokes {
cudaError_t launch_geom_prep(stokes_ctx *c, cudaStream_t s);
cudaError_t launch_pack(stokes_ctx *c, int precision, const double *slp, const double *dlp,
                        cudaStream_t s);
// FP64 partials of split k and target i go to partial[k * n_targets + i].
cudaError_t launch_pair(stokes_ctx *c, int precision, int n_targets, const double2 *tgt,
                        const int2 *skip, int splits, double2 *partial, cudaStream_t s);
cudaError_t launch_self(stokes_ctx *c, const double *slp, cudaStream_t s);
cudaError_t launch_finish_nodes(stokes_ctx *c, int splits, const double *slp, const double *dlp,
                                double jump, double2 *out, cudaStream_t s);
cudaError_t launch_finish_free(stokes_ctx *c, int splits, int n_targets, double2 *out,
                               cudaStream_t s);
cudaError_t launch_pair_batch(stokes_ctx *c, int precision, int slots, cudaStream_t s);
cudaError_t launch_finish_batch(stokes_ctx *c, int precision, const double *dlp, double jump,
                                double2 *out, cudaStream_t s);
int pair_blocks_per_sm(stokes_ctx *c, int precision);
int pair_batch_blocks_per_sm(stokes_ctx *c, int precision);
// double-float path (k_pair_df.cu)
cudaError_t launch_df_init(stokes::DFConst *d, cudaStream_t s);
cudaError_t launch_geom_prep_df(stokes_ctx *c, cudaStream_t s);
cudaError_t launch_pack_df(stokes_ctx *c, const double *slp, const double *dlp, cudaStream_t s);
cudaError_t launch_pair_df(stokes_ctx *c, int n_targets, const double2 *tgt, const int2 *skip,
                           int splits, double2 *partial, cudaStream_t s);
cudaError_t launch_pair_batch_df(stokes_ctx *c, int blocks, cudaStream_t s);
int pair_df_blocks_per_sm(stokes_ctx *c);
int pair_df_batch_blocks_per_sm(stokes_ctx *c);
}  // namespace stokes
