// stokes_internal.cuh -- shared device/host definitions of libstokes (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/stokes.h"

namespace stokes {

constexpr double kPi = 3.14159265358979323846;

// Device status word bits (set by kernels, read by stokes_sync).
constexpr unsigned kStatusNonfinite = 1u;
constexpr unsigned kStatusTimeout = 2u;

// Source tile (one pipeline stage) lengths.
constexpr int kTileF32 = 128;   // FP32 path: 128 sources x 32 B
constexpr int kTileF64 = 64;    // FP64 path: 64 sources x 48 B
constexpr int kStages = 3;      // ring of shared-memory stages per block

// Pair-kernel block shape.
constexpr int kThreadsF32 = 128;
constexpr int kTptF32 = 4;      // default targets per thread
constexpr int kThreadsF64 = 128;
constexpr int kTptF64 = 1;

constexpr int kMaxVesicleNodes = 1024;  // Kress self pass stages one curve in shared memory

// Per-curve description used by the finishing kernel.
struct CurveDev {
  int node_begin;   // first node index
  int n;            // node count
  int kind;         // STOKES_KIND_*
  int dens_begin;   // first row in the kind's density array
  int kress_off;    // offset of the curve's Kress table (vesicles), -1 for walls
};

// Arguments of the pair kernels (both precisions).
struct PairArgs {
  // targets
  int n_targets;
  const double2 *tgt;       // FP64 target points
  const int2 *tgt_skip;     // per target: source-slot range [x, y) skipped at image 0 (or NULL)
  double period;
  // sources (slot order: wall tiles then vesicle tiles, each padded to the tile length)
  int n_tiles;
  int n_wall_tiles;
  int tiles_per_split;
  const void *src_pos;      // FP32: float4 (x_hi, y_hi, x_lo, y_lo); FP64: double2 (x, y)
  const void *src_val;      // FP32: float4 (q1, q2, p1|n1, p2|n2); FP64: double4_32a
  // outputs
  double2 *partial;         // [split][n_targets]
  unsigned *status;
};

}  // namespace stokes

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
  int splits_f32 = 0, splits_f64 = 0;
  int tpt_f32 = stokes::kTptF32;       // targets per thread of the FP32 pair kernel: 1, 2 or 4
  int kgroup_f32 = 4;          // sources summed in FP32 before each Kahan update: 1, 2 or 4

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
  double2 *d_self = nullptr;     // [n_ves_nodes] Kress self term, by vesicle density row
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

  // scratch
  double2 *d_partial = nullptr;
  size_t partial_cap = 0;        // in double2 elements
  unsigned *d_status = nullptr;
  // host-API staging
  double *d_h_slp = nullptr, *d_h_dlp = nullptr, *d_h_out = nullptr;

  int num_sms = 0;

  // phase timing (stokes_set_profiling)
  bool profiling = false;
  bool timed = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

// Launchers implemented in the .cu files.
namespace stokes {
cudaError_t launch_geom_prep(stokes_ctx *c, cudaStream_t s);
cudaError_t launch_pack(stokes_ctx *c, int precision, const double *slp, const double *dlp,
                        cudaStream_t s);
cudaError_t launch_pair(stokes_ctx *c, int precision, int n_targets, const double2 *tgt,
                        const int2 *skip, int splits, cudaStream_t s);
cudaError_t launch_self(stokes_ctx *c, const double *slp, cudaStream_t s);
cudaError_t launch_finish_nodes(stokes_ctx *c, int splits, const double *slp, const double *dlp,
                                double jump, double2 *out, cudaStream_t s);
cudaError_t launch_finish_free(stokes_ctx *c, int splits, int n_targets, double2 *out,
                               cudaStream_t s);
}  // namespace stokes
