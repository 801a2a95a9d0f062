// stokes_abi.cu -- the C ABI of libstokes (host side): validation, layout planning,
// device memory of a context, and the launch sequence of one layer-potential sum.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>

#include "stokes_internal.cuh"

namespace stokes {
cudaError_t launch_kress_table(int n, double *T, cudaStream_t s);
cudaError_t launch_logtab_init(LogTab *t, cudaStream_t s);
int effective_splits(stokes_ctx *c, int precision, int splits);
int pair_blocks_per_sm(stokes_ctx *c, int precision);
void tune_apply_cached(stokes_ctx *c);  // tune.cu: shapes recorded for the geometry's size class
void fmm_geometry_changed(const stokes_ctx *c);  // fmm.cu: invalidates the context's FMM plans
int field_splits(const stokes_ctx *c, int n_targets);  // k_field.cu
cudaError_t launch_wait_timeout_check(stokes_ctx *c, cudaStream_t s);  // k_prep.cu
void noalloc_setup_device(int device);                                 // noalloc.cu
cudaError_t launch_check_log64(stokes_ctx *c, int n, const double *x, double *out,
                               cudaStream_t s);                        // k_prep.cu
cudaError_t launch_field(stokes_ctx *c, int n_targets, const double2 *tgt, const double2 *tnrm,
                         int splits, double *out, cudaStream_t s);
}  // namespace stokes

using namespace stokes;

namespace {

int fail(stokes_ctx *c, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(stokes_ctx *c, int code, const char *fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

int cuda_fail(stokes_ctx *c, cudaError_t e, const char *where) {
  if (e == cudaErrorMemoryAllocation)
    return fail(c, STOKES_ERR_OOM, "%s: %s", where, cudaGetErrorString(e));
  return fail(c, STOKES_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
  } while (0)

template <class T>
void dfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_geometry(stokes_ctx *c) {
  fmm_geometry_changed(c);
  invalidate_node_graph(c);
  dfree(c->d_x);
  dfree(c->d_nrm);
  dfree(c->d_w);
  dfree(c->d_kap);
  dfree(c->d_tgt_skip32);
  dfree(c->d_tgt_skip64);
  dfree(c->d_node_dens);
  dfree(c->d_wall_nodes);
  dfree(c->d_ves_nodes);
  dfree(c->d_tgt_perm);
  dfree(c->d_self);
  dfree(c->d_selfG);
  dfree(c->d_selfG_off);
  c->self_matrix = false;
  dfree(c->d_node_inst);
  dfree(c->d_inst);
  dfree(c->d_items32);
  dfree(c->d_items64);
  dfree(c->d_b_slp);
  dfree(c->d_b_dlp);
  dfree(c->d_b_out);
  for (auto &g : c->graph_exec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  c->n_inst = 1;
  c->inst.clear();
  c->n_items32 = c->n_items64 = 0;
  dfree(c->d_curves);
  dfree(c->d_ves_curve_ids);
  dfree(c->d_kress);
  dfree(c->d_slot_node32);
  dfree(c->d_src_pos32);
  dfree(c->d_src_val32);
  dfree(c->d_slot_node64);
  dfree(c->d_src_pos64);
  dfree(c->d_src_val64);
  dfree(c->d_src_pos_df);
  dfree(c->d_src_val_df);
  dfree(c->d_h_slp);
  dfree(c->d_h_dlp);
  dfree(c->d_h_out);
  c->have_geom = false;
  c->N = 0;
}

template <class T>
cudaError_t dalloc(T *&p, size_t count) {
  return cudaMalloc(reinterpret_cast<void **>(&p), std::max<size_t>(count, 1) * sizeof(T));
}

template <class T>
cudaError_t upload(T *&p, const std::vector<T> &v, cudaStream_t s) {
  cudaError_t e = dalloc(p, v.size());
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int ensure_partial(stokes_ctx *c, size_t elems) {
  if (elems <= c->partial_cap) return STOKES_OK;
  CK(cudaDeviceSynchronize());
  invalidate_node_graph(c);
  dfree(c->d_partial);
  c->partial_cap = 0;
  CK(dalloc(c->d_partial, elems));
  c->partial_cap = elems;
  return STOKES_OK;
}

// Wave model of the source splits.  The pair kernel runs (target blocks x splits) equal-cost
// blocks in waves of `slots` = resident blocks per SM x SMs; the time is ~ waves x (1 / splits),
// so a split count is costed as ceil(tb s / slots) / s plus a small per-split charge.  At least
// 4 tiles per split keep the per-block prologue and the partial traffic small -- unless even
// then the blocks would not fill one wave (small geometries), where splits down to one tile
// each are allowed.  Returns (cost, splits) for every split count that effective_splits leaves
// unchanged, in increasing split order.
std::vector<std::pair<double, int>> split_costs(stokes_ctx *c, int precision) {
  const bool f32 = precision == STOKES_FP32_KAHAN;
  const int per_block = f32 ? kThreadsF32 * c->tpt_f32
                            : precision == STOKES_DOUBLE_FLOAT ? kThreadsDF * kTptDF : kThreadsF64;
  const long slots = long(pair_blocks_per_sm(c, precision)) * std::max(c->num_sms, 1);
  const long tb = (c->N + per_block - 1) / per_block;
  const int n_tiles = f32 ? (c->wall_slots + c->ves_slots_f32) / kTileF32
                          : (c->wall_slots_f64 + c->ves_slots_f64) / kTileF64;
  const int floor_tiles = tb * std::max(1, n_tiles / 4) < slots ? 1 : 4;
  const int smax = std::max(1, std::min(n_tiles / floor_tiles, 256));
  std::vector<std::pair<double, int>> out;
  for (int sp = 1; sp <= smax; ++sp) {
    const int eff = effective_splits(c, precision, sp);
    if (eff != sp) continue;
    const double waves = double((tb * eff + slots - 1) / slots);
    out.emplace_back(waves / eff + 2e-4 * eff, eff);
  }
  return out;
}

// Default source splits: the cheapest count of the wave model (the smallest on ties).
int default_splits(stokes_ctx *c, int precision) {
  int best = 1;
  double best_cost = 1e300;
  for (const auto &cs : split_costs(c, precision))
    if (cs.first < best_cost - 1e-12) {
      best_cost = cs.first;
      best = cs.second;
    }
  return best;
}

int splits_of(const stokes_ctx *c, int precision) {
  return precision == STOKES_FP32_KAHAN ? c->splits_f32
         : precision == STOKES_FP64     ? c->splits_f64
                                        : c->splits_df;
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

int read_status(stokes_ctx *c, cudaStream_t s) {
  unsigned st = 0;
  CK(cudaMemcpyAsync(&st, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (st) {
    CK(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), s));
    CK(cudaStreamSynchronize(s));
    if (st & kStatusBounds)
      return fail(c, STOKES_ERR_BOUNDS, "a device bounds check failed (debug build)");
    if (st & kStatusTimeout)
      return fail(c, STOKES_ERR_TIMEOUT, "a device pipeline wait exceeded its bound");
    return fail(c, STOKES_ERR_NONFINITE, "non-finite input value");
  }
  return STOKES_OK;
}

int check_density_args(stokes_ctx *c, int precision, const double *slp, const double *dlp) {
  if (!c->have_geom) return fail(c, STOKES_ERR_NO_GEOM, "no geometry set");
  if (precision != STOKES_FP64 && precision != STOKES_FP32_KAHAN &&
      precision != STOKES_DOUBLE_FLOAT)
    return fail(c, STOKES_ERR_ARG, "unknown precision %d", precision);
  if (c->n_ves_nodes > 0 && !slp) return fail(c, STOKES_ERR_ARG, "slp_density is NULL");
  if (c->n_wall_nodes > 0 && !dlp) return fail(c, STOKES_ERR_ARG, "dlp_density is NULL");
  return STOKES_OK;
}

int mark(stokes_ctx *c, int k, cudaStream_t s) {
  if (!c->profiling) return STOKES_OK;
  CK(cudaEventRecord(c->ev[k], s));
  if (k == 3) c->timed = true;
  return STOKES_OK;
}

#define MARK(k)                  \
  do {                           \
    int st_ = mark(c, (k), s);   \
    if (st_) return st_;         \
  } while (0)

// Batched instances: the same phases, with the persistent item-table pair kernel.
int run_batch(stokes_ctx *c, int precision, const double *slp, const double *dlp, double jump,
              double *out, cudaStream_t s) {
  MARK(0);
  if (c->n_ves_curves > 0) {
    CK(cudaEventRecord(c->ev_fork, s));
    CK(cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0));
    CK(launch_self(c, slp, c->side_stream));
    CK(cudaEventRecord(c->ev_join, c->side_stream));
  }
  CK(launch_pack(c, precision, slp, dlp, s));
  MARK(1);
  const int blocks = pair_batch_blocks_per_sm(c, precision) * std::max(c->num_sms, 1);
  CK(launch_pair_batch(c, precision, blocks, s));
  MARK(2);
  if (c->n_ves_curves > 0) CK(cudaStreamWaitEvent(s, c->ev_join, 0));
  CK(launch_finish_batch(c, precision, dlp, jump, reinterpret_cast<double2 *>(out), s));
  MARK(3);
  return STOKES_OK;
}

int run_nodes_direct(stokes_ctx *c, int precision, const double *slp, const double *dlp,
                     double jump, double *out, cudaStream_t s) {
  const int splits = splits_of(c, precision);
  MARK(0);
  // fork: the FP64 Kress self pass runs on the side stream beside the pair kernel
  if (c->n_ves_curves > 0) {
    CK(cudaEventRecord(c->ev_fork, s));
    CK(cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0));
    CK(launch_self(c, slp, c->side_stream));
    CK(cudaEventRecord(c->ev_join, c->side_stream));
  }
  CK(launch_pack(c, precision, slp, dlp, s));
  MARK(1);
  CK(launch_pair(c, precision, c->N, c->d_x,
                 precision == STOKES_FP32_KAHAN ? c->d_tgt_skip32 : c->d_tgt_skip64, splits,
                 c->d_partial, s));
  MARK(2);
  if (c->n_ves_curves > 0) CK(cudaStreamWaitEvent(s, c->ev_join, 0));
  CK(launch_finish_nodes(c, splits, slp, dlp, jump, reinterpret_cast<double2 *>(out), s));
  MARK(3);
  return STOKES_OK;
}

// Node sums of geometries up to this size are replayed from a graph in STOKES_GRAPH_SMALL mode
// (there the five launches' host overhead is a visible share of the sum).
constexpr int kGraphSmallMaxN = 65536;

bool use_node_graph(const stokes_ctx *c) {
  if (c->profiling || c->graph_mode == STOKES_GRAPH_OFF) return false;
  return c->graph_mode == STOKES_GRAPH_ALWAYS || c->N <= kGraphSmallMaxN;
}

// The node sum as one graph launch: captured on the context's own stream (joined by the side
// stream of the self pass through the fork/join events) for these pointers, then relaunched on
// the caller's stream while they repeat.  A capture that fails falls back to direct launches.
int run_nodes_graph(stokes_ctx *c, int precision, const double *slp, const double *dlp,
                    double jump, double *out, cudaStream_t s) {
  if (!(c->node_graph && c->ng_precision == precision && c->ng_jump == jump &&
        c->ng_slp == slp && c->ng_dlp == dlp && c->ng_out == out)) {
    invalidate_node_graph(c);
    cudaStream_t cs = c->own_stream;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const int st = run_nodes_direct(c, precision, slp, dlp, jump, out, cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e2 =
        (st == STOKES_OK && e == cudaSuccess) ? cudaGraphInstantiate(&exec, graph, 0) : e;
    if (graph) cudaGraphDestroy(graph);
    if (st != STOKES_OK || e2 != cudaSuccess) {
      cudaGetLastError();  // clear a capture error; the direct path reports its own
      return run_nodes_direct(c, precision, slp, dlp, jump, out, s);
    }
    c->node_graph = exec;
    ++c->graph_captures;
    c->ng_precision = precision;
    c->ng_jump = jump;
    c->ng_slp = slp;
    c->ng_dlp = dlp;
    c->ng_out = out;
  }
  CK(cudaGraphLaunch(c->node_graph, s));
  ++c->graph_replays;
  return STOKES_OK;
}

int run_nodes(stokes_ctx *c, int precision, const double *slp, const double *dlp, double jump,
              double *out, cudaStream_t s) {
  if (c->n_inst > 1) return run_batch(c, precision, slp, dlp, jump, out, s);
  if (use_node_graph(c)) return run_nodes_graph(c, precision, slp, dlp, jump, out, s);
  return run_nodes_direct(c, precision, slp, dlp, jump, out, s);
}

}  // namespace

namespace stokes {
void invalidate_node_graph(stokes_ctx *c) {
  if (c->node_graph) cudaGraphExecDestroy(c->node_graph);
  c->node_graph = nullptr;
  c->ng_precision = -1;
}
}  // namespace stokes

extern "C" {

int stokes_create(int device, stokes_ctx **out) {
  if (!out) return STOKES_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return STOKES_ERR_CUDA;
  stokes_ctx *c = new stokes_ctx();
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void **>(&c->d_status), sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(c->d_status, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void **>(&c->d_logtab), sizeof(LogTab)) != cudaSuccess ||
      launch_logtab_init(c->d_logtab, nullptr) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void **>(&c->d_dfc), sizeof(DFConst)) != cudaSuccess ||
      launch_df_init(c->d_dfc, nullptr) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete c;
    return STOKES_ERR_CUDA;
  }
  noalloc_setup_device(device);
  *out = c;
  return STOKES_OK;
}

int stokes_destroy(stokes_ctx *c) {
  if (!c) return STOKES_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  invalidate_node_graph(c);
  free_geometry(c);
  dfree(c->d_partial);
  dfree(c->d_status);
  dfree(c->d_counter);
  dfree(c->d_logtab);
  dfree(c->d_dfc);
  for (auto &e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  delete c;
  return STOKES_OK;
}

int stokes_last_error(const stokes_ctx *c, char *buf, size_t len) {
  if (!c || !buf || len == 0) return STOKES_ERR_ARG;
  snprintf(buf, len, "%s", c->err.c_str());
  return STOKES_OK;
}

int stokes_num_nodes(const stokes_ctx *c) { return (c && c->have_geom) ? c->N : 0; }

}  // extern "C"

namespace {

// Interleave the low 16 bits of x and y (x in the even bits).
uint32_t morton2(uint32_t x, uint32_t y) {
  auto spread = [](uint32_t v) {
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
  };
  return spread(x) | (spread(y) << 1);
}

// Target order of the FP32 node evaluation: per instance, its wall nodes in node order, then
// its vesicles along a Morton curve of their centroids (quantised to 2^16 steps over the
// bounding box of the instance's nodes), each vesicle's nodes in node order.  Consecutive
// target blocks then cover compact regions.  *radius = 1/8 of the smallest instance extent
// (the block radius admitted to the pair kernel's local frame).
std::vector<int> target_order(int n_inst, const int *inst_curve_off, const int32_t *off,
                              const int32_t *kind, const std::vector<double2> &x,
                              float *radius) {
  std::vector<int> perm;
  perm.reserve(x.size());
  double min_ext = 0.0;
  bool have_ext = false;
  for (int k = 0; k < n_inst; ++k) {
    const int c0 = inst_curve_off[k], c1 = inst_curve_off[k + 1];
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    for (int i = off[c0]; i < off[c1]; ++i) {
      if (!(isfinite(x[i].x) && isfinite(x[i].y))) continue;
      x0 = std::min(x0, x[i].x);
      x1 = std::max(x1, x[i].x);
      y0 = std::min(y0, x[i].y);
      y1 = std::max(y1, x[i].y);
    }
    const double ext = std::max(x1 - x0, y1 - y0);
    if (ext > 0.0 && isfinite(ext)) {
      min_ext = have_ext ? std::min(min_ext, ext) : ext;
      have_ext = true;
    }
    std::vector<std::pair<uint32_t, int>> ves;
    for (int cc = c0; cc < c1; ++cc) {
      if (kind[cc] == STOKES_KIND_WALL) {
        for (int i = off[cc]; i < off[cc + 1]; ++i) perm.push_back(i);
        continue;
      }
      double cx = 0.0, cy = 0.0;
      for (int i = off[cc]; i < off[cc + 1]; ++i) {
        cx += x[i].x;
        cy += x[i].y;
      }
      const double n = double(off[cc + 1] - off[cc]);
      auto q = [](double v, double lo, double e) {
        const double t = e > 0.0 ? (v - lo) / e : 0.0;
        return (isfinite(t) && t > 0.0) ? uint32_t(std::min(t, 1.0) * 65535.0) : 0u;
      };
      const double e = std::max(x1 - x0, y1 - y0);
      ves.emplace_back(morton2(q(cx / n, x0, e), q(cy / n, y0, e)), cc);
    }
    std::stable_sort(ves.begin(), ves.end(),
                     [](const std::pair<uint32_t, int> &a, const std::pair<uint32_t, int> &b) {
                       return a.first < b.first;
                     });
    for (const auto &v : ves)
      for (int i = off[v.second]; i < off[v.second + 1]; ++i) perm.push_back(i);
  }
  *radius = have_ext ? float(min_ext / 8.0) : 0.f;
  return perm;
}

}  // namespace

namespace stokes {

// The k cheapest split counts of the wave model, cheapest first (the autotuner's candidates).
std::vector<int> ranked_splits(stokes_ctx *c, int precision, int k) {
  auto cs = split_costs(c, precision);
  std::stable_sort(cs.begin(), cs.end(),
                   [](const std::pair<double, int> &a, const std::pair<double, int> &b) {
                     return a.first < b.first;
                   });
  std::vector<int> out;
  for (const auto &x : cs) {
    if (int(out.size()) >= k) break;
    out.push_back(x.second);
  }
  return out;
}

// Validate and upload a geometry of n_inst independent instances (instance k owns curves
// [inst_curve_off[k], inst_curve_off[k+1])), and build the source-slot layout: the wall tiles
// of every instance, then the vesicle tiles of every instance, each instance's run padded to
// the tile length with zero-weight dummies.
int set_geometry(stokes_ctx *c, int n_inst, const int *inst_curve_off, const double *periods,
                 int n_curves, const int32_t *curve_offset, const int32_t *curve_kind,
                 const double *nodes, const double *weights, const double *normals,
                 const double *curvature, double mu, cudaStream_t s) {
  if (n_curves < 1 || !curve_offset || !curve_kind)
    return fail(c, STOKES_ERR_ARG, "need n_curves >= 1 and host curve_offset / curve_kind");
  if (!(isfinite(mu) && mu > 0.0)) return fail(c, STOKES_ERR_ARG, "mu must be finite and > 0");
  if (curve_offset[0] != 0) return fail(c, STOKES_ERR_ARG, "curve_offset[0] must be 0");
  if (n_inst < 1 || inst_curve_off[0] != 0 || inst_curve_off[n_inst] != n_curves)
    return fail(c, STOKES_ERR_ARG, "instance curve offsets must run from 0 to n_curves");
  bool any_img = false, any_flat = false;
  for (int k = 0; k < n_inst; ++k) {
    if (inst_curve_off[k + 1] <= inst_curve_off[k])
      return fail(c, STOKES_ERR_ARG, "instance %d has no curves", k);
    if (!(isfinite(periods[k]) && periods[k] >= 0.0))
      return fail(c, STOKES_ERR_ARG, "period of instance %d must be finite and >= 0", k);
    (periods[k] != 0.0 ? any_img : any_flat) = true;
  }
  if (any_img && any_flat)
    return fail(c, STOKES_ERR_ARG, "instances must all have a period > 0 or all have period 0");
  int n_wall = 0, n_ves = 0, max_ves = 0;
  for (int k = 0; k < n_curves; ++k) {
    const int n = curve_offset[k + 1] - curve_offset[k];
    if (n <= 0) return fail(c, STOKES_ERR_ARG, "curve %d is empty or offsets decrease", k);
    if (curve_kind[k] == STOKES_KIND_WALL) {
      n_wall += n;
    } else if (curve_kind[k] == STOKES_KIND_VESICLE) {
      if (n < 4 || (n & 1))
        return fail(c, STOKES_ERR_ODD_N, "vesicle curve %d has %d nodes; the Kress rule needs an even n >= 4", k, n);
      if (n > kMaxVesicleNodes)
        return fail(c, STOKES_ERR_ARG, "vesicle curve %d has %d > %d nodes", k, n, kMaxVesicleNodes);
      n_ves += n;
      max_ves = std::max(max_ves, n);
    } else {
      return fail(c, STOKES_ERR_ARG, "curve %d has unknown kind %d", k, curve_kind[k]);
    }
  }
  const int N = curve_offset[n_curves];
  if (!nodes || !weights || !normals) return fail(c, STOKES_ERR_ARG, "NULL geometry pointer");
  if (n_wall > 0 && !curvature) return fail(c, STOKES_ERR_ARG, "curvature is required when walls are present");
  if (!aligned16(nodes) || !aligned16(normals))
    return fail(c, STOKES_ERR_ARG, "nodes and normals must be 16-byte aligned");

  free_geometry(c);
  c->N = N;
  c->n_curves = n_curves;
  c->n_wall_nodes = n_wall;
  c->n_ves_nodes = n_ves;
  c->max_ves_n = max_ves;
  c->period = periods[0];
  c->mu = mu;
  c->off.assign(curve_offset, curve_offset + n_curves + 1);
  c->kind.assign(curve_kind, curve_kind + n_curves);
  c->n_inst = n_inst;

  // ---- layout planning (host) ----
  auto pad = [](int n, int t) { return (n + t - 1) / t * t; };
  std::vector<InstHost> inst(n_inst);
  std::vector<int> inst_wall(n_inst, 0), inst_ves(n_inst, 0);
  for (int k = 0; k < n_inst; ++k) {
    for (int cc = inst_curve_off[k]; cc < inst_curve_off[k + 1]; ++cc)
      (curve_kind[cc] == STOKES_KIND_WALL ? inst_wall[k] : inst_ves[k]) +=
          curve_offset[cc + 1] - curve_offset[cc];
    InstHost &I = inst[k];
    I = InstHost{};
    I.node_begin = curve_offset[inst_curve_off[k]];
    I.N = curve_offset[inst_curve_off[k + 1]] - I.node_begin;
    I.period = periods[k];
  }
  int t32 = 0, t64 = 0;
  for (int k = 0; k < n_inst; ++k) {  // wall runs
    inst[k].wb32 = t32;
    inst[k].nw32 = pad(inst_wall[k], kTileF32) / kTileF32;
    t32 += inst[k].nw32;
    inst[k].wb64 = t64;
    inst[k].nw64 = pad(inst_wall[k], kTileF64) / kTileF64;
    t64 += inst[k].nw64;
  }
  c->wall_slots = t32 * kTileF32;
  c->wall_slots_f64 = t64 * kTileF64;
  for (int k = 0; k < n_inst; ++k) {  // vesicle runs
    inst[k].vb32 = t32;
    inst[k].nv32 = pad(inst_ves[k], kTileF32) / kTileF32;
    t32 += inst[k].nv32;
    inst[k].vb64 = t64;
    inst[k].nv64 = pad(inst_ves[k], kTileF64) / kTileF64;
    t64 += inst[k].nv64;
  }
  c->ves_slots_f32 = t32 * kTileF32 - c->wall_slots;
  c->ves_slots_f64 = t64 * kTileF64 - c->wall_slots_f64;
  std::vector<int> slot32(size_t(t32) * kTileF32, -1);
  std::vector<int> slot64(size_t(t64) * kTileF64, -1);
  std::vector<int2> skip32(N, make_int2(-1, -1)), skip64(N, make_int2(-1, -1));
  std::vector<int> node_dens(N), node_inst(N), wall_nodes, ves_nodes, ves_ids;
  std::vector<CurveDev> curves(n_curves);
  std::map<int, int> kress_off;
  int kress_len = 0;
  int ws = 0, vs = 0;
  for (int k = 0; k < n_inst; ++k) {
    int wloc = 0, vloc = 0;
    for (int cc = inst_curve_off[k]; cc < inst_curve_off[k + 1]; ++cc) {
      const int b = curve_offset[cc], n = curve_offset[cc + 1] - b;
      CurveDev cd{b, n, curve_kind[cc], 0, -1};
      for (int a = 0; a < n; ++a) node_inst[b + a] = k;
      if (curve_kind[cc] == STOKES_KIND_WALL) {
        cd.dens_begin = ws;
        for (int a = 0; a < n; ++a) {
          slot32[size_t(inst[k].wb32) * kTileF32 + wloc + a] = b + a;
          slot64[size_t(inst[k].wb64) * kTileF64 + wloc + a] = b + a;
          node_dens[b + a] = ws + a;
          wall_nodes.push_back(b + a);
        }
        ws += n;
        wloc += n;
      } else {
        cd.dens_begin = vs;
        const int s32 = inst[k].vb32 * kTileF32 + vloc, s64 = inst[k].vb64 * kTileF64 + vloc;
        for (int a = 0; a < n; ++a) {
          slot32[s32 + a] = b + a;
          slot64[s64 + a] = b + a;
          node_dens[b + a] = vs + a;
          skip32[b + a] = make_int2(s32, s32 + n);
          skip64[b + a] = make_int2(s64, s64 + n);
          ves_nodes.push_back(b + a);
        }
        vs += n;
        vloc += n;
        if (!kress_off.count(n)) {
          kress_off[n] = kress_len;
          kress_len += n;
        }
        cd.kress_off = kress_off[n];
        ves_ids.push_back(cc);
      }
      curves[cc] = cd;
    }
  }
  c->n_wall_curves = n_curves - int(ves_ids.size());
  c->n_ves_curves = int(ves_ids.size());
  c->inst = inst;

  // ---- device buffers ----
  CK(dalloc(c->d_x, N));
  CK(dalloc(c->d_nrm, N));
  CK(dalloc(c->d_w, N));
  CK(dalloc(c->d_kap, N));
  CK(cudaMemcpyAsync(c->d_x, nodes, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(c->d_nrm, normals, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(c->d_w, weights, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  if (curvature)
    CK(cudaMemcpyAsync(c->d_kap, curvature, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  else
    CK(cudaMemsetAsync(c->d_kap, 0, sizeof(double) * N, s));
  CK(upload(c->d_slot_node32, slot32, s));
  CK(upload(c->d_slot_node64, slot64, s));
  CK(upload(c->d_tgt_skip32, skip32, s));
  CK(upload(c->d_tgt_skip64, skip64, s));
  CK(upload(c->d_node_dens, node_dens, s));
  CK(upload(c->d_wall_nodes, wall_nodes, s));
  CK(upload(c->d_ves_nodes, ves_nodes, s));
  CK(upload(c->d_curves, curves, s));
  CK(upload(c->d_ves_curve_ids, ves_ids, s));
  if (n_inst > 1) CK(upload(c->d_node_inst, node_inst, s));
  {
    std::vector<double2> hx(N);
    CK(cudaMemcpyAsync(hx.data(), c->d_x, sizeof(double2) * N, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float radius = 0.f;
    const std::vector<int> perm =
        target_order(n_inst, inst_curve_off, curve_offset, curve_kind, hx, &radius);
    CK(upload(c->d_tgt_perm, perm, s));
    c->local_radius = radius;
  }
  CK(dalloc(c->d_self, n_ves));
  CK(dalloc(c->d_kress, kress_len));
  {  // stored Kress self blocks, when they fit
    std::vector<long long> goff;
    long long total = 0;
    for (int cc : ves_ids) {
      const long long n = curve_offset[cc + 1] - curve_offset[cc];
      goff.push_back(total);
      total += 3 * n * n;
    }
    c->self_matrix = !goff.empty() && total * long(sizeof(double)) <= kSelfMatrixMaxBytes;
    if (c->self_matrix) {
      CK(dalloc(c->d_selfG, size_t(total)));
      CK(upload(c->d_selfG_off, goff, s));
    }
  }
  CK(dalloc(c->d_src_pos32, 2 * slot32.size()));
  CK(dalloc(c->d_src_val32, 2 * slot32.size()));
  CK(dalloc(c->d_src_pos64, slot64.size()));
  CK(dalloc(c->d_src_val64, slot64.size()));
  CK(dalloc(c->d_src_pos_df, 2 * slot64.size()));
  CK(dalloc(c->d_src_val_df, 2 * slot64.size()));
  CK(dalloc(c->d_h_slp, size_t(2) * n_ves));
  CK(dalloc(c->d_h_dlp, size_t(2) * n_wall));
  CK(dalloc(c->d_h_out, size_t(2) * N));
  for (auto &kv : kress_off) CK(launch_kress_table(kv.first, c->d_kress + kv.second, s));
  CK(launch_geom_prep(c, s));
  CK(cudaStreamSynchronize(s));

  c->have_geom = true;
  c->splits_f32 = default_splits(c, STOKES_FP32_KAHAN);
  c->splits_f64 = default_splits(c, STOKES_FP64);
  c->splits_df = default_splits(c, STOKES_DOUBLE_FLOAT);
  tune_apply_cached(c);
  int st = ensure_partial(c, size_t(std::max({c->splits_f32, c->splits_f64, c->splits_df})) * N);
  if (st) return st;
  st = read_status(c, s);
  if (st) {
    free_geometry(c);
    return fail(c, STOKES_ERR_NONFINITE, "non-finite geometry value");
  }
  return STOKES_OK;
}

}  // namespace stokes

extern "C" {

int stokes_geom_set(stokes_ctx *c, int n_curves, const int32_t *curve_offset,
                    const int32_t *curve_kind, const double *nodes, const double *weights,
                    const double *normals, const double *curvature, double period, double mu,
                    void *stream) {
  if (!c) return STOKES_ERR_ARG;
  CK(cudaSetDevice(c->device));
  const int inst_off[2] = {0, n_curves};
  return set_geometry(c, 1, inst_off, &period, n_curves, curve_offset, curve_kind, nodes, weights,
                      normals, curvature, mu, as_stream(stream));
}

int stokes_geom_update(stokes_ctx *c, const double *nodes, const double *weights,
                       const double *normals, const double *curvature, void *stream) {
  if (!c) return STOKES_ERR_ARG;
  if (!c->have_geom) return fail(c, STOKES_ERR_NO_GEOM, "no geometry set");
  if (!nodes || !weights || !normals || !aligned16(nodes) || !aligned16(normals))
    return fail(c, STOKES_ERR_ARG, "nodes, weights and normals must be device pointers (16-byte aligned 2-vectors)");
  if (c->n_wall_nodes > 0 && !curvature)
    return fail(c, STOKES_ERR_ARG, "curvature is required when walls are present");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = as_stream(stream);
  const int N = c->N;
  // FMM and close-evaluation plans hold positions of the old geometry: they no longer apply
  fmm_geometry_changed(c);
  CK(cudaMemcpyAsync(c->d_x, nodes, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(c->d_nrm, normals, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(c->d_w, weights, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  if (curvature) CK(cudaMemcpyAsync(c->d_kap, curvature, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  CK(launch_geom_prep(c, s));
  for (auto &g : c->graph_exec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  return STOKES_OK;
}

int stokes_sum_eval(stokes_ctx *c, int precision, const double *slp, const double *dlp,
                    double jump, double *out, void *stream) {
  if (!c) return STOKES_ERR_ARG;
  int st = check_density_args(c, precision, slp, dlp);
  if (st) return st;
  if (!out || !aligned16(out)) return fail(c, STOKES_ERR_ARG, "out_velocity must be a 16-byte aligned device pointer");
  if (!isfinite(jump)) return fail(c, STOKES_ERR_ARG, "jump must be finite");
  CK(cudaSetDevice(c->device));
  return run_nodes(c, precision, slp, dlp, jump, out, as_stream(stream));
}

int stokes_sum_eval_targets(stokes_ctx *c, int precision, const double *slp, const double *dlp,
                            int n_targets, const double *targets, double *out, void *stream) {
  if (!c) return STOKES_ERR_ARG;
  int st = check_density_args(c, precision, slp, dlp);
  if (st) return st;
  if (n_targets < 0) return fail(c, STOKES_ERR_ARG, "n_targets < 0");
  if (n_targets == 0) return STOKES_OK;
  if (!targets || !out || !aligned16(targets) || !aligned16(out))
    return fail(c, STOKES_ERR_ARG, "targets and out_velocity must be 16-byte aligned device pointers");
  if (c->n_inst > 1)
    return fail(c, STOKES_ERR_ARG, "free-point evaluation needs a single-instance geometry");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = as_stream(stream);
  int splits = splits_of(c, precision);
  st = ensure_partial(c, size_t(splits) * n_targets);
  if (st) return st;
  MARK(0);
  CK(launch_pack(c, precision, slp, dlp, s));
  MARK(1);
  CK(launch_pair(c, precision, n_targets, reinterpret_cast<const double2 *>(targets), nullptr,
                 splits, c->d_partial, s));
  MARK(2);
  CK(launch_finish_free(c, splits, n_targets, reinterpret_cast<double2 *>(out), s));
  MARK(3);
  return STOKES_OK;
}

}  // extern "C"

namespace {

// Pressure (tnrm == NULL) or traction of the layer potentials at free points, FP64.
int field_eval(stokes_ctx *c, const double *slp, const double *dlp, int n_targets,
               const double *targets, const double *tnrm, double *out, void *stream) {
  if (!c) return STOKES_ERR_ARG;
  int st = check_density_args(c, STOKES_FP64, slp, dlp);
  if (st) return st;
  if (n_targets < 0) return fail(c, STOKES_ERR_ARG, "n_targets < 0");
  if (n_targets == 0) return STOKES_OK;
  if (!targets || !out || !aligned16(targets) || (tnrm && !aligned16(tnrm)) ||
      (reinterpret_cast<uintptr_t>(out) & 7u))
    return fail(c, STOKES_ERR_ARG, "targets (and normals) must be 16-byte aligned device pointers, "
                                   "the output 8-byte aligned");
  if (c->n_inst > 1)
    return fail(c, STOKES_ERR_ARG, "free-point evaluation needs a single-instance geometry");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = as_stream(stream);
  const int splits = field_splits(c, n_targets);
  st = ensure_partial(c, size_t(splits) * n_targets);
  if (st) return st;
  CK(launch_pack(c, STOKES_FP64, slp, dlp, s));
  CK(launch_field(c, n_targets, reinterpret_cast<const double2 *>(targets),
                  reinterpret_cast<const double2 *>(tnrm), splits, out, s));
  return STOKES_OK;
}

}  // namespace

extern "C" {

int stokes_check_wait_timeout(stokes_ctx *c, void *stream) {
  if (!c) return STOKES_ERR_ARG;
  CK(cudaSetDevice(c->device));
  CK(launch_wait_timeout_check(c, as_stream(stream)));
  return STOKES_OK;
}

int stokes_check_log64(stokes_ctx *c, const double *x, int n, double *out, void *stream) {
  if (!c) return STOKES_ERR_ARG;
  if (n < 0) return fail(c, STOKES_ERR_ARG, "n < 0");
  if (n == 0) return STOKES_OK;
  if (!x || !out) return fail(c, STOKES_ERR_ARG, "x and out must be device pointers");
  CK(cudaSetDevice(c->device));
  CK(launch_check_log64(c, n, x, out, as_stream(stream)));
  return STOKES_OK;
}

int stokes_sum_eval_pressure(stokes_ctx *c, const double *slp, const double *dlp, int n_targets,
                             const double *targets, double *out_pressure, void *stream) {
  return field_eval(c, slp, dlp, n_targets, targets, nullptr, out_pressure, stream);
}

int stokes_sum_eval_traction(stokes_ctx *c, const double *slp, const double *dlp, int n_targets,
                             const double *targets, const double *target_normals,
                             double *out_traction, void *stream) {
  if (c && !target_normals && n_targets > 0)
    return fail(c, STOKES_ERR_ARG, "target_normals is NULL");
  return field_eval(c, slp, dlp, n_targets, targets, target_normals, out_traction, stream);
}

int stokes_sum_eval_host(stokes_ctx *c, int precision, const double *slp_h, const double *dlp_h,
                         double jump, double *out_h) {
  if (!c) return STOKES_ERR_ARG;
  int st = check_density_args(c, precision, slp_h, dlp_h);
  if (st) return st;
  if (!out_h) return fail(c, STOKES_ERR_ARG, "out_host is NULL");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = c->own_stream;
  if (c->n_ves_nodes)
    CK(cudaMemcpyAsync(c->d_h_slp, slp_h, sizeof(double) * 2 * c->n_ves_nodes, cudaMemcpyHostToDevice, s));
  if (c->n_wall_nodes)
    CK(cudaMemcpyAsync(c->d_h_dlp, dlp_h, sizeof(double) * 2 * c->n_wall_nodes, cudaMemcpyHostToDevice, s));
  st = run_nodes(c, precision, c->d_h_slp, c->d_h_dlp, jump, c->d_h_out, s);
  if (st) return st;
  CK(cudaMemcpyAsync(out_h, c->d_h_out, sizeof(double) * 2 * c->N, cudaMemcpyDeviceToHost, s));
  return read_status(c, s);
}

int stokes_sync(stokes_ctx *c, void *stream) {
  if (!c) return STOKES_ERR_ARG;
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize(as_stream(stream)));
  return read_status(c, as_stream(stream));
}

int stokes_set_launch(stokes_ctx *c, int precision, int splits, int targets_per_thread,
                      int kahan_group) {
  if (!c) return STOKES_ERR_ARG;
  if (!c->have_geom) return fail(c, STOKES_ERR_NO_GEOM, "no geometry set");
  if (precision != STOKES_FP64 && precision != STOKES_FP32_KAHAN &&
      precision != STOKES_DOUBLE_FLOAT)
    return fail(c, STOKES_ERR_ARG, "unknown precision %d", precision);
  if (splits < 0) return fail(c, STOKES_ERR_ARG, "source_splits < 0");
  if (c->n_inst > 1)
    return fail(c, STOKES_ERR_ARG, "batched geometry: use stokes_batch_set_shape");
  if (targets_per_thread != 0 && targets_per_thread != 1 && targets_per_thread != 2 &&
      targets_per_thread != 4)
    return fail(c, STOKES_ERR_ARG, "targets_per_thread must be 0, 1, 2 or 4");
  if (kahan_group != 0 && kahan_group != 1 && kahan_group != 2 && kahan_group != 4 &&
      kahan_group != 8 && kahan_group != 16)
    return fail(c, STOKES_ERR_ARG, "kahan_group must be 0, 1, 2, 4, 8 or 16");
  CK(cudaSetDevice(c->device));
  if (precision == STOKES_FP32_KAHAN) {
    if (targets_per_thread) c->tpt_f32 = targets_per_thread;
    if (kahan_group) c->kgroup_f32 = kahan_group;
  }
  int eff = splits ? effective_splits(c, precision, splits) : default_splits(c, precision);
  int st = ensure_partial(c, size_t(eff) * c->N);
  if (st) return st;
  invalidate_node_graph(c);
  (precision == STOKES_FP32_KAHAN ? c->splits_f32
   : precision == STOKES_FP64    ? c->splits_f64
                                 : c->splits_df) = eff;
  return STOKES_OK;
}

int stokes_set_local_frame(stokes_ctx *c, int on) {
  if (!c) return STOKES_ERR_ARG;
  c->local_frame = on != 0;
  invalidate_node_graph(c);
  return STOKES_OK;
}

int stokes_graph_stats(const stokes_ctx *c, long long *captures, long long *launches) {
  if (!c || !captures || !launches) return STOKES_ERR_ARG;
  *captures = c->graph_captures;
  *launches = c->graph_replays;
  return STOKES_OK;
}

int stokes_time_sums(stokes_ctx *c, int precision, const double *slp, const double *dlp,
                     double jump, double *out, int reps, void *stream, double *ms_per_sum) {
  if (!c || !ms_per_sum || reps < 1) return STOKES_ERR_ARG;
  int st = check_density_args(c, precision, slp, dlp);
  if (st) return st;
  if (!out || !aligned16(out)) return fail(c, STOKES_ERR_ARG, "out_velocity must be a 16-byte aligned device pointer");
  if (!isfinite(jump)) return fail(c, STOKES_ERR_ARG, "jump must be finite");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = as_stream(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int r = 0; r < reps && e == cudaSuccess && st == STOKES_OK; ++r)
    st = run_nodes(c, precision, slp, dlp, jump, out, s);
  if (e == cudaSuccess && st == STOKES_OK) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess && st == STOKES_OK) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess && st == STOKES_OK) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) return st;
  if (e != cudaSuccess) return cuda_fail(c, e, "stokes_time_sums");
  *ms_per_sum = double(ms) / reps;
  return read_status(c, s);
}

int stokes_debug_build(void) {
#ifdef STOKES_DEBUG
  return 1;
#else
  return 0;
#endif
}

int stokes_debug_tighten(stokes_ctx *c, long long elements) {
  if (!c) return STOKES_ERR_ARG;
#ifdef STOKES_DEBUG
  if (elements < 0) return fail(c, STOKES_ERR_ARG, "elements < 0");
  c->debug_tighten = elements;
  invalidate_node_graph(c);
  return STOKES_OK;
#else
  (void)elements;
  return fail(c, STOKES_ERR_ARG, "release build: no device bounds checks to tighten");
#endif
}

int stokes_set_graph_mode(stokes_ctx *c, int mode) {
  if (!c) return STOKES_ERR_ARG;
  if (mode != STOKES_GRAPH_OFF && mode != STOKES_GRAPH_SMALL && mode != STOKES_GRAPH_ALWAYS)
    return fail(c, STOKES_ERR_ARG, "unknown graph mode %d", mode);
  c->graph_mode = mode;
  invalidate_node_graph(c);
  return STOKES_OK;
}

int stokes_get_launch(const stokes_ctx *c, int precision, int *splits, int *targets_per_thread,
                      int *kahan_group) {
  if (!c || !splits || !targets_per_thread || !kahan_group) return STOKES_ERR_ARG;
  const bool f32 = precision == STOKES_FP32_KAHAN;
  *splits = splits_of(c, precision);
  *targets_per_thread = f32 ? c->tpt_f32 : precision == STOKES_DOUBLE_FLOAT ? kTptDF : 1;
  *kahan_group = f32 ? c->kgroup_f32 : 0;
  return STOKES_OK;
}

int stokes_set_profiling(stokes_ctx *c, int on) {
  if (!c) return STOKES_ERR_ARG;
  CK(cudaSetDevice(c->device));
  if (on && !c->ev[0])
    for (auto &e : c->ev) CK(cudaEventCreate(&e));
  c->profiling = on != 0;
  c->timed = false;
  return STOKES_OK;
}

int stokes_last_timing(stokes_ctx *c, double *ms) {
  if (!c || !ms) return STOKES_ERR_ARG;
  if (!c->timed) return fail(c, STOKES_ERR_ARG, "no timed call (enable stokes_set_profiling first)");
  CK(cudaSetDevice(c->device));
  CK(cudaEventSynchronize(c->ev[3]));
  for (int k = 0; k < 3; ++k) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, c->ev[k], c->ev[k + 1]));
    ms[k] = t;
  }
  return STOKES_OK;
}

int stokes_pair_count(const stokes_ctx *c, int n_targets, double *pairs) {
  if (!c || !pairs) return STOKES_ERR_ARG;
  if (!c->have_geom) return STOKES_ERR_NO_GEOM;
  const double img = c->period != 0.0 ? 3.0 : 1.0;
  if (c->n_inst > 1) {
    double p = 0.0;
    for (const auto &I : c->inst) p += img * double(I.N) * double(I.N);
    *pairs = p;
    return STOKES_OK;
  }
  const double nt = n_targets > 0 ? double(n_targets) : double(c->N);
  *pairs = img * nt * double(c->N);
  return STOKES_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batched instances
// ---------------------------------------------------------------------------
namespace {

// Item table of one precision: every instance's (target block x source split) items, with the
// split count chosen so that an item costs about total / (resident blocks x items_per_slot)
// target-tile evaluations; items sorted by cost, largest first, for the work counter.
int build_items(stokes_ctx *c, int precision, size_t *partial_elems) {
  const bool f32 = precision == STOKES_FP32_KAHAN;
  const long B = f32 ? long(kThreadsF32) * c->tpt_f32 : long(kThreadsF64);
  const long slots = long(pair_batch_blocks_per_sm(c, precision)) * std::max(c->num_sms, 1);
  const int ips = f32 ? c->batch_ips32 : c->batch_ips64;
  double total = 0.0;
  for (const auto &I : c->inst) {
    const long T = f32 ? I.nw32 + I.nv32 : I.nw64 + I.nv64;
    total += double((I.N + B - 1) / B) * double(B) * double(T);
  }
  const double target = std::max(1.0, total / double(slots * std::max(ips, 1)));
  const long tps_goal = std::max(1L, long(target / double(B)));
  std::vector<ItemDesc> items;
  long long off = 0;
  for (auto &I : c->inst) {
    const int T = f32 ? I.nw32 + I.nv32 : I.nw64 + I.nv64;
    int splits = int(std::min<long>(T, std::max<long>(1, (T + tps_goal - 1) / tps_goal)));
    const int tps = (T + splits - 1) / splits;
    splits = (T + tps - 1) / tps;
    (f32 ? I.splits32 : I.splits64) = splits;
    (f32 ? I.part_off32 : I.part_off64) = off;
    for (int t0 = 0; t0 < I.N; t0 += int(B)) {
      for (int k = 0; k < splits; ++k) {
        ItemDesc it{};
        it.tgt_begin = I.node_begin + t0;
        it.tgt_count = int(std::min<long>(B, I.N - t0));
        it.vt_begin = k * tps;
        it.vt_end = std::min(T, (k + 1) * tps);
        it.wb = f32 ? I.wb32 : I.wb64;
        it.nw = f32 ? I.nw32 : I.nw64;
        it.vb = f32 ? I.vb32 : I.vb64;
        it.part_off = off + (long long)k * I.N - I.node_begin;
        it.period = I.period;
        items.push_back(it);
      }
    }
    off += (long long)splits * I.N;
  }
  std::stable_sort(items.begin(), items.end(), [](const ItemDesc &x, const ItemDesc &y) {
    return (long long)x.tgt_count * (x.vt_end - x.vt_begin) >
           (long long)y.tgt_count * (y.vt_end - y.vt_begin);
  });
  ItemDesc *&dst = f32 ? c->d_items32 : c->d_items64;
  dfree(dst);
  CK(upload(dst, items, c->own_stream));
  (f32 ? c->n_items32 : c->n_items64) = int(items.size());
  (f32 ? c->batch_part32 : c->batch_part64) = off;
  *partial_elems = size_t(off);
  return STOKES_OK;
}

int build_batch_tables(stokes_ctx *c) {
  size_t p32 = 0, p64 = 0;
  int st = build_items(c, STOKES_FP32_KAHAN, &p32);
  if (st) return st;
  st = build_items(c, STOKES_FP64, &p64);
  if (st) return st;
  dfree(c->d_inst);
  CK(upload(c->d_inst, c->inst, c->own_stream));
  if (!c->d_counter) CK(dalloc(c->d_counter, 1));
  CK(cudaStreamSynchronize(c->own_stream));
  st = ensure_partial(c, std::max(p32, p64));
  if (st) return st;
  for (auto &g : c->graph_exec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  return STOKES_OK;
}

int capture_batch_graph(stokes_ctx *c, int precision, double jump) {
  const int k = precision;
  if (c->graph_exec[k] && c->graph_jump[k] == jump) return STOKES_OK;
  if (c->graph_exec[k]) {
    cudaGraphExecDestroy(c->graph_exec[k]);
    c->graph_exec[k] = nullptr;
  }
  if (!c->d_b_out) {
    CK(dalloc(c->d_b_slp, size_t(2) * std::max(c->n_ves_nodes, 1)));
    CK(dalloc(c->d_b_dlp, size_t(2) * std::max(c->n_wall_nodes, 1)));
    CK(dalloc(c->d_b_out, size_t(2) * c->N));
  }
  const bool prof = c->profiling;
  c->profiling = false;  // events of the timing API stay outside the graph
  cudaStream_t s = c->own_stream;
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int st = run_batch(c, precision, c->d_b_slp, c->d_b_dlp, jump, c->d_b_out, s);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &graph);
  c->profiling = prof;
  if (st) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  const cudaError_t e2 = cudaGraphInstantiate(&c->graph_exec[k], graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaGraphInstantiate");
  c->graph_jump[k] = jump;
  return STOKES_OK;
}

}  // namespace

extern "C" {

int stokes_batch_set(stokes_ctx *c, int n_inst, const int32_t *inst_curve_offset, int n_curves,
                     const int32_t *curve_offset, const int32_t *curve_kind, const double *nodes,
                     const double *weights, const double *normals, const double *curvature,
                     const double *periods, double mu, void *stream) {
  if (!c) return STOKES_ERR_ARG;
  if (n_inst < 1 || !inst_curve_offset || !periods)
    return fail(c, STOKES_ERR_ARG, "need n_inst >= 1 and host inst_curve_offset / periods");
  CK(cudaSetDevice(c->device));
  int st = set_geometry(c, n_inst, inst_curve_offset, periods, n_curves, curve_offset, curve_kind,
                        nodes, weights, normals, curvature, mu, as_stream(stream));
  if (st) return st;
  if (n_inst == 1) return STOKES_OK;
  return build_batch_tables(c);
}

int stokes_batch_set_shape(stokes_ctx *c, int precision, int targets_per_thread,
                           int items_per_slot) {
  if (!c) return STOKES_ERR_ARG;
  if (!c->have_geom || c->n_inst < 2) return fail(c, STOKES_ERR_NO_GEOM, "no batched geometry set");
  if (precision != STOKES_FP64 && precision != STOKES_FP32_KAHAN &&
      precision != STOKES_DOUBLE_FLOAT)
    return fail(c, STOKES_ERR_ARG, "unknown precision %d", precision);
  if (targets_per_thread != 0 && targets_per_thread != 1 && targets_per_thread != 2 &&
      targets_per_thread != 4)
    return fail(c, STOKES_ERR_ARG, "targets_per_thread must be 0, 1, 2 or 4");
  if (items_per_slot < 0 || items_per_slot > 64)
    return fail(c, STOKES_ERR_ARG, "items_per_slot must be in [0, 64]");
  CK(cudaSetDevice(c->device));
  if (precision == STOKES_FP32_KAHAN) {
    if (targets_per_thread) c->tpt_f32 = targets_per_thread;
    if (items_per_slot) c->batch_ips32 = items_per_slot;
  } else if (items_per_slot) {
    c->batch_ips64 = items_per_slot;
  }
  return build_batch_tables(c);
}

int stokes_batch_info(const stokes_ctx *c, int precision, int *n_items, int *blocks,
                      int *targets_per_thread, int *items_per_slot) {
  if (!c || !n_items || !blocks || !targets_per_thread || !items_per_slot) return STOKES_ERR_ARG;
  if (!c->have_geom || c->n_inst < 2) return STOKES_ERR_NO_GEOM;
  const bool f32 = precision == STOKES_FP32_KAHAN;
  *n_items = f32 ? c->n_items32 : c->n_items64;
  *blocks = pair_batch_blocks_per_sm(const_cast<stokes_ctx *>(c), precision) * std::max(c->num_sms, 1);
  *targets_per_thread = f32 ? c->tpt_f32 : precision == STOKES_DOUBLE_FLOAT ? kTptDF : 1;
  *items_per_slot = f32 ? c->batch_ips32 : c->batch_ips64;
  return STOKES_OK;
}

int stokes_batch_eval(stokes_ctx *c, int precision, const double *slp, const double *dlp,
                      double jump, double *out, int use_graph, void *stream) {
  if (!c) return STOKES_ERR_ARG;
  int st = check_density_args(c, precision, slp, dlp);
  if (st) return st;
  if (c->n_inst < 2) return fail(c, STOKES_ERR_NO_GEOM, "no batched geometry set");
  if (!out || !aligned16(out)) return fail(c, STOKES_ERR_ARG, "out_velocity must be a 16-byte aligned device pointer");
  if (!isfinite(jump)) return fail(c, STOKES_ERR_ARG, "jump must be finite");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = as_stream(stream);
  if (!use_graph) return run_batch(c, precision, slp, dlp, jump, out, s);
  st = capture_batch_graph(c, precision, jump);
  if (st) return st;
  if (c->n_ves_nodes)
    CK(cudaMemcpyAsync(c->d_b_slp, slp, sizeof(double) * 2 * c->n_ves_nodes, cudaMemcpyDeviceToDevice, s));
  if (c->n_wall_nodes)
    CK(cudaMemcpyAsync(c->d_b_dlp, dlp, sizeof(double) * 2 * c->n_wall_nodes, cudaMemcpyDeviceToDevice, s));
  CK(cudaGraphLaunch(c->graph_exec[precision], s));
  CK(cudaMemcpyAsync(out, c->d_b_out, sizeof(double) * 2 * c->N, cudaMemcpyDeviceToDevice, s));
  return STOKES_OK;
}

}  // extern "C"
