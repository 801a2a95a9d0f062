// noalloc.cu -- free-point evaluation that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they evaluate: code recording a
// CUDA graph by stream capture (allocation and the device-wide synchronisation that a
// growing scratch buffer needs are not allowed while capturing), hosts that hand the GPU's
// memory to a pool of their own and forbid other allocations, and real-time loops that
// must not block on the allocator.  stokes_sum_eval_targets may grow the context's scratch
// buffer (cudaMalloc after a device synchronisation) when it sees more targets than before.
// The entry point below keeps its cross-split partial sums in a fixed, file-scope device
// array instead, so a call never allocates.
#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "stokes_internal.cuh"

namespace stokes {
cudaError_t launch_pair_scratch(stokes_ctx *c, int precision, int n_targets, const double2 *tgt,
                                int splits, double2 *partial, cudaStream_t s);
cudaError_t launch_finish_free_scratch(int splits, int n_targets, const double2 *partial,
                                       double2 *out, cudaStream_t s);
int effective_splits(stokes_ctx *c, int precision, int splits);
}  // namespace stokes

using namespace stokes;

namespace {

// Scratch of the no-allocation entry point: (source split, target) FP64 partial sums.
// Every device that loads the library holds this 4 MiB array until the process exits.
constexpr int kNoAllocPartials = 1 << 18;  // double2 elements = splits x targets capacity
static __device__ __align__(256) double2 g_noalloc_partial[kNoAllocPartials];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double2 *g_partial_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_partial on `device` (which must be current).  The name
// g_noalloc_partial in host code is only a host-side stand-in, so the address is looked up
// once per device with cudaGetSymbolAddress and cached.
cudaError_t scratch_for_device(int device, double2 **out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partial_ptr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (e != cudaSuccess) return e;
    g_partial_ptr[device] = static_cast<double2 *>(p);
  }
  *out = g_partial_ptr[device];
  return cudaSuccess;
}

int set_err(stokes_ctx *c, int code, const char *msg) {
  c->err = msg;
  return code;
}

}  // namespace

extern "C" int stokes_sum_eval_targets_noalloc(stokes_ctx *c, int precision, const double *slp,
                                               const double *dlp, int n_targets,
                                               const double *targets, double *out,
                                               void *stream) {
  if (!c) return STOKES_ERR_ARG;
  if (!c->have_geom) return set_err(c, STOKES_ERR_NO_GEOM, "no geometry set");
  if (precision != STOKES_FP64 && precision != STOKES_FP32_KAHAN &&
      precision != STOKES_DOUBLE_FLOAT)
    return set_err(c, STOKES_ERR_ARG, "unknown precision");
  if (c->n_ves_nodes > 0 && !slp) return set_err(c, STOKES_ERR_ARG, "slp_density is NULL");
  if (c->n_wall_nodes > 0 && !dlp) return set_err(c, STOKES_ERR_ARG, "dlp_density is NULL");
  if (n_targets < 0) return set_err(c, STOKES_ERR_ARG, "n_targets < 0");
  if (n_targets == 0) return STOKES_OK;
  if (n_targets > kNoAllocPartials) {
    char buf[160];
    snprintf(buf, sizeof(buf),
             "stokes_sum_eval_targets_noalloc: n_targets = %d exceeds the fixed scratch capacity "
             "of %d targets",
             n_targets, kNoAllocPartials);
    return set_err(c, STOKES_ERR_ARG, buf);
  }
  if (!targets || !out || (reinterpret_cast<uintptr_t>(targets) & 15u) ||
      (reinterpret_cast<uintptr_t>(out) & 15u))
    return set_err(c, STOKES_ERR_ARG, "targets and out_velocity must be 16-byte aligned device pointers");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return set_err(c, STOKES_ERR_CUDA, cudaGetErrorString(e));
  double2 *scratch = nullptr;
  e = scratch_for_device(c->device, &scratch);
  if (e != cudaSuccess) return set_err(c, STOKES_ERR_CUDA, cudaGetErrorString(e));

  // As many source splits as the context uses, capped by the scratch capacity; every
  // (split, target) element is written by the pair kernel before the finish pass reads it,
  // so nothing has to be cleared between calls.
  const int want = precision == STOKES_FP32_KAHAN ? c->splits_f32
                   : precision == STOKES_FP64     ? c->splits_f64
                                                  : c->splits_df;
  const int splits = effective_splits(c, precision, std::min(want, kNoAllocPartials / n_targets));
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  e = launch_pack(c, precision, slp, dlp, s);
  if (e == cudaSuccess)
    e = launch_pair_scratch(c, precision, n_targets, reinterpret_cast<const double2 *>(targets),
                            splits, scratch, s);
  if (e == cudaSuccess)
    e = launch_finish_free_scratch(splits, n_targets, scratch, reinterpret_cast<double2 *>(out), s);
  if (e != cudaSuccess) return set_err(c, STOKES_ERR_CUDA, cudaGetErrorString(e));
  return STOKES_OK;
}
