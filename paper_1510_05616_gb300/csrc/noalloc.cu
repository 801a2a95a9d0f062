// noalloc.cu -- free-point evaluation that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they evaluate: hosts that hand all
// of the GPU's memory to a pool of their own and forbid other allocations, plug-ins that run
// inside such a host with a fixed memory budget, and real-time loops that must not block on
// the allocator.  stokes_sum_eval_targets may grow the context's scratch buffer (cudaMalloc
// after a device synchronisation) when it sees more targets than before.  The entry point
// below keeps its cross-split partial sums in a fixed, file-scope device array instead, so a
// call never allocates.
#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "stokes_internal.cuh"

namespace stokes {
cudaError_t launch_finish_free_scratch(int splits, int n_targets, const double2 *partial,
                                       double2 *out, cudaStream_t s);
int effective_splits(stokes_ctx *c, int precision, int splits);
void noalloc_setup_device(int device);
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

// Looks up the device address of g_noalloc_partial on `device` (which must be current) and
// caches it.  The name g_noalloc_partial in host code is only a host-side stand-in, so host
// code must pass this looked-up address to the kernels.
cudaError_t lookup_locked(int device) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
  if (e != cudaSuccess) return e;
  g_partial_ptr[device] = static_cast<double2 *>(p);
  return cudaSuccess;
}

// The cached address for `device` (current), looked up now if no context creation has yet.
cudaError_t scratch_for_device(int device, double2 **out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partial_ptr[device]) {
    const cudaError_t e = lookup_locked(device);
    if (e != cudaSuccess) return e;
  }
  *out = g_partial_ptr[device];
  return cudaSuccess;
}

int set_err(stokes_ctx *c, int code, const char *msg) {
  c->err = msg;
  return code;
}

// Profiling events of the three phases, as the allocating entry point records them.
cudaError_t mark(stokes_ctx *c, int k, cudaStream_t s) {
  if (!c->profiling) return cudaSuccess;
  const cudaError_t e = cudaEventRecord(c->ev[k], s);
  if (e == cudaSuccess && k == 3) c->timed = true;
  return e;
}

}  // namespace

namespace stokes {

// Called by stokes_create with `device` current: (re)reads the array's device address, so a
// context created after a cudaDeviceReset (which unloads the module and with it the array)
// never sees an address from before the reset.  A failed lookup leaves the entry empty; the
// entry point then retries and reports the error itself.
void noalloc_setup_device(int device) {
  if (device < 0 || device >= kMaxDevices) return;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  g_partial_ptr[device] = nullptr;
  (void)lookup_locked(device);
}

}  // namespace stokes

extern "C" int stokes_sum_eval_targets_noalloc(stokes_ctx *c, int precision, const double *slp,
                                               const double *dlp, int n_targets,
                                               const double *targets, double *out,
                                               void *stream) {
  if (!c) return STOKES_ERR_ARG;
  if (!c->have_geom) return set_err(c, STOKES_ERR_NO_GEOM, "no geometry set");
  if (c->n_inst > 1)
    return set_err(c, STOKES_ERR_ARG, "free-point evaluation needs a single-instance geometry");
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
  e = mark(c, 0, s);
  if (e == cudaSuccess) e = launch_pack(c, precision, slp, dlp, s);
  if (e == cudaSuccess) e = mark(c, 1, s);
  if (e == cudaSuccess)
    e = launch_pair(c, precision, n_targets, reinterpret_cast<const double2 *>(targets), nullptr,
                    splits, scratch, s);
  if (e == cudaSuccess) e = mark(c, 2, s);
  if (e == cudaSuccess)
    e = launch_finish_free_scratch(splits, n_targets, scratch, reinterpret_cast<double2 *>(out), s);
  if (e == cudaSuccess) e = mark(c, 3, s);
  if (e != cudaSuccess) return set_err(c, STOKES_ERR_CUDA, cudaGetErrorString(e));
  return STOKES_OK;
}
