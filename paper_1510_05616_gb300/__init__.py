"""GB300-native periodized 2-D Stokes layer-potential sum (Marple, Barnett, Gillman,
Veerapaneni): Python binding of the C ABI in ``include/stokes.h``.

The functions below carry the C names and only marshal arguments (torch tensors -> device
pointers, current CUDA stream -> cudaStream_t); every step of the sum runs in libstokes'
CUDA kernels.  There is no CPU fallback: without the built library or a CUDA device the
calls raise :class:`StokesError`.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# STOKES_LIBRARY=debug selects libstokes_debug.so (device bounds checks, -DSTOKES_DEBUG)
LIB_PATH = os.path.join(HERE, "libstokes_debug.so" if os.environ.get("STOKES_LIBRARY") == "debug"
                        else "libstokes.so")

STOKES_OK = 0
STOKES_ERR_ARG = -1
STOKES_ERR_CUDA = -2
STOKES_ERR_NO_GEOM = -3
STOKES_ERR_ODD_N = -4
STOKES_ERR_NONFINITE = -5
STOKES_ERR_TIMEOUT = -6
STOKES_ERR_NOT_CONVERGED = -7
STOKES_ERR_OOM = -8
STOKES_ERR_BOUNDS = -9

STOKES_FP64 = 0
STOKES_FP32_KAHAN = 1
STOKES_DOUBLE_FLOAT = 2
STOKES_KIND_WALL = 0
STOKES_KIND_VESICLE = 1

STOKES_GUESS_ZERO = 0
STOKES_GUESS_PREVIOUS = 1
STOKES_GUESS_MLP = 2
STOKES_GUESS_USER = 3
STOKES_GUESS_EXTRAPOLATE = 4
STOKES_WARM_BASE_PREVIOUS = 0
STOKES_WARM_BASE_EXTRAPOLATE = 1
STOKES_GRAPH_OFF = 0
STOKES_GRAPH_SMALL = 1
STOKES_GRAPH_ALWAYS = 2
STOKES_WALLS_LU64 = 0
STOKES_WALLS_LU32_REFINE = 1
STOKES_WALLS_FDS = 2
N_FEATURES = 64
N_TARGETS = 48

PRECISIONS = {"fp64": STOKES_FP64, "fp32k": STOKES_FP32_KAHAN, "df": STOKES_DOUBLE_FLOAT}


class StokesError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("libstokes status %d: %s" % (code, msg))
        self.code = code


_lib = None

_c_int, _c_double, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
_SIGNATURES = {
    "stokes_create": [_c_int, ctypes.POINTER(_vp)],
    "stokes_destroy": [_vp],
    "stokes_last_error": [_vp, ctypes.c_char_p, ctypes.c_size_t],
    "stokes_geom_set": [_vp, _c_int, _vp, _vp, _vp, _vp, _vp, _vp, _c_double, _c_double, _vp],
    "stokes_sum_eval": [_vp, _c_int, _vp, _vp, _c_double, _vp, _vp],
    "stokes_geom_update": [_vp, _vp, _vp, _vp, _vp, _vp],
    "stokes_sum_eval_targets": [_vp, _c_int, _vp, _vp, _c_int, _vp, _vp, _vp],
    "stokes_sum_eval_host": [_vp, _c_int, _vp, _vp, _c_double, _vp],
    "stokes_sum_eval_targets_noalloc": [_vp, _c_int, _vp, _vp, _c_int, _vp, _vp, _vp],
    "stokes_sync": [_vp, _vp],
    "stokes_check_wait_timeout": [_vp, _vp],
    "stokes_check_log64": [_vp, _vp, _c_int, _vp, _vp],
    "stokes_set_graph_mode": [_vp, _c_int],
    "stokes_debug_build": [],
    "stokes_graph_stats": [_vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)],
    "stokes_time_sums": [_vp, _c_int, _vp, _vp, _c_double, _vp, _c_int, _vp, ctypes.POINTER(_c_double)],
    "stokes_debug_tighten": [_vp, ctypes.c_longlong],
    "stokes_fmm_create": [_vp, _c_int, _c_int, ctypes.POINTER(_vp)],
    "stokes_fmm_eval": [_vp, _vp, _vp, _c_double, _vp, _vp],
    "stokes_fmm_get_info": [_vp, _vp],
    "stokes_fmm_create_targets": [_vp, _c_int, _c_int, _c_int, _vp, _vp],
    "stokes_fmm_create_targets_only": [_vp, _c_int, _c_int, _c_int, _vp, _vp],
    "stokes_fmm_eval_targets": [_vp, _vp, _vp, _vp, _vp],
    "stokes_fmm_set_eval_order": [_vp, _c_int],
    "stokes_fmm_set_precision": [_vp, _c_int],
    "stokes_fmm_last_error": [_vp, ctypes.c_char_p, ctypes.c_size_t],
    "stokes_fmm_destroy": [_vp],
    "stokes_close_create": [_vp, _c_double, _c_int, ctypes.POINTER(_vp)],
    "stokes_close_eval": [_vp, _vp, _vp, _vp],
    "stokes_close_get_info": [_vp, _vp],
    "stokes_close_last_error": [_vp, ctypes.c_char_p, ctypes.c_size_t],
    "stokes_close_destroy": [_vp],
    "stokes_num_nodes": [_vp],
    "stokes_set_launch": [_vp, _c_int, _c_int, _c_int, _c_int],
    "stokes_get_launch": [_vp, _c_int, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                          ctypes.POINTER(_c_int)],
    "stokes_pair_count": [_vp, _c_int, ctypes.POINTER(_c_double)],
    "stokes_set_profiling": [_vp, _c_int],
    "stokes_batch_set": [_vp, _c_int, _vp, _c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _c_double,
                         _vp],
    "stokes_batch_eval": [_vp, _c_int, _vp, _vp, _c_double, _vp, _c_int, _vp],
    "stokes_batch_set_shape": [_vp, _c_int, _c_int, _c_int],
    "stokes_batch_info": [_vp, _c_int] + [ctypes.POINTER(_c_int)] * 4,
    "stokes_sim_create": [_c_int, ctypes.POINTER(_vp)],
    "stokes_sim_destroy": [_vp],
    "stokes_sim_last_error": [_vp, ctypes.c_char_p, ctypes.c_size_t],
    "stokes_sim_set_walls": [_vp, _c_int, _vp, _vp, _vp, _vp, _c_double, _c_double, _c_int, _c_int,
                             _c_double],
    "stokes_sim_set_vesicles": [_vp, _c_int, _c_int, _vp, _c_double, _c_double, _c_double],
    "stokes_sim_channel_response": [_vp, _vp, _c_double, _vp],
    "stokes_sim_set_wall_solver": [_vp, _c_int],
    "stokes_sim_set_block_refinement": [_vp, _c_int],
    "stokes_sim_set_precond_precision": [_vp, _c_int],
    "stokes_sim_set_precond_refresh": [_vp, _c_int],
    "stokes_sim_set_precond_tensor": [_vp, _c_int],
    "stokes_sim_set_inner_tolerance": [_vp, _c_double],
    "stokes_sim_set_residual_fmm": [_vp, _c_int, _c_int],
    "stokes_sim_set_sweep_fmm": [_vp, _c_int],
    "stokes_sim_set_close_eval": [_vp, _c_double, _c_int],
    "stokes_sim_set_warm_modes": [_vp, _c_int],
    "stokes_sim_set_warm_history": [_vp, _c_int],
    "stokes_sim_set_warm_base": [_vp, _c_int],
    "stokes_sim_get_warm_modes": [_vp, ctypes.POINTER(_c_int)],
    "stokes_sim_empty_channel_pressure": [_vp, _c_double, _vp, _c_int, _vp, _vp],
    "stokes_sum_eval_pressure": [_vp, _vp, _vp, _c_int, _vp, _vp, _vp],
    "stokes_sum_eval_traction": [_vp, _vp, _vp, _c_int, _vp, _vp, _vp, _vp],
    "stokes_sim_wall_stats": [_vp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_double)],
    "stokes_sim_set_fds_params": [_vp, _c_double, _c_int, _c_int],
    "stokes_sim_wall_solve": [_vp, _vp, _c_int],
    "stokes_sim_fds_info": [_vp, _vp],
    "stokes_sim_set_fds_recompress": [_vp, _c_int],
    "stokes_sim_empty_channel": [_vp, _c_double, _vp, _c_int, _vp, _vp],
    "vesicle_step_warmstart": [_vp, _c_double, _c_double, _c_int, _vp, _vp, _c_double, _c_int,
                               _c_int, _vp],
    "stokes_sim_last_features": [_vp, _vp, _vp],
    "stokes_mlp_create": [_c_int, _c_int, _c_int, _c_int, ctypes.POINTER(_vp)],
    "stokes_mlp_destroy": [_vp],
    "stokes_mlp_last_error": [_vp, ctypes.c_char_p, ctypes.c_size_t],
    "stokes_mlp_num_params": [_vp],
    "stokes_mlp_get_dims": [_vp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)],
    "stokes_mlp_set_params": [_vp, _vp],
    "stokes_mlp_get_params": [_vp, _vp],
    "stokes_mlp_set_normalization": [_vp, _vp],
    "stokes_mlp_get_normalization": [_vp, _vp],
    "stokes_mlp_fit_normalization": [_vp, _c_int, _vp, _vp],
    "stokes_mlp_forward": [_vp, _c_int, _vp, _vp],
    "stokes_mlp_loss_grad": [_vp, _c_int, _vp, _vp, _vp, _c_int, _vp, _vp],
    "stokes_mlp_train_step": [_vp, _c_int, _vp, _vp, _vp, _c_int, ctypes.c_float, _vp],
    "stokes_sim_get_state": [_vp, _vp, _vp, _vp],
    "stokes_sim_set_state": [_vp, _vp, _vp],
    "stokes_sim_sizes": [_vp] + [ctypes.POINTER(_c_int)] * 3,
    "stokes_sim_set_restart": [_vp, _c_int],
    "stokes_sim_get_history": [_vp, _vp, _vp, _vp, _vp],
    "stokes_sim_set_history": [_vp, _vp, _vp, _vp, _vp],
    "stokes_mlp_get_adam": [_vp, _vp, _vp, ctypes.POINTER(_c_int)],
    "stokes_mlp_set_adam": [_vp, _vp, _vp, _c_int],
    "stokes_last_timing": [_vp, ctypes.POINTER(_c_double)],
    "stokes_set_local_frame": [_vp, _c_int],
    "stokes_autotune": [_vp, _c_int, _c_int, _vp, _vp],
    "stokes_tune_lookup": [_c_int] * 6 + [_vp],
    "stokes_tune_save": [ctypes.c_char_p],
    "stokes_tune_load": [ctypes.c_char_p],
    "stokes_tune_clear": [],
}


def library_path() -> str:
    return LIB_PATH


def load() -> ctypes.CDLL:
    """Load the in-tree libstokes.so (built by ``build.build()``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise StokesError(STOKES_ERR_CUDA, "%s is not built" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, argt in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = argt
            fn.restype = _c_int
        _lib = lib
    return _lib


def _err(h) -> str:
    buf = ctypes.create_string_buffer(512)
    if h:
        load().stokes_last_error(h, buf, 512)
    return buf.value.decode(errors="replace")


def _check(h, code: int):
    if code != STOKES_OK:
        raise StokesError(code, _err(h))
    return code


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return _vp(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dptr(t, name, shape_tail=None, allow_none=False):
    import torch
    if t is None:
        if allow_none:
            return None
        raise StokesError(STOKES_ERR_ARG, "%s is None" % name)
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise StokesError(STOKES_ERR_ARG, "%s must be a CUDA float64 tensor" % name)
    if not t.is_contiguous():
        raise StokesError(STOKES_ERR_ARG, "%s must be contiguous" % name)
    if shape_tail is not None and tuple(t.shape[1:]) != tuple(shape_tail):
        raise StokesError(STOKES_ERR_ARG, "%s has shape %s" % (name, tuple(t.shape)))
    return _vp(t.data_ptr()) if t.numel() else None


# ---------------------------------------------------------------------------
# C-named functions (argument marshalling only)
# ---------------------------------------------------------------------------
def stokes_create(device: int = 0):
    h = _vp()
    code = load().stokes_create(int(device), ctypes.byref(h))
    if code != STOKES_OK:
        raise StokesError(code, "stokes_create(device=%d) failed" % device)
    return h


def stokes_destroy(h):
    return _check(h, load().stokes_destroy(h))


def stokes_geom_set(h, curve_offset, curve_kind, nodes, weights, normals, curvature, period,
                    mu, stream=None):
    import numpy as np
    off = np.ascontiguousarray(curve_offset, dtype=np.int32)
    kind = np.ascontiguousarray(curve_kind, dtype=np.int32)
    code = load().stokes_geom_set(
        h, int(kind.shape[0]), _vp(off.ctypes.data), _vp(kind.ctypes.data),
        _dptr(nodes, "nodes", (2,)), _dptr(weights, "weights"), _dptr(normals, "normals", (2,)),
        _dptr(curvature, "curvature", allow_none=True), float(period), float(mu), _stream(stream))
    return _check(h, code)


def stokes_geom_update(h, nodes, weights, normals, curvature=None, stream=None):
    code = load().stokes_geom_update(h, _dptr(nodes, "nodes", (2,)), _dptr(weights, "weights"),
                                     _dptr(normals, "normals", (2,)),
                                     _dptr(curvature, "curvature", allow_none=True), _stream(stream))
    return _check(h, code)


def stokes_sum_eval(h, precision, slp_density, dlp_density, jump, out_velocity, stream=None):
    code = load().stokes_sum_eval(h, int(precision),
                                  _dptr(slp_density, "slp_density", (2,), True),
                                  _dptr(dlp_density, "dlp_density", (2,), True), float(jump),
                                  _dptr(out_velocity, "out_velocity", (2,)), _stream(stream))
    return _check(h, code)


def stokes_sum_eval_targets(h, precision, slp_density, dlp_density, targets, out_velocity,
                            stream=None):
    n = int(targets.shape[0])
    code = load().stokes_sum_eval_targets(h, int(precision),
                                          _dptr(slp_density, "slp_density", (2,), True),
                                          _dptr(dlp_density, "dlp_density", (2,), True), n,
                                          _dptr(targets, "targets", (2,), True),
                                          _dptr(out_velocity, "out_velocity", (2,), True),
                                          _stream(stream))
    return _check(h, code)


def stokes_sum_eval_targets_noalloc(h, precision, slp_density, dlp_density, targets,
                                    out_velocity, stream=None):
    """Free-point evaluation that allocates no device memory (for callers that cannot call
    cudaMalloc, e.g. while recording a CUDA graph); at most 262,144 targets."""
    n = int(targets.shape[0])
    code = load().stokes_sum_eval_targets_noalloc(h, int(precision),
                                                  _dptr(slp_density, "slp_density", (2,), True),
                                                  _dptr(dlp_density, "dlp_density", (2,), True),
                                                  n, _dptr(targets, "targets", (2,), True),
                                                  _dptr(out_velocity, "out_velocity", (2,), True),
                                                  _stream(stream))
    return _check(h, code)


def stokes_sum_eval_host(h, precision, slp_density_host, dlp_density_host, jump, out_host):
    """Host-buffer evaluation: NumPy (or pinned torch CPU) float64 arrays."""
    import numpy as np

    def hp(a, name):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            if a.dtype.__str__() != "torch.float64" or not a.is_contiguous() or a.is_cuda:
                raise StokesError(STOKES_ERR_ARG, "%s must be a contiguous CPU float64 tensor" % name)
            return _vp(a.data_ptr()) if a.numel() else None
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
            raise StokesError(STOKES_ERR_ARG, "%s must be a C-contiguous float64 array" % name)
        return _vp(a.ctypes.data) if a.size else None

    code = load().stokes_sum_eval_host(h, int(precision), hp(slp_density_host, "slp"),
                                       hp(dlp_density_host, "dlp"), float(jump),
                                       hp(out_host, "out"))
    return _check(h, code)


def stokes_last_error(h) -> str:
    return _err(h)


def stokes_sync(h, stream=None):
    return _check(h, load().stokes_sync(h, _stream(stream)))


def stokes_check_wait_timeout(h, stream=None):
    return _check(h, load().stokes_check_wait_timeout(h, _stream(stream)))


def stokes_check_log64(h, x, out, stream=None):
    """out[i] = the FP64 pair kernels' logarithm of x[i] (device float64 tensors, same length)."""
    n = int(x.numel())
    if int(out.numel()) != n:
        raise StokesError(STOKES_ERR_ARG, "x and out must have the same length")
    return _check(h, load().stokes_check_log64(h, _dptr(x, "x"), n, _dptr(out, "out"),
                                               _stream(stream)))


class FmmInfo(ctypes.Structure):
    _fields_ = [("order", _c_int), ("levels", _c_int), ("sources", _c_int),
                ("source_cells", _c_int), ("target_cells", _c_int), ("m2l_pairs", _c_double),
                ("near_pairs", _c_double), ("plan_ms", _c_double), ("device_bytes", _c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def stokes_fmm_create(h, order=24, leaf_size=32):
    """FMM plan for the context's current geometry (see stokes.h)."""
    f = _vp()
    code = load().stokes_fmm_create(h, int(order), int(leaf_size), ctypes.byref(f))
    if code != STOKES_OK:
        raise StokesError(code, _err(h))
    return f


def _fmm_err(f) -> str:
    buf = ctypes.create_string_buffer(512)
    if f:
        load().stokes_fmm_last_error(f, buf, 512)
    return buf.value.decode(errors="replace")


def stokes_fmm_create_targets(h, targets, order=24, leaf_size=32):
    """FMM plan of context h that also evaluates at the free points `targets` (device, (T, 2))."""
    f = _vp()
    code = load().stokes_fmm_create_targets(h, int(order), int(leaf_size), int(targets.shape[0]),
                                            _dptr(targets, "targets", (2,)), ctypes.byref(f))
    if code != STOKES_OK:
        raise StokesError(code, _err(h))
    return f


def stokes_fmm_create_targets_only(h, targets, order=24, leaf_size=32):
    """FMM plan of context h whose only targets are the free points `targets` (device, (T, 2))."""
    f = _vp()
    code = load().stokes_fmm_create_targets_only(h, int(order), int(leaf_size),
                                                 int(targets.shape[0]),
                                                 _dptr(targets, "targets", (2,)), ctypes.byref(f))
    if code != STOKES_OK:
        raise StokesError(code, _err(h))
    return f


def stokes_fmm_eval_targets(f, slp_density, dlp_density, out_velocity, stream=None):
    """Velocity at the plan's free targets into out_velocity (device, (T, 2))."""
    code = load().stokes_fmm_eval_targets(f, _dptr(slp_density, "slp_density", (2,), True),
                                          _dptr(dlp_density, "dlp_density", (2,), True),
                                          _dptr(out_velocity, "out_velocity", (2,)), _stream(stream))
    if code != STOKES_OK:
        raise StokesError(code, _fmm_err(f))
    return code


def stokes_fmm_eval(f, slp_density, dlp_density, jump, out_velocity, stream=None):
    code = load().stokes_fmm_eval(f, _dptr(slp_density, "slp_density", (2,), True),
                                  _dptr(dlp_density, "dlp_density", (2,), True), float(jump),
                                  _dptr(out_velocity, "out_velocity", (2,)), _stream(stream))
    if code != STOKES_OK:
        raise StokesError(code, _fmm_err(f))
    return code


def stokes_fmm_set_eval_order(f, order):
    """Truncate the following evaluations of plan f at `order` (0: the plan's order)."""
    code = load().stokes_fmm_set_eval_order(f, int(order))
    if code != STOKES_OK:
        raise StokesError(code, _fmm_err(f))
    return code


def stokes_fmm_set_precision(f, precision):
    """Arithmetic of the following evaluations: STOKES_FP64 or STOKES_FP32_KAHAN (FP32 expansions
    and direct pairs)."""
    code = load().stokes_fmm_set_precision(f, int(precision))
    if code != STOKES_OK:
        raise StokesError(code, _fmm_err(f))
    return code


def stokes_fmm_get_info(f):
    info = FmmInfo()
    code = load().stokes_fmm_get_info(f, ctypes.byref(info))
    if code != STOKES_OK:
        raise StokesError(code, "stokes_fmm_get_info")
    return info.as_dict()


def stokes_fmm_last_error(f) -> str:
    return _fmm_err(f)


def stokes_fmm_destroy(f):
    return load().stokes_fmm_destroy(f)


class CloseInfo(ctypes.Structure):
    _fields_ = [("upsample", _c_int), ("pairs", _c_int), ("targets", _c_int),
                ("vesicles", _c_int), ("factor", _c_double), ("plan_ms", _c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def stokes_close_create(h, factor=5.0, upsample=16):
    """Close-evaluation plan for the context's current geometry (see stokes.h)."""
    f = _vp()
    code = load().stokes_close_create(h, float(factor), int(upsample), ctypes.byref(f))
    if code != STOKES_OK:
        raise StokesError(code, _err(h))
    return f


def stokes_close_last_error(f) -> str:
    buf = ctypes.create_string_buffer(512)
    if f:
        load().stokes_close_last_error(f, buf, 512)
    return buf.value.decode(errors="replace")


def stokes_close_eval(f, slp_density, out_velocity, stream=None):
    """Adds the close-evaluation correction to out_velocity (the node sum)."""
    code = load().stokes_close_eval(f, _dptr(slp_density, "slp_density", (2,), True),
                                    _dptr(out_velocity, "out_velocity", (2,)), _stream(stream))
    if code != STOKES_OK:
        raise StokesError(code, stokes_close_last_error(f))
    return code


def stokes_close_get_info(f):
    info = CloseInfo()
    code = load().stokes_close_get_info(f, ctypes.byref(info))
    if code != STOKES_OK:
        raise StokesError(code, "stokes_close_get_info")
    return info.as_dict()


def stokes_close_destroy(f):
    return load().stokes_close_destroy(f)


def stokes_num_nodes(h) -> int:
    return int(load().stokes_num_nodes(h))


def stokes_set_launch(h, precision, source_splits=0, targets_per_thread=0, kahan_group=0):
    return _check(h, load().stokes_set_launch(h, int(precision), int(source_splits),
                                              int(targets_per_thread), int(kahan_group)))


def stokes_graph_stats(h):
    """(graphs captured, graph launches) of the context's node sums."""
    a, b = ctypes.c_longlong(), ctypes.c_longlong()
    _check(h, load().stokes_graph_stats(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def stokes_time_sums(h, precision, slp_density, dlp_density, jump, out_velocity, reps=20,
                     stream=None):
    """Device time per node sum (ms) of `reps` sums issued back to back by the library."""
    ms = _c_double()
    _check(h, load().stokes_time_sums(h, int(precision), _dptr(slp_density, "slp_density", (2,), True),
                                      _dptr(dlp_density, "dlp_density", (2,), True), float(jump),
                                      _dptr(out_velocity, "out_velocity", (2,)), int(reps),
                                      _stream(stream), ctypes.byref(ms)))
    return float(ms.value)


def stokes_debug_build() -> bool:
    """True when the loaded library is the debug build (device bounds checks)."""
    return bool(load().stokes_debug_build())


def stokes_debug_tighten(h, elements):
    """Debug build: the bounds checks treat the last `elements` partial-sum elements as out
    of range (the buffers keep their size)."""
    return _check(h, load().stokes_debug_tighten(h, int(elements)))


def stokes_set_graph_mode(h, mode=STOKES_GRAPH_SMALL):
    """Node sums replayed from a captured CUDA graph: STOKES_GRAPH_OFF / _SMALL / _ALWAYS."""
    return _check(h, load().stokes_set_graph_mode(h, int(mode)))


def stokes_set_local_frame(h, on: bool = True):
    return _check(h, load().stokes_set_local_frame(h, int(bool(on))))


def stokes_get_launch(h, precision):
    """(source_splits, targets_per_thread, kahan_group) of the current launch shape."""
    a, b, c = _c_int(), _c_int(), _c_int()
    _check(h, load().stokes_get_launch(h, int(precision), ctypes.byref(a), ctypes.byref(b),
                                       ctypes.byref(c)))
    return a.value, b.value, c.value


def stokes_set_profiling(h, on: bool = True):
    return _check(h, load().stokes_set_profiling(h, int(bool(on))))


def stokes_last_timing(h):
    """(pack_ms, pair_ms, finish_ms) of the last profiled call."""
    ms = (_c_double * 3)()
    _check(h, load().stokes_last_timing(h, ms))
    return tuple(float(v) for v in ms)


def stokes_pair_count(h, n_targets: int = 0) -> float:
    v = _c_double()
    _check(h, load().stokes_pair_count(h, int(n_targets), ctypes.byref(v)))
    return float(v.value)


def stokes_batch_set(h, inst_curve_offset, curve_offset, curve_kind, nodes, weights, normals,
                     curvature, periods, mu, stream=None):
    import numpy as np
    ioff = np.ascontiguousarray(inst_curve_offset, dtype=np.int32)
    off = np.ascontiguousarray(curve_offset, dtype=np.int32)
    kind = np.ascontiguousarray(curve_kind, dtype=np.int32)
    per = np.ascontiguousarray(periods, dtype=np.float64)
    code = load().stokes_batch_set(
        h, int(ioff.shape[0] - 1), _vp(ioff.ctypes.data), int(kind.shape[0]), _vp(off.ctypes.data),
        _vp(kind.ctypes.data), _dptr(nodes, "nodes", (2,)), _dptr(weights, "weights"),
        _dptr(normals, "normals", (2,)), _dptr(curvature, "curvature", allow_none=True),
        _vp(per.ctypes.data), float(mu), _stream(stream))
    return _check(h, code)


def stokes_batch_eval(h, precision, slp_density, dlp_density, jump, out_velocity, use_graph=True,
                      stream=None):
    code = load().stokes_batch_eval(h, int(precision),
                                    _dptr(slp_density, "slp_density", (2,), True),
                                    _dptr(dlp_density, "dlp_density", (2,), True), float(jump),
                                    _dptr(out_velocity, "out_velocity", (2,)),
                                    int(bool(use_graph)), _stream(stream))
    return _check(h, code)


def stokes_batch_set_shape(h, precision, targets_per_thread=0, items_per_slot=0):
    return _check(h, load().stokes_batch_set_shape(h, int(precision), int(targets_per_thread),
                                                   int(items_per_slot)))


def stokes_batch_info(h, precision):
    """(n_items, blocks, targets_per_thread, items_per_slot) of the batched launch."""
    v = [_c_int() for _ in range(4)]
    _check(h, load().stokes_batch_info(h, int(precision), *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


class TuneResult(ctypes.Structure):
    _fields_ = [("precision", _c_int), ("source_splits", _c_int),
                ("targets_per_thread", _c_int), ("kahan_group", _c_int),
                ("items_per_slot", _c_int), ("candidates", _c_int), ("best_ms", _c_double),
                ("initial_ms", _c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def stokes_autotune(h, precision, repeats=5, stream=None):
    """Time the candidate launch shapes, apply the fastest and record it for the size class."""
    r = TuneResult()
    _check(h, load().stokes_autotune(h, int(precision), int(repeats), _vp(ctypes.addressof(r)),
                                     _stream(stream)))
    return r.as_dict()


def stokes_tune_lookup(num_sms, precision, n_inst, n_nodes, n_wall_nodes, n_ves_nodes):
    """The recorded shape of a size class as a dict, or None."""
    r = TuneResult()
    code = load().stokes_tune_lookup(int(num_sms), int(precision), int(n_inst), int(n_nodes),
                                     int(n_wall_nodes), int(n_ves_nodes), _vp(ctypes.addressof(r)))
    if code < 0:
        raise StokesError(code, "stokes_tune_lookup: bad argument")
    return r.as_dict() if code == 1 else None


def stokes_tune_save(path):
    code = load().stokes_tune_save(os.fsencode(path))
    if code != STOKES_OK:
        raise StokesError(code, "stokes_tune_save: cannot write %s" % path)
    return code


def stokes_tune_load(path):
    code = load().stokes_tune_load(os.fsencode(path))
    if code != STOKES_OK:
        raise StokesError(code, "stokes_tune_load: cannot read or parse %s" % path)
    return code


def stokes_tune_clear():
    return load().stokes_tune_clear()


# ---------------------------------------------------------------------------
# channel response and time stepping
# ---------------------------------------------------------------------------
class StepStats(ctypes.Structure):
    _fields_ = [("iterations", _c_int), ("residual", _c_double), ("setup_ms", _c_double),
                ("gmres_ms", _c_double), ("total_ms", _c_double), ("refinements", _c_int),
                ("accurate_residuals", _c_int), ("fmm_plan_ms", _c_double),
                ("precond_refresh", _c_int), ("response_plan_ms", _c_double),
                ("plan_wait_ms", _c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _sim_err(h) -> str:
    buf = ctypes.create_string_buffer(512)
    if h:
        load().stokes_sim_last_error(h, buf, 512)
    return buf.value.decode(errors="replace")


def _sim_check(h, code):
    if code != STOKES_OK:
        raise StokesError(code, _sim_err(h))
    return code


def _host(a, name, dtype="float64"):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, _vp(a.ctypes.data)


def stokes_sim_create(device: int = 0):
    h = _vp()
    code = load().stokes_sim_create(int(device), ctypes.byref(h))
    if code != STOKES_OK:
        raise StokesError(code, "stokes_sim_create(device=%d) failed" % device)
    return h


def stokes_sim_destroy(h):
    return _sim_check(h, load().stokes_sim_destroy(h))


def stokes_sim_last_error(h) -> str:
    return _sim_err(h)


def stokes_sim_set_walls(h, n_per_wall, nodes, weights, normals, curvature, period, mu, K=32,
                         M=128, proxy_radius=None):
    keep = [_host(a, "w") for a in (nodes, weights, normals, curvature)]
    code = load().stokes_sim_set_walls(h, int(n_per_wall), *[p for _, p in keep], float(period),
                                       float(mu), int(K), int(M),
                                       float(period if proxy_radius is None else proxy_radius))
    return _sim_check(h, code)


def stokes_sim_set_vesicles(h, V, n, x, kappa_b, mu, period):
    a, p = _host(x, "x")
    return _sim_check(h, load().stokes_sim_set_vesicles(h, int(V), int(n), p, float(kappa_b),
                                                        float(mu), float(period)))


def stokes_sim_empty_channel_pressure(h, p_drive, v_walls, targets, p_out):
    return _sim_check(h, load().stokes_sim_empty_channel_pressure(
        h, float(p_drive), _dptr(v_walls, "v_walls", (2,), True), int(targets.shape[0]),
        _dptr(targets, "targets", (2,)), _dptr(p_out, "p_out")))


def stokes_sum_eval_pressure(h, slp_density, dlp_density, targets, out_pressure, stream=None):
    """Pressure of the layer potentials at free points (FP64), shape (T,)."""
    code = load().stokes_sum_eval_pressure(
        h, _dptr(slp_density, "slp_density", (2,), True), _dptr(dlp_density, "dlp_density", (2,), True),
        int(targets.shape[0]), _dptr(targets, "targets", (2,)), _dptr(out_pressure, "out_pressure"),
        _stream(stream))
    return _check(h, code)


def stokes_sum_eval_traction(h, slp_density, dlp_density, targets, target_normals, out_traction,
                             stream=None):
    """Traction of the layer potentials at free points with normals (FP64), shape (T, 2)."""
    code = load().stokes_sum_eval_traction(
        h, _dptr(slp_density, "slp_density", (2,), True), _dptr(dlp_density, "dlp_density", (2,), True),
        int(targets.shape[0]), _dptr(targets, "targets", (2,)),
        _dptr(target_normals, "target_normals", (2,)), _dptr(out_traction, "out_traction", (2,)),
        _stream(stream))
    return _check(h, code)


def stokes_sim_set_wall_solver(h, mode):
    """STOKES_WALLS_FDS (the fast direct solver, default), STOKES_WALLS_LU32_REFINE or
    STOKES_WALLS_LU64; read at the next set_walls."""
    return _sim_check(h, load().stokes_sim_set_wall_solver(h, int(mode)))


class FdsInfo(ctypes.Structure):
    _fields_ = [("levels", _c_int), ("max_rank", _c_int), ("root_size", _c_int),
                ("neighbour_rank", _c_int), ("sections", _c_int), ("host_ms", _c_double),
                ("device_ms", _c_double), ("device_bytes", _c_double),
                ("solve_bytes", _c_double), ("walls_setup_ms", _c_double),
                ("neighbour_col_rank", _c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def stokes_sim_wall_solve(h, X):
    """X (device, (4 n_w,) or (nrhs, 4 n_w) rows = right-hand sides) <- A^-1 X in place."""
    if X.dim() == 1:
        nrhs = 1
    else:
        nrhs = int(X.shape[0])
    return _sim_check(h, load().stokes_sim_wall_solve(h, _dptr(X, "X", None), nrhs))


def stokes_sim_set_fds_params(h, tol=1e-12, leaf_nodes=64, n_proxy=64):
    """Interpolative-decomposition tolerance, HBS leaf size and proxy count (next set_walls)."""
    return _sim_check(h, load().stokes_sim_set_fds_params(h, float(tol), int(leaf_nodes), int(n_proxy)))


def stokes_sim_set_fds_recompress(h, on=True):
    """Column recompression of the neighbour factors (Sec. 4.2 remark), read at the next set_walls."""
    return _sim_check(h, load().stokes_sim_set_fds_recompress(h, int(on)))


def stokes_sim_fds_info(h):
    """Statistics of the last set_walls (fast direct solver ranks and timings) as a dict."""
    info = FdsInfo()
    _sim_check(h, load().stokes_sim_fds_info(h, ctypes.byref(info)))
    return info.as_dict()


def stokes_sim_set_block_refinement(h, sweeps):
    return _sim_check(h, load().stokes_sim_set_block_refinement(h, int(sweeps)))


def stokes_sim_set_precond_refresh(h, on=True):
    """Newton-Schulz refresh of the FP32 preconditioner inverse from the previous step's."""
    return _sim_check(h, load().stokes_sim_set_precond_refresh(h, int(on)))


def stokes_sim_set_precond_tensor(h, on=True):
    """FP32 preconditioner GEMMs (assembly, refresh) by cuBLAS's BF16x9 FP32 emulation."""
    return _sim_check(h, load().stokes_sim_set_precond_tensor(h, int(on)))


def stokes_sim_set_precond_precision(h, precision):
    return _sim_check(h, load().stokes_sim_set_precond_precision(h, int(precision)))


def stokes_sim_set_inner_tolerance(h, tol):
    return _sim_check(h, load().stokes_sim_set_inner_tolerance(h, float(tol)))


def stokes_sim_set_warm_modes(h, modes):
    """Fourier modes nm of the warm-start features (4 nm) and targets (3 nm)."""
    return _sim_check(h, load().stokes_sim_set_warm_modes(h, int(modes)))


def stokes_sim_get_warm_modes(h) -> int:
    v = _c_int()
    _sim_check(h, load().stokes_sim_get_warm_modes(h, ctypes.byref(v)))
    return int(v.value)


def stokes_sim_set_warm_history(h, on=True):
    """Features also carry the previous solution and its last change (10 nm features)."""
    return _sim_check(h, load().stokes_sim_set_warm_history(h, int(bool(on))))


def stokes_sim_set_warm_base(h, base):
    """STOKES_WARM_BASE_PREVIOUS or STOKES_WARM_BASE_EXTRAPOLATE: what the learned change is
    added to (and what the targets are relative to)."""
    return _sim_check(h, load().stokes_sim_set_warm_base(h, int(base)))


def feature_dims(modes: int, history: bool = False):
    """(features, targets) per vesicle for `modes` warm-start modes (with history features)."""
    return 4 * int(modes) + (6 * int(modes) if history else 0), 3 * int(modes)


def stokes_sim_set_close_eval(h, factor, upsample=16):
    """Steps add the close-evaluation correction of vesicle pairs closer than factor h (0: off)."""
    return _sim_check(h, load().stokes_sim_set_close_eval(h, float(factor), int(upsample)))


def stokes_sim_set_residual_fmm(h, order, leaf_size=32):
    """FP32-Kahan steps: FP64-accurate vesicle sums by the FMM of `order` (0 = double-float)."""
    return _sim_check(h, load().stokes_sim_set_residual_fmm(h, int(order), int(leaf_size)))


def stokes_sim_set_sweep_fmm(h, order):
    """FP32-Kahan steps: the Krylov sweeps' vesicle sums by the step's FMM plan at `order` (0 = direct)."""
    return _sim_check(h, load().stokes_sim_set_sweep_fmm(h, int(order)))


def stokes_sim_wall_stats(h):
    """(refinement sweeps, relative residual) of the last wall solve."""
    a, b = _c_int(), _c_double()
    _sim_check(h, load().stokes_sim_wall_stats(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def stokes_sim_channel_response(h, f, p_drive, u_resp):
    return _sim_check(h, load().stokes_sim_channel_response(h, _dptr(f, "f", (2,)), float(p_drive),
                                                            _dptr(u_resp, "u_resp", (2,))))


def stokes_sim_empty_channel(h, p_drive, v_walls, targets, u_out):
    return _sim_check(h, load().stokes_sim_empty_channel(
        h, float(p_drive), _dptr(v_walls, "v_walls", (2,), True), int(targets.shape[0]),
        _dptr(targets, "targets", (2,)), _dptr(u_out, "u_out", (2,))))


def vesicle_step_warmstart(h, dt, p_drive, guess_mode=STOKES_GUESS_ZERO, model=None, guess=None,
                           tol=1e-10, max_iter=300, precision=STOKES_FP64):
    st = StepStats()
    code = load().vesicle_step_warmstart(h, float(dt), float(p_drive), int(guess_mode),
                                         model if model else None,
                                         _dptr(guess, "guess", None, True), float(tol),
                                         int(max_iter), int(precision), ctypes.byref(st))
    _sim_check(h, code)
    return st.as_dict()


def _fptr(t, name, allow_none=False):
    import torch
    if t is None:
        if allow_none:
            return None
        raise StokesError(STOKES_ERR_ARG, "%s is None" % name)
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype not in (torch.float32, torch.int32) \
            or not t.is_contiguous():
        raise StokesError(STOKES_ERR_ARG, "%s must be a contiguous CUDA float32/int32 tensor" % name)
    return _vp(t.data_ptr()) if t.numel() else None


def stokes_sim_last_features(h, features, targets):
    return _sim_check(h, load().stokes_sim_last_features(h, _fptr(features, "features", True),
                                                         _fptr(targets, "targets", True)))


def _mlp_err(h):
    buf = ctypes.create_string_buffer(512)
    if h:
        load().stokes_mlp_last_error(h, buf, 512)
    return buf.value.decode(errors="replace")


def _mlp_check(h, code):
    if code != STOKES_OK:
        raise StokesError(code, _mlp_err(h))
    return code


def stokes_mlp_create(device, n_in, n_hidden, n_out):
    h = _vp()
    code = load().stokes_mlp_create(int(device), int(n_in), int(n_hidden), int(n_out), ctypes.byref(h))
    if code != STOKES_OK:
        raise StokesError(code, "stokes_mlp_create failed")
    return h


def stokes_mlp_destroy(h):
    return _mlp_check(h, load().stokes_mlp_destroy(h))


def stokes_mlp_last_error(h):
    return _mlp_err(h)


def stokes_mlp_num_params(h):
    return int(load().stokes_mlp_num_params(h))


def stokes_mlp_set_params(h, theta):
    a, p = _host(theta, "theta", "float32")
    if a.size != stokes_mlp_num_params(h):
        raise StokesError(STOKES_ERR_ARG, "theta must hold %d floats" % stokes_mlp_num_params(h))
    return _mlp_check(h, load().stokes_mlp_set_params(h, p))


def stokes_mlp_get_params(h):
    import numpy as np
    out = np.zeros(stokes_mlp_num_params(h), dtype=np.float32)
    _mlp_check(h, load().stokes_mlp_get_params(h, _vp(out.ctypes.data)))
    return out


def stokes_mlp_set_normalization(h, norm):
    a, p = _host(norm, "norm", "float32")
    d_in, _, d_out = stokes_mlp_get_dims(h)
    if a.size != 2 * (d_in + d_out):
        raise StokesError(STOKES_ERR_ARG, "norm must hold 2 (n_in + n_out) = %d floats"
                          % (2 * (d_in + d_out)))
    return _mlp_check(h, load().stokes_mlp_set_normalization(h, p))


def stokes_mlp_get_dims(h):
    """(n_in, n_hidden, n_out) of the network."""
    a, b, c = _c_int(), _c_int(), _c_int()
    _mlp_check(h, load().stokes_mlp_get_dims(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def stokes_mlp_get_normalization(h, n_in=None, n_out=None):
    """(mu_in, sd_in, mu_out, sd_out) concatenated; the sizes come from the network itself."""
    import numpy as np
    d_in, _, d_out = stokes_mlp_get_dims(h)
    if (n_in is not None and n_in != d_in) or (n_out is not None and n_out != d_out):
        raise StokesError(STOKES_ERR_ARG, "the network maps %d -> %d" % (d_in, d_out))
    out = np.zeros(2 * (d_in + d_out), dtype=np.float32)
    _mlp_check(h, load().stokes_mlp_get_normalization(h, _vp(out.ctypes.data)))
    return out


def stokes_mlp_fit_normalization(h, X, T):
    return _mlp_check(h, load().stokes_mlp_fit_normalization(h, int(X.shape[0]), _fptr(X, "X"),
                                                             _fptr(T, "T")))


def stokes_mlp_forward(h, X, Y):
    return _mlp_check(h, load().stokes_mlp_forward(h, int(X.shape[0]), _fptr(X, "X"), _fptr(Y, "Y")))


def stokes_mlp_loss_grad(h, X, T, idx=None, batch=None):
    """(loss, gradient as a NumPy array) of rows idx (CUDA int32) or the first `batch` rows."""
    import numpy as np
    b = int(idx.shape[0]) if idx is not None else int(batch if batch else X.shape[0])
    g = np.zeros(stokes_mlp_num_params(h), dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    _mlp_check(h, load().stokes_mlp_loss_grad(h, int(X.shape[0]), _fptr(X, "X"), _fptr(T, "T"),
                                              _fptr(idx, "idx", True), b, _vp(g.ctypes.data),
                                              _vp(loss.ctypes.data)))
    return float(loss[0]), g


def stokes_mlp_train_step(h, X, T, idx, lr):
    import numpy as np
    loss = np.zeros(1, dtype=np.float32)
    _mlp_check(h, load().stokes_mlp_train_step(h, int(X.shape[0]), _fptr(X, "X"), _fptr(T, "T"),
                                               _fptr(idx, "idx"), int(idx.shape[0]), float(lr),
                                               _vp(loss.ctypes.data)))
    return float(loss[0])


def stokes_sim_get_history(h):
    """(L0 (V,), A0 (V,), zprev (3 n V,), bprev (3 n V,)) as NumPy arrays."""
    import numpy as np
    V, n, _ = stokes_sim_sizes(h)
    L0, A0 = np.zeros(V), np.zeros(V)
    zp, bp = np.zeros(3 * n * V), np.zeros(3 * n * V)
    _sim_check(h, load().stokes_sim_get_history(h, _vp(L0.ctypes.data), _vp(A0.ctypes.data),
                                                _vp(zp.ctypes.data), _vp(bp.ctypes.data)))
    return L0, A0, zp, bp


def stokes_sim_set_history(h, L0, A0, zprev, bprev):
    keep = [_host(a, "history") for a in (L0, A0, zprev, bprev)]
    return _sim_check(h, load().stokes_sim_set_history(h, *[p for _, p in keep]))


def stokes_mlp_get_adam(h):
    """(first moments, second moments, step count) of the network's Adam state."""
    import numpy as np
    n = stokes_mlp_num_params(h)
    mm, vv, t = np.zeros(n, dtype=np.float32), np.zeros(n, dtype=np.float32), _c_int()
    _mlp_check(h, load().stokes_mlp_get_adam(h, _vp(mm.ctypes.data), _vp(vv.ctypes.data),
                                             ctypes.byref(t)))
    return mm, vv, t.value


def stokes_mlp_set_adam(h, m, v, t):
    import numpy as np
    mm = np.ascontiguousarray(m, dtype=np.float32)
    vv = np.ascontiguousarray(v, dtype=np.float32)
    if mm.size != stokes_mlp_num_params(h) or vv.size != mm.size:
        raise StokesError(STOKES_ERR_ARG, "Adam moments must hold %d floats each" % stokes_mlp_num_params(h))
    return _mlp_check(h, load().stokes_mlp_set_adam(h, _vp(mm.ctypes.data), _vp(vv.ctypes.data),
                                                    int(t)))


def stokes_sim_set_restart(h, restart):
    return _sim_check(h, load().stokes_sim_set_restart(h, int(restart)))


def stokes_sim_sizes(h):
    v = [_c_int() for _ in range(3)]
    _sim_check(h, load().stokes_sim_sizes(h, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def stokes_sim_get_state(h):
    """(positions (V n, 2), tension (V n), last solution (3 n V)) as NumPy arrays."""
    import numpy as np
    V, n, _ = stokes_sim_sizes(h)
    x = np.zeros((V * n, 2))
    sg = np.zeros(V * n)
    sol = np.zeros(3 * V * n)
    _sim_check(h, load().stokes_sim_get_state(h, _vp(x.ctypes.data), _vp(sg.ctypes.data),
                                              _vp(sol.ctypes.data)))
    return x, sg, sol


def stokes_sim_set_state(h, x=None, sigma=None):
    kx = _host(x, "x") if x is not None else (None, None)
    ks = _host(sigma, "sigma") if sigma is not None else (None, None)
    return _sim_check(h, load().stokes_sim_set_state(h, kx[1], ks[1]))


# ---------------------------------------------------------------------------
# convenience wrappers
# ---------------------------------------------------------------------------
class StokesSum:
    """One libstokes context with a geometry resident on the GPU.

    ``geom`` is any object with ``curve_offset``, ``curve_kind``, ``nodes``, ``weights``,
    ``normals``, ``curvature`` (NumPy), ``period`` and ``mu`` (e.g. ``inputs.Geometry``).
    """

    def __init__(self, geom=None, device: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise StokesError(STOKES_ERR_CUDA, "no CUDA device: libstokes runs on the GPU only")
        self.device = torch.device("cuda", device)
        self.h = stokes_create(device)
        self.N = 0
        if geom is not None:
            self.set_geometry(geom)

    def set_geometry(self, geom):
        import torch
        dev = self.device
        t = lambda a: torch.as_tensor(a, dtype=torch.float64).to(dev).contiguous()
        self._geom_tensors = (t(geom.nodes), t(geom.weights), t(geom.normals), t(geom.curvature))
        x, w, n, k = self._geom_tensors
        stokes_geom_set(self.h, geom.curve_offset, geom.curve_kind, x, w, n, k, geom.period,
                        geom.mu)
        self.N = stokes_num_nodes(self.h)

    def eval(self, slp, dlp, precision="fp32k", jump=0.0, out=None, sync=True):
        import torch
        prec = PRECISIONS.get(precision, precision)
        if out is None:
            out = torch.empty((self.N, 2), dtype=torch.float64, device=self.device)
        stokes_sum_eval(self.h, prec, slp, dlp, jump, out)
        if sync:
            stokes_sync(self.h)
        return out

    def eval_targets(self, slp, dlp, targets, precision="fp32k", out=None, sync=True):
        import torch
        prec = PRECISIONS.get(precision, precision)
        if out is None:
            out = torch.empty((int(targets.shape[0]), 2), dtype=torch.float64, device=self.device)
        stokes_sum_eval_targets(self.h, prec, slp, dlp, targets, out)
        if sync:
            stokes_sync(self.h)
        return out

    def close(self):
        if getattr(self, "h", None):
            stokes_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StokesBatch:
    """Many independent channel instances evaluated by one persistent launch.

    ``geoms`` is a list of geometry objects (as for :class:`StokesSum`) sharing one ``mu``.
    Densities and results are the instances' arrays stacked in order (vesicle rows of all
    instances, wall rows of all instances, node rows of all instances).
    """

    def __init__(self, geoms, device: int = 0):
        import numpy as np
        import torch
        if not torch.cuda.is_available():
            raise StokesError(STOKES_ERR_CUDA, "no CUDA device: libstokes runs on the GPU only")
        self.device = torch.device("cuda", device)
        self.h = stokes_create(device)
        curves = [c for g in geoms for c in g.curves]
        ioff = np.zeros(len(geoms) + 1, dtype=np.int32)
        ioff[1:] = np.cumsum([len(g.curves) for g in geoms])
        off = np.zeros(len(curves) + 1, dtype=np.int32)
        off[1:] = np.cumsum([c.n for c in curves])
        kind = np.array([c.kind for c in curves], dtype=np.int32)
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).to(self.device)
        cat = lambda name: np.concatenate([getattr(c, name) for c in curves])
        self._geom_tensors = (t(cat("nodes")), t(cat("weights")), t(cat("normals")),
                              t(cat("curvature")))
        x, w, n, k = self._geom_tensors
        stokes_batch_set(self.h, ioff, off, kind, x, w, n, k, [g.period for g in geoms],
                         geoms[0].mu)
        self.N = int(off[-1])
        self.sizes = [g.n_nodes for g in geoms]

    @staticmethod
    def stack(per_instance):
        import numpy as np
        return np.ascontiguousarray(np.concatenate([np.asarray(a).reshape(-1, 2) for a in per_instance]))

    def eval(self, slp, dlp, precision="fp32k", jump=0.0, use_graph=True, out=None, sync=True):
        import torch
        prec = PRECISIONS.get(precision, precision)
        if out is None:
            out = torch.empty((self.N, 2), dtype=torch.float64, device=self.device)
        stokes_batch_eval(self.h, prec, slp, dlp, jump, out, use_graph)
        if sync:
            stokes_sync(self.h)
        return out

    def close(self):
        if getattr(self, "h", None):
            stokes_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
