"""The no-allocation free-point entry point agrees with stokes_sum_eval_targets.

stokes_sum_eval_targets_noalloc serves callers that cannot allocate device memory where they
evaluate: hosts that own every byte of device memory through their own pool, plug-ins on a
fixed memory budget inside such a host, and real-time loops that must not block on the
allocator.  Its scratch is a fixed array inside the library.  This file is collected last so
that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from paper_1510_05616_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32k": 1e-6, "df": 1e-12}
CAPACITY = 1 << 18  # targets the fixed scratch array holds at one source split


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_05616_gb300 import build
    build.build()
    import paper_1510_05616_gb300 as P
    return P


def _cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _targets(rng, n):
    return np.stack([rng.uniform(-1.0, 7.0, n), rng.uniform(-0.55, 0.55, n)], 1)


def _compare(P, s, pc, ts, td, tg, tol):
    import torch
    n = tg.shape[0]
    ref = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    out = torch.full((n, 2), float("nan"), dtype=torch.float64, device="cuda")
    P.stokes_sum_eval_targets(s.h, pc, ts, td, tg, ref)
    P.stokes_sum_eval_targets_noalloc(s.h, pc, ts, td, tg, out)
    P.stokes_sync(s.h)
    r, o = ref.cpu().numpy(), out.cpu().numpy()
    err = np.abs(o - r).max(0) / np.abs(r).max(0)
    assert np.all(err <= tol), (n, err)


@pytest.mark.parametrize("prec", ["fp64", "fp32k", "df"])
def test_noalloc_matches_allocating_entry_point(P, prec):
    g, slp, dlp = I.workload("small_n1280")
    s = P.StokesSum(g)
    pc = P.PRECISIONS[prec]
    rng = np.random.default_rng(17)
    # two calls in a row with different targets and densities: no state may leak between them
    for n, scale in ((3001, 1.0), (777, -0.5)):
        _compare(P, s, pc, _cuda(scale * slp), _cuda(scale * dlp), _cuda(_targets(rng, n)),
                 TOL[prec])
    s.close()


@pytest.mark.parametrize("prec", ["fp32k", "df"])
def test_noalloc_at_capacity_uses_fewer_splits(P, prec):
    # At the full capacity only one source split fits the array, whatever the context's
    # split count is; the result must still equal the allocating entry point's.
    g, slp, dlp = I.workload("mid_n16k")
    s = P.StokesSum(g)
    pc = P.PRECISIONS[prec]
    splits = P.stokes_get_launch(s.h, pc)[0]
    assert splits > 1  # the context itself splits the sources
    rng = np.random.default_rng(5)
    _compare(P, s, pc, _cuda(slp), _cuda(dlp), _cuda(_targets(rng, CAPACITY)), TOL[prec])
    _compare(P, s, pc, _cuda(-slp), _cuda(2.0 * dlp), _cuda(_targets(rng, 5000)), TOL[prec])
    s.close()


def test_noalloc_rejects_too_many_targets(P):
    import torch
    g, slp, dlp = I.workload("small_n1280")
    s = P.StokesSum(g)
    n = CAPACITY + 1
    tg = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    out = torch.empty_like(tg)
    with pytest.raises(P.StokesError) as e:
        P.stokes_sum_eval_targets_noalloc(s.h, P.STOKES_FP64, _cuda(slp), _cuda(dlp), tg, out)
    assert e.value.code == P.STOKES_ERR_ARG and "capacity" in str(e.value)
    s.close()


def test_noalloc_rejects_batched_context(P):
    import torch
    ws = [I.workload("small_n1280"), I.workload("small_n1280", seed=7)]
    b = P.StokesBatch([w[0] for w in ws])
    nv = sum(w[1].shape[0] for w in ws)
    nw = sum(w[2].shape[0] for w in ws)
    ts = torch.zeros((nv, 2), dtype=torch.float64, device="cuda")
    td = torch.zeros((nw, 2), dtype=torch.float64, device="cuda")
    tg = torch.zeros((10, 2), dtype=torch.float64, device="cuda")
    out = torch.empty_like(tg)
    with pytest.raises(P.StokesError) as e:
        P.stokes_sum_eval_targets_noalloc(b.h, P.STOKES_FP32_KAHAN, ts, td, tg, out)
    assert e.value.code == P.STOKES_ERR_ARG and "single-instance" in str(e.value)
    b.close()


def test_noalloc_records_phase_timing(P):
    g, slp, dlp = I.workload("small_n1280")
    s = P.StokesSum(g)
    rng = np.random.default_rng(3)
    tg = _cuda(_targets(rng, 2048))
    import torch
    out = torch.empty_like(tg)
    P.stokes_set_profiling(s.h, True)
    P.stokes_sum_eval_targets_noalloc(s.h, P.STOKES_FP32_KAHAN, _cuda(slp), _cuda(dlp), tg, out)
    P.stokes_sync(s.h)
    ms = P.stokes_last_timing(s.h)
    assert len(ms) == 3 and all(np.isfinite(ms)) and all(m >= 0.0 for m in ms) and ms[1] > 0.0
    s.close()
