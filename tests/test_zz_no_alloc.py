"""The no-allocation free-point entry point agrees with stokes_sum_eval_targets.

stokes_sum_eval_targets_noalloc serves callers that cannot allocate device memory where they
evaluate (stream capture, host-owned memory pools, real-time loops); its scratch is a fixed
array inside the library.  This file is collected last so that a failure here leaves every
other test already run.
"""
import math

import numpy as np
import pytest

from paper_1510_05616_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32k": 1e-6, "df": 1e-12}


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


@pytest.mark.parametrize("prec", ["fp64", "fp32k", "df"])
def test_noalloc_matches_allocating_entry_point(P, prec):
    import torch
    g, slp, dlp = I.workload("small_n1280")
    s = P.StokesSum(g)
    pc = P.PRECISIONS[prec]
    rng = np.random.default_rng(17)
    # two calls in a row with different targets and densities: no state may leak between them
    for n, scale in ((3001, 1.0), (777, -0.5)):
        tg = _cuda(_targets(rng, n))
        ts, td = _cuda(scale * slp), _cuda(scale * dlp)
        ref = torch.empty((n, 2), dtype=torch.float64, device="cuda")
        out = torch.full((n, 2), float("nan"), dtype=torch.float64, device="cuda")
        P.stokes_sum_eval_targets(s.h, pc, ts, td, tg, ref)
        P.stokes_sum_eval_targets_noalloc(s.h, pc, ts, td, tg, out)
        P.stokes_sync(s.h)
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        err = np.abs(o - r).max(0) / np.abs(r).max(0)
        assert np.all(err <= TOL[prec]), (n, err)
    s.close()


def test_noalloc_rejects_too_many_targets(P):
    import torch
    g, slp, dlp = I.workload("small_n1280")
    s = P.StokesSum(g)
    n = (1 << 18) + 1
    tg = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    out = torch.empty_like(tg)
    with pytest.raises(P.StokesError) as e:
        P.stokes_sum_eval_targets_noalloc(s.h, P.STOKES_FP64, _cuda(slp), _cuda(dlp), tg, out)
    assert e.value.code == P.STOKES_ERR_ARG and "capacity" in str(e.value)
    s.close()
