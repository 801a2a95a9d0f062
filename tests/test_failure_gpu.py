"""Failure handling on the GPU without faulting it: the pair kernels' bounded pipeline wait
gives up after its limit and reports a timeout that the host reads, leaving the context
usable; bad inputs come back as status codes; a wildly wrong warm start still converges."""
import numpy as np
import pytest

from paper_1510_05616_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_05616_gb300 import build
    build.build()
    import paper_1510_05616_gb300 as P
    return P


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def test_bounded_wait_times_out_and_context_survives(P, oracle_mod):
    import time
    g, slp, dlp = I.workload("small_n1280")
    s = P.StokesSum(g)
    t0 = time.perf_counter()
    P.stokes_check_wait_timeout(s.h)
    with pytest.raises(P.StokesError) as e:
        P.stokes_sync(s.h)
    assert e.value.code == P.STOKES_ERR_TIMEOUT
    assert 0.3 < time.perf_counter() - t0 < 30.0
    P.stokes_sync(s.h)  # the status was cleared
    out = s.eval(dev(slp), dev(dlp), precision="fp32k").cpu().numpy()
    ref = oracle_mod.sum_nodes(g, slp, dlp)
    assert np.abs(out - ref).max() / np.abs(ref).max() < 1e-6
    s.close()


def test_nonfinite_density_is_reported_and_context_survives(P, oracle_mod):
    g, slp, dlp = I.workload("small_n1280")
    s = P.StokesSum(g)
    bad = slp.copy()
    bad[3, 1] = np.nan
    with pytest.raises(P.StokesError) as e:
        s.eval(dev(bad), dev(dlp), precision="fp32k")
    assert e.value.code == P.STOKES_ERR_NONFINITE
    out = s.eval(dev(slp), dev(dlp), precision="fp64").cpu().numpy()
    ref = oracle_mod.sum_nodes(g, slp, dlp)
    assert np.abs(out - ref).max() / np.abs(ref).max() < 1e-12
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32k"])
def test_wild_warm_start_still_converges(P, prec):
    """A deliberately bad initial guess (noise 1e3 times the solution's size) costs iterations
    but GMRES still ends on the FP64-accurate residual bound at the same solution."""
    g = I.channel(96, I.WALL_SHAPE_SMALL, 3, 32, 0.04, 3, mu=1.0)
    walls = [c for c in g.curves if c.kind == I.KIND_DLP]
    ves = [c for c in g.curves if c.kind == I.KIND_SLP]
    x0 = np.vstack([c.nodes for c in ves])

    def sim():
        h = P.stokes_sim_create(0)
        lo, up = walls
        P.stokes_sim_set_walls(h, lo.n, np.vstack([lo.nodes, up.nodes]),
                               np.concatenate([lo.weights, up.weights]),
                               np.vstack([lo.normals, up.normals]),
                               np.concatenate([lo.curvature, up.curvature]), g.period, 1.0, 24, 96)
        P.stokes_sim_set_vesicles(h, len(ves), ves[0].n, x0, 0.01, 1.0, g.period)
        return h

    h = sim()
    st0 = P.vesicle_step_warmstart(h, 1e-3, 0.5, tol=1e-10, max_iter=400,
                                   precision=P.PRECISIONS[prec])
    _, _, sol0 = P.stokes_sim_get_state(h)
    P.stokes_sim_destroy(h)
    rng = np.random.default_rng(9)
    wild = 1e3 * np.abs(sol0).max() * rng.normal(size=sol0.shape)
    h = sim()
    st1 = P.vesicle_step_warmstart(h, 1e-3, 0.5, P.STOKES_GUESS_USER, guess=dev(wild), tol=1e-10,
                                   max_iter=400, precision=P.PRECISIONS[prec])
    _, _, sol1 = P.stokes_sim_get_state(h)
    P.stokes_sim_destroy(h)
    assert st0["residual"] <= 1e-10 and st1["residual"] <= 1e-10
    assert st1["iterations"] >= st0["iterations"]
    assert np.abs(sol1 - sol0).max() <= 1e-5 * np.abs(sol0).max()
