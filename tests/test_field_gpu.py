"""GPU parity of the pressure and traction outputs (FP64, through the C ABI) against the
pinned NumPy oracle of oracle/sim_oracle.py, and the channel's pressure against the exact
Poiseuille flow (Sec. 5.1)."""
import math

import numpy as np
import pytest

from paper_1510_05616_gb300 import inputs as I

pytestmark = pytest.mark.gpu
MU = 0.7
D = 2 * math.pi


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_05616_gb300 import build
    build.build()
    import paper_1510_05616_gb300 as P
    return P


@pytest.fixture(scope="module")
def S():
    from oracle import sim_oracle
    return sim_oracle


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _interior_points(g, n, rng):
    """Random points inside the channel, off the walls by a margin, away from the vesicles."""
    lo = next(c for c in g.curves if c.kind == I.KIND_DLP)
    ves = np.vstack([c.nodes for c in g.curves if c.kind == I.KIND_SLP]) if g.n_slp else np.zeros((0, 2))
    out = []
    while len(out) < n:
        x = rng.uniform(0, g.period)
        ylo = np.interp(x, lo.nodes[:, 0], lo.nodes[:, 1])
        y = rng.uniform(ylo + 0.15, -ylo - 0.15)
        if len(ves) and np.hypot(ves[:, 0] - x, ves[:, 1] - y).min() < 0.1:
            continue
        out.append((x, y))
    return np.array(out)


def _fields(P, g, slp, dlp, pts, nrm):
    import torch
    s = P.StokesSum(g)
    p = torch.zeros(len(pts), dtype=torch.float64, device="cuda")
    t = torch.zeros((len(pts), 2), dtype=torch.float64, device="cuda")
    P.stokes_sum_eval_pressure(s.h, dev(slp) if g.n_slp else None, dev(dlp) if g.n_dlp else None,
                               dev(pts), p)
    P.stokes_sum_eval_traction(s.h, dev(slp) if g.n_slp else None, dev(dlp) if g.n_dlp else None,
                               dev(pts), dev(nrm), t)
    P.stokes_sync(s.h)
    s.close()
    return p.cpu().numpy(), t.cpu().numpy()


def _oracle(S, g, slp, dlp, pts, nrm):
    kind = np.concatenate([np.full(c.n, c.kind) for c in g.curves])
    return S.layer_fields(g.nodes, g.weights, g.normals, kind,
                          slp if g.n_slp else np.zeros((0, 2)), dlp if g.n_dlp else np.zeros((0, 2)),
                          g.period, g.mu, pts, nrm)


@pytest.mark.parametrize("case", ["channel", "no_images", "walls_only", "vesicles_only", "ragged"])
def test_fields_match_oracle(P, S, case):
    rng = np.random.default_rng(11)
    if case == "ragged":
        g = I.channel(100, I.WALL_SHAPE_SMALL, 5, 18, 0.03, 12, mu=MU)
    else:
        g = I.channel(256, I.WALL_SHAPE_SMALL, 6, 32, 0.04, 13, mu=MU)
    pts = _interior_points(g, 300, rng)
    if case == "no_images":
        g = I.Geometry(g.curves, 0.0, MU)
    elif case == "walls_only":
        g = I.Geometry([c for c in g.curves if c.kind == I.KIND_DLP], D, MU)
    elif case == "vesicles_only":
        g = I.Geometry([c for c in g.curves if c.kind == I.KIND_SLP], D, MU)
    slp, dlp = I.densities(g, 14)
    nrm = rng.normal(size=pts.shape)
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    p, t = _fields(P, g, slp, dlp, pts, nrm)
    pr, tr = _oracle(S, g, slp, dlp, pts, nrm)
    assert np.abs(p - pr).max() / np.abs(pr).max() < 1e-12
    assert np.abs(t - tr).max() / np.abs(tr).max() < 1e-12


def test_field_arguments(P):
    import torch
    g = I.channel(64, I.WALL_SHAPE_SMALL, 2, 16, 0.04, 3, mu=MU)
    slp, dlp = I.densities(g, 3)
    s = P.StokesSum(g)
    pts = dev(np.array([[1.0, 0.0], [2.0, 0.1]]))
    p = torch.zeros(2, dtype=torch.float64, device="cuda")
    P.stokes_sum_eval_pressure(s.h, dev(slp), dev(dlp), pts[:0], p)  # empty: no-op
    assert P.load().stokes_sum_eval_traction(s.h, None, None, 2, None, None, None, None) == P.STOKES_ERR_ARG
    with pytest.raises(P.StokesError):
        P.stokes_sum_eval_pressure(s.h, None, dev(dlp), pts, p)  # vesicles need slp
    s.close()


def test_channel_pressure_is_poiseuille(P, S):
    """The GPU pressure of the pressure-driven channel has the exact Poiseuille differences
    (the additive constant is the representation's) to round-off, and matches the oracle's
    refined block solve."""
    import torch
    lo, up = I.wall_curves(128, I.WALL_SHAPE_SMALL)
    pd = 2 * MU * D * 0.2
    ue = lambda q: np.stack([-(pd / (2 * MU * D)) * q[:, 1] ** 2, 0 * q[:, 1]], 1)
    xw = np.vstack([lo.nodes, up.nodes])
    pts = np.array([[0.8, 0.0], [3.2, 0.0], [4.8, 0.0], [2.0, 0.5], [5.0, -0.4]])
    h = P.stokes_sim_create(0)
    P.stokes_sim_set_walls(h, lo.n, xw, np.concatenate([lo.weights, up.weights]),
                           np.vstack([lo.normals, up.normals]),
                           np.concatenate([lo.curvature, up.curvature]), D, MU, 32, 128)
    out = torch.zeros(len(pts), dtype=torch.float64, device="cuda")
    P.stokes_sim_empty_channel_pressure(h, pd, dev(ue(xw)), dev(pts), out)
    p = out.cpu().numpy()
    P.stokes_sim_destroy(h)
    off = p + pd * pts[:, 0] / D
    assert np.abs(off - off.mean()).max() / pd < 1e-11
    W = S.Walls(lo, up, D, MU, K=32, M=128)
    _, gv = S.empty_channel_rhs(W, pd)
    tau, c = W.solve_refined(ue(xw).reshape(-1), gv)
    ref = W.pressure(tau, c, pts)
    # the proxy weights c are not unique (more proxies than side conditions): solutions with
    # the same velocity may differ in the pressure's additive constant
    dp = p - ref
    assert np.abs(dp - dp.mean()).max() / pd < 1e-11
