"""Pins of the pressure and traction oracle (oracle/sim_oracle.py: slp_pressure, dlp_pressure,
layer_fields, Walls.pressure).

The pressure kernels Q, P (Eq. (Q), (P)) are pinned by the Stokes equations themselves,
grad p = mu Laplacian u, with u from the velocity kernels and derivatives by finite
differences; the summed fields of a channel with vesicles by the same identity and by the
traction sigma(u, p) n (Eq. (Tup)) against finite differences of the separately pinned C
velocity oracle; the channel's pressure by the exact Poiseuille flow (Sec. 5.1).
"""
import math
import warnings

import numpy as np
import pytest

from paper_1510_05616_gb300 import inputs as I

warnings.filterwarnings("ignore", category=RuntimeWarning)
PI = math.pi
MU = 0.7
D = 2 * PI


@pytest.fixture(scope="module")
def S():
    from oracle import sim_oracle
    return sim_oracle


def _grad(f, x, h):
    return np.stack([(f(x + e) - f(x - e)) / (2 * h) for e in (np.array([h, 0.0]), np.array([0.0, h]))], -1)


def _lap(f, x, h):
    out = -4.0 * f(x)
    for e in (np.array([h, 0.0]), np.array([0.0, h])):
        out = out + f(x + e) + f(x - e)
    return out / (h * h)


def test_pressure_kernels_satisfy_stokes(S):
    """grad (Q F) = mu Lap (S F) and grad (P F) = mu Lap (D F), away from the source."""
    rng = np.random.default_rng(1)
    for _ in range(6):
        x, y = rng.normal(size=2), rng.normal(size=2)
        ny = rng.normal(size=2)
        ny /= np.linalg.norm(ny)
        for F in np.eye(2):
            gq = _grad(lambda z: S.slp_pressure(z, y) @ F, x, 1e-5)
            lq = MU * _lap(lambda z: S.stokeslet(z, y, MU) @ F, x, 1e-3)
            assert np.allclose(gq, lq, rtol=1e-5, atol=1e-6 * np.abs(gq).max())
            gp = _grad(lambda z: S.dlp_pressure(z, y, ny, MU) @ F, x, 1e-5)
            lp = MU * _lap(lambda z: S.stresslet(z, y, ny) @ F, x, 1e-3)
            assert np.allclose(gp, lp, rtol=1e-5, atol=1e-6 * np.abs(gp).max())


def test_pressure_kernels_far_field_and_sign(S):
    """Q is the pressure of a point force F: p = F . r / (2 pi r^2), largest ahead of the force;
    P of a double layer falls off like 1/r^2."""
    y = np.zeros(2)
    F = np.array([1.0, 0.0])
    assert S.slp_pressure(np.array([1.0, 0.0]), y) @ F == pytest.approx(1 / (2 * PI))
    assert S.slp_pressure(np.array([-1.0, 0.0]), y) @ F == pytest.approx(-1 / (2 * PI))
    ny = np.array([0.0, 1.0])
    a = np.abs(S.dlp_pressure(np.array([10.0, 3.0]), y, ny, MU)).max()
    b = np.abs(S.dlp_pressure(np.array([20.0, 6.0]), y, ny, MU)).max()
    assert a / b == pytest.approx(4.0, rel=1e-12)


def _channel(seed=5):
    g = I.channel(96, I.WALL_SHAPE_SMALL, 3, 32, 0.05, seed, mu=MU)
    slp, dlp = I.densities(g, seed)
    kind = np.concatenate([np.full(c.n, c.kind) for c in g.curves])
    return g, slp, dlp, kind


def test_layer_fields_satisfy_stokes_with_the_c_velocity(S, oracle_mod):
    """The summed pressure (images, weights, both kinds) against grad p = mu Lap u, with u
    from the independent C oracle at free points."""
    g, slp, dlp, kind = _channel()
    pts = np.array([[0.7, 0.1], [3.3, -0.2], [5.9, 0.3]])
    h = 2e-3

    def u(z):
        return oracle_mod.sum_free(g, slp, dlp, np.atleast_2d(z))[0]

    def p(z):
        return S.layer_fields(g.nodes, g.weights, g.normals, kind, slp, dlp, D, MU, z)[0][0]

    for x in pts:
        gp = _grad(p, x, 1e-5)
        lu = MU * _lap(u, x, h)
        assert np.allclose(gp, lu, rtol=1e-4, atol=1e-5 * np.abs(lu).max())


def test_layer_traction_is_sigma_n_of_the_c_velocity(S, oracle_mod):
    """T = -p n + mu (grad u + grad u^T) n (Eq. (Tup)) with u from the C oracle."""
    g, slp, dlp, kind = _channel(7)
    pts = np.array([[1.1, 0.0], [4.2, 0.25]])
    rng = np.random.default_rng(2)
    nrm = rng.normal(size=pts.shape)
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    p, t = S.layer_fields(g.nodes, g.weights, g.normals, kind, slp, dlp, D, MU, pts, nrm)
    for k, x in enumerate(pts):
        gu = _grad(lambda z: oracle_mod.sum_free(g, slp, dlp, np.atleast_2d(z))[0], x, 1e-5)
        ref = -p[k] * nrm[k] + MU * ((gu + gu.T) @ nrm[k])
        assert np.allclose(t[k], ref, rtol=1e-6, atol=1e-7 * np.abs(ref).max())


def test_layer_fields_period_translation(S):
    """Translating sources and targets together by any vector changes nothing."""
    g, slp, dlp, kind = _channel(9)
    pts = np.array([[2.0, 0.1], [4.0, -0.3]])
    nrm = np.array([[1.0, 0.0], [0.0, 1.0]])
    p0, t0 = S.layer_fields(g.nodes, g.weights, g.normals, kind, slp, dlp, D, MU, pts, nrm)
    sh = np.array([0.37, -1.1])
    p1, t1 = S.layer_fields(g.nodes + sh, g.weights, g.normals, kind, slp, dlp, D, MU, pts + sh, nrm)
    assert np.allclose(p0, p1, rtol=1e-12, atol=1e-12 * np.abs(p0).max())
    assert np.allclose(t0, t1, rtol=1e-12, atol=1e-12 * np.abs(t0).max())


def test_poiseuille_pressure(S):
    """Exact flow u = (-p_drive/(2 mu d) y^2, 0), p = -p_drive x / d + const: the channel's
    pressure (least-squares solve of the discretised system) has the exact differences."""
    lo, up = I.wall_curves(128, I.WALL_SHAPE_SMALL)
    W = S.Walls(lo, up, D, MU, K=32, M=128)
    pd = 2 * MU * D * 0.2
    ue = lambda q: np.stack([-(pd / (2 * MU * D)) * q[:, 1] ** 2, 0 * q[:, 1]], 1)
    _, gvec = S.empty_channel_rhs(W, pd)
    tau, c = W.solve_lstsq(ue(W.x).reshape(-1), gvec)
    pts = np.array([[0.8, 0.0], [3.2, 0.0], [4.8, 0.0], [2.0, 0.5], [5.0, -0.4]])
    p = W.pressure(tau, c, pts)
    pe = -pd * pts[:, 0] / D
    off = p - pe
    assert np.abs(off - off.mean()).max() / pd < 1e-10
