"""Pins of the FP64 CPU oracle against what the paper's setting and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an integral identity of Stokes potential theory, an invariance, or a
discrete symmetry.  Together they are chosen so that a dropped term, a wrong
sign, a wrong index or a transposed operand in the oracle fails at least one.
"""
import math

import numpy as np
import pytest

from paper_1510_05616_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

EMPTY = np.zeros((0, 2))


def _as_kind(c, kind):
    return I.Curve(kind, c.nodes, c.weights, c.normals, c.curvature, c.tparam)


def _shapes():
    """A circle, an ellipse and a Fourier-perturbed ellipse, 128 nodes each."""
    pert = ((2, 0.01, 0.3), (3, -0.007, 1.1), (5, 0.004, 2.0))
    return [
        I.closed_curve(128, 1.0, 1.0, (0.2, -0.1), 0.0),
        I.closed_curve(128, 1.0, 0.6, (0.3, -0.2), 0.4),
        I.closed_curve(128, 0.9, 0.55, (-0.1, 0.25), 1.3, pert),
    ]


INSIDE = lambda c: c.nodes.mean(0) + np.array([[0.0, 0.0], [0.15, 0.05], [-0.1, -0.12]])
OUTSIDE = np.array([[3.0, 1.0], [-2.0, 0.5], [0.3, 2.4]])


# ---------------------------------------------------------------------------
# Kress product-rule weights (Sec. 3.2): the rule integrates log(4 sin^2(t/2))
# against trigonometric polynomials exactly; its Fourier coefficients are
# int_0^{2pi} log(4 sin^2(t/2)) e^{ipt} dt = -2 pi / |p| (p != 0), 0 (p = 0).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [4, 8, 64, 128, 256])
def test_kress_weights_fourier_closed_form(oracle_mod, n):
    R = oracle_mod.kress_weights(n)
    F = np.fft.fft(R)
    p = np.arange(n)
    p = np.minimum(p, n - p)
    exact = np.where(p == 0, 0.0, -2 * math.pi / np.maximum(p, 1))
    assert np.abs(F - exact).max() < 1e-12 * n


def test_kress_rejects_odd_n(oracle_mod):
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.kress_weights(63)


# ---------------------------------------------------------------------------
# Pair kernels, Eq. (S) and Eq. (D)
# ---------------------------------------------------------------------------
def test_stokeslet_symmetry_and_scaling(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(20):
        x, y = rng.normal(size=2), rng.normal(size=2)
        mu = rng.uniform(0.3, 3.0)
        S = oracle_mod.stokeslet(x, y, mu)
        assert np.allclose(S, S.T, rtol=0, atol=1e-15)
        assert np.allclose(S, oracle_mod.stokeslet(y, x, mu), rtol=0, atol=1e-15)
        assert np.allclose(S * mu, oracle_mod.stokeslet(x, y, 1.0), rtol=1e-14, atol=1e-15)


def test_stokeslet_special_values(oracle_mod):
    # |r| = 1 along x: log term vanishes, r r^T / r^2 = e1 e1^T.
    S = oracle_mod.stokeslet([1.0, 0.0], [0.0, 0.0], 1.0)
    assert np.allclose(S, np.array([[1.0, 0.0], [0.0, 0.0]]) / (4 * math.pi), atol=1e-16)
    # |r| = e along y: log(1/r) = -1 on the diagonal.
    S = oracle_mod.stokeslet([0.0, math.e], [0.0, 0.0], 1.0)
    assert np.allclose(S, np.array([[-1.0, 0.0], [0.0, 0.0]]) / (4 * math.pi), atol=1e-16)


def test_stresslet_symmetry_and_special_values(oracle_mod):
    rng = np.random.default_rng(2)
    for _ in range(20):
        x, y = rng.normal(size=2), rng.normal(size=2)
        n = rng.normal(size=2)
        n /= np.linalg.norm(n)
        D = oracle_mod.stresslet(x, y, n)
        assert np.allclose(D, D.T, atol=1e-15)
        # odd under r -> -r: D(y, x) with the same normal is -D(x, y)
        assert np.allclose(oracle_mod.stresslet(y, x, n), -D, atol=1e-15)
        # tangential source displacement: r . n = 0 gives zero
        t = np.array([-n[1], n[0]])
        assert np.abs(oracle_mod.stresslet(y + 0.7 * t, y, n)).max() < 1e-15
    D = oracle_mod.stresslet([2.0, 0.0], [0.0, 0.0], [1.0, 0.0])
    assert np.allclose(D, np.array([[1.0, 0.0], [0.0, 0.0]]) / (2 * math.pi), atol=1e-16)


# ---------------------------------------------------------------------------
# Double-layer identities on closed curves (Eq. (JR), Sec. 2.3 diagonal limit)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", range(3))
def test_dlp_constant_density_jump(oracle_mod, shape):
    c = _as_kind(_shapes()[shape], I.KIND_DLP)
    g = I.Geometry([c], 0.0, 1.0)
    tau = np.tile([0.7, -1.3], (c.n, 1))
    on = oracle_mod.sum_nodes(g, EMPTY, tau)
    assert np.abs(on + 0.5 * tau).max() < 1e-12          # PV + curvature diagonal
    lim = oracle_mod.sum_nodes(g, EMPTY, tau, jump=-0.5)
    assert np.abs(lim + tau).max() < 1e-12               # interior limit, Eq. (JR)
    inn = oracle_mod.sum_free(g, EMPTY, tau, INSIDE(c))
    assert np.abs(inn + tau[:3]).max() < 1e-12
    out = oracle_mod.sum_free(g, EMPTY, tau, OUTSIDE)
    assert np.abs(out).max() < 1e-12


@pytest.mark.parametrize("shape", range(3))
def test_dlp_rigid_rotation(oracle_mod, shape):
    """A rigid rotation has zero traction, so Green's formula gives D[u] = -u inside."""
    c = _as_kind(_shapes()[shape], I.KIND_DLP)
    g = I.Geometry([c], 0.0, 1.0)
    rot = lambda p: np.stack([-p[:, 1], p[:, 0]], 1)
    u = rot(c.nodes)
    assert np.abs(oracle_mod.sum_nodes(g, EMPTY, u) + 0.5 * u).max() < 1e-12
    pts = INSIDE(c)
    assert np.abs(oracle_mod.sum_free(g, EMPTY, u, pts) + rot(pts)).max() < 1e-12
    assert np.abs(oracle_mod.sum_free(g, EMPTY, u, OUTSIDE)).max() < 1e-12


def test_dlp_curvature_diagonal_sign(oracle_mod):
    """Dropping or flipping the curvature diagonal breaks the constant-density identity."""
    c = _as_kind(_shapes()[1], I.KIND_DLP)
    tau = np.tile([0.4, 1.1], (c.n, 1))
    g = I.Geometry([c], 0.0, 1.0)
    on = oracle_mod.sum_nodes(g, EMPTY, tau)
    flat = I.Geometry([I.Curve(I.KIND_DLP, c.nodes, c.weights, c.normals, 0 * c.curvature, c.tparam)], 0.0)
    assert np.abs(oracle_mod.sum_nodes(flat, EMPTY, tau) + 0.5 * tau).max() > 1e-4
    assert np.abs(on + 0.5 * tau).max() < 1e-12


# ---------------------------------------------------------------------------
# Single layer with the Kress self rule (Sec. 3.2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", range(3))
def test_slp_of_normal_vanishes(oracle_mod, shape):
    """int S(x, y) n(y) ds_y = 0 everywhere: the stokeslet is divergence free."""
    c = _shapes()[shape]
    g = I.Geometry([c], 0.0, 0.7)
    assert np.abs(oracle_mod.sum_nodes(g, c.normals, EMPTY)).max() < 1e-12
    assert np.abs(oracle_mod.sum_free(g, c.normals, EMPTY, INSIDE(c))).max() < 1e-12
    assert np.abs(oracle_mod.sum_free(g, c.normals, EMPTY, OUTSIDE)).max() < 1e-12


def _stokeslet_flow(pts, y0, F, mu):
    r = pts - y0
    rr = (r * r).sum(1)
    return ((np.log(1 / np.sqrt(rr))[:, None] * F + r * ((r @ F) / rr)[:, None]) / (4 * math.pi * mu))


def _stokeslet_traction(pts, nrm, y0, F):
    """Traction of the stokeslet flow, Eq. (K): -(1/pi) r (r.F) (r.n_x) / r^4."""
    r = pts - y0
    rr = (r * r).sum(1)
    return -(1 / math.pi) * r * ((r @ F) * (r * nrm).sum(1) / rr**2)[:, None]


@pytest.mark.parametrize("shape", range(3))
@pytest.mark.parametrize("mu", [1.0, 0.7])
def test_green_representation(oracle_mod, shape, mu):
    """u = S[f] - D[u] inside, u/2 on the curve, 0 outside, for an exterior stokeslet flow."""
    c = _shapes()[shape]
    y0, F = np.array([2.5, 1.0]), np.array([0.8, -0.5])
    u = _stokeslet_flow(c.nodes, y0, F, mu)
    f = _stokeslet_traction(c.nodes, c.normals, y0, F)
    gs = I.Geometry([c], 0.0, mu)
    gd = I.Geometry([_as_kind(c, I.KIND_DLP)], 0.0, mu)
    on = oracle_mod.sum_nodes(gs, f, EMPTY) - oracle_mod.sum_nodes(gd, EMPTY, u)
    assert np.abs(on - 0.5 * u).max() < 1e-12
    pin = INSIDE(c)
    val = oracle_mod.sum_free(gs, f, EMPTY, pin) - oracle_mod.sum_free(gd, EMPTY, u, pin)
    assert np.abs(val - _stokeslet_flow(pin, y0, F, mu)).max() < 1e-12
    val = oracle_mod.sum_free(gs, f, EMPTY, OUTSIDE) - oracle_mod.sum_free(gd, EMPTY, u, OUTSIDE)
    assert np.abs(val).max() < 1e-12


def test_kress_self_is_spectral(oracle_mod):
    """Green's identity on the curve converges spectrally in n (the product rule is exact
    on the log part); a plain trapezoid self rule would stall at O(h log h)."""
    y0, F, mu = np.array([2.0, 0.7]), np.array([0.3, 1.0]), 1.0
    errs = []
    for n in (16, 32, 64):
        c = I.closed_curve(n, 1.0, 0.7, (0.0, 0.0), 0.2)
        u = _stokeslet_flow(c.nodes, y0, F, mu)
        f = _stokeslet_traction(c.nodes, c.normals, y0, F)
        on = oracle_mod.sum_nodes(I.Geometry([c], 0.0, mu), f, EMPTY) \
            - oracle_mod.sum_nodes(I.Geometry([_as_kind(c, I.KIND_DLP)], 0.0, mu), EMPTY, u)
        errs.append(np.abs(on - 0.5 * u).max())
    assert errs[1] < 1e-2 * errs[0] and errs[2] < 1e-4 * errs[1] + 1e-14


# ---------------------------------------------------------------------------
# Periodic channel: images, invariances, symmetry
# ---------------------------------------------------------------------------
def _tiny_channel(seed=7, n_w=64, n_ves=3, n_v=16):
    g = I.channel(n_w, I.WALL_SHAPE_SMALL, n_ves, n_v, 0.05, seed)
    slp, dlp = I.densities(g, seed)
    return g, slp, dlp


def _tiled(g):
    """The cell's curves copied to shifts -d, 0, +d as separate curves, images off."""
    d = g.period
    order = [0, -1, 1]
    cs = [I.Curve(c.kind, c.nodes + np.array([m * d, 0.0]), c.weights, c.normals, c.curvature, c.tparam)
          for m in order for c in g.curves]
    return I.Geometry(cs, 0.0, g.mu)


def test_images_equal_explicit_tiling(oracle_mod):
    g, slp, dlp = _tiny_channel()
    per = oracle_mod.sum_nodes(g, slp, dlp)
    t = _tiled(g)
    til = oracle_mod.sum_nodes(t, np.vstack([slp] * 3), np.vstack([dlp] * 3),
                               select=np.arange(g.n_nodes))
    assert np.abs(per - til).max() < 1e-13 * np.abs(per).max()
    # and the images matter: switching them off changes the answer
    off = oracle_mod.sum_nodes(g, slp, dlp, period=0.0)
    assert np.abs(per - off).max() > 1e-3 * np.abs(per).max()


@pytest.mark.parametrize("shift", [(0.37, -0.21), (2 * math.pi, 0.0), (-1.3, 4.0)])
def test_translation_invariance(oracle_mod, shift):
    g, slp, dlp = _tiny_channel()
    a = oracle_mod.sum_nodes(g, slp, dlp)
    b = oracle_mod.sum_nodes(g.translated(shift), slp, dlp)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_slp_reciprocity(oracle_mod):
    """sum_i w_i g_i . (S f)_i = sum_j w_j f_j . (S g)_j for the full discrete periodic
    single-layer operator, Kress self blocks included (R_k even in k; L, M symmetric)."""
    g = I.channel(64, I.WALL_SHAPE_SMALL, 5, 32, 0.05, 11)
    ves = I.Geometry([c for c in g.curves if c.kind == I.KIND_SLP], g.period, 0.8)
    rng = np.random.default_rng(5)
    f = rng.normal(size=(ves.n_nodes, 2))
    h = rng.normal(size=(ves.n_nodes, 2))
    Sf = oracle_mod.sum_nodes(ves, f, EMPTY)
    Sh = oracle_mod.sum_nodes(ves, h, EMPTY)
    w = ves.weights[:, None]
    lhs, rhs = (w * h * Sf).sum(), (w * f * Sh).sum()
    assert abs(lhs - rhs) < 1e-13 * (np.abs(w * h * Sf).sum())


def test_slp_scales_as_inverse_mu_dlp_independent(oracle_mod):
    g, slp, dlp = _tiny_channel()
    a = oracle_mod.sum_nodes(g, slp, 0 * dlp, mu=1.0)
    b = oracle_mod.sum_nodes(g, slp, 0 * dlp, mu=0.25)
    assert np.abs(4 * a - b).max() < 1e-13 * np.abs(b).max()
    c = oracle_mod.sum_nodes(g, 0 * slp, dlp, mu=1.0)
    e = oracle_mod.sum_nodes(g, 0 * slp, dlp, mu=0.25)
    assert np.abs(c - e).max() < 1e-15 * np.abs(c).max()


def test_linearity_and_selection(oracle_mod):
    g, slp, dlp = _tiny_channel()
    full = oracle_mod.sum_nodes(g, slp, dlp)
    parts = oracle_mod.sum_nodes(g, slp, 0 * dlp) + oracle_mod.sum_nodes(g, 0 * slp, dlp)
    assert np.abs(full - parts).max() < 1e-13 * np.abs(full).max()
    sel = np.array([0, 5, g.n_nodes - 1, 70, 64])
    assert np.array_equal(oracle_mod.sum_nodes(g, slp, dlp, select=sel), full[sel])


def test_thread_count_does_not_change_bits(oracle_mod):
    g, slp, dlp = _tiny_channel()
    a = oracle_mod.sum_nodes(g, slp, dlp, threads=1)
    b = oracle_mod.sum_nodes(g, slp, dlp, threads=4)
    assert np.array_equal(a, b)


def test_free_targets_match_far_nodes(oracle_mod):
    """A wall-only geometry evaluated at a free point equals the node sum minus nothing when
    the point is a node of a different curve: check via the vesicle-free channel."""
    g, slp, dlp = _tiny_channel(n_ves=0)
    # free point = a vesicle-free interior point; compare with explicit image sum of Eq. (D)
    p = np.array([[1.0, 0.2]])
    val = oracle_mod.sum_free(g, EMPTY, dlp, p)[0]
    acc = np.zeros(2)
    for m in (-1, 0, 1):
        for y, n, w, t in zip(g.nodes, g.normals, g.weights, dlp):
            acc += oracle_mod.stresslet(p[0], y + np.array([m * g.period, 0.0]), n) @ (w * t)
    assert np.abs(val - acc).max() < 1e-14 * np.abs(acc).max()


def test_bad_inputs_rejected(oracle_mod):
    c = I.closed_curve(15, 1.0, 0.6)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.sum_nodes(I.Geometry([c], 0.0), np.ones((15, 2)), EMPTY)


def test_empty_geometry(oracle_mod):
    g = I.Geometry([], 2 * math.pi)
    assert oracle_mod.sum_nodes(g, EMPTY, EMPTY).shape == (0, 2)
    assert np.array_equal(oracle_mod.sum_free(g, EMPTY, EMPTY, np.ones((3, 2))), np.zeros((3, 2)))
