"""Pins of the close-evaluation oracle (single layer of a closed curve at targets near it)
against closed forms, the divergence theorem and the plain sum far away."""
import math

import numpy as np
import pytest

from oracle import close_oracle as C
from oracle import sim_oracle as S

PI = math.pi


def circle(n, R=0.7):
    t = 2 * PI * np.arange(n) / n
    return np.stack([R * np.cos(t), R * np.sin(t)], 1), t


def ellipse(n, a=0.9, b=0.5, eps=0.05):
    t = 2 * PI * np.arange(n) / n
    rho = 1 + eps * np.cos(3 * t)
    return np.stack([a * rho * np.cos(t), b * rho * np.sin(t)], 1), t


def test_upsampling_is_exact_for_trigonometric_polynomials():
    """Resampling reproduces a trigonometric polynomial (Nyquist cosine included) and its
    derivative at the fine points."""
    n, K = 16, 4
    f = lambda t: 1 + np.cos(3 * t) + 0.5 * np.sin(5 * t) + 0.3 * np.cos(8 * t)
    df = lambda t: -3 * np.sin(3 * t) + 2.5 * np.cos(5 * t) - 2.4 * np.sin(8 * t)
    t = 2 * PI * np.arange(n) / n
    tf = 2 * PI * np.arange(n * K) / (n * K)
    assert np.abs(C.upsample(f(t), K) - f(tf)).max() < 1e-13
    assert np.abs(C.upsample(f(t), K, derivative=True) - df(tf)).max() < 1e-12
    t7 = 2 * PI * np.arange(15) / 15  # odd n: no Nyquist mode
    tf7 = 2 * PI * np.arange(45) / 45
    g = lambda t: np.sin(2 * t) - np.cos(7 * t)
    assert np.abs(C.upsample(g(t7), 3) - g(tf7)).max() < 1e-13


def _constant_density_exact(z, R, e, mu):
    """Single layer of the constant density e on the circle of radius R, complex arithmetic.
    int log|x - y| ds is 2 pi R log R inside (mean-value property) and 2 pi R log|z| outside;
    (r . e) r / |r|^2 = e/2 + conj(e) r / (2 conj(r)), and int r / conj(r) ds (a contour integral
    in e^{i theta}) is 0 inside and 2 pi R (z - R^2 / conj(z)) / conj(z) outside."""
    E = e[0] + 1j * e[1]
    if abs(z) < R:
        u = -2 * PI * R * math.log(R) * E + PI * R * E
    else:
        u = (-2 * PI * R * math.log(abs(z)) * E + PI * R * E
             + PI * R * np.conj(E) * (z - R * R / np.conj(z)) / np.conj(z))
    return u / (4 * PI * mu)


@pytest.mark.parametrize("frac", [0.1, 1 / 3, 1.0])
def test_constant_density_on_a_circle(frac):
    """Closed forms inside and outside, at a fraction of the node spacing from the curve; the
    plain n-point sum misses them by orders of magnitude at the closest distance."""
    n, R, mu = 32, 0.7, 0.8
    x, _ = circle(n, R)
    e = np.array([0.3, -0.8])
    h = 2 * PI * R / n
    ang = np.array([0.05, 1.3, 2.9, 4.4])
    pts, ref = [], []
    for side in (-1, 1):
        rr = R + side * frac * h
        for a in ang:
            z = rr * complex(math.cos(a), math.sin(a))
            pts.append([z.real, z.imag])
            ref.append(_constant_density_exact(z, R, e, mu))
    pts = np.array(pts)
    ref = np.array(ref)
    u = C.close_slp(x, np.tile(e, (n, 1)), pts, mu, K=128)
    err = np.abs(u[:, 0] + 1j * u[:, 1] - ref).max() / np.abs(ref).max()
    assert err < 1e-11, err
    if frac == 0.1:  # the plain trapezoid sum at the same targets
        w = np.full(n, h)
        plain = np.einsum("tjab,jb->ta", S.stokeslet(pts[:, None, :], x[None], mu) * w[None, :, None, None],
                          np.tile(e, (n, 1)))
        perr = np.abs(plain[:, 0] + 1j * plain[:, 1] - ref).max() / np.abs(ref).max()
        assert perr > 1e-3, perr


@pytest.mark.parametrize("shape,tol", [("circle", 1e-12), ("ellipse", 1e-9)])
def test_single_layer_of_the_normal_vanishes(shape, tol):
    """The stokeslet is divergence-free in the source point, so the single layer of the unit
    normal vanishes off the curve, inside and outside (divergence theorem); close targets."""
    n = 32 if shape == "circle" else 128
    x, t = circle(n) if shape == "circle" else ellipse(n)
    dy = C.upsample(x, 1, derivative=True)
    nrm = np.stack([dy[:, 1], -dy[:, 0]], 1) / np.sqrt((dy * dy).sum(1))[:, None]  # outward (ccw)
    h = np.sqrt((np.diff(np.vstack([x, x[:1]]), axis=0) ** 2).sum(1)).max()
    idx = np.arange(0, n, n // 8)
    mid = 0.5 * (x[idx] + x[(idx + 1) % n])
    nm = nrm[idx]
    pts = np.vstack([mid + 0.2 * h * nm, mid - 0.2 * h * nm, mid + 2 * h * nm, mid - 2 * h * nm])
    u = C.close_slp(x, nrm, pts, 1.0, K=128)
    scale = np.abs(C.close_slp(x, np.tile([1.0, 0.0], (n, 1)), pts, 1.0, K=128)).max()
    assert np.abs(u).max() / scale < tol, np.abs(u).max() / scale


@pytest.mark.parametrize("k", [0, 1, 3, 7])
def test_log_potential_of_circle_modes(k):
    """int log|x - y| cos(k theta') ds on the circle of radius R: 2 pi R log max(r, R) for k = 0,
    -(pi R / k) (r/R)^k cos(k theta) inside and -(pi R / k) (R/r)^k cos(k theta) outside."""
    n, R = 32, 0.7
    x, t = circle(n, R)
    h = 2 * PI * R / n
    pts, ref = [], []
    for rr in (R - 0.1 * h, R + 0.1 * h, 0.3 * R, 2 * R):
        for a in (0.2, 2.1, 4.0):
            pts.append([rr * math.cos(a), rr * math.sin(a)])
            if k == 0:
                ref.append(2 * PI * R * math.log(max(rr, R)))
            else:
                q = (rr / R) ** k if rr < R else (R / rr) ** k
                ref.append(-(PI * R / k) * q * math.cos(k * a))
    got = C.log_potential(x, np.cos(k * t), np.array(pts), K=128)
    ref = np.array(ref)
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-12


def test_far_targets_match_the_plain_sum():
    """Six node spacings away the plain n-point trapezoid sum (weights from the step oracle's
    spectral speed) is already converged: both agree to round-off."""
    n, mu = 64, 0.9
    x, t = ellipse(n)
    rng = np.random.default_rng(3)
    f = np.zeros((n, 2))
    for kk in range(0, 9):
        f += np.outer(np.cos(kk * t), rng.normal(size=2)) + np.outer(np.sin(kk * t), rng.normal(size=2))
    _, w = S.curve_normals_weights(x)
    h = w.max()
    cx = x.mean(0)
    ang = np.linspace(0, 2 * PI, 9)[:-1]
    pts = np.stack([cx[0] + 1.2 * np.cos(ang) + 6 * h * np.cos(ang),
                    cx[1] + 0.8 * np.sin(ang) + 6 * h * np.sin(ang)], 1)
    plain = np.einsum("tjab,jb->ta", S.stokeslet(pts[:, None, :], x[None], mu) * w[None, :, None, None], f)
    u = C.close_slp(x, f, pts, mu, K=8)
    assert np.abs(u - plain).max() / np.abs(plain).max() < 1e-11


def test_converges_in_the_upsampling():
    """At a tenth of the node spacing the plain sum (K = 1) is off by percents; the error against
    the K = 128 value falls monotonically with K, faster than geometrically, to round-off."""
    n, mu = 64, 1.0
    x, t = ellipse(n)
    f = np.stack([1 + 0.5 * np.cos(2 * t), np.sin(3 * t)], 1)
    dy = C.upsample(x, 1, derivative=True)
    nrm = np.stack([dy[:, 1], -dy[:, 0]], 1) / np.sqrt((dy * dy).sum(1))[:, None]
    h = np.sqrt((dy * dy).sum(1)).max() * 2 * PI / n
    pts = np.vstack([x[::8] + 0.1 * h * nrm[::8], x[::8] - 0.1 * h * nrm[::8]])
    Ks = (1, 2, 4, 8, 16, 32, 64, 128)
    us = [C.close_slp(x, f, pts, mu, K=K) for K in Ks]
    e = [np.abs(u - us[-1]).max() / np.abs(us[-1]).max() for u in us[:-1]]
    assert e[0] > 1e-2, e
    assert all(e[i + 1] < e[i] for i in range(len(e) - 1)), e
    assert e[-1] < 1e-13 and e[-2] < 1e-10, e
