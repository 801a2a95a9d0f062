"""Brute-force pin of the FP64 oracle: the same discrete sum assembled as dense operators in
extended precision (``numpy.longdouble``) on tiny geometries (N <= 40), agreeing to 1e-14.

This restatement is written independently of ``oracle/stokes_oracle.c``: it forms the full
stokeslet and stresslet matrices of every (target, source, image) triple at once with masks for
the skipped pairs (own curve at m = 0 for vesicles, own node at m = 0 for walls; Eq. (S),
Eq. (D), the near-image sums of Eq. (Dnr) and Eq. (utotrep)), adds the Nystrom diagonal of
Sec. 2.3 and the Kress self block of Sec. 3.2 as matrices, and applies them to the densities --
no per-target loop and no FP64 rounding, so a dropped term, a wrong sign or index, or
accumulated FP64 rounding in the oracle would show.
"""
import numpy as np
import pytest

from paper_1510_05616_gb300 import inputs as I

LD = np.longdouble
PI = 4 * np.arctan(LD(1))


def _ld(a):
    return np.asarray(a, dtype=LD)


def kress_R(n):
    j = np.arange(n, dtype=LD)
    p = np.arange(1, n // 2, dtype=LD)
    acc = (np.cos(2 * PI * np.outer(j, p) / n) / p).sum(1)
    return -(4 * PI / n) * acc - (4 * PI / (LD(n) * n)) * np.where(np.arange(n) % 2, -1, 1)


def brute_force(geom, slp, dlp, jump=0.0):
    x = _ld(geom.nodes)
    w = _ld(geom.weights)
    nr = _ld(geom.normals)
    kap = _ld(geom.curvature)
    off = geom.curve_offset
    N = x.shape[0]
    curve = np.repeat(np.arange(len(off) - 1), np.diff(off))
    is_slp = ~geom.kind_mask(I.KIND_DLP)
    dens = np.zeros((N, 2), dtype=LD)
    dens[is_slp] = _ld(slp).reshape(-1, 2)
    dens[~is_slp] = _ld(dlp).reshape(-1, 2)
    mu = LD(geom.mu)
    d = LD(geom.period)
    images = (-1, 0, 1) if geom.period != 0 else (0,)
    # operator K[i, a, j, b]: velocity component a at node i per density component b at node j
    K = np.zeros((N, 2, N, 2), dtype=LD)
    eye = np.eye(2, dtype=LD)
    for m in images:
        r = x[:, None, :] - (x[None, :, :] + np.array([m * d, LD(0)], dtype=LD))
        rr = (r * r).sum(-1)
        skip = np.zeros((N, N), dtype=bool)
        if m == 0:
            skip = (curve[:, None] == curve[None, :]) & is_slp[None, :]
            skip |= np.eye(N, dtype=bool) & ~is_slp[None, :]
        rr_safe = np.where(skip, LD(1), rr)
        rrT = r[..., :, None] * r[..., None, :] / rr_safe[..., None, None]
        S = (-LD(0.5) * np.log(rr_safe))[..., None, None] * eye + rrT
        S = S * (w / (4 * PI * mu))[None, :, None, None]
        rn = (r * nr[None, :, :]).sum(-1)
        D = rrT * (rn / (PI * rr_safe))[..., None, None] * w[None, :, None, None]
        blk = np.where(is_slp[None, :, None, None], S, D)
        blk[skip] = 0
        K += blk.transpose(0, 2, 1, 3)
    # Nystrom diagonal of the walls and the jump
    for i in np.nonzero(~is_slp)[0]:
        t = np.array([-nr[i, 1], nr[i, 0]], dtype=LD)
        K[i, :, i, :] += -kap[i] / (2 * PI) * w[i] * np.outer(t, t) + LD(jump) * eye
    # Kress self blocks of the vesicles
    for c in range(len(off) - 1):
        b, e = off[c], off[c + 1]
        if not is_slp[b]:
            continue
        n = e - b
        R = kress_R(n)
        h = 2 * PI / n
        s = w[b:e] / h
        for a in range(n):
            for k in range(n):
                if k == a:
                    L = np.log(s[k] * s[k])
                    t = np.array([-nr[b + k, 1], nr[b + k, 0]], dtype=LD)
                    M = np.outer(t, t)
                else:
                    r = x[b + a] - x[b + k]
                    rr = (r * r).sum()
                    sn = np.sin(PI * (a - k) / n)
                    L = np.log(rr / (4 * sn * sn))
                    M = np.outer(r, r) / rr
                coef = (-LD(0.5) * R[(a - k) % n] + h * (-LD(0.5) * L)) * eye + h * M
                K[b + a, :, b + k, :] += coef * s[k] / (4 * PI * mu)
    return np.einsum("iajb,jb->ia", K, dens)


def _tiny(n_w, n_vs, period, seed):
    rng = np.random.default_rng(seed)
    curves = list(I.wall_curves(n_w, I.WALL_SHAPE_SMALL)) if n_w else []
    xs = np.linspace(0.8, 5.2, max(len(n_vs), 1))
    for k, n in enumerate(n_vs):
        curves.append(I.closed_curve(n, 0.35, 0.22, center=(xs[k], rng.uniform(-0.3, 0.3)),
                                     angle=rng.uniform(0, np.pi),
                                     pert=((3, 0.02, 0.4),) if k % 2 else ()))
    g = I.Geometry(curves, period, mu=0.7)
    slp = rng.normal(size=(g.n_slp, 2))
    dlp = rng.normal(size=(g.n_dlp, 2))
    return g, slp, dlp


CASES = [  # (wall nodes per wall, vesicle node counts, period)
    (12, (8, 8), 2 * np.pi),
    (8, (6, 10, 8), 2 * np.pi),
    (0, (16, 12, 8), 2 * np.pi),
    (16, (), 2 * np.pi),
    (10, (10, 10), 0.0),
]


@pytest.mark.parametrize("n_w,n_vs,period", CASES)
@pytest.mark.parametrize("jump", [0.0, -0.5])
def test_oracle_equals_extended_precision_brute_force(oracle_mod, n_w, n_vs, period, jump):
    g, slp, dlp = _tiny(n_w, n_vs, period, seed=n_w + 7 * len(n_vs))
    assert g.n_nodes <= 40
    ref = brute_force(g, slp, dlp, jump)
    out = oracle_mod.sum_nodes(g, slp, dlp, jump=jump)
    err = np.abs(out - ref.astype(np.float64)).max(0) / np.abs(ref.astype(np.float64)).max(0)
    assert np.all(err <= 1e-14), err


def test_brute_force_catches_a_planted_mistake(oracle_mod):
    """The comparison is sharp: a flipped sign of one wall normal (as a wrong orientation in
    either side would be) moves the result by far more than the bound."""
    g, slp, dlp = _tiny(12, (8, 8), 2 * np.pi, seed=3)
    ref = brute_force(g, slp, dlp).astype(np.float64)
    g.curves[0].normals[5] *= -1.0
    out = oracle_mod.sum_nodes(g, slp, dlp)
    assert np.abs(out - ref).max() / np.abs(ref).max() > 1e-6
