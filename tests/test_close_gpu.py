"""GPU close evaluation of the vesicles' single layer at nearby nodes against the close oracle."""
import math

import numpy as np
import pytest

from paper_1510_05616_gb300 import inputs as I

pytestmark = pytest.mark.gpu
PI = math.pi
MU = 0.8


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


def vesicle(n, c, a, b, rot):
    from oracle import close_oracle as C
    t = 2 * PI * np.arange(n) / n
    rho = 1 + 0.05 * np.cos(3 * t)
    p = np.stack([a * rho * np.cos(t), b * rho * np.sin(t)], 1)
    R = np.array([[math.cos(rot), -math.sin(rot)], [math.sin(rot), math.cos(rot)]])
    p = p @ R.T + np.asarray(c)
    dy = C.upsample(p, 1, derivative=True)
    sp = np.sqrt((dy * dy).sum(1))
    nrm = np.stack([dy[:, 1], -dy[:, 0]], 1) / sp[:, None]
    return I.Curve(I.KIND_SLP, p, sp * 2 * PI / n, nrm, np.zeros(n), t)


def expected_correction(geo, slp, factor, K):
    """Per node: sum over vesicle images within factor h (own vesicle at m = 0 excluded) of the
    oracle's resampled single layer minus the plain n-point sum."""
    from oracle import close_oracle as C
    from oracle import sim_oracle as S
    x = geo.nodes
    d = geo.period
    out = np.zeros((len(x), 2))
    ves_rows, r = [], 0
    for ci, c in enumerate(geo.curves):
        if c.kind == I.KIND_SLP:
            ves_rows.append((ci, r))
            r += c.n
    off = geo.curve_offset
    pairs = 0
    for i in range(len(x)):
        own = int(np.searchsorted(off, i, side="right") - 1)
        for ci, r0 in ves_rows:
            c = geo.curves[ci]
            f = slp[r0:r0 + c.n]
            for m in ((-1, 0, 1) if d else (0,)):
                if ci == own and m == 0:
                    continue
                xs = c.nodes + np.array([m * d, 0.0])
                h = np.sqrt((np.diff(np.vstack([xs, xs[:1]]), axis=0) ** 2).sum(1)).max()
                if np.sqrt(((xs - x[i]) ** 2).sum(1)).min() >= factor * h:
                    continue
                pairs += 1
                fine = C.close_slp(xs, f, x[i:i + 1], MU, K=K)[0]
                plain = np.einsum("jab,jb->a", S.stokeslet(x[i][None], xs, MU) * c.weights[:, None, None], f)
                out[i] += fine - plain
    return out, pairs


def run_close(P, geo, slp, dlp, factor, K):
    s = P.StokesSum(geo)
    base = s.eval(dev(slp), dev(dlp) if dlp is not None else None, precision="fp64")
    out = base.clone()
    cl = P.stokes_close_create(s.h, factor, K)
    P.stokes_close_eval(cl, dev(slp), out)
    P.stokes_sync(s.h)
    info = P.stokes_close_get_info(cl)
    P.stokes_close_destroy(cl)
    s.close()
    return (out - base).cpu().numpy(), info


def density(n_total, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n_total, 2))


@pytest.mark.parametrize("case", ["two_vesicles", "through_the_image"])
def test_close_correction_matches_oracle(P, case):
    """Vesicles a fraction of a node spacing apart (directly, or only through the +-d image):
    the added correction equals the oracle's resampled-minus-plain single layer."""
    n, K, factor = 64, 16, 5.0
    if case == "two_vesicles":
        A = vesicle(n, (0.0, 0.0), 0.3, 0.15, 0.0)
        B = vesicle(n, (0.62, 0.02), 0.3, 0.15, 0.2)
        geo = I.Geometry([A, B], 0.0, MU, {})
    else:
        d = 2 * PI
        A = vesicle(n, (0.32, 0.0), 0.3, 0.15, 0.0)
        B = vesicle(n, (d - 0.31, 0.01), 0.3, 0.15, -0.1)
        geo = I.Geometry([A, B], d, MU, {})
    slp = density(2 * n, 7)
    corr, info = run_close(P, geo, slp, None, factor, K)
    ref, pairs = expected_correction(geo, slp, factor, K)
    assert info["pairs"] == pairs > 0, (info, pairs)
    assert np.abs(corr - ref).max() <= 1e-9 * np.abs(ref).max(), (np.abs(corr - ref).max(), np.abs(ref).max())


def test_close_correction_at_wall_nodes(P):
    """A vesicle just above the lower wall: the wall nodes near it get the correction too."""
    n_w, n = 256, 64
    lo, up = I.wall_curves(n_w, I.WALL_SHAPE_SMALL)
    x0 = 1.0
    y_wall = -(1 + 0.3 * math.sin(x0))
    hv = 2 * PI * 0.3 / n
    V = vesicle(n, (x0, y_wall + 0.155 + 1.0 * hv), 0.3, 0.15, 0.0)
    geo = I.Geometry([lo, up, V], 2 * PI, MU, {})
    slp = density(n, 11)
    dlp = density(2 * n_w, 12)
    corr, info = run_close(P, geo, slp, dlp, 5.0, 16)
    ref, pairs = expected_correction(geo, slp, 5.0, 16)
    assert info["pairs"] == pairs > 0
    assert np.abs(corr[:2 * n_w]).max() > 0  # wall targets corrected
    assert np.abs(corr - ref).max() <= 1e-9 * np.abs(ref).max()


def test_no_pairs_at_the_paper_gaps(P):
    """Inputs keep vesicles 5 node spacings from everything: at factor 2 nothing is close and the
    node sum is left untouched."""
    g, slp, dlp = I.workload("small_n1280")
    corr, info = run_close(P, g, slp, dlp, 2.0, 8)
    assert info["pairs"] == 0 and np.abs(corr).max() == 0.0


def test_close_argument_errors(P):
    import torch
    g, slp, dlp = I.workload("small_n1280")
    s = P.StokesSum(g)
    for factor, K in ((0.0, 8), (5.0, 0), (5.0, 128)):  # K n > 4096 at n = 64
        with pytest.raises(P.StokesError):
            P.stokes_close_create(s.h, factor, K)
    cl = P.stokes_close_create(s.h, 5.0, 8)
    out = torch.zeros((s.N, 2), dtype=torch.float64, device="cuda")
    s.set_geometry(g)
    with pytest.raises(P.StokesError) as e:
        P.stokes_close_eval(cl, dev(slp), out)
    assert e.value.code == P.STOKES_ERR_NO_GEOM
    P.stokes_close_destroy(cl)
    s.close()
