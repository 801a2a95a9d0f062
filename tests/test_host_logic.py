"""Host logic of the library, on the CPU: the FMM plan (tree, interaction and near lists), the
fast direct solver's compression (HBS tables, neighbour sections) and the close-pair search,
each driven by a small harness (tests/host/*.cu) that includes the library source, runs its
host part and emulates the device passes with the same arithmetic; the results are checked
against the oracles, not against the library."""
import concurrent.futures as cf
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1510_05616_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PI = math.pi


@pytest.fixture(scope="module")
def bins():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tempfile.mkdtemp(prefix="stokes_host_")
    names = {"fmm_plan_check": [], "fmm_plan_threads_check": [],
             "fds_host_check": ["-lcublas", "-lcusolver"], "close_pairs_check": []}

    def build(name):
        exe = os.path.join(out, name)
        cmd = [nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
               "-gencode", "arch=compute_103a,code=sm_103a", os.path.join(HERE, "host", name + ".cu"),
               "-o", exe] + names[name]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        return name, exe

    with cf.ThreadPoolExecutor(4) as ex:
        paths = dict(ex.map(build, names))
    yield paths
    shutil.rmtree(out, ignore_errors=True)


def run(exe, *args):
    r = subprocess.run([exe, *map(str, args)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    return r.stdout


# ---------------------------------------------------------------------------
# FMM plan and passes
# ---------------------------------------------------------------------------
def _fmm_case(path):
    g, slp, dlp = I.workload("small_n1280")
    x, n, w = g.nodes, g.normals, g.weights
    wall = g.kind_mask(I.KIND_DLP)
    vi, wi = np.cumsum(~wall) - 1, np.cumsum(wall) - 1
    vals = np.zeros((len(x), 4))
    for i in range(len(x)):
        if wall[i]:
            t = dlp[wi[i]] * w[i] / PI
            vals[i] = [t[0], t[1], n[i, 0], n[i, 1]]
        else:
            q = slp[vi[i]] * w[i] / (4 * PI * g.mu)
            vals[i] = [q[0], q[1], -0.5 * q[0], -0.5 * q[1]]
    order = list(np.where(wall)[0]) + [-1] + list(np.where(~wall)[0]) + [-1]  # with padding slots
    with open(path, "wb") as f:
        np.array([len(x), len(order), int(wall.sum()) + 1], np.int32).tofile(f)
        np.array([g.period], np.float64).tofile(f)
        x.astype(np.float64).tofile(f)
        np.array(order, np.int32).tofile(f)
        vals.tofile(f)
    # direct sum over the nodes and their +-d images, coincident pairs skipped
    src = np.vstack([x + [m * g.period, 0.0] for m in (-1, 0, 1)])
    v = np.tile(vals, (3, 1))
    sw = np.tile(wall, 3)
    r = x[:, None, :] - src[None]
    rr = (r * r).sum(-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(rr > 0, 1.0 / rr, 0.0)
        lg = np.where(rr > 0, -0.5 * np.log(np.where(rr > 0, rr, 1.0)), 0.0)
    rq = (r * v[None, :, :2]).sum(-1)
    rn = (r * v[None, :, 2:]).sum(-1)
    cs = np.where(sw[None], rn * rq * inv * inv, rq * inv)
    u = (cs[..., None] * r).sum(1)
    u += np.where(sw[None, :, None], 0.0, lg[..., None] * v[None, :, :2]).sum(1)
    return u


@pytest.mark.parametrize("order,leaf,tol", [(20, 32, 1e-6), (28, 8, 1e-9), (28, 200, 1e-9)])
def test_fmm_plan_and_passes(bins, tmp_path, order, leaf, tol):
    """The plan's invariants hold (the harness exits non-zero otherwise) and its passes give the
    direct sum over the images to the expansion error, for deep, medium and shallow trees."""
    case, out = tmp_path / "case.bin", tmp_path / "u.bin"
    ref = _fmm_case(case)
    txt = run(bins["fmm_plan_check"], case, order, leaf, out)
    assert "invariant_violations 0" in txt
    u = np.fromfile(out).reshape(-1, 2)
    err = (np.abs(u - ref).max(0) / np.abs(ref).max(0)).max()
    assert err < tol, (order, leaf, err)


def test_fmm_plan_threads_build_the_same_plan(bins):
    """The plan's key order (a radix sort) equals a stable sort's, ties and 64-bit keys
    included, and the plan built on 2, 3 and 4 host threads equals the one-thread plan in every
    array, bit for bit, for seeded random geometries from 80 to 200,000 source slots (the
    threaded path starts at 4,096 items), periodic and not, with padding slots."""
    txt = run(bins["fmm_plan_threads_check"])
    print(txt)
    assert "ok: order_by_key equals std::stable_sort" in txt, txt
    assert "ok: 36 threaded plans identical" in txt, txt


# ---------------------------------------------------------------------------
# fast direct solver: host factorization
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("recompress", [0, 1])
@pytest.mark.parametrize("n_w,shape", [(96, I.WALL_SHAPE_SMALL), (512, I.WALL_SHAPE_LARGE)])
def test_fds_host_factorization_solves_the_oracle_operator(bins, tmp_path, n_w, shape, recompress):
    """The HBS tables and neighbour sections, applied as the device would, solve the oracle's
    dense wall operator to ~1e-10; with the column recompression (the remark closing Sec. 4.2)
    A_m(J, J_c) C reproduces R = A_m(J, :) to near the decompositions' 1e-12 tolerance."""
    from oracle import sim_oracle as S
    lo, up = I.wall_curves(n_w, shape)
    d, mu = 2 * PI, 0.7
    A = S.Walls(lo, up, d, mu).A()
    rng = np.random.default_rng(n_w)
    b = rng.normal(size=(3, A.shape[0]))
    case, out = tmp_path / "walls.bin", tmp_path / "x.bin"
    with open(case, "wb") as f:
        np.array([n_w, 3], np.int32).tofile(f)
        np.array([d], np.float64).tofile(f)
        np.vstack([lo.nodes, up.nodes]).tofile(f)
        np.concatenate([lo.weights, up.weights]).tofile(f)
        np.vstack([lo.normals, up.normals]).tofile(f)
        np.concatenate([lo.curvature, up.curvature]).tofile(f)
        b.tofile(f)
    txt = run(bins["fds_host_check"], case, out, recompress)
    assert "levels" in txt
    f = txt.split()
    col_rank, r_dev = int(f[f.index("col_rank") + 1]), float(f[f.index("r_dev") + 1])
    rank = int(f[f.index("neighbour_rank") + 1])
    if recompress:
        assert 0 < col_rank < 2 * rank and r_dev < 1e-11, txt
    else:
        assert col_rank == 0, txt
    x = np.fromfile(out).reshape(3, -1)
    res = np.abs(x @ A.T - b).max(1) / np.abs(b).max(1)
    assert res.max() < 1e-9, res


# ---------------------------------------------------------------------------
# close evaluation: pair search and correction
# ---------------------------------------------------------------------------
def _vesicle(n, c, a, b, rot):
    t = 2 * PI * np.arange(n) / n
    rho = 1 + 0.05 * np.cos(3 * t)
    p = np.stack([a * rho * np.cos(t), b * rho * np.sin(t)], 1)
    R = np.array([[math.cos(rot), -math.sin(rot)], [math.sin(rot), math.cos(rot)]])
    return p @ R.T + np.asarray(c)


@pytest.mark.parametrize("period", [0.0, 2 * PI])
def test_close_pairs_and_correction(bins, tmp_path, period):
    """The pair search finds the node-vesicle pairs within factor h (own vesicle at m = 0 excluded,
    images included) and the emulated passes add the close oracle's resampled-minus-plain
    single layer."""
    from oracle import close_oracle as C
    from oracle import sim_oracle as S
    n, K, factor = 64, 16, 5.0
    if period == 0.0:
        A, B = _vesicle(n, (0, 0), 0.3, 0.15, 0.0), _vesicle(n, (0.62, 0.02), 0.3, 0.15, 0.2)
    else:
        A, B = _vesicle(n, (0.32, 0), 0.3, 0.15, 0.0), _vesicle(n, (period - 0.31, 0.01), 0.3, 0.15, -0.1)
    x = np.vstack([A, B])
    f = np.random.default_rng(3).normal(size=(2 * n, 2))
    w = np.concatenate([np.sqrt((C.upsample(V, 1, derivative=True) ** 2).sum(1)) * 2 * PI / n for V in (A, B)])
    case, out = tmp_path / "close.bin", tmp_path / "corr.bin"
    with open(case, "wb") as fh:
        np.array([2 * n, n, 2], np.int32).tofile(fh)
        np.array([period, factor], np.float64).tofile(fh)
        np.array([K], np.int32).tofile(fh)
        x.tofile(fh)
        f.tofile(fh)
        w.tofile(fh)
    txt = run(bins["close_pairs_check"], case, out)
    corr = np.fromfile(out).reshape(-1, 2)
    ref = np.zeros_like(corr)
    pairs = 0
    for i in range(2 * n):
        for v in range(2):
            for m in ((-1, 0, 1) if period else (0,)):
                if v == i // n and m == 0:
                    continue
                xs = x[v * n:(v + 1) * n] + [m * period, 0.0]
                h = np.sqrt((np.diff(np.vstack([xs, xs[:1]]), axis=0) ** 2).sum(1)).max()
                if np.sqrt(((xs - x[i]) ** 2).sum(1)).min() >= factor * h:
                    continue
                pairs += 1
                fine = C.close_slp(xs, f[v * n:(v + 1) * n], x[i:i + 1], 1.0, K=K)[0]
                plain = np.einsum("jab,jb->a", S.stokeslet(x[i][None], xs, 1.0) * w[v * n:(v + 1) * n, None, None],
                                  f[v * n:(v + 1) * n])
                ref[i] += fine - plain
    assert ("pairs %d " % pairs) in txt and pairs > 0, (txt, pairs)
    assert np.abs(corr - ref).max() <= 1e-9 * np.abs(ref).max()
