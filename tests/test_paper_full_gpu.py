"""Every node of the paper-scale channel (N = 128,768) against the FP64 oracle.

The oracle (the plain FP64 double loop) runs once over all 128,768 targets -- 4.97e10
pair-images, under a minute on the host's cores -- and is cached by a hash of its inputs
(``oracle/full_nodes.py``).  The GPU evaluates the same inputs in all three precisions, the
FP32-Kahan path in the launch shape its autotuner picks (the benchmark's configuration) and in
the default shape.  Bounds: max-norm relative error per component, wall and vesicle targets
separately: 1e-6 (FP32-Kahan), 1e-12 (FP64, double-float).

The FP32 path evaluates compact target blocks in a block-local frame whose rounding is largest
for the closest pairs of nodes on different curves, which a random sample can miss; every node
is checked here, the nodes with the closest foreign sources among them, and the worst node's
distance to its nearest foreign source is reported.
"""
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


@pytest.fixture(scope="module")
def paper():
    from oracle import full_nodes as F
    from oracle import oracle as O
    O.build()
    g, slp, dlp = I.workload("paper_n128k")
    ref, key, secs = F.sum_nodes_cached(g, slp, dlp)
    print("oracle over all %d nodes: key %s, %.1f s (%d threads; 0 s = cached)"
          % (g.n_nodes, key, secs, O.max_threads()))
    return g, slp, dlp, ref, foreign_distance(g)


def foreign_distance(g):
    """Per node, the distance to the nearest source node on another curve (images included)."""
    from scipy.spatial import cKDTree
    x = g.nodes.reshape(-1, 2)
    off = np.asarray(g.curve_offset)
    lens = np.diff(off)
    curve = np.repeat(np.arange(len(off) - 1), lens)
    wall = g.kind_mask(I.KIND_DLP)
    shifts = (-g.period, 0.0, g.period)
    dist = np.full(x.shape[0], np.inf)
    # each wall: one tree of its three images, queried by every node not on it
    for c in np.unique(curve[wall]):
        tree = cKDTree(np.concatenate([x[off[c]:off[c + 1]] + [s, 0.0] for s in shifts]))
        other = curve != c
        dist[other] = np.minimum(dist[other], tree.query(x[other], k=1)[0])
    # all vesicles: one tree; the k = (longest vesicle + 1) nearest always hold a node of
    # another curve, since only the target's own curve's m = 0 copy can crowd them
    ves = np.nonzero(~wall)[0]
    if ves.size:
        tiled = np.concatenate([x[ves] + [s, 0.0] for s in shifts])
        owner = np.tile(curve[ves], 3)
        k = min(int(lens[np.unique(curve[ves])].max()) + 1, tiled.shape[0])
        tree = cKDTree(tiled)
        for lo in range(0, x.shape[0], 16384):
            d, j = tree.query(x[lo:lo + 16384], k=k)
            d = np.where(owner[j] == curve[lo:lo + 16384, None], np.inf, d.reshape(j.shape))
            dist[lo:lo + 16384] = np.minimum(dist[lo:lo + 16384], d.min(1))
    return dist


def _errors(out, ref, mask):
    scale = np.abs(ref[mask]).max(0)
    return np.abs(out[mask] - ref[mask]).max(0) / scale


def _eval(P, g, slp, dlp, prec, tune):
    import torch
    s = P.StokesSum(g)
    pc = P.PRECISIONS[prec]
    if tune:
        P.stokes_autotune(s.h, pc, repeats=2)
    shape = P.stokes_get_launch(s.h, pc)
    ts = torch.as_tensor(slp, device="cuda")
    td = torch.as_tensor(dlp, device="cuda")
    out = s.eval(ts, td, precision=prec).cpu().numpy()
    s.close()
    return out, shape


@pytest.mark.parametrize("prec,tune", [("fp32k", True), ("fp32k", False), ("df", False),
                                       ("fp64", False)])
def test_every_node_of_the_paper_channel(P, paper, prec, tune):
    g, slp, dlp, ref, dfor = paper
    out, shape = _eval(P, g, slp, dlp, prec, tune)
    wall = g.kind_mask(I.KIND_DLP)
    per_node = np.abs(out - ref).max(1) / np.abs(ref).max()
    worst = int(np.argmax(per_node))
    close = dfor <= np.quantile(dfor, 0.01)
    report = {"launch": shape, "wall": _errors(out, ref, wall).tolist(),
              "vesicle": _errors(out, ref, ~wall).tolist(),
              "closest_1pct": _errors(out, ref, close).tolist(),
              "worst_node": worst, "worst_kind": "wall" if wall[worst] else "vesicle",
              "worst_rel": float(per_node[worst]),
              "worst_node_foreign_distance": float(dfor[worst]),
              "min_foreign_distance": float(dfor.min())}
    print("%s%s: %s" % (prec, " (autotuned)" if tune else "", report))
    assert np.isfinite(out).all()
    for name, m in (("wall", wall), ("vesicle", ~wall), ("closest 1%", close)):
        e = _errors(out, ref, m)
        assert np.all(e <= TOL[prec]), "%s %s targets: rel err %s (%s)" % (prec, name, e, report)
