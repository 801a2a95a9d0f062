"""GPU parity: libstokes (through its C ABI) against the FP64 CPU oracle on the same inputs.

Tolerances (max-norm relative error per output component, over wall targets and over
vesicle targets separately): 1e-12 for the FP64 path and for the double-float path, 1e-6 for
the FP32 Kahan path.
"""
import math

import numpy as np
import pytest

from paper_1510_05616_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32k": 1e-6, "df": 1e-12}
EMPTY = np.zeros((0, 2))


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_05616_gb300 import build
    build.build()
    import paper_1510_05616_gb300 as P
    return P


def rel_err(out, ref, mask=None):
    """Per component max |out - ref| / max |ref| (over the rows selected by mask)."""
    if mask is not None:
        out, ref = out[mask], ref[mask]
    if ref.shape[0] == 0:
        return np.zeros(2)
    scale = np.abs(ref).max(0)
    scale[scale == 0] = 1.0
    return np.abs(out - ref).max(0) / scale


def check(out, ref, geom, prec, select=None):
    wall = geom.kind_mask(I.KIND_DLP)
    if select is not None:
        wall = wall[select]
    for name, m in (("wall", wall), ("vesicle", ~wall)):
        e = rel_err(out, ref, m)
        assert np.all(e <= TOL[prec]), "%s %s targets: rel err %s" % (prec, name, e)


def dev(P, a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def run(P, geom, slp, dlp, prec, jump=0.0, splits=None):
    s = P.StokesSum(geom)
    if splits:
        P.stokes_set_launch(s.h, P.PRECISIONS[prec], splits)
    out = s.eval(dev(P, slp), dev(P, dlp), precision=prec, jump=jump).cpu().numpy()
    s.close()
    return out


# ---------------------------------------------------------------------------
# workloads of the paper's setting
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small(oracle_mod):
    g, slp, dlp = I.workload("small_n1280")
    return g, slp, dlp, oracle_mod.sum_nodes(g, slp, dlp)


@pytest.fixture(scope="module")
def mid(oracle_mod):
    g, slp, dlp = I.workload("mid_n16k")
    return g, slp, dlp, oracle_mod.sum_nodes(g, slp, dlp)


@pytest.fixture(scope="module")
def paper(oracle_mod):
    g, slp, dlp = I.workload("paper_n128k")
    rng = np.random.default_rng(3)
    off = g.curve_offset
    # curve ends, both walls' first/last nodes, and random wall / vesicle nodes
    sel = {0, off[1] - 1, off[1], off[2] - 1, off[2], off[3] - 1, off[-2], g.n_nodes - 1}
    sel |= set(rng.integers(0, off[2], 96).tolist())
    sel |= set(rng.integers(off[2], g.n_nodes, 160).tolist())
    sel = np.array(sorted(sel), dtype=np.int32)
    return g, slp, dlp, sel, oracle_mod.sum_nodes(g, slp, dlp, select=sel)


@pytest.mark.parametrize("prec", ["fp64", "fp32k", "df"])
def test_small_channel_full(P, small, prec):
    g, slp, dlp, ref = small
    check(run(P, g, slp, dlp, prec), ref, g, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32k", "df"])
def test_mid_channel_full(P, mid, prec):
    g, slp, dlp, ref = mid
    check(run(P, g, slp, dlp, prec), ref, g, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32k", "df"])
def test_paper_scale_sampled(P, paper, prec):
    """N = 128,768 in the bench's launch configuration; oracle at sampled nodes."""
    g, slp, dlp, sel, ref = paper
    out = run(P, g, slp, dlp, prec)
    check(out[sel], ref, g, prec, select=sel)


# ---------------------------------------------------------------------------
# ragged and degenerate geometries
# ---------------------------------------------------------------------------
def _ragged(seed=21, n_w=100, nvs=(36, 50, 18, 64, 8)):
    rng = np.random.default_rng(seed)
    lower, upper = I.wall_curves(n_w, I.WALL_SHAPE_SMALL)
    ves = []
    xs = np.linspace(0.3, 2 * math.pi - 0.3, len(nvs))
    for k, n in enumerate(nvs):
        ves.append(I.closed_curve(n, 0.18, 0.11, (xs[k], 0.3 * rng.uniform(-1, 1)), rng.uniform(0, 6)))
    # interleave kinds to exercise the slot permutation
    curves = [ves[0], lower, ves[1], ves[2], upper] + ves[3:]
    g = I.Geometry(curves, 2 * math.pi, 0.8)
    slp, dlp = I.densities(g, seed)
    return g, slp, dlp


@pytest.mark.parametrize("prec", ["fp64", "fp32k", "df"])
@pytest.mark.parametrize("period", [2 * math.pi, 0.0])
@pytest.mark.parametrize("jump", [0.0, -0.5])
def test_ragged_interleaved(P, oracle_mod, prec, period, jump):
    g, slp, dlp = _ragged()
    g.period = period
    ref = oracle_mod.sum_nodes(g, slp, dlp, jump=jump)
    check(run(P, g, slp, dlp, prec, jump=jump), ref, g, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32k", "df"])
def test_walls_only_and_vesicles_only(P, oracle_mod, prec):
    g, slp, dlp = _ragged()
    walls = I.Geometry([c for c in g.curves if c.kind == I.KIND_DLP], g.period)
    ves = I.Geometry([c for c in g.curves if c.kind == I.KIND_SLP], g.period, 0.8)
    check(run(P, walls, EMPTY, dlp, prec), oracle_mod.sum_nodes(walls, EMPTY, dlp), walls, prec)
    check(run(P, ves, slp, EMPTY, prec), oracle_mod.sum_nodes(ves, slp, EMPTY), ves, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32k", "df"])
def test_single_tiny_vesicle(P, oracle_mod, prec):
    c = I.closed_curve(4, 0.3, 0.2, (0.1, 0.2), 0.5)
    g = I.Geometry([c], 1.0, 1.0)
    f = np.array([[1.0, 0.5], [-0.2, 0.3], [0.7, -1.0], [0.1, 0.1]])
    check(run(P, g, f, EMPTY, prec), oracle_mod.sum_nodes(g, f, EMPTY), g, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32k", "df"])
@pytest.mark.parametrize("splits", [1, 3, 1000])
def test_split_count_does_not_change_result(P, small, prec, splits):
    g, slp, dlp, ref = small
    check(run(P, g, slp, dlp, prec, splits=splits), ref, g, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32k", "df"])
def test_free_targets(P, oracle_mod, prec):
    g, slp, dlp = _ragged()
    rng = np.random.default_rng(9)
    tg = np.stack([rng.uniform(-1, 7, 1001), rng.uniform(-0.6, 0.6, 1001)], 1)
    ref = oracle_mod.sum_free(g, slp, dlp, tg)
    s = P.StokesSum(g)
    out = s.eval_targets(dev(P, slp), dev(P, dlp), dev(P, tg), precision=prec).cpu().numpy()
    s.close()
    # free points can sit close to a curve, where terms are large: compare per component globally
    e = rel_err(out, ref)
    assert np.all(e <= TOL[prec]), e


def test_host_api_matches_device_api(P, small):
    g, slp, dlp, ref = small
    s = P.StokesSum(g)
    for prec in ("fp64", "fp32k", "df"):
        out_h = np.zeros((g.n_nodes, 2))
        P.stokes_sum_eval_host(s.h, P.PRECISIONS[prec], slp, dlp, 0.0, out_h)
        out_d = s.eval(dev(P, slp), dev(P, dlp), precision=prec).cpu().numpy()
        assert np.array_equal(out_h, out_d)
    s.close()


def test_deterministic_repeat(P, small):
    g, slp, dlp, _ = small
    a = run(P, g, slp, dlp, "fp32k")
    b = run(P, g, slp, dlp, "fp32k")
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "fp32k", "df"])
def test_translation_by_period(P, small, prec):
    g, slp, dlp, ref = small
    check(run(P, g.translated((2 * math.pi, 0.0)), slp, dlp, prec), ref, g, prec)


# ---------------------------------------------------------------------------
# failure handling (host-detected or reported through the device status word)
# ---------------------------------------------------------------------------
def test_errors_are_reported(P, small):
    import torch
    g, slp, dlp, _ = small
    s = P.StokesSum()
    out = torch.empty((g.n_nodes, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(P.StokesError) as e:
        P.stokes_sum_eval(s.h, P.STOKES_FP64, dev(P, slp), dev(P, dlp), 0.0, out)
    assert e.value.code == P.STOKES_ERR_NO_GEOM
    s.set_geometry(g)
    with pytest.raises(P.StokesError) as e:
        P.stokes_sum_eval(s.h, 7, dev(P, slp), dev(P, dlp), 0.0, out)
    assert e.value.code == P.STOKES_ERR_ARG
    bad = slp.copy()
    bad[3, 1] = np.nan
    P.stokes_sum_eval(s.h, P.STOKES_FP32_KAHAN, dev(P, bad), dev(P, dlp), 0.0, out)
    with pytest.raises(P.StokesError) as e:
        P.stokes_sync(s.h)
    assert e.value.code == P.STOKES_ERR_NONFINITE
    # the status word is cleared: a clean call succeeds afterwards
    s.eval(dev(P, slp), dev(P, dlp), precision="fp32k")
    odd = I.Geometry([I.closed_curve(15, 0.3, 0.2)], 1.0)
    with pytest.raises(P.StokesError) as e:
        s.set_geometry(odd)
    assert e.value.code == P.STOKES_ERR_ODD_N
    s.close()


@pytest.mark.parametrize("tpt", [1, 2, 4])
@pytest.mark.parametrize("kg", [1, 2, 4, 8, 16])
def test_fp32_launch_shapes(P, oracle_mod, tpt, kg):
    """Every compiled FP32 kernel shape (targets per thread x Kahan group) meets the bound,
    on the ragged interleaved geometry (partial target blocks, padded tiles)."""
    g, slp, dlp = _ragged()
    ref = oracle_mod.sum_nodes(g, slp, dlp)
    s = P.StokesSum(g)
    P.stokes_set_launch(s.h, P.STOKES_FP32_KAHAN, 0, tpt, kg)
    assert P.stokes_get_launch(s.h, P.STOKES_FP32_KAHAN)[1:] == (tpt, kg)
    out = s.eval(dev(P, slp), dev(P, dlp), precision="fp32k").cpu().numpy()
    s.close()
    check(out, ref, g, "fp32k")


def test_launch_knob_validation(P, small):
    g, slp, dlp, _ = small
    s = P.StokesSum(g)
    for bad in ((0, 3, 0), (0, 0, 3), (-1, 0, 0)):
        with pytest.raises(P.StokesError) as e:
            P.stokes_set_launch(s.h, P.STOKES_FP32_KAHAN, *bad)
        assert e.value.code == P.STOKES_ERR_ARG
    s.close()


@pytest.mark.parametrize("tpt", [2, 4])
@pytest.mark.parametrize("workload", ["mid", "paper"])
def test_local_frame_on_and_off(P, mid, paper, workload, tpt):
    """The FP32 stokeslet tiles in the block-local frame (default) and in the (hi, lo) form
    both meet the bound; the two differ (so the local frame is really taken) by rounding only."""
    if workload == "mid":
        g, slp, dlp, ref = mid
        sel = None
    else:
        g, slp, dlp, sel, ref = paper
    s = P.StokesSum(g)
    P.stokes_set_launch(s.h, P.STOKES_FP32_KAHAN, 0, tpt, 4)
    on = s.eval(dev(P, slp), dev(P, dlp), precision="fp32k").cpu().numpy()
    P.stokes_set_local_frame(s.h, False)
    off = s.eval(dev(P, slp), dev(P, dlp), precision="fp32k").cpu().numpy()
    P.stokes_set_local_frame(s.h, True)
    again = s.eval(dev(P, slp), dev(P, dlp), precision="fp32k").cpu().numpy()
    s.close()
    if sel is not None:
        on, off, again = on[sel], off[sel], again[sel]
    check(on, ref, g, "fp32k", select=sel)
    check(off, ref, g, "fp32k", select=sel)
    assert np.array_equal(on, again)
    assert not np.array_equal(on, off)
    assert np.abs(on - off).max() <= 1e-6 * np.abs(ref).max()


# ---------------------------------------------------------------------------
# node sums replayed from a captured CUDA graph
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["fp64", "fp32k", "df"])
def test_graph_replay_equals_direct_launches(P, oracle_mod, small, prec):
    """The graph-replayed node sum is bit-identical to the direct launches, is recaptured when the
    pointers, the launch shape or the partial buffer change, and stays equal to the oracle."""
    import torch
    g, slp, dlp, ref = small
    s = P.StokesSum(g)
    pc = P.PRECISIONS[prec]
    ts, td = dev(P, slp), dev(P, dlp)
    out_d = torch.empty((g.n_nodes, 2), dtype=torch.float64, device="cuda")
    P.stokes_set_graph_mode(s.h, P.STOKES_GRAPH_OFF)
    P.stokes_sum_eval(s.h, pc, ts, td, 0.0, out_d)
    P.stokes_set_graph_mode(s.h, P.STOKES_GRAPH_ALWAYS)
    o = torch.empty_like(out_d)
    outs = []
    for k in range(3):  # one capture, three launches of it
        o.fill_(float("nan"))
        P.stokes_sum_eval(s.h, pc, ts, td, 0.0, o)
        P.stokes_sync(s.h)
        outs.append(o.clone())
    for x in outs:
        assert torch.equal(x, out_d)
    assert P.stokes_graph_stats(s.h) == (1, 3)
    outs[0] = torch.empty_like(out_d)  # a new output pointer: captured anew
    P.stokes_sum_eval(s.h, pc, ts, td, 0.0, outs[0])
    P.stokes_sync(s.h)
    assert torch.equal(outs[0], out_d) and P.stokes_graph_stats(s.h) == (2, 4)
    # new densities in the same buffers: the replay reads them
    ts.mul_(-2.0)
    td.mul_(0.5)
    P.stokes_sum_eval(s.h, pc, ts, td, 0.0, outs[0])
    P.stokes_set_graph_mode(s.h, P.STOKES_GRAPH_OFF)
    P.stokes_sum_eval(s.h, pc, ts, td, 0.0, out_d)
    P.stokes_sync(s.h)
    assert torch.equal(outs[0], out_d)
    # a new launch shape and a grown partial buffer (free targets) drop the graph
    P.stokes_set_graph_mode(s.h, P.STOKES_GRAPH_ALWAYS)
    P.stokes_set_launch(s.h, pc, 3)
    P.stokes_sum_eval(s.h, pc, ts, td, 0.0, outs[1])
    tg = dev(P, np.stack([np.linspace(0.1, 6.0, 50000), np.zeros(50000)], 1))
    ft = torch.empty_like(tg)
    P.stokes_sum_eval_targets(s.h, pc, ts, td, tg, ft)
    P.stokes_sum_eval(s.h, pc, ts, td, 0.0, outs[2])
    P.stokes_sync(s.h)
    s.close()
    o1, o2 = outs[1].cpu().numpy(), outs[2].cpu().numpy()
    assert np.array_equal(o1, o2)
    check(o1, oracle_mod.sum_nodes(g, -2.0 * slp, 0.5 * dlp), g, prec)


def test_graph_mode_argument(P, small):
    g, slp, dlp, _ = small
    s = P.StokesSum(g)
    with pytest.raises(P.StokesError) as e:
        P.stokes_set_graph_mode(s.h, 7)
    assert e.value.code == P.STOKES_ERR_ARG
    s.close()
