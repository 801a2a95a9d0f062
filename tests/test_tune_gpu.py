"""Launch-shape autotuner on the GPU: it times real candidate shapes, applies the fastest,
records it for the geometry's size class, and never changes results beyond rounding (checked
against the FP64 oracle at the parity tolerances)."""
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
    P.stokes_tune_clear()
    yield P
    P.stokes_tune_clear()


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def check(out, ref, geom, prec):
    wall = geom.kind_mask(I.KIND_DLP)
    for name, m in (("wall", wall), ("vesicle", ~wall)):
        if not m.any():
            continue
        scale = np.abs(ref[m]).max(0)
        scale[scale == 0] = 1.0
        e = np.abs(out[m] - ref[m]).max(0) / scale
        assert np.all(e <= TOL[prec]), "%s %s: %s" % (prec, name, e)


@pytest.fixture(scope="module")
def mid(oracle_mod):
    g, s, d = I.workload("mid_n16k")
    return g, s, d, oracle_mod.sum_nodes(g, s, d)


@pytest.fixture(scope="module")
def small(oracle_mod):
    g, s, d = I.workload("small_n1280")
    return g, s, d, oracle_mod.sum_nodes(g, s, d)


def test_autotune_fp32k_applies_records_and_keeps_parity(P, mid):
    import torch
    g, s, d, ref = mid
    P.stokes_tune_clear()
    a = P.StokesSum(g)
    initial = P.stokes_get_launch(a.h, P.STOKES_FP32_KAHAN)
    r = P.stokes_autotune(a.h, P.STOKES_FP32_KAHAN, repeats=3)
    assert r["candidates"] >= 9
    assert r["targets_per_thread"] in (1, 2, 4) and r["kahan_group"] in (2, 4, 8)
    assert r["source_splits"] >= 1
    assert 0.0 < r["best_ms"] <= r["initial_ms"]
    assert P.stokes_get_launch(a.h, P.STOKES_FP32_KAHAN) == (
        r["source_splits"], r["targets_per_thread"], r["kahan_group"])
    out = a.eval(dev(s), dev(d), precision="fp32k").cpu().numpy()
    check(out, ref, g, "fp32k")
    # a second context with a geometry of the same size class starts from the tuned shape
    b = P.StokesSum(g)
    assert P.stokes_get_launch(b.h, P.STOKES_FP32_KAHAN) == (
        r["source_splits"], r["targets_per_thread"], r["kahan_group"])
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n_wall = int(g.kind_mask(I.KIND_DLP).sum())
    found = P.stokes_tune_lookup(sms, P.STOKES_FP32_KAHAN, 1, g.n_nodes, n_wall, g.n_nodes - n_wall)
    assert found is not None and found["source_splits"] == r["source_splits"]
    # with the table cleared a new context is back at the wave model's default
    P.stokes_tune_clear()
    c = P.StokesSum(g)
    P.stokes_set_launch(c.h, P.STOKES_FP32_KAHAN, 0, initial[1], initial[2])
    assert P.stokes_get_launch(c.h, P.STOKES_FP32_KAHAN) == initial
    for h in (a, b, c):
        h.close()


@pytest.mark.parametrize("prec", ["fp64", "df"])
def test_autotune_fp64_and_double_float(P, small, prec):
    g, s, d, ref = small
    P.stokes_tune_clear()
    a = P.StokesSum(g)
    r = P.stokes_autotune(a.h, P.PRECISIONS[prec], repeats=3)
    assert r["candidates"] >= 1 and r["kahan_group"] == 0
    assert 0.0 < r["best_ms"] <= r["initial_ms"]
    assert P.stokes_get_launch(a.h, P.PRECISIONS[prec])[0] == r["source_splits"]
    out = a.eval(dev(s), dev(d), precision=prec).cpu().numpy()
    check(out, ref, g, prec)
    a.close()
    P.stokes_tune_clear()


def test_autotune_batched_ensemble(P, oracle_mod):
    e = I.ensemble(count=6, size_scale=0.12, seed=91)
    refs = [oracle_mod.sum_nodes(g, s, d) for g, s, d in e]
    geoms = [g for g, _, _ in e]
    P.stokes_tune_clear()
    b = P.StokesBatch(geoms)
    r = P.stokes_autotune(b.h, P.STOKES_FP32_KAHAN, repeats=3)
    assert r["candidates"] >= 15 and r["items_per_slot"] in (1, 2, 4, 8, 16)
    info = P.stokes_batch_info(b.h, P.STOKES_FP32_KAHAN)
    assert (info[2], info[3]) == (r["targets_per_thread"], r["items_per_slot"])
    ts = dev(P.StokesBatch.stack([s for _, s, _ in e]))
    td = dev(P.StokesBatch.stack([d for _, _, d in e]))
    for use_graph in (False, True):
        out = b.eval(ts, td, precision="fp32k", use_graph=use_graph).cpu().numpy()
        offs = np.cumsum([0] + [g.n_nodes for g in geoms])
        for k, (g, ref) in enumerate(zip(geoms, refs)):
            check(out[offs[k]:offs[k + 1]], ref, g, "fp32k")
    # a new batch of the same ensemble starts from the recorded shape
    b2 = P.StokesBatch(geoms)
    info2 = P.stokes_batch_info(b2.h, P.STOKES_FP32_KAHAN)
    assert (info2[2], info2[3]) == (r["targets_per_thread"], r["items_per_slot"])
    b.close()
    b2.close()
    P.stokes_tune_clear()


def test_autotune_argument_errors(P, small):
    g, _, _, _ = small
    a = P.StokesSum(g)
    with pytest.raises(P.StokesError):
        P.stokes_autotune(a.h, 9)
    with pytest.raises(P.StokesError):
        P.stokes_autotune(a.h, P.STOKES_FP32_KAHAN, repeats=51)
    a.close()
    e = P.StokesSum(None)
    with pytest.raises(P.StokesError) as ei:
        P.stokes_autotune(e.h, P.STOKES_FP32_KAHAN)
    assert ei.value.code == P.STOKES_ERR_NO_GEOM
    e.close()


def test_autotuned_shape_at_paper_scale_keeps_parity(P, oracle_mod):
    """N = 128,768 in the launch configuration the benchmark times: the autotuner's shape for
    this geometry (tuned here as in the benchmark), checked against the FP64 oracle on sampled
    nodes of both kinds."""
    g, s, d = I.workload("paper_n128k")
    rng = np.random.default_rng(5)
    off = g.curve_offset
    sel = np.unique(np.concatenate([rng.integers(0, off[2], 120), rng.integers(off[2], g.n_nodes, 200),
                                    [0, off[1] - 1, off[2], g.n_nodes - 1]])).astype(np.int32)
    ref = oracle_mod.sum_nodes(g, s, d, select=sel)
    P.stokes_tune_clear()
    a = P.StokesSum(g)
    r = P.stokes_autotune(a.h, P.STOKES_FP32_KAHAN, repeats=3)
    assert P.stokes_get_launch(a.h, P.STOKES_FP32_KAHAN) == (
        r["source_splits"], r["targets_per_thread"], r["kahan_group"])
    out = a.eval(dev(s), dev(d), precision="fp32k").cpu().numpy()[sel]
    a.close()
    P.stokes_tune_clear()
    wall = g.kind_mask(I.KIND_DLP)[sel]
    for m in (wall, ~wall):
        e = np.abs(out[m] - ref[m]).max(0) / np.abs(ref[m]).max(0)
        assert np.all(e <= TOL["fp32k"]), e
