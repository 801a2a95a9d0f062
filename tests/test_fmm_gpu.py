"""GPU fast multipole evaluation of the layer-potential sum at the nodes against the FP64 oracle
and the direct GPU sums."""
import numpy as np
import pytest

from paper_1510_05616_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


def rel(a, b):
    """Per-component max-norm relative error."""
    return float((np.abs(a - b).max(0) / np.abs(b).max(0)).max())


def fmm_eval(P, s, slp, dlp, order, leaf=32, jump=0.0):
    import torch
    f = P.stokes_fmm_create(s.h, order, leaf)
    try:
        out = torch.zeros((s.N, 2), dtype=torch.float64, device="cuda")
        P.stokes_fmm_eval(f, slp, dlp, jump, out)
        P.stokes_sync(s.h)
        return out.cpu().numpy(), P.stokes_fmm_get_info(f)
    finally:
        P.stokes_fmm_destroy(f)


def test_fmm_matches_oracle_and_converges(P):
    """On the small channel the FMM sum equals the FP64 oracle's discrete sum to the expansion
    error, which falls with the order (about 0.45 per order): ~1e-7 at order 20, ~1e-10 at 28."""
    from oracle import oracle as O
    g, slp, dlp = I.workload("small_n1280")
    ref = O.sum_nodes(g, slp, dlp)
    s = P.StokesSum(g)
    errs = {}
    for order in (12, 20, 28):
        u, info = fmm_eval(P, s, dev(slp), dev(dlp), order)
        errs[order] = rel(u, ref)
        assert info["order"] == order and info["levels"] >= 1
        assert info["sources"] == 3 * g.n_nodes
    s.close()
    assert errs[12] > errs[20] > errs[28], errs
    assert errs[20] < 1e-6 and errs[28] < 1e-9, errs


@pytest.mark.parametrize("leaf", [8, 32, 200])
def test_fmm_leaf_sizes_match_direct_fp64(P, leaf):
    """Shallow and deep trees give the same sum as the FP64 direct GPU sum (16k channel)."""
    g, slp, dlp = I.workload("mid_n16k")
    s = P.StokesSum(g)
    ref = s.eval(dev(slp), dev(dlp), precision="fp64").cpu().numpy()
    u, info = fmm_eval(P, s, dev(slp), dev(dlp), 28, leaf)
    s.close()
    assert rel(u, ref) < 1e-9, (leaf, rel(u, ref), info)


def test_fmm_jump_no_images_and_single_kinds(P):
    """The jump term, a geometry without images (period 0) and walls-only / vesicles-only
    geometries all match the direct FP64 sum."""
    g, slp, dlp = I.workload("small_n1280")
    cases = []
    cases.append((g, slp, dlp, -0.5))
    g0 = I.Geometry(g.curves, 0.0, g.mu, dict(g.meta))
    cases.append((g0, slp, dlp, 0.0))
    walls = [c for c in g.curves if c.kind == I.KIND_DLP]
    ves = [c for c in g.curves if c.kind == I.KIND_SLP]
    cases.append((I.Geometry(walls, g.period, g.mu, {}), None, dlp, -0.5))
    cases.append((I.Geometry(ves, g.period, g.mu, {}), slp, None, 0.0))
    for geo, sl, dl, jump in cases:
        s = P.StokesSum(geo)
        ts = dev(sl) if sl is not None else None
        td = dev(dl) if dl is not None else None
        ref = s.eval(ts, td, precision="fp64", jump=jump).cpu().numpy()
        u, _ = fmm_eval(P, s, ts, td, 28, jump=jump)
        s.close()
        assert rel(u, ref) < 1e-9, (geo.period, jump, sl is None, dl is None, rel(u, ref))


def test_fmm_plan_and_argument_errors(P):
    import torch
    g, slp, dlp = I.workload("small_n1280")
    s = P.StokesSum(g)
    for order, leaf in ((3, 32), (41, 32), (20, 2)):
        with pytest.raises(P.StokesError):
            P.stokes_fmm_create(s.h, order, leaf)
    f = P.stokes_fmm_create(s.h, 20, 32)
    out = torch.zeros((s.N, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(P.StokesError):  # the walls' density is missing
        P.stokes_fmm_eval(f, dev(slp), None, 0.0, out)
    s.set_geometry(g)                    # a new geometry: the plan no longer applies
    with pytest.raises(P.StokesError) as e:
        P.stokes_fmm_eval(f, dev(slp), dev(dlp), 0.0, out)
    assert e.value.code == P.STOKES_ERR_NO_GEOM
    P.stokes_fmm_destroy(f)
    # moved nodes (stokes_geom_update) invalidate a plan as well: it holds the old positions
    f = P.stokes_fmm_create(s.h, 20, 32)
    x, w, n, k = (dev(a) for a in (g.nodes + [0.01, 0.0], g.weights, g.normals, g.curvature))
    P.stokes_geom_update(s.h, x, w, n, k)
    with pytest.raises(P.StokesError) as e:
        P.stokes_fmm_eval(f, dev(slp), dev(dlp), 0.0, out)
    assert e.value.code == P.STOKES_ERR_NO_GEOM
    P.stokes_fmm_destroy(f)
    s.close()


def test_fmm_eval_order_truncates_the_plan(P):
    """A plan evaluated below its order (stokes_fmm_set_eval_order) computes what a plan made
    at that order computes -- the tree and lists do not depend on the order -- to the last bit,
    and 0 or the plan's own order restores the full evaluation; orders outside [4, plan] are
    refused."""
    import torch
    g, slp, dlp = I.workload("mid_n16k")
    s = P.StokesSum(g)
    ts, td = dev(slp), dev(dlp)
    u14, _ = fmm_eval(P, s, ts, td, 14)
    u36, _ = fmm_eval(P, s, ts, td, 36)
    f = P.stokes_fmm_create(s.h, 36, 32)
    out = torch.zeros((s.N, 2), dtype=torch.float64, device="cuda")
    try:
        for bad in (3, 37, -1):
            with pytest.raises(P.StokesError):
                P.stokes_fmm_set_eval_order(f, bad)
        P.stokes_fmm_set_eval_order(f, 14)
        P.stokes_fmm_eval(f, ts, td, 0.0, out)
        P.stokes_sync(s.h)
        assert np.array_equal(out.cpu().numpy(), u14)
        for full in (0, 36):
            P.stokes_fmm_set_eval_order(f, full)
            P.stokes_fmm_eval(f, ts, td, 0.0, out)
            P.stokes_sync(s.h)
            assert np.array_equal(out.cpu().numpy(), u36)
        assert P.stokes_fmm_get_info(f)["order"] == 36
    finally:
        P.stokes_fmm_destroy(f)
        s.close()


def test_fmm_fp32_evaluation(P):
    """FP32 arithmetic for the expansions and the directly summed pairs
    (stokes_fmm_set_precision) moves an order-14 evaluation by about FP32 rounding (~1e-6),
    below its truncation error (~2e-5 here): its error against the double-float direct sum stays
    within 10 % of the FP64 evaluation's (and at order 10 within 10 % as well), and switching
    back gives the FP64 result bit for bit.  Other precisions are refused."""
    import torch
    g, slp, dlp = I.workload("mid_n16k")
    s = P.StokesSum(g)
    ts, td = dev(slp), dev(dlp)
    ref = s.eval(ts, td, precision="df").cpu().numpy()
    out = torch.zeros((s.N, 2), dtype=torch.float64, device="cuda")
    errs = {}
    for order in (10, 14):
        f = P.stokes_fmm_create(s.h, order, 32)
        res = {}
        try:
            with pytest.raises(P.StokesError):
                P.stokes_fmm_set_precision(f, P.STOKES_DOUBLE_FLOAT)
            for prec in (P.STOKES_FP64, P.STOKES_FP32_KAHAN, P.STOKES_FP64):
                P.stokes_fmm_set_precision(f, prec)
                P.stokes_fmm_eval(f, ts, td, 0.0, out)
                P.stokes_sync(s.h)
                res.setdefault(prec, []).append(out.cpu().numpy())
        finally:
            P.stokes_fmm_destroy(f)
        e64, e32 = rel(res[P.STOKES_FP64][0], ref), rel(res[P.STOKES_FP32_KAHAN][0], ref)
        errs[order] = (e64, e32)
        assert np.array_equal(res[P.STOKES_FP64][0], res[P.STOKES_FP64][1])
    s.close()
    print("FMM FP64 / FP32 evaluation errors:", errs)
    for order, (e64, e32) in errs.items():
        assert e64 < 1e-3 and abs(e32 - e64) <= 0.1 * e64 + 2e-6, (order, e64, e32)


@pytest.mark.parametrize("kind", ["vesicles", "walls"])
def test_fmm_free_targets_match_direct_free_point_sum(P, kind):
    """A plan with free targets (stokes_fmm_create_targets) gives, at those points, the direct
    free-point sum of stokes_sum_eval_targets (double-float) to the expansion error: the
    vesicles' single layer at the walls' nodes, and the walls' double layer at the vesicles'
    nodes -- the two sums of the channel response.  The same plan's node evaluation still meets
    the direct node sum to the expansion error (the free targets widen the forest, so its tree
    -- and the truncation error -- differs from the nodes-only plan's).  A targets-only plan
    (stokes_fmm_create_targets_only) gives the free-point sum to the same bound and refuses a
    node evaluation."""
    import torch
    g, slp, dlp = I.workload("mid_n16k")
    ves = [c for c in g.curves if c.kind == I.KIND_SLP]
    walls = [c for c in g.curves if c.kind == I.KIND_DLP]
    if kind == "vesicles":
        gs, other, ds, dd = I.Geometry(ves, g.period, g.mu, {}), walls, dev(slp), None
    else:
        gs, other, ds, dd = I.Geometry(walls, g.period, g.mu, {}), ves, None, dev(dlp)
    tg = dev(np.vstack([c.nodes for c in other]))
    s = P.StokesSum(gs)
    ref = s.eval_targets(ds, dd, tg, precision="df").cpu().numpy()
    node_ref = s.eval(ds, dd, precision="df").cpu().numpy()
    f = P.stokes_fmm_create_targets(s.h, tg, 28, 32)
    try:
        out = torch.zeros_like(tg)
        P.stokes_fmm_eval_targets(f, ds, dd, out)
        nodes = torch.zeros((s.N, 2), dtype=torch.float64, device="cuda")
        P.stokes_fmm_eval(f, ds, dd, 0.0, nodes)
        P.stokes_sync(s.h)
        err = rel(out.cpu().numpy(), ref)
        assert err < 1e-9, err
        assert rel(nodes.cpu().numpy(), node_ref) < 1e-9
        cells_all = P.stokes_fmm_get_info(f)["target_cells"]
    finally:
        P.stokes_fmm_destroy(f)
    # a plan whose target tree holds the free points alone: the same sums, fewer target cells
    ft = P.stokes_fmm_create_targets_only(s.h, tg, 28, 32)
    try:
        out2 = torch.zeros_like(tg)
        P.stokes_fmm_eval_targets(ft, ds, dd, out2)
        P.stokes_sync(s.h)
        err2 = rel(out2.cpu().numpy(), ref)
        assert err2 < 1e-9, err2
        cells = P.stokes_fmm_get_info(ft)["target_cells"]
        with pytest.raises(P.StokesError):  # the nodes are not targets of this plan
            P.stokes_fmm_eval(ft, ds, dd, 0.0, torch.zeros((s.N, 2), dtype=torch.float64,
                                                           device="cuda"))
    finally:
        P.stokes_fmm_destroy(ft)
    f0 = P.stokes_fmm_create(s.h, 20, 32)
    assert cells < cells_all, (cells, cells_all)
    with pytest.raises(P.StokesError):  # no free targets in this plan
        P.stokes_fmm_eval_targets(f0, ds, dd, torch.zeros_like(tg))
    P.stokes_fmm_destroy(f0)
    s.close()
    print("free targets (%s sources): %.2e; targets-only plan %.2e, %d target cells"
          % (kind, err, err2, cells))


def test_fmm_high_order_converges(P):
    """Orders above 30 (shared memory sized by the order) keep converging: at order 36 the FMM
    meets the double-float direct sum to 1e-11 on the 16k channel."""
    g, slp, dlp = I.workload("mid_n16k")
    s = P.StokesSum(g)
    ref = s.eval(dev(slp), dev(dlp), precision="df").cpu().numpy()
    errs = {}
    for order in (28, 36, 40):
        u, _ = fmm_eval(P, s, dev(slp), dev(dlp), order)
        errs[order] = float((np.abs(u - ref).max(0) / np.abs(ref).max(0)).max())
    s.close()
    print("FMM order -> error vs double-float:", errs)
    assert errs[36] < errs[28] and errs[36] < 1e-11 and errs[40] < 1e-11, errs


def test_fmm_paper_channel(P):
    """At N = 128,768 the FMM sum (order 28) equals the FP64-accurate double-float direct sum."""
    g, slp, dlp = I.workload("paper_n128k")
    s = P.StokesSum(g)
    ref = s.eval(dev(slp), dev(dlp), precision="df").cpu().numpy()
    u, info = fmm_eval(P, s, dev(slp), dev(dlp), 28)
    s.close()
    assert rel(u, ref) < 1e-9, (rel(u, ref), info)
