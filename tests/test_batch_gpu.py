"""Batched ensemble: many independent channels in one persistent (graph-captured) launch,
checked instance by instance against the FP64 oracle and against single-instance runs."""
import math

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


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def split_rows(out, geoms):
    offs = np.cumsum([0] + [g.n_nodes for g in geoms])
    return [out[offs[k]:offs[k + 1]] for k in range(len(geoms))]


def check_instance(out, ref, geom, prec, sel=None):
    wall = geom.kind_mask(I.KIND_DLP)
    if sel is not None:
        wall = wall[sel]
    for name, m in (("wall", wall), ("vesicle", ~wall)):
        if not m.any():
            continue
        scale = np.abs(ref[m]).max(0)
        scale[scale == 0] = 1.0
        e = np.abs(out[m] - ref[m]).max(0) / scale
        assert np.all(e <= TOL[prec]), "%s %s: %s" % (prec, name, e)


@pytest.fixture(scope="module")
def ens(oracle_mod):
    e = I.ensemble(count=9, size_scale=0.12, seed=77)
    refs = [oracle_mod.sum_nodes(g, s, d) for g, s, d in e]
    return e, refs


def _batch(P, e):
    return P.StokesBatch([g for g, _, _ in e])


def _dens(P, e):
    return dev(P.StokesBatch.stack([s for _, s, _ in e])), dev(P.StokesBatch.stack([d for _, _, d in e]))


@pytest.mark.parametrize("prec", ["fp64", "fp32k", "df"])
@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_oracle(P, ens, prec, use_graph):
    e, refs = ens
    b = _batch(P, e)
    ts, td = _dens(P, e)
    out = b.eval(ts, td, precision=prec, use_graph=use_graph).cpu().numpy()
    b.close()
    geoms = [g for g, _, _ in e]
    for o, r, g in zip(split_rows(out, geoms), refs, geoms):
        check_instance(o, r, g, prec)


def test_graph_equals_direct_and_is_repeatable(P, ens):
    e, _ = ens
    b = _batch(P, e)
    ts, td = _dens(P, e)
    for prec in ("fp32k", "fp64", "df"):
        a = b.eval(ts, td, precision=prec, use_graph=False).cpu().numpy()
        g1 = b.eval(ts, td, precision=prec, use_graph=True).cpu().numpy()
        g2 = b.eval(ts, td, precision=prec, use_graph=True).cpu().numpy()
        assert np.array_equal(a, g1) and np.array_equal(g1, g2)
    b.close()


def test_batch_matches_single_instance_runs(P, ens):
    e, _ = ens
    b = _batch(P, e)
    ts, td = _dens(P, e)
    geoms = [g for g, _, _ in e]
    outs = {p: split_rows(b.eval(ts, td, precision=p).cpu().numpy(), geoms)
            for p in ("fp64", "fp32k", "df")}
    b.close()
    for k, (g, s, d) in enumerate(e):
        one = P.StokesSum(g)
        for p, tol in (("fp64", 1e-13), ("fp32k", 1e-6), ("df", 1e-13)):
            ref = one.eval(dev(s), dev(d), precision=p).cpu().numpy()
            err = np.abs(outs[p][k] - ref).max(0) / np.abs(ref).max(0)
            assert np.all(err <= tol), (k, p, err)
        one.close()


@pytest.mark.parametrize("tpt,ips", [(1, 1), (2, 16), (4, 4), (4, 64)])
def test_batch_shapes(P, ens, tpt, ips):
    e, refs = ens
    b = _batch(P, e)
    P.stokes_batch_set_shape(b.h, P.STOKES_FP32_KAHAN, tpt, ips)
    P.stokes_batch_set_shape(b.h, P.STOKES_FP64, 0, ips)
    n_items, blocks, t, i = P.stokes_batch_info(b.h, P.STOKES_FP32_KAHAN)
    assert (t, i) == (tpt, ips) and n_items >= len(e) and blocks > 0
    ts, td = _dens(P, e)
    geoms = [g for g, _, _ in e]
    for prec in ("fp32k", "fp64"):
        out = b.eval(ts, td, precision=prec).cpu().numpy()
        for o, r, g in zip(split_rows(out, geoms), refs, geoms):
            check_instance(o, r, g, prec)
    b.close()


def test_batch_jump_recaptures_graph(P, ens, oracle_mod):
    e, refs = ens
    b = _batch(P, e)
    ts, td = _dens(P, e)
    geoms = [g for g, _, _ in e]
    out = b.eval(ts, td, precision="fp64", jump=-0.5).cpu().numpy()
    for o, (g, s, d) in zip(split_rows(out, geoms), e):
        check_instance(o, oracle_mod.sum_nodes(g, s, d, jump=-0.5), g, "fp64")
    out = b.eval(ts, td, precision="fp64", jump=0.0).cpu().numpy()
    for o, r, g in zip(split_rows(out, geoms), refs, geoms):
        check_instance(o, r, g, "fp64")
    b.close()


def test_batch_rejects_mixed_periods(P, ens):
    e, _ = ens
    g0 = e[0][0]
    g1 = I.Geometry(e[1][0].curves, 0.0, g0.mu)
    with pytest.raises(P.StokesError) as err:
        P.StokesBatch([g0, g1])
    assert err.value.code == P.STOKES_ERR_ARG


def test_free_targets_refused_on_batch(P, ens):
    import torch
    e, _ = ens
    b = _batch(P, e)
    ts, td = _dens(P, e)
    tg = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(P.StokesError):
        P.stokes_sum_eval_targets(b.h, P.STOKES_FP64, ts, td, tg, torch.empty_like(tg))
    b.close()


def test_full_ensemble_sampled(P, oracle_mod):
    """The 64-channel ensemble at full size in the bench's launch configuration; the oracle
    checks per instance the ends of both walls, the first and last vesicle node and 32 random
    wall and 32 random vesicle nodes (the relative error is taken over that sample)."""
    import os
    e = I.ensemble(workers=min(16, os.cpu_count() or 1))
    geoms = [g for g, _, _ in e]
    b = _batch(P, e)
    ts, td = _dens(P, e)
    rng = np.random.default_rng(5)
    outs = {p: split_rows(b.eval(ts, td, precision=p).cpu().numpy(), geoms) for p in ("fp32k", "fp64")}
    b.close()
    for k, (g, s, d) in enumerate(e):
        off = g.curve_offset
        sel = np.unique(np.concatenate([[0, off[1] - 1, off[2] - 1, off[2], g.n_nodes - 1],
                                        rng.integers(0, off[2], 32),
                                        rng.integers(off[2], g.n_nodes, 32)])).astype(np.int32)
        ref = oracle_mod.sum_nodes(g, s, d, select=sel)
        for p in ("fp32k", "fp64"):
            check_instance(outs[p][k][sel], ref, g, p, sel)
