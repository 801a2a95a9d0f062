"""GPU channel response and semi-implicit step against the NumPy FP64 oracle."""
import math
import warnings

import numpy as np
import pytest

from paper_1510_05616_gb300 import inputs as I

pytestmark = pytest.mark.gpu
warnings.filterwarnings("ignore", category=RuntimeWarning)
PI = math.pi
D = 2 * PI
MU = 0.7


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
def S():
    from oracle import sim_oracle
    return sim_oracle


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def make_sim(P, walls=None, ves=None, kappa_b=1.0, K=24, M=96, period=D):
    h = P.stokes_sim_create(0)
    if walls is not None:
        lo, up = walls
        P.stokes_sim_set_walls(h, lo.n, np.vstack([lo.nodes, up.nodes]),
                               np.concatenate([lo.weights, up.weights]),
                               np.vstack([lo.normals, up.normals]),
                               np.concatenate([lo.curvature, up.curvature]), period, MU, K, M)
    if ves is not None:
        x = np.vstack([c.nodes for c in ves])
        P.stokes_sim_set_vesicles(h, len(ves), ves[0].n, x, kappa_b, MU, period)
    return h


def _case(seed=3, n_w=96, n_ves=3, n_v=16):
    g = I.channel(n_w, I.WALL_SHAPE_SMALL, n_ves, n_v, 0.05, seed)
    walls = [c for c in g.curves if c.kind == I.KIND_DLP]
    ves = [c for c in g.curves if c.kind == I.KIND_SLP]
    return walls, ves


PTS = np.array([[0.8, 0.0], [3.2, 0.0], [4.8, 0.0], [2.0, 0.5], [5.0, -0.4]])


@pytest.mark.parametrize("sweeps", [3, 0])
def test_poiseuille_on_gpu(P, S, sweeps):
    """The GPU block solve reproduces the exact Poiseuille flow: to round-off with the default
    three refinement sweeps, at the paper's accuracy level (the truncation of S^+) without them;
    and it agrees with the oracle's solve of the same kind."""
    import torch
    lo, up = I.wall_curves(128, I.WALL_SHAPE_SMALL)
    pd = 2 * MU * D * 0.2
    ue = lambda p: np.stack([-(pd / (2 * MU * D)) * p[:, 1] ** 2, 0 * p[:, 1]], 1)
    h = P.stokes_sim_create(0)
    P.stokes_sim_set_block_refinement(h, sweeps)
    xw = np.vstack([lo.nodes, up.nodes])
    P.stokes_sim_set_walls(h, lo.n, xw, np.concatenate([lo.weights, up.weights]),
                           np.vstack([lo.normals, up.normals]),
                           np.concatenate([lo.curvature, up.curvature]), D, MU, 32, 128)
    out = torch.zeros((len(PTS), 2), dtype=torch.float64, device="cuda")
    P.stokes_sim_empty_channel(h, pd, dev(ue(xw)), dev(PTS), out)
    u = out.cpu().numpy()
    P.stokes_sim_destroy(h)
    scale = np.abs(ue(xw)).max()
    # without the refinement the truncation of S^+ (singular values below 1e-13 sigma_max)
    # leaves ~1e-5 of the data in the side-point rows (Sec. 4.1's block solve)
    tol = 1e-12 if sweeps else 1e-5
    assert np.abs(u - ue(PTS)).max() / scale < tol
    W = S.Walls(lo, up, D, MU, K=32, M=128)
    _, g = S.empty_channel_rhs(W, pd)
    tau, c = (W.solve_refined(ue(xw).reshape(-1), g, sweeps=sweeps) if sweeps
              else W.solve(ue(xw).reshape(-1), g))
    ref = W.velocity(tau, c, PTS)
    assert np.abs(u - ref).max() / scale < tol


def test_channel_response_parity(P, S):
    import torch
    walls, ves = _case()
    rng = np.random.default_rng(4)
    f = rng.normal(size=(sum(c.n for c in ves), 2))
    h = make_sim(P, walls, ves)
    out = torch.zeros_like(dev(f))
    P.stokes_sim_channel_response(h, dev(f), 0.8, out)
    u = out.cpu().numpy()
    P.stokes_sim_destroy(h)
    W = S.Walls(walls[0], walls[1], D, MU, K=24, M=96)
    xv = np.vstack([c.nodes for c in ves])
    wv = np.concatenate([S.curve_normals_weights(c.nodes)[1] for c in ves])
    v, g = S.vesicle_rhs(W, xv, wv, f, 0.8)
    tau, c = W.solve_refined(v, g)
    ref = W.velocity(tau, c, xv)
    # both sides refine the block solve to round-off, so the truncation of S^+ no longer
    # separates them
    assert np.abs(u - ref).max() / np.abs(ref).max() < 1e-9


def _oracle_step(S, ves_x, dt, walls=None, p_drive=0.0, period=D, kappa_b=1.0, K=24, M=96,
                 close=None):
    L0 = [S.perimeter(x) for x in ves_x]
    A0 = [S.area(x) for x in ves_x]
    W = S.Walls(walls[0], walls[1], D, MU, K=K, M=M) if walls is not None else None
    sig = [np.zeros(x.shape[0]) for x in ves_x]
    return S.step(ves_x, sig, L0, A0, dt, kappa_b, MU, period, W, p_drive, close=close)


@pytest.mark.parametrize("period", [D, 0.0])
def test_free_step_parity(P, S, period):
    """No walls: one step of GPU GMRES (FP64 sums) equals the oracle's direct solve."""
    _, ves = _case(n_ves=3, n_v=16)
    dt = 1e-3
    h = make_sim(P, None, ves, period=period)
    st = P.vesicle_step_warmstart(h, dt, 0.0, tol=1e-12, max_iter=200)
    x, sg, sol = P.stokes_sim_get_state(h)
    P.stokes_sim_destroy(h)
    ox, osg, u, sig, _ = _oracle_step(S, [c.nodes for c in ves], dt, period=period)
    assert st["residual"] <= 1e-12 and st["iterations"] > 0
    n = ves[0].n
    gu = np.concatenate([np.stack([sol[3 * n * v:3 * n * v + n], sol[3 * n * v + n:3 * n * v + 2 * n]], 1)
                         for v in range(len(ves))])
    assert np.abs(gu - u).max() < 1e-8 * np.abs(u).max()
    assert np.abs(sg - sig).max() < 1e-8 * np.abs(sig).max()
    assert np.abs(x - np.vstack(ox)).max() < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "df"])
def test_channel_step_parity(P, S, prec):
    """One step with walls: GPU GMRES to a 1e-13 residual against the oracle's dense direct
    solve of the same system (both FP64-accurate), so what is left is round-off amplified by
    the step system's conditioning, not the solver tolerance: 1e-9 relative on u and sigma."""
    walls, ves = _case(n_ves=2, n_v=16, n_w=64)
    dt, pd = 1e-3, 0.5
    h = make_sim(P, walls, ves)
    st = P.vesicle_step_warmstart(h, dt, pd, tol=1e-13, max_iter=400, precision=P.PRECISIONS[prec])
    x, sg, sol = P.stokes_sim_get_state(h)
    P.stokes_sim_destroy(h)
    assert st["residual"] <= 1e-13
    ox, osg, u, sig, ures = _oracle_step(S, [c.nodes for c in ves], dt, walls, pd)
    n = ves[0].n
    gu = np.concatenate([np.stack([sol[3 * n * v:3 * n * v + n], sol[3 * n * v + n:3 * n * v + 2 * n]], 1)
                         for v in range(len(ves))])
    eu = np.abs(gu - u).max() / np.abs(u).max()
    es = np.abs(sg - sig).max() / np.abs(sig).max()
    ex = np.abs(x - np.vstack(ox)).max()
    print("%s step with walls: u %.2e, sigma %.2e, x %.2e (GMRES %d its, residual %.1e)"
          % (prec, eu, es, ex, st["iterations"], st["residual"]))
    assert eu < 1e-9 and es < 1e-9
    assert ex < 1e-11


@pytest.mark.parametrize("prec", ["fp64", "fp32k"])
def test_step_with_close_evaluation_matches_oracle(P, S, prec):
    """Two vesicles half a node spacing apart: with close evaluation on, one step (FP64 sums,
    or FP32-Kahan sweeps inside FP64-accurate refinement) equals the oracle's step whose
    single-layer operator carries the close oracle's correction; without it the step differs
    from that by far more."""
    from types import SimpleNamespace
    n = 32
    t = 2 * PI * np.arange(n) / n
    A = np.stack([0.3 * np.cos(t), 0.15 * np.sin(t)], 1)
    h = np.sqrt((np.diff(np.vstack([A, A[:1]]), axis=0) ** 2).sum(1)).max()
    B = A @ np.array([[np.cos(0.3), np.sin(0.3)], [-np.sin(0.3), np.cos(0.3)]]) + [0.6 + 0.5 * h, 0.02]
    ves = [SimpleNamespace(nodes=X, n=n) for X in (A, B)]
    dt, factor, K = 1e-3, 5.0, 16
    ox, osg, u, sig, _ = _oracle_step(S, [A, B], dt, period=0.0, close=(factor, K))
    res = {}
    for on in (True, False):
        h_sim = make_sim(P, None, ves, period=0.0)
        if on:
            P.stokes_sim_set_close_eval(h_sim, factor, K)
        st = P.vesicle_step_warmstart(h_sim, dt, 0.0, tol=1e-12, max_iter=300,
                                      precision=P.PRECISIONS[prec])
        x, sg, sol = P.stokes_sim_get_state(h_sim)
        P.stokes_sim_destroy(h_sim)
        gu = np.concatenate([np.stack([sol[3 * n * v:3 * n * v + n], sol[3 * n * v + n:3 * n * v + 2 * n]], 1)
                             for v in range(2)])
        res[on] = (np.abs(gu - u).max() / np.abs(u).max(), np.abs(sg - sig).max() / np.abs(sig).max(),
                   np.abs(x - np.vstack(ox)).max(), st["residual"])
    print("close step (%s): with %s, without %s" % (prec, res[True], res[False]))
    assert res[True][3] <= 1e-12
    assert res[True][0] < 1e-8 and res[True][1] < 1e-8 and res[True][2] < 1e-10
    assert res[False][0] > 100 * res[True][0]


def test_fmm_residual_step_matches_double_float_step(P):
    """Mixed-precision steps on the 16k channel whose FP64-accurate vesicle sums (right-hand
    side, refinement residuals) come from the FMM (order 36, plan rebuilt every step) agree
    with the same steps on double-float direct sums: solutions to 1e-8, positions to 1e-10."""
    from paper_1510_05616_gb300 import warmstart as WS
    g = I.workload("mid_n16k")[0]
    dt, pd, kb = 1e-3, 2 * 2 * PI * 0.2, 0.01
    a = WS.Simulation(g, kappa_b=kb, restart=200)
    b = WS.Simulation(g, kappa_b=kb, restart=200, residual_fmm=36)
    for k in range(2):
        sa = a.step(dt, pd, "zero" if k == 0 else "previous", precision=P.STOKES_FP32_KAHAN)
        sb = b.step(dt, pd, "zero" if k == 0 else "previous", precision=P.STOKES_FP32_KAHAN)
        assert sa["residual"] <= 1e-10 and sb["residual"] <= 1e-10
        assert sb["accurate_residuals"] >= 1 and sb["fmm_plan_ms"] > 0.0
        assert sa["fmm_plan_ms"] == 0.0
        xa, siga, za = a.state()
        xb, sigb, zb = b.state()
        ez = np.abs(za - zb).max() / np.abs(za).max()
        ex = np.abs(xa - xb).max()
        print("step %d: FMM vs double-float residuals: solution %.2e, positions %.2e; "
              "its %d / %d, step %.1f / %.1f ms, plan %.1f ms"
              % (k, ez, ex, sa["iterations"], sb["iterations"], sa["total_ms"], sb["total_ms"],
                 sb["fmm_plan_ms"]))
        assert ez <= 1e-8 and ex <= 1e-10
    a.close()
    b.close()


@pytest.mark.parametrize("resid", [36, 0])
def test_fmm_sweep_step_matches_direct_sweep_step(P, resid):
    """Mixed-precision steps on the 16k channel whose Krylov sweeps take their vesicle sums from
    the step's FMM plan (order 20; with FMM residuals at order 36 or double-float residuals)
    end on the same FP64-accurate residual bound at the same solution as the steps with
    FP32-Kahan direct sweeps: solutions to 1e-8, positions to 1e-10."""
    from paper_1510_05616_gb300 import warmstart as WS
    g = I.workload("mid_n16k")[0]
    dt, pd, kb = 1e-3, 2 * 2 * PI * 0.2, 0.01
    a = WS.Simulation(g, kappa_b=kb, restart=200, residual_fmm=resid)
    b = WS.Simulation(g, kappa_b=kb, restart=200, residual_fmm=resid, sweep_fmm=20)
    for k in range(2):
        sa = a.step(dt, pd, "zero" if k == 0 else "previous", precision=P.STOKES_FP32_KAHAN)
        sb = b.step(dt, pd, "zero" if k == 0 else "previous", precision=P.STOKES_FP32_KAHAN)
        assert sa["residual"] <= 1e-10 and sb["residual"] <= 1e-10
        assert sb["fmm_plan_ms"] > 0.0
        xa, siga, za = a.state()
        xb, sigb, zb = b.state()
        ez = np.abs(za - zb).max() / np.abs(za).max()
        ex = np.abs(xa - xb).max()
        print("step %d (residuals %s): FMM vs direct sweeps: solution %.2e, positions %.2e; "
              "its %d / %d, step %.1f / %.1f ms"
              % (k, resid or "df", ez, ex, sa["iterations"], sb["iterations"], sa["total_ms"],
                 sb["total_ms"]))
        assert ez <= 1e-8 and ex <= 1e-10
    a.close()
    b.close()


def test_precond_refresh_step_matches_factorised_step(P):
    """Mixed-precision steps on the 16k channel whose preconditioner inverse is refreshed from the
    previous step's by Newton-Schulz (stokes_sim_set_precond_refresh) end on the same
    FP64-accurate residual bound at the same solution as the steps that factorise every block:
    solutions to 1e-8, positions to 1e-10.  The first step factorises (0 products); while the
    shapes relax fast the previous inverse is rejected and the blocks are factorised (reported
    as 0); once they settle the refresh is taken (>= 1 product).  The steps run until three
    have been refreshed, and at least one must be."""
    from paper_1510_05616_gb300 import warmstart as WS
    g = I.workload("mid_n16k")[0]
    dt, pd, kb = 1e-3, 2 * 2 * PI * 0.2, 0.01
    a = WS.Simulation(g, kappa_b=kb, restart=200, residual_fmm=36)
    b = WS.Simulation(g, kappa_b=kb, restart=200, residual_fmm=36, precond_refresh=True)
    refreshed = []
    for k in range(40):
        sa = a.step(dt, pd, "zero" if k == 0 else "previous", precision=P.STOKES_FP32_KAHAN)
        sb = b.step(dt, pd, "zero" if k == 0 else "previous", precision=P.STOKES_FP32_KAHAN)
        assert sa["residual"] <= 1e-10 and sb["residual"] <= 1e-10
        assert sa["precond_refresh"] == 0
        refreshed.append(sb["precond_refresh"])
        xa, siga, za = a.state()
        xb, sigb, zb = b.state()
        ez = np.abs(za - zb).max() / np.abs(za).max()
        ex = np.abs(xa - xb).max()
        print("step %d: refresh products %d; solution %.2e, positions %.2e; its %d / %d"
              % (k, sb["precond_refresh"], ez, ex, sa["iterations"], sb["iterations"]))
        assert ez <= 1e-8 and ex <= 1e-10
        if sum(r > 0 for r in refreshed) >= 3:
            break
    assert refreshed[0] == 0 and any(r > 0 for r in refreshed[1:]), refreshed
    h = P.stokes_sim_create(0)
    with pytest.raises(P.StokesError):
        P.stokes_sim_set_precond_refresh(h, 2)
    P.stokes_sim_destroy(h)
    a.close()
    b.close()


def test_precond_tensor_step_matches_plain_gemm_step(P):
    """Mixed-precision steps on the 16k channel whose FP32 preconditioner GEMMs run as cuBLAS's
    BF16x9 FP32 emulation (stokes_sim_set_precond_tensor), factorised and then refreshed by
    Newton-Schulz, end on the same FP64-accurate residual bound at the same solution as the
    steps with plain SGEMMs: solutions to 1e-8, positions to 1e-10, iteration counts within 2."""
    from paper_1510_05616_gb300 import warmstart as WS
    g = I.workload("mid_n16k")[0]
    dt, pd, kb = 1e-3, 2 * 2 * PI * 0.2, 0.01
    a = WS.Simulation(g, kappa_b=kb, restart=200, residual_fmm=36, precond_refresh=True)
    b = WS.Simulation(g, kappa_b=kb, restart=200, residual_fmm=36, precond_refresh=True,
                      precond_tensor=True)
    for k in range(3):
        sa = a.step(dt, pd, "zero" if k == 0 else "previous", precision=P.STOKES_FP32_KAHAN)
        sb = b.step(dt, pd, "zero" if k == 0 else "previous", precision=P.STOKES_FP32_KAHAN)
        assert sa["residual"] <= 1e-10 and sb["residual"] <= 1e-10
        xa, siga, za = a.state()
        xb, sigb, zb = b.state()
        ez = np.abs(za - zb).max() / np.abs(za).max()
        ex = np.abs(xa - xb).max()
        print("step %d: solution %.2e, positions %.2e; its %d / %d; refresh %d / %d"
              % (k, ez, ex, sa["iterations"], sb["iterations"], sa["precond_refresh"],
                 sb["precond_refresh"]))
        assert ez <= 1e-8 and ex <= 1e-10
        assert abs(sa["iterations"] - sb["iterations"]) <= 2
    h = P.stokes_sim_create(0)
    with pytest.raises(P.StokesError):
        P.stokes_sim_set_precond_tensor(h, 2)
    P.stokes_sim_destroy(h)
    a.close()
    b.close()


def test_residual_fmm_and_warm_modes_arguments(P):
    h = P.stokes_sim_create(0)
    for bad in ((3, 32), (41, 32), (20, 2)):
        with pytest.raises(P.StokesError):
            P.stokes_sim_set_residual_fmm(h, *bad)
    P.stokes_sim_set_residual_fmm(h, 0)
    for bad in (3, 41, -2):
        with pytest.raises(P.StokesError):
            P.stokes_sim_set_sweep_fmm(h, bad)
    P.stokes_sim_set_sweep_fmm(h, 0)
    for bad in (2, 15, 66):
        with pytest.raises(P.StokesError):
            P.stokes_sim_set_warm_modes(h, bad)
    P.stokes_sim_set_warm_modes(h, 32)
    assert P.stokes_sim_get_warm_modes(h) == 32
    P.stokes_sim_destroy(h)


def test_warm_start_with_solution_converges_at_once(P):
    import torch
    walls, ves = _case(n_ves=3, n_v=16)
    h = make_sim(P, walls, ves)
    x0 = np.vstack([c.nodes for c in ves])
    st0 = P.vesicle_step_warmstart(h, 1e-3, 0.5, tol=1e-10, max_iter=200)
    _, _, sol = P.stokes_sim_get_state(h)
    P.stokes_sim_set_state(h, x0, np.zeros(len(x0)))
    st1 = P.vesicle_step_warmstart(h, 1e-3, 0.5, P.STOKES_GUESS_USER, guess=dev(sol), tol=1e-10, max_iter=200)
    P.stokes_sim_destroy(h)
    assert st0["iterations"] >= 3 and st1["iterations"] <= 1


def test_several_steps_conserve_area_and_length(P, S):
    walls, ves = _case(n_ves=3, n_v=32, n_w=96)
    h = make_sim(P, walls, ves)
    x0 = [c.nodes for c in ves]
    A0 = [S.area(x) for x in x0]
    L0 = [S.perimeter(x) for x in x0]
    for _ in range(5):
        P.vesicle_step_warmstart(h, 1e-3, 1.0, tol=1e-10, max_iter=300)
    x, _, _ = P.stokes_sim_get_state(h)
    P.stokes_sim_destroy(h)
    for v in range(3):
        xv = x[32 * v:32 * (v + 1)]
        # area is restored exactly by App. B, then moved by the Fourier re-interpolation of App. C
        assert abs(S.area(xv) - A0[v]) < 1e-8 * A0[v]
        assert abs(S.perimeter(xv) - L0[v]) < 1e-4 * L0[v]


def test_sim_errors(P):
    h = P.stokes_sim_create(0)
    with pytest.raises(P.StokesError) as e:
        P.vesicle_step_warmstart(h, 1e-3, 0.0)
    assert e.value.code == P.STOKES_ERR_NO_GEOM
    with pytest.raises(P.StokesError):
        P.stokes_sim_set_vesicles(h, 1, 15, np.zeros((15, 2)), 1.0, 1.0, 0.0)
    P.stokes_sim_destroy(h)


def test_mixed_precision_step_meets_fp64_tolerance(P):
    """FP32-Kahan Krylov iterations wrapped in FP64 refinement reach the same FP64 residual
    bound as the all-FP64 solve."""
    walls, ves = _case(n_ves=4, n_v=32, n_w=96)
    x0 = np.vstack([c.nodes for c in ves])
    h = make_sim(P, walls, ves)
    st64 = P.vesicle_step_warmstart(h, 1e-3, 0.5, tol=1e-11, max_iter=300)
    _, _, sol64 = P.stokes_sim_get_state(h)
    P.stokes_sim_set_state(h, x0, np.zeros(len(x0)))
    st32 = P.vesicle_step_warmstart(h, 1e-3, 0.5, tol=1e-11, max_iter=300,
                                    precision=P.STOKES_FP32_KAHAN)
    _, _, sol32 = P.stokes_sim_get_state(h)
    P.stokes_sim_destroy(h)
    assert st32["residual"] <= 1e-11 and st32["refinements"] >= 1
    # both meet the FP64 residual bound; the stiff system (condition ~1e5) lets two such
    # iterates differ by about cond x tol in the solution
    assert np.abs(sol32 - sol64).max() < 1e-4 * np.abs(sol64).max()


@pytest.mark.parametrize("guess", ["user_exact", "user_rough"])
def test_mixed_precision_step_with_warm_start(P, guess):
    """A warm-started FP32-Kahan step (whose first residual is taken with the FP32 operator)
    still ends on an FP64-accurate residual below tol, at the FP64 step's solution."""
    walls, ves = _case(n_ves=4, n_v=32, n_w=96)
    x0 = np.vstack([c.nodes for c in ves])
    h = make_sim(P, walls, ves)
    P.vesicle_step_warmstart(h, 1e-3, 0.5, tol=1e-11, max_iter=300)
    _, _, sol64 = P.stokes_sim_get_state(h)
    g = sol64 if guess == "user_exact" else sol64 * (1.0 + 1e-3 * np.cos(np.arange(sol64.size)))
    P.stokes_sim_set_state(h, x0, np.zeros(len(x0)))
    st = P.vesicle_step_warmstart(h, 1e-3, 0.5, P.STOKES_GUESS_USER, guess=dev(g), tol=1e-11,
                                  max_iter=300, precision=P.STOKES_FP32_KAHAN)
    _, _, sol32 = P.stokes_sim_get_state(h)
    P.stokes_sim_destroy(h)
    assert st["residual"] <= 1e-11 and st["refinements"] >= 1
    assert np.abs(sol32 - sol64).max() < 1e-4 * np.abs(sol64).max()


def test_double_float_step_matches_fp64_step(P):
    """Every sum of the step in double-float: the same iterations and, the operator agreeing
    with FP64 to ~1e-13, the same solution up to that times the conditioning (~1e5)."""
    walls, ves = _case(n_ves=4, n_v=32, n_w=96)
    x0 = np.vstack([c.nodes for c in ves])
    h = make_sim(P, walls, ves)
    st64 = P.vesicle_step_warmstart(h, 1e-3, 0.5, tol=1e-11, max_iter=300)
    x64, _, sol64 = P.stokes_sim_get_state(h)
    P.stokes_sim_set_state(h, x0, np.zeros(len(x0)))
    stdf = P.vesicle_step_warmstart(h, 1e-3, 0.5, tol=1e-11, max_iter=300,
                                    precision=P.STOKES_DOUBLE_FLOAT)
    xdf, _, soldf = P.stokes_sim_get_state(h)
    P.stokes_sim_destroy(h)
    assert stdf["residual"] <= 1e-11
    assert abs(stdf["iterations"] - st64["iterations"]) <= 1
    assert np.abs(soldf - sol64).max() < 1e-7 * np.abs(sol64).max()
    # x^{k+1} = x^k + dt u (then the area correction and reparameterization, both Lipschitz ~1)
    assert np.abs(xdf - x64).max() < 2 * 1e-3 * 1e-7 * np.abs(sol64).max()


def test_wall_solvers_agree(P, S):
    """The FP32-LU + FP64-refinement wall solver (default) reaches the FP64 solution: every
    solve ends with an FP64 residual below 1e-13 and the channel response equals the FP64-LU
    solver's up to the truncation of the Schur complement's pseudo-inverse."""
    import torch
    walls, ves = _case(n_w=256)
    rng = np.random.default_rng(8)
    f = rng.normal(size=(sum(c.n for c in ves), 2))
    xw = np.vstack([walls[0].nodes, walls[1].nodes])
    outs = {}
    for mode in (P.STOKES_WALLS_LU64, P.STOKES_WALLS_LU32_REFINE):
        h = P.stokes_sim_create(0)
        P.stokes_sim_set_wall_solver(h, mode)
        lo, up = walls
        P.stokes_sim_set_walls(h, lo.n, xw, np.concatenate([lo.weights, up.weights]),
                               np.vstack([lo.normals, up.normals]),
                               np.concatenate([lo.curvature, up.curvature]), D, MU, 24, 96)
        refs, res = P.stokes_sim_wall_stats(h)  # the solve for W = A^-1 B
        if mode == P.STOKES_WALLS_LU32_REFINE:
            assert 1 <= refs <= 6 and res < 1e-13, (refs, res)
        else:
            assert (refs, res) == (0, 0.0)
        P.stokes_sim_set_vesicles(h, len(ves), ves[0].n, np.vstack([c.nodes for c in ves]), 1.0,
                                  MU, D)
        out = torch.zeros_like(dev(f))
        P.stokes_sim_channel_response(h, dev(f), 0.8, out)
        refs, res = P.stokes_sim_wall_stats(h)
        if mode == P.STOKES_WALLS_LU32_REFINE:  # single inner sweeps under the block refinement
            assert (refs, res) == (1, -1.0), (refs, res)
        pts = torch.zeros((len(PTS), 2), dtype=torch.float64, device="cuda")
        P.stokes_sim_empty_channel(h, 0.8, None, dev(PTS), pts)
        outs[mode] = (out.cpu().numpy(), pts.cpu().numpy())
        P.stokes_sim_destroy(h)
    # with the refined block solve both reach the discrete system's solution
    for a, b in zip(outs[P.STOKES_WALLS_LU64], outs[P.STOKES_WALLS_LU32_REFINE]):
        assert np.abs(a - b).max() / np.abs(a).max() < 1e-10
    with pytest.raises(P.StokesError):
        h = P.stokes_sim_create(0)
        try:
            P.stokes_sim_set_wall_solver(h, 7)
        finally:
            P.stokes_sim_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "fp32k"])
def test_fp32_preconditioner_keeps_the_solution(P, prec):
    """The FP32-factored block preconditioner (default) is one fixed FP64 operator: the step
    solves to the same FP64 tolerance as with the FP64 factorization, to the same solution."""
    walls, ves = _case(n_ves=3, n_v=32, n_w=96)
    out = {}
    for pc in (P.STOKES_FP64, P.STOKES_FP32_KAHAN):
        h = make_sim(P, walls, ves)
        P.stokes_sim_set_precond_precision(h, pc)
        st = P.vesicle_step_warmstart(h, 1e-3, 0.5, tol=1e-11, max_iter=300,
                                      precision=P.PRECISIONS[prec])
        x, sg, sol = P.stokes_sim_get_state(h)
        P.stokes_sim_destroy(h)
        assert st["residual"] <= 1e-11
        out[pc] = (st["iterations"], sol)
    (i64, s64), (i32, s32) = out[P.STOKES_FP64], out[P.STOKES_FP32_KAHAN]
    assert abs(i32 - i64) <= 3
    assert np.abs(s32 - s64).max() <= 1e-6 * np.abs(s64).max()
    h = P.stokes_sim_create(0)
    with pytest.raises(P.StokesError):
        P.stokes_sim_set_precond_precision(h, P.STOKES_DOUBLE_FLOAT)
    P.stokes_sim_destroy(h)
