"""Warm-start network kernels against the FP64 oracle, and the gain of the trained network."""
import math

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


@pytest.fixture(scope="module")
def M():
    from oracle import mlp_oracle
    return mlp_oracle


def cuda32(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _net(P, rng, n_in=64, H=96, n_out=48):
    h = P.stokes_mlp_create(0, n_in, H, n_out)
    n = P.stokes_mlp_num_params(h)
    theta = (rng.normal(scale=0.15, size=n)).astype(np.float32)
    P.stokes_mlp_set_params(h, theta)
    norm = np.concatenate([rng.normal(size=n_in), rng.uniform(0.5, 2, n_in),
                           rng.normal(size=n_out), rng.uniform(0.5, 2, n_out)]).astype(np.float32)
    P.stokes_mlp_set_normalization(h, norm)
    return h, theta, norm, (n_in, H, n_out)


def test_forward_and_gradient_match_oracle(P, M):
    rng = np.random.default_rng(0)
    h, theta, norm, dims = _net(P, rng)
    n_in, H, n_out = dims
    B = 37  # ragged against the 32-wide GEMM tiles
    X = rng.normal(size=(B, n_in)).astype(np.float32)
    T = rng.normal(size=(B, n_out)).astype(np.float32)
    mu_i, sd_i = norm[:n_in], norm[n_in:2 * n_in]
    mu_o, sd_o = norm[2 * n_in:2 * n_in + n_out], norm[2 * n_in + n_out:]
    xh = (X.astype(np.float64) - mu_i) / sd_i
    th = (T.astype(np.float64) - mu_o) / sd_o
    # forward
    import torch
    Y = torch.empty((B, n_out), dtype=torch.float32, device="cuda")
    P.stokes_mlp_forward(h, cuda32(X), Y)
    yo, _ = M.forward(theta.astype(np.float64), dims, xh)
    ref = mu_o + sd_o * yo
    assert np.abs(Y.cpu().numpy() - ref).max() < 1e-4 * np.abs(ref).max()
    # loss and gradient
    loss, g = P.stokes_mlp_loss_grad(h, cuda32(X), cuda32(T), batch=B)
    lo, go = M.loss_and_grad(theta.astype(np.float64), dims, xh, th)
    assert abs(loss - lo) < 1e-5 * lo
    assert np.abs(g - go).max() < 1e-4 * np.abs(go).max()
    P.stokes_mlp_destroy(h)


def test_gather_and_adam_step_match_oracle(P, M):
    rng = np.random.default_rng(1)
    h, theta, norm, dims = _net(P, rng, H=40)
    n_in, H, n_out = dims
    rows = 300
    X = rng.normal(size=(rows, n_in)).astype(np.float32)
    T = rng.normal(size=(rows, n_out)).astype(np.float32)
    idx = rng.permutation(rows)[:64].astype(np.int32)
    import torch
    lr = 1e-3
    loss0, g_gpu = P.stokes_mlp_loss_grad(h, cuda32(X), cuda32(T), torch.as_tensor(idx, device="cuda"))
    mu_i, sd_i = norm[:n_in], norm[n_in:2 * n_in]
    mu_o, sd_o = norm[2 * n_in:2 * n_in + n_out], norm[2 * n_in + n_out:]
    lo, go = M.loss_and_grad(theta.astype(np.float64), dims, (X[idx] - mu_i) / sd_i, (T[idx] - mu_o) / sd_o)
    assert abs(loss0 - lo) < 1e-5 * lo
    P.stokes_mlp_train_step(h, cuda32(X), cuda32(T), torch.as_tensor(idx, device="cuda"), lr)
    th1 = P.stokes_mlp_get_params(h)
    ref, _, _ = M.adam(theta.astype(np.float64), g_gpu.astype(np.float64), np.zeros(len(theta)),
                       np.zeros(len(theta)), 1, lr)
    assert np.abs(th1 - ref).max() < 1e-6
    P.stokes_mlp_destroy(h)


def test_trained_warm_start_beats_the_previous_step_guess(P):
    """On the 16k channel (2 x 4096 wall nodes, 128 vesicles x 64 nodes, bending modulus 0.01,
    dt = 1e-3, double-float matvecs, GMRES to 1e-10): trained on two plain runs of other
    channels, the network with history features (its guess: the previous solution plus the
    predicted change) needs fewer GMRES iterations than the previous-step guess -- and than
    the paper's zero guess -- over 20 held-out steps of an unseen channel."""
    from paper_1510_05616_gb300 import warmstart as WS
    n_w, modes, nv, n_v, area = I.WORKLOADS["mid_n16k"]
    dt, pd, kb = 1e-3, 2.0 * 2 * math.pi * 0.2, 0.01
    import torch
    Xs, Ts = [], []
    for seed in (1000, 1001):
        sim = WS.Simulation(I.channel(n_w, modes, nv, n_v, area, seed), kappa_b=kb, restart=200,
                            history=True)
        X, T, _ = WS.collect(sim, 41, dt, pd, precision=P.STOKES_DOUBLE_FLOAT)
        Xs.append(X)
        Ts.append(T)
        sim.close()
    X, T = torch.cat(Xs), torch.cat(Ts)
    net = WS.WarmStartNet(hidden=256, seed=0, history=True)
    losses = net.fit(X, T, epochs=40, batch=256, lr=2e-3)
    assert losses[-1] < 0.2 * losses[0]
    sim = WS.Simulation(I.channel(n_w, modes, nv, n_v, area, 2000), kappa_b=kb, restart=200,
                        history=True)
    x0, s0, _ = sim.state()
    res = WS.evaluate(sim, x0, s0, 20, dt, pd, model=net, guesses=("zero", "previous", "mlp"),
                      precision=P.STOKES_DOUBLE_FLOAT)
    sim.close()
    net.close()
    its = {k: v["mean_iterations"] for k, v in res.items()}
    print("mean GMRES iterations over 20 held-out steps:", its)
    assert its["mlp"] < its["previous"] < its["zero"], its
