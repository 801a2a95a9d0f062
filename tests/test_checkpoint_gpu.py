"""Checkpoint / resume: a time-stepping run saved after k steps and continued in a new
simulation is bit-identical to the uninterrupted run (FP64), and a network checkpoint
(parameters, normalisation, Adam state) resumes training bit-identically."""
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


@pytest.mark.parametrize("prec", ["fp64", "fp32k"])
def test_run_resumes_bit_identically(P, prec, tmp_path):
    from paper_1510_05616_gb300 import warmstart as WS
    g = I.channel(96, I.WALL_SHAPE_SMALL, 3, 32, 0.04, 5, mu=1.0)
    kw = dict(tol=1e-10, precision=P.PRECISIONS[prec])
    a = WS.Simulation(g, kappa_b=0.01)
    for k in range(4):
        a.step(1e-3, 0.5, "previous" if k else "zero", **kw)
    xa, sa, _ = a.state()
    a.close()
    b = WS.Simulation(g, kappa_b=0.01)
    for k in range(2):
        b.step(1e-3, 0.5, "previous" if k else "zero", **kw)
    b.save(tmp_path / "run.npz", step=2)
    b.close()
    c = WS.Simulation(g, kappa_b=0.01)
    assert c.restore(tmp_path / "run.npz") == 2
    for _ in range(2):
        c.step(1e-3, 0.5, "previous", **kw)
    xc, sc, _ = c.state()
    c.close()
    assert np.array_equal(xa, xc) and np.array_equal(sa, sc)


def test_restore_rejects_other_sizes(P, tmp_path):
    from paper_1510_05616_gb300 import warmstart as WS
    g = I.channel(96, I.WALL_SHAPE_SMALL, 3, 32, 0.04, 5, mu=1.0)
    h = I.channel(96, I.WALL_SHAPE_SMALL, 2, 32, 0.04, 6, mu=1.0)
    a = WS.Simulation(g, kappa_b=0.01)
    a.save(tmp_path / "a.npz")
    a.close()
    b = WS.Simulation(h, kappa_b=0.01)
    with pytest.raises(ValueError):
        b.restore(tmp_path / "a.npz")
    b.close()


def test_network_training_resumes_bit_identically(P, tmp_path):
    import torch
    from paper_1510_05616_gb300 import warmstart as WS
    rng = np.random.default_rng(3)
    X = torch.as_tensor(rng.normal(size=(1024, P.N_FEATURES)).astype(np.float32), device="cuda")
    T = torch.as_tensor(rng.normal(size=(1024, P.N_TARGETS)).astype(np.float32), device="cuda")
    a = WS.WarmStartNet(hidden=64, seed=1)
    a.fit(X, T, epochs=4, batch=128, seed=2, lr_decay=1.0)
    b = WS.WarmStartNet(hidden=64, seed=1)
    b.fit(X, T, epochs=2, batch=128, seed=2, lr_decay=1.0)
    b.save(tmp_path / "net.npz")
    b.close()
    c = WS.WarmStartNet(hidden=64, seed=7)
    c.load(tmp_path / "net.npz")
    c.fit(X, T, epochs=4, batch=128, seed=2, lr_decay=1.0, start_epoch=2)
    assert np.array_equal(P.stokes_mlp_get_params(a.h), P.stokes_mlp_get_params(c.h))
    a.close()
    c.close()
