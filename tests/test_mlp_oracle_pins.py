"""Pins of the warm-start network oracle: the backward pass against central finite
differences of the forward pass (FP64), BF16 rounding against its definition, Adam against
its closed form for one step."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def M():
    from oracle import mlp_oracle
    return mlp_oracle


def test_bf16_rounding(M):
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.140625, 1e-30, 65504.0], dtype=np.float32)
    r = M.bf16_round(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # tie rounds to even mantissa
    assert r[2] == 1.0 + 2 ** -7            # above the half-way point rounds up
    assert r[3] == -3.140625
    # every result has a zero low half word and is within half a BF16 ulp
    u = r.astype(np.float32).view(np.uint32)
    assert np.all((u & 0xFFFF) == 0)
    assert np.all(np.abs(r - v) <= np.abs(v) * 2.0 ** -8 + 1e-38)


def test_backward_matches_finite_differences(M):
    rng = np.random.default_rng(0)
    dims = (5, 7, 3)
    n = sum(int(np.prod(s)) for s in M.shapes(*dims))
    # weights exactly representable in BF16, so the rounding is the identity here
    theta = M.bf16_round(rng.normal(scale=0.5, size=n))
    x = rng.normal(size=(4, 5))
    t = rng.normal(size=(4, 3))
    _, g = M.loss_and_grad(theta, dims, x, t)
    eps = 1e-6
    # finite differences only on bias entries (keeps every perturbed weight representable)
    offs = np.cumsum([0] + [int(np.prod(s)) for s in M.shapes(*dims)])
    for blk in (1, 3, 5):
        for k in range(offs[blk], offs[blk + 1]):
            tp, tm = theta.copy(), theta.copy()
            tp[k] += eps
            tm[k] -= eps
            fd = (M.loss_and_grad(tp, dims, x, t)[0] - M.loss_and_grad(tm, dims, x, t)[0]) / (2 * eps)
            assert abs(fd - g[k]) < 1e-7 * max(1.0, abs(fd))


def test_weight_gradient_matches_finite_differences_without_rounding(M, monkeypatch):
    monkeypatch.setattr(M, "bf16_round", lambda w: np.asarray(w, dtype=np.float64))
    rng = np.random.default_rng(1)
    dims = (4, 6, 2)
    n = sum(int(np.prod(s)) for s in M.shapes(*dims))
    theta = rng.normal(scale=0.5, size=n)
    x = rng.normal(size=(3, 4))
    t = rng.normal(size=(3, 2))
    _, g = M.loss_and_grad(theta, dims, x, t)
    eps = 1e-6
    for k in rng.choice(n, 25, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        fd = (M.loss_and_grad(tp, dims, x, t)[0] - M.loss_and_grad(tm, dims, x, t)[0]) / (2 * eps)
        assert abs(fd - g[k]) < 1e-7 * max(1.0, abs(fd))


def test_adam_first_step_closed_form(M):
    """At t = 1 the bias-corrected update is -lr g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = M.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
