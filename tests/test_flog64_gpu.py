"""The FP64 pair kernels' table-driven logarithm against CUDA's log and NumPy's.

The kernel-side log (Tang's table-driven method: breakpoint a_k from the top 7 mantissa bits,
log a_k from a table, log1p(u) by its Taylor series to u^7) feeds every FP64 stokeslet and the
Kress self pass (Eq. (S), Sec. 3.2).  Checked directly over the squared distances the kernels
pass (1e-150 .. 1e6), densely around 1 (where e ln 2 and log a_k cancel), at powers of two and
at the table's breakpoints and their neighbours.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1510_05616_gb300 as P
    h = P.stokes_create(0)
    yield P, h
    P.stokes_destroy(h)


def _points():
    rng = np.random.default_rng(1510)
    parts = [10.0 ** rng.uniform(-150.0, 6.0, 200_000),
             rng.uniform(0.5, 2.0, 200_000),
             1.0 + rng.uniform(-1e-6, 1e-6, 20_000),
             2.0 ** np.arange(-480, 20, dtype=np.float64)]
    a = 1.0 + (np.arange(128) + 0.5) / 128.0  # the breakpoints, and each side of them
    for e in (-40, -1, 0, 1, 13):
        b = a * 2.0 ** e
        parts += [b, np.nextafter(b, 0.0), np.nextafter(b, np.inf)]
    return np.concatenate(parts)


def test_flog64_matches_cuda_log(ctx):
    import torch
    P, h = ctx
    x = _points()
    xd = torch.as_tensor(x, device="cuda")
    out = torch.empty_like(xd)
    P.stokes_check_log64(h, xd, out)
    P.stokes_sync(h)
    got = out.cpu().numpy()
    ref_cuda = torch.log(xd).cpu().numpy()
    ref_np = np.log(x)
    # absolute error within 4 ulp of max(1, |log x|): the table value, the series and the
    # two final roundings each contribute at most about half an ulp of that size
    bound = 4.0 * 2.0 ** -52 * np.maximum(1.0, np.abs(ref_np))
    for ref in (ref_cuda, ref_np):
        err = np.abs(got - ref)
        worst = int(np.argmax(err / bound))
        assert np.all(err <= bound), (x[worst], got[worst], ref[worst])
    # and nothing systematic: the mean signed error is far below one ulp of the values
    assert abs(np.mean((got - ref_np) / np.maximum(1.0, np.abs(ref_np)))) < 2.0 ** -53


def test_flog64_rejects_bad_arguments(ctx):
    import torch
    P, h = ctx
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(P.StokesError) as e:
        P.stokes_check_log64(h, x, torch.empty(3, dtype=torch.float64, device="cuda"))
    assert e.value.code == P.STOKES_ERR_ARG
