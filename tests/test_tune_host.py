"""Host-side logic of the launch-shape autotuner: the process-wide table of tuned shapes by
geometry size class, its lookup and its text file (no GPU needed)."""
import math

import pytest


@pytest.fixture(scope="module")
def P():
    from paper_1510_05616_gb300 import build
    build.build()
    import paper_1510_05616_gb300 as P
    P.load()
    yield P
    P.stokes_tune_clear()


def bucket(x):
    """Half-octave size bucket: ceil(2 log2 x)."""
    return math.ceil(2.0 * math.log2(x) - 1e-9) if x > 0 else -1


def line(sms, prec, n_inst, n, nw, nv, splits, tpt, kg, ips, ms):
    return "%d %d %d %d %d %d %d %d %d %d %g\n" % (
        sms, prec, bucket(n_inst), bucket(n), bucket(nw), bucket(nv), splits, tpt, kg, ips, ms)


def test_table_load_lookup_save_round_trip(P, tmp_path):
    P.stokes_tune_clear()
    f = tmp_path / "shapes.txt"
    f.write_text("# comment\n\n"
                 + line(152, P.STOKES_FP32_KAHAN, 1, 128768, 32768, 96000, 12, 4, 4, 0, 20.9)
                 + line(152, P.STOKES_FP64, 1, 128768, 32768, 96000, 7, 1, 0, 0, 2100.0)
                 + line(152, P.STOKES_FP32_KAHAN, 64, 1855968, 500000, 1355968, 0, 2, 0, 8, 90.0))
    P.stokes_tune_load(str(f))
    r = P.stokes_tune_lookup(152, P.STOKES_FP32_KAHAN, 1, 128768, 32768, 96000)
    assert r is not None
    assert (r["source_splits"], r["targets_per_thread"], r["kahan_group"]) == (12, 4, 4)
    assert r["candidates"] == 0 and abs(r["best_ms"] - 20.9) < 1e-9
    # the same half-octave bucket of every count finds the entry ...
    assert P.stokes_tune_lookup(152, P.STOKES_FP32_KAHAN, 1, 120000, 31000, 93000) is not None
    # ... another bucket, another SM count, another precision or instance count does not
    assert P.stokes_tune_lookup(152, P.STOKES_FP32_KAHAN, 1, 60000, 32768, 96000) is None
    assert P.stokes_tune_lookup(148, P.STOKES_FP32_KAHAN, 1, 128768, 32768, 96000) is None
    assert P.stokes_tune_lookup(152, P.STOKES_DOUBLE_FLOAT, 1, 128768, 32768, 96000) is None
    assert P.stokes_tune_lookup(152, P.STOKES_FP32_KAHAN, 2, 128768, 32768, 96000) is None
    b = P.stokes_tune_lookup(152, P.STOKES_FP32_KAHAN, 64, 1855968, 500000, 1355968)
    assert (b["targets_per_thread"], b["items_per_slot"]) == (2, 8)
    # save, clear, reload: the same entries come back
    g = tmp_path / "saved.txt"
    P.stokes_tune_save(str(g))
    P.stokes_tune_clear()
    assert P.stokes_tune_lookup(152, P.STOKES_FP64, 1, 128768, 32768, 96000) is None
    P.stokes_tune_load(str(g))
    d = P.stokes_tune_lookup(152, P.STOKES_FP64, 1, 128768, 32768, 96000)
    assert d["source_splits"] == 7 and abs(d["best_ms"] - 2100.0) < 1e-6
    assert len([ln for ln in g.read_text().splitlines() if not ln.startswith("#")]) == 3
    P.stokes_tune_clear()


@pytest.mark.parametrize("bad", [
    "152 1 0 34 30 34 12 4 4\n",            # too few fields
    "152 1 0 34 30 34 12 3 4 0 1.0\n",      # targets_per_thread 3
    "152 7 0 34 30 34 12 4 4 0 1.0\n",      # unknown precision
    "152 1 0 34 30 34 12 4 4 99 1.0\n",     # items_per_slot beyond 64
    "0 1 0 34 30 34 12 4 4 0 1.0\n",        # no SMs
    "152 1 0 34 30 34 12 4 4 0 1.0 x\n",    # trailing junk
])
def test_malformed_file_is_rejected_and_changes_nothing(P, tmp_path, bad):
    P.stokes_tune_clear()
    good = tmp_path / "good.txt"
    good.write_text(line(152, P.STOKES_FP64, 1, 1280, 1024, 256, 3, 1, 0, 0, 1.0))
    P.stokes_tune_load(str(good))
    f = tmp_path / "bad.txt"
    f.write_text(line(152, P.STOKES_FP32_KAHAN, 1, 1280, 1024, 256, 2, 2, 2, 0, 1.0) + bad)
    with pytest.raises(P.StokesError):
        P.stokes_tune_load(str(f))
    assert P.stokes_tune_lookup(152, P.STOKES_FP32_KAHAN, 1, 1280, 1024, 256) is None
    assert P.stokes_tune_lookup(152, P.STOKES_FP64, 1, 1280, 1024, 256)["source_splits"] == 3
    P.stokes_tune_clear()


def test_missing_file_and_bad_lookup_arguments(P, tmp_path):
    with pytest.raises(P.StokesError):
        P.stokes_tune_load(str(tmp_path / "absent.txt"))
    with pytest.raises(P.StokesError):
        P.stokes_tune_save(str(tmp_path / "no_such_dir" / "x.txt"))
    for args in [(0, 1, 1, 10, 0, 10), (152, 5, 1, 10, 0, 10), (152, 1, 0, 10, 0, 10),
                 (152, 1, 1, 0, 0, 0), (152, 1, 1, 10, -1, 10)]:
        with pytest.raises(P.StokesError):
            P.stokes_tune_lookup(*args)


def test_autotune_without_context_is_rejected(P):
    import ctypes
    assert P.load().stokes_autotune(None, 1, 5, None, None) == P.STOKES_ERR_ARG
