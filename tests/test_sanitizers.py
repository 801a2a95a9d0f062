"""AddressSanitizer + UndefinedBehaviorSanitizer builds of the host code, run on the CPU.

* The FP64 oracle (``oracle/stokes_oracle.c``) under a small driver (``tests/host/oracle_main.c``)
  that calls every entry point, including the argument checks, with exact-size buffers; its
  results must equal the regular build's bit for bit.
* The library's host code that runs without a GPU -- the FMM plan, the fast direct solver's
  host factorization and the close-pair search, through the harnesses of
  ``tests/test_host_logic.py`` -- on one case each.
Any invalid access, overflow, misaligned or out-of-range conversion stops the program with a
non-zero exit (``-fno-sanitize-recover=all``).
* The FMM plan build on several host threads (``tests/host/fmm_plan_threads_check.cu``) under
  ThreadSanitizer: a data race between the threads stops it (``halt_on_error=1``).  The device kernels are not covered here: they
check their own bounds and report through the device status word.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1510_05616_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SAN = ["-fsanitize=address,undefined", "-fno-omit-frame-pointer", "-fno-sanitize-recover=all"]
ENV = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0:halt_on_error=1",
           UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1", TSAN_OPTIONS="halt_on_error=1",
           OMP_NUM_THREADS="2")


def _run(cmd, **kw):
    r = subprocess.run(cmd, capture_output=True, text=True, env=ENV, timeout=900, **kw)
    assert r.returncode == 0, (cmd[0], r.returncode, r.stdout[-3000:], r.stderr[-6000:])
    assert "runtime error" not in r.stderr and "ERROR: AddressSanitizer" not in r.stderr, r.stderr
    return r.stdout


@pytest.fixture(scope="module")
def san_bins():
    gcc = shutil.which("gcc")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not gcc:
        pytest.skip("gcc not available")
    out = tempfile.mkdtemp(prefix="stokes_san_")
    jobs = {"oracle_main": [gcc, "-O1", "-g", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                            *SAN, os.path.join(HERE, "host", "oracle_main.c"),
                            os.path.join(ROOT, "oracle", "stokes_oracle.c"), "-o",
                            os.path.join(out, "oracle_main"), "-lm"]}
    if os.path.exists(nvcc):
        libs = {"fmm_plan_check": [], "fds_host_check": ["-lcublas", "-lcusolver"],
                "close_pairs_check": []}
        for name, extra in libs.items():
            jobs[name] = [nvcc, "-O1", "-g", "-std=c++17", "--expt-relaxed-constexpr",
                          "-I", os.path.join(ROOT, "include"),
                          "-gencode", "arch=compute_103a,code=sm_103a",
                          # nvcc splits -Xcompiler= at commas: one flag per sanitizer
                          "-Xcompiler=-fsanitize=address,-fsanitize=undefined,"
                          "-fno-omit-frame-pointer,-fno-sanitize-recover=all",
                          os.path.join(HERE, "host", name + ".cu"), "-o", os.path.join(out, name),
                          "-lasan", "-lubsan"] + extra
        jobs["fmm_plan_threads_tsan"] = [
            nvcc, "-O1", "-g", "-std=c++17", "--expt-relaxed-constexpr",
            "-I", os.path.join(ROOT, "include"), "-gencode", "arch=compute_103a,code=sm_103a",
            "-Xcompiler=-fsanitize=thread,-fno-omit-frame-pointer",
            os.path.join(HERE, "host", "fmm_plan_threads_check.cu"),
            "-o", os.path.join(out, "fmm_plan_threads_tsan"), "-ltsan"]

    def build(item):
        name, cmd = item
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, (name, r.stderr[-3000:])
        return name, os.path.join(out, name)

    with cf.ThreadPoolExecutor(4) as ex:
        paths = dict(ex.map(build, jobs.items()))
    yield paths
    shutil.rmtree(out, ignore_errors=True)


def _oracle_case(path, g, slp, dlp, sel, free, jump):
    with open(path, "wb") as f:
        np.array([g.n_nodes, len(g.curves), len(sel), len(free)], np.int32).tofile(f)
        np.array([g.period, g.mu, jump], np.float64).tofile(f)
        g.curve_offset.astype(np.int32).tofile(f)
        g.curve_kind.astype(np.int32).tofile(f)
        for a in (g.nodes, g.weights, g.normals, g.curvature, slp, dlp):
            np.ascontiguousarray(a, np.float64).tofile(f)
        np.asarray(sel, np.int32).tofile(f)
        np.ascontiguousarray(free, np.float64).tofile(f)


@pytest.mark.parametrize("period,jump", [(2 * np.pi, 0.0), (2 * np.pi, -0.5), (0.0, 0.0)])
def test_oracle_under_sanitizers(san_bins, oracle_mod, tmp_path, period, jump):
    g, slp, dlp = I.workload("small_n1280")
    g = I.Geometry(g.curves, period, g.mu)
    rng = np.random.default_rng(11)
    sel = np.sort(rng.choice(g.n_nodes, 57, replace=False))
    free = np.stack([rng.uniform(0, 6, 33), rng.uniform(-0.6, 0.6, 33)], 1)
    case, out = tmp_path / "case.bin", tmp_path / "out.bin"
    _oracle_case(case, g, slp, dlp, sel, free, jump)
    _run([san_bins["oracle_main"], str(case), str(out)])
    raw = np.fromfile(out, dtype=np.uint8)
    n_ves = g.curves[[c.kind for c in g.curves].index(I.KIND_SLP)].n
    nd = 2 * g.n_nodes + 2 * len(sel) + 2 * len(free) + n_ves
    vals = raw[:8 * nd].view(np.float64)
    status = raw[8 * nd:].view(np.int32)
    u_all = vals[:2 * g.n_nodes].reshape(-1, 2)
    u_sel = vals[2 * g.n_nodes:2 * g.n_nodes + 2 * len(sel)].reshape(-1, 2)
    u_free = vals[2 * g.n_nodes + 2 * len(sel):2 * g.n_nodes + 2 * len(sel) + 2 * len(free)].reshape(-1, 2)
    R = vals[nd - n_ves:]
    assert list(status) == [0, 0, 0, 0, -4, -1]
    # the sanitized build computes exactly what the regular one does
    assert np.array_equal(u_all, oracle_mod.sum_nodes(g, slp, dlp, jump=jump))
    assert np.array_equal(u_sel, u_all[sel])
    assert np.array_equal(u_free, oracle_mod.sum_free(g, slp, dlp, free))
    assert np.array_equal(R, oracle_mod.kress_weights(n_ves))


def test_host_logic_under_sanitizers(san_bins, tmp_path):
    if "fmm_plan_check" not in san_bins:
        pytest.skip("nvcc not available")
    import test_host_logic as H
    # FMM plan and emulated passes
    case, out = tmp_path / "case.bin", tmp_path / "u.bin"
    ref = H._fmm_case(case)
    txt = _run([san_bins["fmm_plan_check"], str(case), "20", "32", str(out)])
    assert "invariant_violations 0" in txt
    u = np.fromfile(out).reshape(-1, 2)
    assert (np.abs(u - ref).max(0) / np.abs(ref).max(0)).max() < 1e-6


def test_fmm_plan_threads_under_thread_sanitizer(san_bins):
    """The threaded FMM plan build, on the four smaller cases of its host check (80 to 33,000
    source slots; the threads start at 4,096 items), races nowhere and still equals the
    one-thread plan."""
    if "fmm_plan_threads_tsan" not in san_bins:
        pytest.skip("nvcc not available")
    r = subprocess.run([san_bins["fmm_plan_threads_tsan"], "4"], capture_output=True, text=True,
                       env=ENV, timeout=900)
    assert r.returncode == 0, (r.returncode, r.stdout[-2000:], r.stderr[-6000:])
    assert "ThreadSanitizer" not in r.stderr, r.stderr[-6000:]
    assert "ok: 24 threaded plans identical" in r.stdout, r.stdout


def test_fds_host_under_sanitizers(san_bins, tmp_path):
    if "fds_host_check" not in san_bins:
        pytest.skip("nvcc not available")
    from oracle import sim_oracle as S
    n_w = 96
    lo, up = I.wall_curves(n_w, I.WALL_SHAPE_SMALL)
    A = S.Walls(lo, up, 2 * np.pi, 0.7).A()
    b = np.random.default_rng(1).normal(size=(2, A.shape[0]))
    case, out = tmp_path / "walls.bin", tmp_path / "x.bin"
    with open(case, "wb") as f:
        np.array([n_w, 2], np.int32).tofile(f)
        np.array([2 * np.pi], np.float64).tofile(f)
        np.vstack([lo.nodes, up.nodes]).tofile(f)
        np.concatenate([lo.weights, up.weights]).tofile(f)
        np.vstack([lo.normals, up.normals]).tofile(f)
        np.concatenate([lo.curvature, up.curvature]).tofile(f)
        b.tofile(f)
    _run([san_bins["fds_host_check"], str(case), str(out)])
    x = np.fromfile(out).reshape(2, -1)
    assert (np.abs(x @ A.T - b).max(1) / np.abs(b).max(1)).max() < 1e-9


def test_close_pairs_under_sanitizers(san_bins, tmp_path):
    if "close_pairs_check" not in san_bins:
        pytest.skip("nvcc not available")
    import test_host_logic as H
    # the harness's own case of two close vesicles through the period
    H.test_close_pairs_and_correction({"close_pairs_check": san_bins["close_pairs_check"]},
                                      tmp_path, 2 * np.pi)
