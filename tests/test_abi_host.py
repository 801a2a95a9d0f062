"""CPU-side checks of the C ABI: the library builds, loads and exports every declared call."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"STOKES_API\s+int\s+(\w+)\s*\(", src)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1510_05616_gb300 import build
    build.build()
    import paper_1510_05616_gb300 as P
    return P.load()


def test_header_declares_calls():
    names = _declared()
    for must in ("stokes_create", "stokes_geom_set", "stokes_sum_eval", "stokes_sum_eval_targets",
                 "stokes_sum_eval_host", "stokes_sync"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_debug_library_exports_the_same_and_says_so(lib):
    """libstokes_debug.so (device bounds checks) is the same ABI; only it reports a debug
    build, and only it accepts stokes_debug_tighten."""
    import ctypes
    from paper_1510_05616_gb300 import build
    dbg = ctypes.CDLL(build.LIB_DEBUG)
    missing = [n for n in _declared() if not hasattr(dbg, n)]
    assert not missing, missing
    assert dbg.stokes_debug_build() == 1 and lib.stokes_debug_build() == 0


def test_binding_names_match_abi():
    import paper_1510_05616_gb300 as P
    for n in _declared():
        assert callable(getattr(P, n, None)), n


def test_null_handle_is_rejected_without_gpu(lib):
    import ctypes
    import paper_1510_05616_gb300 as P
    assert lib.stokes_sum_eval(None, 0, None, None, 0.0, None, None) == P.STOKES_ERR_ARG
    assert lib.stokes_destroy(None) == P.STOKES_OK
    assert lib.stokes_num_nodes(None) == 0
    h = ctypes.c_void_p()
    # no GPU in a CPU-only run: creation must fail cleanly, never fall back
    if not os.environ.get("CUDA_VISIBLE_DEVICES_FORCE"):
        import torch
        if not torch.cuda.is_available():
            assert lib.stokes_create(0, ctypes.byref(h)) == P.STOKES_ERR_CUDA


def test_binding_refuses_without_cuda():
    import torch
    import paper_1510_05616_gb300 as P
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(P.StokesError):
        P.StokesSum(None)


def test_binding_constants_match_header_enums():
    """Every STOKES_* enumerator of the header has the same value in the Python binding."""
    import paper_1510_05616_gb300 as P
    src = open(os.path.join(ROOT, "include", "stokes.h")).read()
    found = re.findall(r"\b(STOKES_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)
    assert len(found) >= 15
    for name, value in found:
        assert getattr(P, name) == int(value), name


def test_binding_structs_match_header_layout(tmp_path):
    """Every result struct of the header (stokes_fmm_info, stokes_close_info,
    stokes_tune_result, stokes_fds_info, stokes_step_stats) has the binding's ctypes layout:
    the same field names in the same order, and the same size and offset of every field as the
    C compiler gives them (a field added on one side only would shift the rest)."""
    import ctypes
    import shutil
    import subprocess
    import paper_1510_05616_gb300 as P
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    src = open(os.path.join(ROOT, "include", "stokes.h")).read()
    structs = {m.group(2): re.findall(r"^\s*(?:int|double)\s+([\w\s,]+);", m.group(1), re.M)
               for m in re.finditer(r"typedef struct \{(.*?)\}\s*(stokes_\w+);", src, re.S)}
    fields = {k: [n.strip() for decl in v for n in decl.split(",")] for k, v in structs.items()}
    binding = {"stokes_fmm_info": P.FmmInfo, "stokes_close_info": P.CloseInfo,
               "stokes_tune_result": P.TuneResult, "stokes_fds_info": P.FdsInfo,
               "stokes_step_stats": P.StepStats}
    assert set(fields) == set(binding), sorted(fields)
    prog = ['#include <stdio.h>', '#include <stddef.h>', '#include "stokes.h"', "int main(void) {"]
    for name, names in fields.items():
        prog.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f in names:
            prog.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    prog.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(prog))
    exe = tmp_path / "layout"
    r = subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in binding.items():
        assert [f for f, _ in cls._fields_] == fields[name], name
        assert ctypes.sizeof(cls) == got[(name, "size")], name
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == got[(name, f)], (name, f)
