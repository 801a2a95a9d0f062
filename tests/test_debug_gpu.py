"""The debug library (libstokes_debug.so: every source-tile, target, density-row and partial-sum
index of the pair, pack and finishing kernels checked against its buffer, failures recorded in
the status word, nothing trapped) on a tiny ragged geometry, in a child process that loads it.

It must compute what the release library computes (same oracle bounds) with no check firing,
in all three precisions, for node and free-target sums and the batched launch; and when the
checks are told that the last N partial-sum elements are out of range (the buffers keep their
size, so no access leaves its allocation) they must fire and stokes_sync must report
STOKES_ERR_BOUNDS.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT); sys.path.insert(0, ROOT + "/tests")
import paper_1510_05616_gb300 as P
from oracle import oracle as O
from test_parity_gpu import _ragged
assert P.stokes_debug_build()
g, slp, dlp = _ragged()
ref = O.sum_nodes(g, slp, dlp)
out = {}
s = P.StokesSum(g)
ts, td = torch.as_tensor(slp, device="cuda"), torch.as_tensor(dlp, device="cuda")
for prec in ("fp64", "fp32k", "df"):
    u = s.eval(ts, td, precision=prec).cpu().numpy()   # eval syncs: a failed check raises
    out[prec] = float((np.abs(u - ref).max(0) / np.abs(ref).max(0)).max())
tg = np.stack([np.linspace(0.2, 6.0, 333), np.full(333, 0.05)], 1)
ft = s.eval_targets(ts, td, torch.as_tensor(tg, device="cuda"), precision="fp32k").cpu().numpy()
fr = O.sum_free(g, slp, dlp, tg)
out["free_fp32k"] = float((np.abs(ft - fr).max(0) / np.abs(fr).max(0)).max())
b = P.StokesBatch([g, g])
ub = b.eval(torch.cat([ts, ts]), torch.cat([td, td]), precision="fp32k").cpu().numpy()
out["batch_fp32k"] = float((np.abs(ub - np.vstack([ref, ref])).max(0) / np.abs(ref).max(0)).max())
b.close()
P.stokes_debug_tighten(s.h, g.n_nodes)
try:
    s.eval(ts, td, precision="fp32k")
    out["tightened"] = "no error"
except P.StokesError as e:
    out["tightened"] = e.code
P.stokes_debug_tighten(s.h, 0)
u = s.eval(ts, td, precision="fp32k").cpu().numpy()
out["after"] = float((np.abs(u - ref).max(0) / np.abs(ref).max(0)).max())
s.close()
print("RESULT " + json.dumps(out))
"""


def test_debug_library_checks_bounds():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_05616_gb300 import build
    build.build()
    env = dict(os.environ, STOKES_LIBRARY="debug")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    print(res)
    assert res["fp64"] <= 1e-12 and res["df"] <= 1e-12 and res["fp32k"] <= 1e-6
    assert res["free_fp32k"] <= 1e-6 and res["batch_fp32k"] <= 1e-6
    assert res["tightened"] == -9  # STOKES_ERR_BOUNDS
    assert res["after"] <= 1e-6    # the context is usable again
