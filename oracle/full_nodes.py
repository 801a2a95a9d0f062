"""FP64 oracle velocities at every node of a named workload, cached by a hash of the inputs.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the tests and the benchmark's CPU leg
use it; the product path never does.  It calls nothing but ``oracle.oracle.sum_nodes`` -- the
plain FP64 double loop of ``stokes_oracle.c`` (Eq. (S), Eq. (D), the near-image sums of
Eq. (Dnr) and Eq. (utotrep), the Nystrom diagonal of Sec. 2.3 and the Kress rule of Sec. 3.2)
-- over all targets, with OpenMP over targets only.

The key is the SHA-256 of every array the oracle reads (nodes, weights, normals, curvature,
curve offsets and kinds, densities, period, mu, jump), so a cached result is reused only for
bit-identical inputs: a platform whose input generator rounds one value differently gets a
fresh oracle run, never another platform's numbers.  The cache directory is
``$STOKES_ORACLE_CACHE`` or ``oracle/_cache`` (not committed).

Usage: ``python -m oracle.full_nodes paper_n128k`` writes the cache entry and prints its key.
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def cache_dir() -> str:
    d = os.environ.get("STOKES_ORACLE_CACHE") or os.path.join(HERE, "_cache")
    os.makedirs(d, exist_ok=True)
    return d


def input_key(geom, slp, dlp, jump: float = 0.0) -> str:
    h = hashlib.sha256()
    for a in (geom.nodes, geom.weights, geom.normals, geom.curvature,
              np.asarray(geom.curve_offset, dtype=np.int64),
              np.asarray(geom.curve_kind, dtype=np.int64), slp, dlp,
              np.array([geom.period, geom.mu, jump], dtype=np.float64)):
        a = np.ascontiguousarray(a)
        h.update(str(a.dtype).encode() + str(a.shape).encode())
        h.update(a.tobytes())
    return h.hexdigest()[:32]


def sum_nodes_cached(geom, slp, dlp, jump: float = 0.0, threads: int = 0):
    """(velocity at every node (N, 2), key, seconds spent in the oracle (0 when cached))."""
    key = input_key(geom, slp, dlp, jump)
    path = os.path.join(cache_dir(), "nodes_%s.npy" % key)
    if os.path.exists(path):
        out = np.load(path)
        if out.shape == (geom.n_nodes, 2):
            return out, key, 0.0
    t0 = time.perf_counter()
    out = O.sum_nodes(geom, slp, dlp, jump=jump, threads=threads)
    dt = time.perf_counter() - t0
    tmp = path + ".tmp%d.npy" % os.getpid()
    np.save(tmp, out)
    os.replace(tmp, path)
    return out, key, dt


def main(argv):
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_1510_05616_gb300 import inputs as I
    name = argv[1] if len(argv) > 1 else "paper_n128k"
    g, slp, dlp = I.workload(name)
    O.build()
    out, key, dt = sum_nodes_cached(g, slp, dlp)
    print("%s: N = %d, key %s, oracle %.1f s on %d threads" % (name, g.n_nodes, key, dt,
                                                               O.max_threads()))


if __name__ == "__main__":
    main(sys.argv)
