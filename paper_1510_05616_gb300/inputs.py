"""Seeded synthetic inputs: periodic channel walls, vesicles and smooth densities.

This module is the only code shared by the CUDA path and the CPU oracle.  It
builds *inputs* (curve samples, quadrature weights, normals, curvature and
density values) and holds none of the layer-potential arithmetic.

Geometry follows the paper's setting (Sec. 2.2-2.3, Sec. 3):

* The unit cell has period ``d`` along x (lattice vector (d, 0)).  The upper
  wall U is y = f(t), the lower wall D is y = -f(t), with x(t) = t d / (2 pi),
  t in [0, 2 pi), sampled by the periodic trapezoid rule (Sec. 2.3): N nodes
  t_j = 2 pi j / N, weights w_j = |x'(t_j)| 2 pi / N.
* Normals point out of the fluid domain, so the fluid lies on the side
  opposite n (the interior-limit convention x - h n of Eq. (JR)): the upper
  wall's normal points up, the lower wall's points down, a vesicle's normal
  points out of the vesicle.
* Curvature kappa = -(x'' . n) / |x'|^2, which is +1 on the unit circle with
  outward normal; with this sign the Nystrom diagonal of the double layer is
  -kappa / (2 pi) t t^T (Sec. 2.3).
* Vesicles are closed curves sampled at n equispaced parameter values
  theta_k = 2 pi k / n (the Kress product rule needs an equispaced parameter).

Seeding: ``numpy.random.SeedSequence(seed)`` is split into one child stream
for the vesicle shapes and placement, one for the vesicle (single-layer)
densities and one for the wall (double-layer) densities; within each, curves
draw in a fixed order (walls lower then upper; vesicles by index).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi
SEED_BASE = 1510056160

KIND_DLP = 0  # wall curve: double-layer (stresslet) source
KIND_SLP = 1  # vesicle curve: single-layer (stokeslet) source


@dataclass
class Curve:
    kind: int
    nodes: np.ndarray      # (n, 2)
    weights: np.ndarray    # (n,)
    normals: np.ndarray    # (n, 2) unit, pointing out of the fluid domain
    curvature: np.ndarray  # (n,)
    tparam: np.ndarray     # (n,) node parameter in [0, 2 pi)

    @property
    def n(self) -> int:
        return int(self.nodes.shape[0])

    def spacing(self) -> float:
        """Largest distance between consecutive nodes (vesicles closed, walls open)."""
        pts = self.nodes if self.kind == KIND_DLP else np.vstack([self.nodes, self.nodes[:1]])
        d = np.diff(pts, axis=0)
        return float(np.max(np.hypot(d[:, 0], d[:, 1])))


@dataclass
class Geometry:
    curves: list
    period: float
    mu: float = 1.0
    meta: dict = field(default_factory=dict)

    @property
    def curve_offset(self) -> np.ndarray:
        off = np.zeros(len(self.curves) + 1, dtype=np.int32)
        off[1:] = np.cumsum([c.n for c in self.curves])
        return off

    @property
    def curve_kind(self) -> np.ndarray:
        return np.array([c.kind for c in self.curves], dtype=np.int32)

    def _cat(self, name):
        if not self.curves:
            shape = (0, 2) if name in ("nodes", "normals") else (0,)
            return np.zeros(shape)
        return np.ascontiguousarray(np.concatenate([getattr(c, name) for c in self.curves]))

    @property
    def nodes(self):
        return self._cat("nodes")

    @property
    def weights(self):
        return self._cat("weights")

    @property
    def normals(self):
        return self._cat("normals")

    @property
    def curvature(self):
        return self._cat("curvature")

    @property
    def tparam(self):
        return self._cat("tparam")

    @property
    def n_nodes(self) -> int:
        return int(sum(c.n for c in self.curves))

    def kind_mask(self, kind: int) -> np.ndarray:
        """Boolean mask over nodes selecting curves of the given kind."""
        return np.concatenate([np.full(c.n, c.kind == kind) for c in self.curves]) if self.curves \
            else np.zeros(0, dtype=bool)

    @property
    def n_slp(self) -> int:
        return int(sum(c.n for c in self.curves if c.kind == KIND_SLP))

    @property
    def n_dlp(self) -> int:
        return int(sum(c.n for c in self.curves if c.kind == KIND_DLP))

    def translated(self, shift) -> "Geometry":
        sx, sy = float(shift[0]), float(shift[1])
        cs = [Curve(c.kind, c.nodes + np.array([sx, sy]), c.weights.copy(), c.normals.copy(),
                    c.curvature.copy(), c.tparam.copy()) for c in self.curves]
        return Geometry(cs, self.period, self.mu, dict(self.meta))


# --------------------------------------------------------------------------
# walls
# --------------------------------------------------------------------------

def wall_profile(t, modes):
    """f(t) = 1 + sum_k a_k sin(k t) and its first two t-derivatives."""
    f = np.ones_like(t)
    f1 = np.zeros_like(t)
    f2 = np.zeros_like(t)
    for k, a in modes:
        f += a * np.sin(k * t)
        f1 += a * k * np.cos(k * t)
        f2 -= a * k * k * np.sin(k * t)
    return f, f1, f2


def wall_curves(n_w: int, modes, period: float = TWO_PI):
    """Lower wall D (y = -f) and upper wall U (y = +f), each with n_w nodes."""
    t = TWO_PI * np.arange(n_w) / n_w
    f, f1, f2 = wall_profile(t, modes)
    a = period / TWO_PI  # dx/dt
    s = np.sqrt(a * a + f1 * f1)
    w = s * TWO_PI / n_w
    kap = -f2 * a / s**3  # same value on both walls with their outward normals
    x = a * t
    upper = Curve(KIND_DLP, np.stack([x, f], 1), w.copy(),
                  np.stack([-f1 / s, a / s], 1), kap.copy(), t.copy())
    lower = Curve(KIND_DLP, np.stack([x, -f], 1), w.copy(),
                  np.stack([-f1 / s, -a / s], 1), kap.copy(), t.copy())
    return lower, upper


# --------------------------------------------------------------------------
# closed curves (vesicles and test shapes)
# --------------------------------------------------------------------------

def _radial_factor(theta, pert):
    """rho(theta) = 1 + sum a_k cos(k theta + phi_k) and its derivatives."""
    r = np.ones_like(theta)
    r1 = np.zeros_like(theta)
    r2 = np.zeros_like(theta)
    for k, a, ph in pert:
        r += a * np.cos(k * theta + ph)
        r1 -= a * k * np.sin(k * theta + ph)
        r2 -= a * k * k * np.cos(k * theta + ph)
    return r, r1, r2


def _shape_xy(theta, a, b, pert):
    """Body-frame point and derivatives of (a cos, b sin) * rho(theta)."""
    c, s = np.cos(theta), np.sin(theta)
    r, r1, r2 = _radial_factor(theta, pert)
    e0 = np.stack([a * c, b * s], 1)
    e1 = np.stack([-a * s, b * c], 1)
    e2 = -e0
    p = e0 * r[:, None]
    p1 = e1 * r[:, None] + e0 * r1[:, None]
    p2 = e2 * r[:, None] + 2 * e1 * r1[:, None] + e0 * r2[:, None]
    return p, p1, p2


def _area(a, b, pert, m=128):
    th = TWO_PI * np.arange(m) / m
    p, p1, _ = _shape_xy(th, a, b, pert)
    return 0.5 * np.mean(p[:, 0] * p1[:, 1] - p[:, 1] * p1[:, 0]) * TWO_PI


def _perimeter(a, b, pert, m=2048):
    th = TWO_PI * np.arange(m) / m
    _, p1, _ = _shape_xy(th, a, b, pert)
    return np.mean(np.hypot(p1[:, 0], p1[:, 1])) * TWO_PI


_NU_TABLE = None


def ellipse_ratio_for_reduced_area(nu: float) -> float:
    """Axis ratio b/a of an ellipse whose reduced area 4 pi A / L^2 is nu."""
    global _NU_TABLE
    if _NU_TABLE is None:
        ratios = np.linspace(0.05, 1.0, 4000)
        nus = np.array([4 * math.pi * (math.pi * q) / _perimeter(1.0, q, (), m=256) ** 2
                        for q in ratios])
        _NU_TABLE = (nus, ratios)
    nus, ratios = _NU_TABLE
    return float(np.interp(nu, nus, ratios))


def closed_curve(n: int, a: float, b: float, center=(0.0, 0.0), angle: float = 0.0,
                 pert=(), kind: int = KIND_SLP) -> Curve:
    """Counter-clockwise closed curve center + Rot(angle) (a cos, b sin) rho(theta)."""
    th = TWO_PI * np.arange(n) / n
    p, p1, p2 = _shape_xy(th, a, b, pert)
    ca, sa = math.cos(angle), math.sin(angle)
    rot = np.array([[ca, -sa], [sa, ca]])
    x = p @ rot.T + np.asarray(center, dtype=float)
    x1 = p1 @ rot.T
    x2 = p2 @ rot.T
    s = np.hypot(x1[:, 0], x1[:, 1])
    nrm = np.stack([x1[:, 1] / s, -x1[:, 0] / s], 1)  # outward for CCW orientation
    kap = -(x2[:, 0] * nrm[:, 0] + x2[:, 1] * nrm[:, 1]) / s**2
    return Curve(kind, x, s * TWO_PI / n, nrm, kap, th)


def vesicle_shape(rng, n: int, area: float, nu_range=(0.65, 0.9), pert_modes=(2, 8),
                  pert_amp=0.02):
    """Random vesicle in its body frame: (a, b, pert) with enclosed area ``area``."""
    nu = rng.uniform(*nu_range)
    ratio = ellipse_ratio_for_reduced_area(nu)
    pert = tuple((k, rng.uniform(-pert_amp, pert_amp) / k, rng.uniform(0, TWO_PI))
                 for k in range(pert_modes[0], pert_modes[1] + 1))
    a0 = 1.0
    s = math.sqrt(area / _area(a0, ratio, pert))
    return a0 * s, ratio * s, pert


# --------------------------------------------------------------------------
# vesicle placement in the channel
# --------------------------------------------------------------------------

def _wall_tree(walls, period):
    from scipy.spatial import cKDTree
    pts = np.vstack([c.nodes for c in walls])
    if period > 0:
        pts = np.vstack([pts + np.array([m * period, 0.0]) for m in (-1, 0, 1)])
    return cKDTree(pts)


def place_vesicles(rng, walls, modes, period, count, n_v, area, gap_factor=5.0,
                   max_attempts=20000):
    """Random sequential placement with node-to-node gaps >= gap_factor * h.

    h is the larger node spacing of the two curves involved.  Vesicles may
    straddle the cell's side edges; distances use the +-d images.
    """
    tree = _wall_tree(walls, period)
    h_wall = max(c.spacing() for c in walls)
    placed = []
    cen = np.zeros((count, 2))
    bnd = np.zeros(count)
    hs = np.zeros(count)
    shifts = np.array([-period, 0.0, period])
    for v in range(count):
        for _attempt in range(max_attempts):
            a, b, pert = vesicle_shape(rng, n_v, area)
            ang = rng.uniform(0, TWO_PI)
            xc = rng.uniform(0, period)
            f, _, _ = wall_profile(np.array([xc * TWO_PI / period]), modes)
            rad = max(a, b) * 1.1
            yspan = f[0] - rad
            if yspan <= 0:
                continue
            yc = rng.uniform(-yspan, yspan)
            cv = closed_curve(n_v, a, b, (xc, yc), ang, pert, KIND_SLP)
            h_v = cv.spacing()
            # inside the channel
            fx, _, _ = wall_profile(cv.nodes[:, 0] * TWO_PI / period, modes)
            if np.any(np.abs(cv.nodes[:, 1]) >= fx):
                continue
            gap = gap_factor * max(h_v, h_wall)
            dmin, _ = tree.query(cv.nodes, k=1)
            if np.min(dmin) < gap:
                continue
            bound = np.max(np.hypot(*(cv.nodes - np.array([xc, yc])).T))
            ok = True
            if v:
                g2 = gap_factor * np.maximum(h_v, hs[:v])
                dx = xc - (cen[:v, 0][:, None] + shifts[None, :])
                dy = (yc - cen[:v, 1])[:, None]
                jj, mm = np.nonzero(np.hypot(dx, dy) <= (bound + bnd[:v] + g2)[:, None])
                if jj.size:
                    from scipy.spatial import cKDTree
                    others = np.concatenate([placed[j].nodes + np.array([shifts[m], 0.0])
                                             for j, m in zip(jj, mm)])
                    thr = np.concatenate([np.full(placed[j].n, g2[j]) for j in jj])
                    dist, _ = cKDTree(cv.nodes).query(others, k=1)
                    ok = bool(np.all(dist >= thr))
            if ok:
                placed.append(cv)
                cen[v] = (xc, yc)
                bnd[v] = bound
                hs[v] = h_v
                break
        else:
            raise RuntimeError("vesicle placement failed; volume fraction too high")
    return placed


# --------------------------------------------------------------------------
# densities
# --------------------------------------------------------------------------

def fourier_density(rng, tparam, n_modes: int = 16):
    """Per component sum_{k=0}^{K} a_k cos(k t) + b_k sin(k t); a_0 ~ N(0,1),
    a_k, b_k ~ N(0, 1/k^2) for k >= 1."""
    out = np.zeros((tparam.shape[0], 2))
    for comp in range(2):
        v = np.full_like(tparam, rng.normal())
        for k in range(1, n_modes + 1):
            v += rng.normal(0, 1.0 / k) * np.cos(k * tparam) + rng.normal(0, 1.0 / k) * np.sin(k * tparam)
        out[:, comp] = v
    return out


def densities(geom: Geometry, seed: int):
    """(slp_density, dlp_density): rows follow the node order of each kind."""
    ss = np.random.SeedSequence(seed)
    _, s_slp, s_dlp = ss.spawn(3)
    r_slp = np.random.Generator(np.random.PCG64(s_slp))
    r_dlp = np.random.Generator(np.random.PCG64(s_dlp))
    slp = [fourier_density(r_slp, c.tparam) for c in geom.curves if c.kind == KIND_SLP]
    dlp = [fourier_density(r_dlp, c.tparam) for c in geom.curves if c.kind == KIND_DLP]
    slp = np.ascontiguousarray(np.concatenate(slp)) if slp else np.zeros((0, 2))
    dlp = np.ascontiguousarray(np.concatenate(dlp)) if dlp else np.zeros((0, 2))
    return slp, dlp


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

WALL_SHAPE_SMALL = ((1, 0.3),)              # y = +-(1 + 0.3 sin x)
WALL_SHAPE_LARGE = ((1, 0.4), (3, 0.15))    # y = +-(1 + 0.4 sin x + 0.15 sin 3x)
CELL_AREA = 2.0 * TWO_PI                    # |Omega| = integral of 2 f over one period

WORKLOADS = {
    # name: (wall nodes, wall shape, vesicles, nodes per vesicle, vesicle area)
    "small_n1280": (512, WALL_SHAPE_SMALL, 4, 64, math.pi * 0.25**2),
    "mid_n16k": (4096, WALL_SHAPE_SMALL, 128, 64, 0.15 * CELL_AREA / 128),
    "paper_n128k": (16384, WALL_SHAPE_LARGE, 750, 128, 0.15 * CELL_AREA / 750),
    # a 4x larger channel of the same shape and fill (scaling of the sum beyond the paper's size)
    "large_n512k": (65536, WALL_SHAPE_LARGE, 3072, 128, 0.15 * CELL_AREA / 3072),
}
WORKLOAD_SEED = {"small_n1280": SEED_BASE + 0, "mid_n16k": SEED_BASE + 1, "paper_n128k": SEED_BASE + 2,
                 "large_n512k": SEED_BASE + 5}


def channel(n_w, modes, n_ves, n_v, area, seed, period=TWO_PI, mu=1.0, gap_factor=5.0) -> Geometry:
    ss = np.random.SeedSequence(seed)
    s_geo, _, _ = ss.spawn(3)
    rng = np.random.Generator(np.random.PCG64(s_geo))
    lower, upper = wall_curves(n_w, modes, period)
    ves = place_vesicles(rng, [lower, upper], modes, period, n_ves, n_v, area,
                         gap_factor=gap_factor) if n_ves else []
    return Geometry([lower, upper] + ves, period, mu,
                    dict(n_w=n_w, modes=modes, n_ves=n_ves, n_v=n_v, area=area, seed=seed))


_CACHE: dict = {}


def workload(name: str, seed: int | None = None):
    """(geometry, slp_density, dlp_density) for a named workload."""
    seed = WORKLOAD_SEED[name] if seed is None else seed
    key = (name, seed)
    if key not in _CACHE:
        n_w, modes, nv, n_v, area = WORKLOADS[name]
        g = channel(n_w, modes, nv, n_v, area, seed)
        g.meta["name"] = name
        slp, dlp = densities(g, seed)
        _CACHE[key] = (g, slp, dlp)
    return _CACHE[key]


ENSEMBLE_GAP = 2.0  # node gap >= 2h: 5h with 32-node vesicles at 15% fill nears jamming


def _ensemble_member(args):
    n_w, modes, nv, n_v, area, s = args
    g = channel(n_w, modes, nv, n_v, area, s, gap_factor=ENSEMBLE_GAP)
    slp, dlp = densities(g, s)
    return g, slp, dlp


def ensemble(count: int = 64, seed: int = SEED_BASE + 3, size_scale: float = 1.0,
             workers: int = 0):
    """Independent channel instances of mixed sizes (batched workload).

    Wall nodes per wall from {1024, 2048, 4096, 8192}, vesicle counts
    U[10, 400], nodes per vesicle from {32, 64, 128, 256}, volume fraction
    U[0.05, 0.15]; walls alternate between the small and large shapes.
    ``size_scale`` < 1 shrinks node and vesicle counts for quick tests.  The
    instances are independent, so ``workers`` > 1 builds them in a process pool
    (spawned, so it is safe after CUDA has been initialised); the result does not
    depend on ``workers``.
    """
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))
    jobs = []
    for i in range(count):
        n_w = int(rng.choice([1024, 2048, 4096, 8192]))
        nv = int(rng.integers(10, 401))
        n_v = int(rng.choice([32, 64, 128, 256]))
        phi = rng.uniform(0.05, 0.15)
        area = phi * CELL_AREA / nv  # vesicle size of the full-size instance
        if size_scale != 1.0:
            n_w = max(64, int(n_w * size_scale) // 32 * 32)
            nv = max(1, int(nv * size_scale))
            n_v = max(16, int(n_v * size_scale) // 2 * 2)
        modes = WALL_SHAPE_SMALL if i % 2 == 0 else WALL_SHAPE_LARGE
        jobs.append((n_w, modes, nv, n_v, area, int(rng.integers(0, 2**31))))
    if workers and workers > 1 and count > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_ensemble_member, jobs))
    return [_ensemble_member(j) for j in jobs]
