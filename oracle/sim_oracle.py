"""FP64 NumPy oracle of the channel response and the semi-implicit vesicle step.

TEST INFRASTRUCTURE ONLY: used by the tests, the package smoke check and the benchmark's
CPU-baseline leg, never by the product path; it imports nothing from the CUDA package.

Channel response (Sec. 2.2, 2.3 and the three-step procedure of Sec. 3.1):
  representation u = D^near tau + sum_m c_m S(., y_m) (Eq. (urep)) with proxy stokeslets y_m
  on a circle of radius R_p around the cell centre (Eq. (phi)); the extended linear system
  [A B; C Q][tau; c] = [v; g] (Eq. (BIEU), (BIED), (BIEgu), (BIEgT)) is assembled densely
  and solved by the block elimination of Sec. 4.1, c = S^+ (g - C A^-1 v),
  tau = A^-1 v - A^-1 B c with S = Q - C A^-1 B and S^+ a pseudo-inverse.
  Side points L are K Gauss-Legendre nodes across the inlet at x = 0, R = L + d; their
  normal is (1, 0).  The pressure drive enters as g_T = p_drive n, p_drive being the
  pressure drop over one period (flow towards +x for p_drive > 0).

Semi-implicit step (Sec. 3.2, Eq. (tsteplinsys) with the arc-length correction
Eq. (ALC), App. A; area correction App. B; reparameterization App. C, Algorithm 2):
  dense assembly of the full single-layer operator over all vesicles (Kress self blocks
  and +-d images) and of the Fourier differentiation operators, one direct solve.
"""
from __future__ import annotations

import math

import numpy as np

PI = math.pi


# ---------------------------------------------------------------------------
# kernels (Sec. 2.1)
# ---------------------------------------------------------------------------
def stokeslet(x, y, mu):
    """S(x, y), Eq. (S): (1/(4 pi mu)) (log(1/r) I + r r^T / r^2); x, y (..., 2) -> (..., 2, 2)."""
    r = np.asarray(x, float) - np.asarray(y, float)
    rr = (r * r).sum(-1)
    out = np.einsum("...i,...j->...ij", r, r) / rr[..., None, None]
    out += (np.log(1.0 / np.sqrt(rr)))[..., None, None] * np.eye(2)
    return out / (4 * PI * mu)


def stresslet(x, y, ny):
    """D(x, y), Eq. (D): (1/pi) r r^T (r . n_y) / r^4."""
    r = np.asarray(x, float) - np.asarray(y, float)
    rr = (r * r).sum(-1)
    rn = (r * ny).sum(-1)
    return np.einsum("...i,...j->...ij", r, r) * (rn / (PI * rr * rr))[..., None, None]


def slp_pressure(x, y):
    """Q(x, y), Eq. (Q): pressure at x of the stokeslet at y, (1/(2 pi)) r / r^2 (row vector)."""
    r = np.asarray(x, float) - np.asarray(y, float)
    rr = (r * r).sum(-1)
    return r / (2 * PI * rr[..., None])


def dlp_pressure(x, y, ny, mu):
    """P(x, y), Eq. (P): pressure at x of the double layer at y, (mu/pi)(-n_y/r^2 + 2 (r.n_y) r/r^4)."""
    r = np.asarray(x, float) - np.asarray(y, float)
    ny = np.broadcast_to(ny, r.shape)
    rr = (r * r).sum(-1)
    rn = (r * ny).sum(-1)
    return (mu / PI) * (-ny / rr[..., None] + 2 * (rn / (rr * rr))[..., None] * r)


def layer_fields(src, w, nrm, kind, slp, dlp, period, mu, pts, pts_normals=None):
    """Pressure and (with target normals) traction at free points of the near-image layer
    potentials: sum over images m = -1, 0, 1 and every source j of Q w f (vesicle sources,
    Eq. (Q)) + P w tau (wall sources, Eq. (P)), and K w f + T w tau (Eq. (K), (T)); plain
    trapezoid rule, nothing skipped (the targets lie off the curves).  src (N, 2), kind (N,)
    0 = wall, 1 = vesicle; slp / dlp are the densities of the vesicle / wall nodes in node order."""
    pts = np.atleast_2d(np.asarray(pts, float))
    ves = kind == 1
    dens = np.zeros_like(src)
    dens[ves] = slp
    dens[~ves] = dlp
    q = w[:, None] * dens
    p = np.zeros(len(pts))
    t = np.zeros_like(pts) if pts_normals is not None else None
    images = (-1, 0, 1) if period != 0.0 else (0,)
    for m in images:
        y = src + np.array([m * period, 0.0])
        p += np.einsum("pji,ji->p", slp_pressure(pts[:, None], y[None, ves]), q[ves])
        p += np.einsum("pji,ji->p", dlp_pressure(pts[:, None], y[None, ~ves], nrm[None, ~ves], mu), q[~ves])
        if t is not None:
            nx = pts_normals[:, None, :]
            t += np.einsum("pjik,jk->pi", slp_traction(pts[:, None], y[None, ves], nx), q[ves])
            t += np.einsum("pjik,jk->pi", dlp_traction(pts[:, None], y[None, ~ves], nx,
                                                       nrm[None, ~ves], mu), q[~ves])
    return p, t


def slp_traction(x, y, nx):
    """K(x, y), Eq. (K): traction at x (normal n_x) of the stokeslet at y: -(1/pi) r r^T (r.n_x)/r^4."""
    r = np.asarray(x, float) - np.asarray(y, float)
    rr = (r * r).sum(-1)
    rn = (r * nx).sum(-1)
    return -np.einsum("...i,...j->...ij", r, r) * (rn / (PI * rr * rr))[..., None, None]


def dlp_traction(x, y, nx, ny, mu):
    """T(x, y), Eq. (T): traction at x (normal n_x) of the double layer at y (normal n_y)."""
    r = np.asarray(x, float) - np.asarray(y, float)
    nx = np.broadcast_to(nx, r.shape)
    ny = np.broadcast_to(ny, r.shape)
    rr = (r * r).sum(-1)
    # dipole functions: d_x = (r . n_x) / r^2 (target), d_y = (r . n_y) / r^2 (source); with
    # this reading the formula of Eq. (T) is the traction of the (D, P) pair of Eq. (D), (P)
    dx = (r * nx).sum(-1) / rr
    dy = (r * ny).sum(-1) / rr
    nn = (nx * ny).sum(-1)
    rrT = np.einsum("...i,...k->...ik", r, r) / rr[..., None, None]
    out = ((nn / rr - 8 * dx * dy)[..., None, None] * rrT
           + (dx * dy)[..., None, None] * np.eye(2)
           + np.einsum("...i,...k->...ik", nx, ny) / rr[..., None, None]
           + dx[..., None, None] * np.einsum("...k,...i->...ik", r, ny) / rr[..., None, None]
           + dy[..., None, None] * np.einsum("...i,...k->...ik", r, nx) / rr[..., None, None])
    return (mu / PI) * out


# ---------------------------------------------------------------------------
# channel response
# ---------------------------------------------------------------------------
class Walls:
    """Both walls of one cell (nodes (N_w, 2) each; lower first), side and proxy points."""

    def __init__(self, lower, upper, period, mu, K=32, M=128, Rp=None):
        self.curves = [lower, upper]
        self.x = np.vstack([lower.nodes, upper.nodes])
        self.w = np.concatenate([lower.weights, upper.weights])
        self.n = np.vstack([lower.normals, upper.normals])
        self.kap = np.concatenate([lower.curvature, upper.curvature])
        self.d = float(period)
        self.mu = float(mu)
        # side wall L across the inlet at x = 0 (between the two walls' first nodes)
        ylo, yhi = lower.nodes[0, 1], upper.nodes[0, 1]
        assert abs(lower.nodes[0, 0]) < 1e-14 and abs(upper.nodes[0, 0]) < 1e-14
        t, _ = np.polynomial.legendre.leggauss(K)
        self.L = np.stack([np.zeros(K), 0.5 * (ylo + yhi) + 0.5 * (yhi - ylo) * t], 1)
        self.R = self.L + np.array([self.d, 0.0])
        self.side_n = np.array([1.0, 0.0])
        Rp = self.d if Rp is None else Rp
        th = 2 * PI * np.arange(M) / M
        self.proxy = np.stack([0.5 * self.d + Rp * np.cos(th), Rp * np.sin(th)], 1)
        self.K, self.M = K, M

    # --- blocks -----------------------------------------------------------
    def A(self):
        """-1/2 I + D^near on the walls (Nystrom, curvature diagonal), Eq. (BIEU)/(BIED)."""
        x, n, w = self.x, self.n, self.w
        Nt = x.shape[0]
        A = np.zeros((Nt, 2, Nt, 2))
        for m in (-1, 0, 1):
            y = x + np.array([m * self.d, 0.0])
            blk = stresslet(x[:, None, :], y[None, :, :], n[None, :, :]) * w[None, :, None, None]
            if m == 0:
                idx = np.arange(Nt)
                t = np.stack([-n[:, 1], n[:, 0]], 1)
                blk[idx, idx] = (-self.kap / (2 * PI) * w)[:, None, None] * np.einsum("ni,nj->nij", t, t)
            A += blk.transpose(0, 2, 1, 3)
        A = A.reshape(2 * Nt, 2 * Nt) - 0.5 * np.eye(2 * Nt)
        return A

    def B(self):
        blk = stokeslet(self.x[:, None, :], self.proxy[None, :, :], self.mu)
        return blk.transpose(0, 2, 1, 3).reshape(2 * self.x.shape[0], 2 * self.M)

    def C(self):
        """Velocity and traction discrepancy of D^near tau between R and L, Eq. (BIEgu)/(BIEgT)."""
        x, n, w = self.x, self.n, self.w
        sh = np.array([self.d, 0.0])
        dv = (stresslet(self.R[:, None, :], (x - sh)[None, :, :], n[None, :, :])
              - stresslet(self.L[:, None, :], (x + sh)[None, :, :], n[None, :, :])) * w[None, :, None, None]
        dt = (dlp_traction(self.R[:, None, :], (x - sh)[None, :, :], self.side_n, n[None, :, :], self.mu)
              - dlp_traction(self.L[:, None, :], (x + sh)[None, :, :], self.side_n, n[None, :, :], self.mu)) \
            * w[None, :, None, None]
        K, Nt = self.K, x.shape[0]
        return np.vstack([dv.transpose(0, 2, 1, 3).reshape(2 * K, 2 * Nt),
                          dt.transpose(0, 2, 1, 3).reshape(2 * K, 2 * Nt)])

    def Q(self):
        y = self.proxy
        dv = stokeslet(self.R[:, None, :], y[None], self.mu) - stokeslet(self.L[:, None, :], y[None], self.mu)
        dt = slp_traction(self.R[:, None, :], y[None], self.side_n) - slp_traction(self.L[:, None, :], y[None], self.side_n)
        K = self.K
        return np.vstack([dv.transpose(0, 2, 1, 3).reshape(2 * K, 2 * self.M),
                          dt.transpose(0, 2, 1, 3).reshape(2 * K, 2 * self.M)])

    def solve(self, v, g, rcond=1e-13):
        """Block solve of Sec. 4.1: c = S^+ (g - C A^-1 v), tau = A^-1 (v - B c)."""
        A, B, C, Q = self.A(), self.B(), self.C(), self.Q()
        Av = np.linalg.solve(A, v)
        AB = np.linalg.solve(A, B)
        S = Q - C @ AB
        c = np.linalg.pinv(S, rcond=rcond) @ (g - C @ Av)
        tau = Av - AB @ c
        return tau.reshape(-1, 2), c.reshape(-1, 2)

    def solve_refined(self, v, g, sweeps=3, rcond=1e-13):
        """The block solve followed by `sweeps` residual corrections on the whole extended
        system: r = [v; g] - [A B; C Q][tau; c], (dtau, dc) = block solve of r.  The truncated
        pseudo-inverse leaves a residual in the side-point rows; the corrections remove it."""
        A, B, C, Q = self.A(), self.B(), self.C(), self.Q()
        tau, c = (z.reshape(-1) for z in self.solve(v, g, rcond))
        for _ in range(sweeps):
            rv = v - A @ tau - B @ c
            rg = g - C @ tau - Q @ c
            dt, dc = self.solve(rv, rg, rcond)
            tau, c = tau + dt.reshape(-1), c + dc.reshape(-1)
        return tau.reshape(-1, 2), c.reshape(-1, 2)

    def solve_lstsq(self, v, g):
        """Minimum-norm least-squares solve of the whole rectangular system (SVD); used to pin
        the discretisation itself, independently of the block elimination."""
        big = np.block([[self.A(), self.B()], [self.C(), self.Q()]])
        z = np.linalg.lstsq(big, np.concatenate([v, g]), rcond=1e-16)[0]
        n = self.x.size
        return z[:n].reshape(-1, 2), z[n:].reshape(-1, 2)

    # --- evaluation ---------------------------------------------------------
    def velocity(self, tau, c, pts):
        """u = D^near tau + sum_m c_m S(., y_m) at free points, Eq. (urep)."""
        pts = np.atleast_2d(pts)
        u = np.zeros_like(pts, dtype=float)
        for m in (-1, 0, 1):
            y = self.x + np.array([m * self.d, 0.0])
            u += np.einsum("pjik,jk->pi", stresslet(pts[:, None], y[None], self.n[None]) * self.w[None, :, None, None], tau)
        u += np.einsum("pmik,mk->pi", stokeslet(pts[:, None], self.proxy[None], self.mu), c)
        return u

    def pressure(self, tau, c, pts):
        """p = P^near tau + sum_m c_m . Q(., y_m) at free points (pressure of Eq. (urep))."""
        pts = np.atleast_2d(pts)
        p = np.zeros(len(pts))
        for m in (-1, 0, 1):
            y = self.x + np.array([m * self.d, 0.0])
            P = dlp_pressure(pts[:, None], y[None], self.n[None], self.mu) * self.w[None, :, None]
            p += np.einsum("pji,ji->p", P, tau)
        p += np.einsum("pmi,mi->p", slp_pressure(pts[:, None], self.proxy[None]), c)
        return p

    def traction(self, tau, c, pts, nrm):
        """Traction of (D^near tau + proxy stokeslets) at pts with normal nrm (Eq. (T), (K))."""
        pts = np.atleast_2d(pts)
        out = np.zeros_like(pts, dtype=float)
        for m in (-1, 0, 1):
            y = self.x + np.array([m * self.d, 0.0])
            T = dlp_traction(pts[:, None], y[None], nrm, self.n[None], self.mu) * self.w[None, :, None, None]
            out += np.einsum("pjik,jk->pi", T, tau)
        out += np.einsum("pmik,mk->pi", slp_traction(pts[:, None], self.proxy[None], nrm), c)
        return out


def vesicle_rhs(walls: Walls, xv, wv, f, p_drive):
    """Data (v, g) of the channel response to vesicle forces f at nodes xv (weights wv),
    Eq. (vesU)-(vesgT): v = -S^near f on the walls, g_u = -S_{gamma-d} f|_R + S_{gamma+d} f|_L,
    g_T = -K(S_{gamma-d} f)|_R + K(S_{gamma+d} f)|_L + p_drive n."""
    d = walls.d
    q = f * wv[:, None]
    v = np.zeros_like(walls.x)
    for m in (-1, 0, 1):
        y = xv + np.array([m * d, 0.0])
        v -= np.einsum("pjik,jk->pi", stokeslet(walls.x[:, None], y[None], walls.mu), q)
    sh = np.array([d, 0.0])
    gu = (-np.einsum("pjik,jk->pi", stokeslet(walls.R[:, None], (xv - sh)[None], walls.mu), q)
          + np.einsum("pjik,jk->pi", stokeslet(walls.L[:, None], (xv + sh)[None], walls.mu), q))
    gt = (-np.einsum("pjik,jk->pi", slp_traction(walls.R[:, None], (xv - sh)[None], walls.side_n), q)
          + np.einsum("pjik,jk->pi", slp_traction(walls.L[:, None], (xv + sh)[None], walls.side_n), q))
    gt = gt + p_drive * walls.side_n
    return v.reshape(-1), np.concatenate([gu.reshape(-1), gt.reshape(-1)])


def empty_channel_rhs(walls: Walls, p_drive):
    """Data of the pure pressure-driven problem: v = 0, g_u = 0, g_T = p_drive n."""
    v = np.zeros(walls.x.size)
    gt = np.tile(p_drive * walls.side_n, (walls.K, 1))
    return v, np.concatenate([np.zeros(2 * walls.K), gt.reshape(-1)])


# ---------------------------------------------------------------------------
# vesicle geometry operators (Sec. 3.2, App. A-C)
# ---------------------------------------------------------------------------
def fourier_diff(n):
    """First-derivative Fourier differentiation matrix for n (even) equispaced nodes on [0, 2pi):
    D_jk = (1/2) (-1)^(j-k) cot((j-k) pi / n), D_jj = 0 (the Nyquist mode is dropped)."""
    j = np.arange(n)
    diff = j[:, None] - j[None, :]
    D = np.zeros((n, n))
    m = diff != 0
    D[m] = 0.5 * ((-1.0) ** diff[m]) / np.tan(diff[m] * PI / n)
    return D


def arclength_ops(x):
    """Speed s = |x_alpha|, d/ds = diag(1/s) D, unit tangent x_s, for one closed curve (n, 2)."""
    n = x.shape[0]
    D = fourier_diff(n)
    xa = D @ x
    s = np.hypot(xa[:, 0], xa[:, 1])
    Ds = D / s[:, None]
    xs = xa / s[:, None]
    return s, Ds, xs


def kress_self_matrix(x, w, nrm, mu):
    """Kress product-rule matrix of the self single layer (2n x 2n, rows (node, comp))."""
    n = x.shape[0]
    h = 2 * PI / n
    s = w / h
    j = np.arange(n)
    R = np.array([-(4 * PI / n) * sum(math.cos(2 * PI * p * k / n) / p for p in range(1, n // 2))
                  - (4 * PI / n ** 2) * (-1) ** k for k in range(n)])
    G = np.zeros((n, 2, n, 2))
    t = np.stack([-nrm[:, 1], nrm[:, 0]], 1)
    for a in range(n):
        for k in range(n):
            if k == a:
                L = math.log(s[a] ** 2)
                M = np.outer(t[a], t[a])
            else:
                r = x[a] - x[k]
                rr = r @ r
                L = math.log(rr / (4 * math.sin(PI * (a - k) / n) ** 2))
                M = np.outer(r, r) / rr
            coef = -0.5 * R[(a - k) % n] + h * (-0.5 * L)
            G[a, :, k, :] = (coef * np.eye(2) + h * M) * s[k] / (4 * PI * mu)
    return G.reshape(2 * n, 2 * n)


def curve_normals_weights(x):
    """Outward normals (for counter-clockwise curves) and trapezoid weights from the nodes."""
    s, _, xs = arclength_ops(x)
    n = x.shape[0]
    return np.stack([xs[:, 1], -xs[:, 0]], 1), s * 2 * PI / n


def slp_operator(xs_list, period, mu):
    """Full single-layer matrix S^near_{gamma,gamma} over all vesicles (node rows (v, k, comp)):
    Kress self blocks, plain trapezoid for other vesicles and for every +-d image."""
    nodes = np.vstack(xs_list)
    ws, ns = [], []
    for x in xs_list:
        nr, w = curve_normals_weights(x)
        ns.append(nr)
        ws.append(w)
    w_all = np.concatenate(ws)
    N = nodes.shape[0]
    S = np.zeros((N, N, 2, 2))
    off = np.cumsum([0] + [x.shape[0] for x in xs_list])
    shifts = (-1, 0, 1) if period else (0,)
    for m in shifts:
        y = nodes + np.array([m * period, 0.0])
        with np.errstate(divide="ignore", invalid="ignore"):
            blk = stokeslet(nodes[:, None], y[None], mu) * w_all[None, :, None, None]
        if m == 0:
            for v in range(len(xs_list)):
                blk[off[v]:off[v + 1], off[v]:off[v + 1]] = 0.0
        S += blk
    S = S.transpose(0, 2, 1, 3)
    for v, x in enumerate(xs_list):
        G = kress_self_matrix(x, ws[v], ns[v], mu).reshape(x.shape[0], 2, x.shape[0], 2)
        S[off[v]:off[v + 1], :, off[v]:off[v + 1], :] += G
    return S.reshape(2 * N, 2 * N)


def close_correction(xs_list, period, mu, factor, K):
    """Close evaluation of the single-layer operator (the near-pair reading of Sec. 3.2; see
    close_oracle): the dense matrix C (rows and columns (node, comp), like slp_operator) to add to
    it.  For every node x_i and every vesicle image m (own vesicle at m = 0 excluded) whose nodes
    come closer to x_i than factor h (h its largest node spacing), the row block of x_i gets the
    close oracle's single layer of the interpolated vesicle minus the plain n-point sum, column
    by column (unit densities)."""
    from oracle import close_oracle as C
    nodes = np.vstack(xs_list)
    ws = [curve_normals_weights(x)[1] for x in xs_list]
    off = np.cumsum([0] + [x.shape[0] for x in xs_list])
    N = nodes.shape[0]
    out = np.zeros((2 * N, 2 * N))
    shifts = (-1, 0, 1) if period else (0,)
    owner = np.repeat(np.arange(len(xs_list)), np.diff(off))
    for i in range(N):
        for b, xb in enumerate(xs_list):
            nb = xb.shape[0]
            for m in shifts:
                if b == owner[i] and m == 0:
                    continue
                xs = xb + np.array([m * period, 0.0])
                h = np.sqrt((np.diff(np.vstack([xs, xs[:1]]), axis=0) ** 2).sum(1)).max()
                if np.sqrt(((xs - nodes[i]) ** 2).sum(1)).min() >= factor * h:
                    continue
                plain = stokeslet(nodes[i][None], xs, mu) * ws[b][:, None, None]  # (nb, 2, 2)
                for j in range(nb):
                    for c in range(2):
                        e = np.zeros((nb, 2))
                        e[j, c] = 1.0
                        fine = C.close_slp(xs, e, nodes[i:i + 1], mu, K=K)[0]
                        out[2 * i:2 * i + 2, 2 * (off[b] + j) + c] += fine - plain[j][:, c]
    return out


def perimeter(x):
    s, _, _ = arclength_ops(x)
    return s.mean() * 2 * PI


def area(x):
    """Enclosed area A = int x y_alpha d alpha (App. B) by the trapezoid rule (spectral)."""
    D = fourier_diff(x.shape[0])
    return np.mean(x[:, 0] * (D @ x[:, 1])) * 2 * PI


def area_correct(x, A0):
    """App. B: x + c n with n = (y_a, -x_a) and c the root closest to 0 of
    A(x) - c int x x_aa + c int (y_a)^2 - c^2 int y_a x_aa = A0 (integrals over alpha)."""
    n = x.shape[0]
    D = fourier_diff(n)
    xa = D @ x
    xaa = D @ xa
    I = lambda g: np.mean(g) * 2 * PI
    a0 = I(x[:, 0] * xa[:, 1]) - A0
    a1 = -I(x[:, 0] * xaa[:, 0]) + I(xa[:, 1] ** 2)
    a2 = -I(xa[:, 1] * xaa[:, 0])
    if abs(a2) < 1e-300:
        c = -a0 / a1
    else:
        disc = a1 * a1 - 4 * a2 * a0
        roots = np.array([(-a1 + math.sqrt(disc)) / (2 * a2), (-a1 - math.sqrt(disc)) / (2 * a2)])
        c = roots[np.argmin(np.abs(roots))]
    return x + c * np.stack([xa[:, 1], -xa[:, 0]], 1)


def fourier_interp(x, alpha):
    """Trigonometric interpolant of the n (even) samples x (n, k) at parameters alpha; the
    Nyquist mode enters as a cosine, so the samples are reproduced exactly."""
    n = x.shape[0]
    X = np.fft.fft(x, axis=0) / n
    k = np.fft.fftfreq(n, 1.0 / n)
    keep = np.ones(n, bool)
    keep[n // 2] = False
    out = (np.exp(1j * np.outer(alpha, k[keep])) @ X[keep]).real
    return out + np.outer(np.cos(n // 2 * np.asarray(alpha)), X[n // 2].real)


def arclength_samples(x):
    """s(2 pi j / n), j = 0..n, of s(alpha) = int_0^alpha |x_beta| d beta from the Fourier
    series of the speed (App. C); the Nyquist term integrates to 0 at the samples."""
    n = x.shape[0]
    s_al, _, _ = arclength_ops(x)
    C = np.fft.fft(s_al) / n
    k = np.fft.fftfreq(n, 1.0 / n)
    a = 2 * PI * np.arange(n) / n
    m = (k != 0) & (np.arange(n) != n // 2)
    sj = C[0].real * a + ((np.exp(1j * np.outer(a, k[m])) - 1.0) @ (C[m] / (1j * k[m]))).real
    return np.append(sj, C[0].real * 2 * PI)


def reparametrize(x):
    """App. C, Algorithm 2: nearly equal arc-length nodes by inverting s(alpha) piecewise
    linearly at s(2 pi) k / n, then Fourier interpolation of x at the new parameters."""
    n = x.shape[0]
    sj = arclength_samples(x)
    total = sj[n]
    astar = np.zeros(n)
    j = 0
    for q in range(1, n):
        target = total / n * q
        while not (sj[j] <= target < sj[j + 1]):
            j += 1
        astar[q] = 2 * PI / n * (j + (target - sj[j]) / (sj[j + 1] - sj[j]))
    return fourier_interp(x, astar)


# ---------------------------------------------------------------------------
# semi-implicit step (Eq. (tsteplinsys) with Eq. (ALC))
# ---------------------------------------------------------------------------
def forces(x, sigma, kappa_b):
    """Bending -kappa_B x_ssss and tension (sigma x_s)_s of one vesicle (d/ds applied 4 times)."""
    _, Ds, xs = arclength_ops(x)
    xssss = Ds @ (Ds @ (Ds @ (Ds @ x)))
    return -kappa_b * xssss, Ds @ (sigma[:, None] * xs)


def step_system(ves_x, dt, kappa_b, mu, period, L0, close=None):
    """Dense matrix of Eq. (tsteplinsys) (unknowns: u of every node (node, comp), then sigma
    of every node) and the arc-length-corrected constraint right-hand side.  close =
    (factor, K) adds the close-evaluation correction to the single-layer operator."""
    sizes = [x.shape[0] for x in ves_x]
    N = sum(sizes)
    Sop = slp_operator(ves_x, period, mu)
    if close is not None:
        Sop = Sop + close_correction(ves_x, period, mu, *close)
    D4 = np.zeros((2 * N, 2 * N))
    Tsig = np.zeros((2 * N, N))
    Xds = np.zeros((N, 2 * N))
    rhs2 = np.zeros(N)
    o = 0
    for v, x in enumerate(ves_x):
        n = x.shape[0]
        _, Ds, xs = arclength_ops(x)
        Ds4 = Ds @ Ds @ Ds @ Ds
        for c in range(2):
            idx = 2 * (o + np.arange(n)) + c
            D4[np.ix_(idx, idx)] = Ds4
            Tsig[idx, o:o + n] = Ds @ np.diag(xs[:, c])
            Xds[o:o + n, idx] = xs[:, c][:, None] * Ds
        Lk = perimeter(x)
        rhs2[o:o + n] = (L0[v] - Lk) / (dt * Lk)
        o += n
    M = np.block([[np.eye(2 * N) + dt * kappa_b * Sop @ D4, -Sop @ Tsig],
                  [Xds, np.zeros((N, N))]])
    return M, Sop, rhs2


def step(ves_x, sigma, L0, A0, dt, kappa_b, mu, period, walls=None, p_drive=0.0,
         reparam=True, close=None, corrections=True):
    """One semi-implicit step of Algorithm 1: forces, channel response (explicit), the
    solve of Eq. (tsteplinsys) with Eq. (ALC), x <- x + dt u, area correction, reparam.
    corrections=False takes the uncorrected scheme the appendices compare against: the
    plain inextensibility constraint x_s . u_s = 0 (Eq. (ALC) with L_0 = L_k, App. A) and no
    area correction (App. B).
    Returns (new positions, new tensions, u, sigma_{k+1}, u_resp)."""
    if not corrections:
        L0 = [perimeter(x) for x in ves_x]
    sizes = [x.shape[0] for x in ves_x]
    fb, f = [], []
    for x, sg in zip(ves_x, sigma):
        b, t = forces(x, sg, kappa_b)
        fb.append(b)
        f.append(b + t)
    fb = np.vstack(fb)
    f = np.vstack(f)
    M, Sop, rhs2 = step_system(ves_x, dt, kappa_b, mu, period, L0, close)
    xv = np.vstack(ves_x)
    if walls is not None:
        wv = np.concatenate([curve_normals_weights(x)[1] for x in ves_x])
        v, g = vesicle_rhs(walls, xv, wv, f, p_drive)
        tau, c = walls.solve_refined(v, g)
        u_resp = walls.velocity(tau, c, xv)
    else:
        u_resp = np.zeros_like(xv)
    rhs1 = Sop @ fb.reshape(-1) + u_resp.reshape(-1)
    z = np.linalg.solve(M, np.concatenate([rhs1, rhs2]))
    N = xv.shape[0]
    u = z[:2 * N].reshape(N, 2)
    sig_new = z[2 * N:]
    out_x, out_s = [], []
    o = 0
    for v, x in enumerate(ves_x):
        n = x.shape[0]
        xn = x + dt * u[o:o + n]
        if corrections:
            xn = area_correct(xn, A0[v])
        if reparam:
            xn = reparametrize(xn)
        out_x.append(xn)
        out_s.append(sig_new[o:o + n])
        o += n
    return out_x, out_s, u, sig_new, u_resp
