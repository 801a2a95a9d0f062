"""Learned warm start of the semi-implicit vesicle step: data, training, evaluation.

Orchestration only: every numerical step runs in libstokes (the time step, the feature and
target transforms, the network's forward/backward/Adam kernels).  PyTorch holds the device
buffers; the shuffles are seeded NumPy permutations passed to the training kernels.
"""
from __future__ import annotations

import time

import numpy as np

from . import (STOKES_FP64, STOKES_GUESS_EXTRAPOLATE, STOKES_GUESS_MLP, STOKES_GUESS_PREVIOUS,
               STOKES_GUESS_ZERO, STOKES_WARM_BASE_EXTRAPOLATE, STOKES_WARM_BASE_PREVIOUS,
               feature_dims, stokes_sim_set_warm_base, stokes_mlp_create, stokes_sim_set_residual_fmm,
               stokes_sim_set_sweep_fmm, stokes_sim_set_precond_refresh, stokes_sim_set_precond_tensor,
               stokes_sim_set_warm_history, stokes_sim_set_warm_modes, stokes_mlp_destroy, stokes_sim_set_restart,
               stokes_mlp_fit_normalization, stokes_mlp_get_adam, stokes_mlp_get_normalization,
               stokes_mlp_get_params, stokes_mlp_num_params, stokes_mlp_set_adam,
               stokes_mlp_set_normalization, stokes_mlp_set_params,
               stokes_mlp_train_step, stokes_sim_create, stokes_sim_destroy,
               stokes_sim_get_history, stokes_sim_get_state, stokes_sim_last_features,
               stokes_sim_set_history, stokes_sim_set_state, stokes_sim_set_wall_solver,
               stokes_sim_set_vesicles, stokes_sim_set_walls, stokes_sim_sizes,
               vesicle_step_warmstart)

GUESS_NAMES = {"zero": STOKES_GUESS_ZERO, "previous": STOKES_GUESS_PREVIOUS, "mlp": STOKES_GUESS_MLP,
               "extrapolate": STOKES_GUESS_EXTRAPOLATE}
BASES = {"previous": STOKES_WARM_BASE_PREVIOUS, "extrapolate": STOKES_WARM_BASE_EXTRAPOLATE}


class Simulation:
    """A channel with vesicles (from an inputs.Geometry) on the GPU."""

    def __init__(self, geom, kappa_b=1.0, K=32, M=128, device=0, restart=80, wall_solver=None,
                 modes=16, residual_fmm=0, history=False, base="previous", sweep_fmm=0,
                 precond_refresh=False, precond_tensor=False):
        walls = [c for c in geom.curves if c.kind == 0]
        ves = [c for c in geom.curves if c.kind == 1]
        self.h = stokes_sim_create(device)
        self.mu, self.period = geom.mu, geom.period
        if wall_solver is not None:  # else the library's default (the fast direct solver)
            stokes_sim_set_wall_solver(self.h, wall_solver)
        if walls:
            lo, up = walls
            stokes_sim_set_walls(self.h, lo.n, np.vstack([lo.nodes, up.nodes]),
                                 np.concatenate([lo.weights, up.weights]),
                                 np.vstack([lo.normals, up.normals]),
                                 np.concatenate([lo.curvature, up.curvature]), geom.period,
                                 geom.mu, K, M)
        self.x0 = np.vstack([c.nodes for c in ves])
        stokes_sim_set_vesicles(self.h, len(ves), ves[0].n, self.x0, kappa_b, geom.mu, geom.period)
        self.V, self.n, _ = stokes_sim_sizes(self.h)
        if restart != 80:
            stokes_sim_set_restart(self.h, restart)
        self.modes = int(modes)
        self.history = bool(history)
        self.base = base
        stokes_sim_set_warm_modes(self.h, self.modes)
        stokes_sim_set_warm_history(self.h, self.history)
        stokes_sim_set_warm_base(self.h, BASES[base])
        if residual_fmm:  # mixed-precision steps take their FP64-accurate vesicle sums by FMM
            stokes_sim_set_residual_fmm(self.h, residual_fmm)
        if sweep_fmm:  # ... and their Krylov sweeps' sums from the same plan at a lower order
            stokes_sim_set_sweep_fmm(self.h, sweep_fmm)
        if precond_refresh:  # Newton-Schulz refresh of the preconditioner inverse
            stokes_sim_set_precond_refresh(self.h, True)
        if precond_tensor:  # ... and its GEMMs by BF16x9 FP32 emulation on the tensor cores
            stokes_sim_set_precond_tensor(self.h, True)

    def step(self, dt, p_drive, guess="zero", model=None, tol=1e-10, max_iter=500,
             precision=STOKES_FP64):
        return vesicle_step_warmstart(self.h, dt, p_drive, GUESS_NAMES[guess], model, None, tol,
                                      max_iter, precision)

    def state(self):
        return stokes_sim_get_state(self.h)

    def set_state(self, x, sigma):
        stokes_sim_set_state(self.h, x, sigma)

    def save(self, path, step=0):
        """Checkpoint of the run (positions, tension, initial perimeters and areas, previous
        solution and right-hand side, step index) to an .npz file."""
        x, sigma, _ = stokes_sim_get_state(self.h)
        L0, A0, zprev, bprev = stokes_sim_get_history(self.h)
        np.savez(path, x=x, sigma=sigma, L0=L0, A0=A0, zprev=zprev, bprev=bprev,
                 step=np.int64(step), V=np.int64(self.V), n=np.int64(self.n))

    def restore(self, path):
        """Continue a checkpointed run (same walls and vesicle count); returns its step index."""
        with np.load(path) as z:
            if int(z["V"]) != self.V or int(z["n"]) != self.n:
                raise ValueError("checkpoint of %d x %d vesicles, simulation has %d x %d"
                                 % (int(z["V"]), int(z["n"]), self.V, self.n))
            stokes_sim_set_state(self.h, z["x"], z["sigma"])  # clears the history ...
            stokes_sim_set_history(self.h, z["L0"], z["A0"], z["zprev"], z["bprev"])  # ... restored here
            return int(z["step"])

    def features(self, feat, targ):
        stokes_sim_last_features(self.h, feat, targ)

    def close(self):
        if getattr(self, "h", None):
            stokes_sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def collect(sim: Simulation, steps, dt, p_drive, guess="previous", tol=1e-10,
            precision=STOKES_FP64):
    """Run plain steps; return device tensors (features, targets) of the vesicle states and the
    per-step statistics.  Every precision solves to the same FP64 tolerance.  The run's first
    step has no previous solution (its "change" would be the whole solution, far outside what a
    warm start ever predicts), and with the extrapolation base the second step's target is still
    a first difference, so those states are left out: (steps - skip) V rows."""
    import torch
    V = sim.V
    skip = 2 if sim.base == "extrapolate" else 1
    nf, nt = feature_dims(sim.modes, sim.history)
    X = torch.empty((max(steps - skip, 0) * V, nf), dtype=torch.float32, device="cuda")
    T = torch.empty((max(steps - skip, 0) * V, nt), dtype=torch.float32, device="cuda")
    stats = []
    for k in range(steps):
        stats.append(sim.step(dt, p_drive, "zero" if k == 0 else guess, tol=tol,
                              precision=precision))
        if k >= skip:
            sim.features(X[(k - skip) * V:(k - skip + 1) * V], T[(k - skip) * V:(k - skip + 1) * V])
    return X, T, stats


class WarmStartNet:
    """The 4 nm -> H -> H -> 3 nm network (nm warm-start modes; 64 -> H -> H -> 48 at the default
    16); parameters initialised from a seeded NumPy draw."""

    def __init__(self, hidden=256, seed=0, device=0, modes=16, history=False):
        # (a network is used with the feature set and base guess of the data it was fitted to)
        nf, nt = feature_dims(modes, history)
        self.h = stokes_mlp_create(device, nf, hidden, nt)
        self.hidden = hidden
        self.modes = int(modes)
        self.history = bool(history)
        rng = np.random.default_rng(seed)
        theta = []
        for fan_in, fan_out in ((nf, hidden), (hidden, hidden), (hidden, nt)):
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            theta.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
            theta.append(np.zeros(fan_out))
        stokes_mlp_set_params(self.h, np.concatenate(theta).astype(np.float32))
        assert stokes_mlp_num_params(self.h) == sum(t.size for t in theta)

    def save(self, path):
        """Parameters, input/output normalisation and Adam state to an .npz file."""
        theta = stokes_mlp_get_params(self.h)
        norm = stokes_mlp_get_normalization(self.h, *feature_dims(self.modes, self.history))
        m, v, t = stokes_mlp_get_adam(self.h)
        np.savez(path, theta=theta, norm=norm, adam_m=m, adam_v=v, adam_t=np.int64(t),
                 hidden=np.int64(self.hidden))

    def load(self, path):
        with np.load(path) as z:
            if int(z["hidden"]) != self.hidden:
                raise ValueError("checkpoint of a %d-wide network" % int(z["hidden"]))
            stokes_mlp_set_params(self.h, z["theta"])  # resets Adam ...
            stokes_mlp_set_normalization(self.h, z["norm"])
            stokes_mlp_set_adam(self.h, z["adam_m"], z["adam_v"], int(z["adam_t"]))  # ... restored

    def fit(self, X, T, epochs=30, batch=256, lr=2e-3, seed=1, lr_decay=0.97, start_epoch=0):
        """Adam on shuffled minibatches; returns the per-epoch mean losses.  start_epoch > 0
        resumes a checkpointed fit (same data and seed): the normalisation is kept and the
        shuffles and learning rate continue where epoch start_epoch begins."""
        import torch
        rng = np.random.default_rng(seed)
        rows = X.shape[0]
        if start_epoch == 0:
            stokes_mlp_fit_normalization(self.h, X, T)
        for _ in range(start_epoch):
            rng.permutation(rows)
        lr *= lr_decay ** start_epoch
        losses = []
        for ep in range(start_epoch, epochs):
            perm = torch.as_tensor(rng.permutation(rows).astype(np.int32), device="cuda")
            tot, cnt = 0.0, 0
            for b0 in range(0, rows - batch + 1, batch):
                tot += stokes_mlp_train_step(self.h, X, T, perm[b0:b0 + batch], lr)
                cnt += 1
            losses.append(tot / max(cnt, 1))
            lr *= lr_decay
        return losses

    def close(self):
        if getattr(self, "h", None):
            stokes_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def evaluate(sim: Simulation, x_start, sigma_start, steps, dt, p_drive, model=None,
             guesses=("zero", "previous", "mlp"), tol=1e-10, precision=STOKES_FP64):
    """From the same start state, run `steps` steps per guess kind; iterations and times."""
    out = {}
    for gname in guesses:
        if gname == "mlp" and model is None:
            continue
        sim.set_state(x_start, sigma_start)
        its, tms, gms, refs, accs = [], [], [], [], []
        for k in range(steps):
            # the first step of a run has no previous solution (nothing to extrapolate from):
            # every warm start starts from zero there (the library itself falls back to the
            # previous solution while an extrapolation lacks its second one)
            g = "zero" if (gname in ("previous", "mlp", "extrapolate") and k == 0) else gname
            t0 = time.perf_counter()
            st = sim.step(dt, p_drive, g, model=model.h if model is not None else None, tol=tol,
                          precision=precision)
            tms.append(1e3 * (time.perf_counter() - t0))
            its.append(st["iterations"])
            gms.append(st["gmres_ms"])
            refs.append(st["refinements"])
            accs.append(st["accurate_residuals"])
        out[gname] = {"iterations": its, "mean_iterations": float(np.mean(its)),
                      "step_ms": float(np.mean(tms)), "gmres_ms": float(np.mean(gms)),
                      "mean_refinements": float(np.mean(refs)),
                      "mean_accurate_residuals": float(np.mean(accs))}
    return out
