"""Gradients of a final overlap with respect to the layer potentials.

``overlap_loss(theta1, theta2, ...)`` evolves phi_0 by nsteps steps of the
layer-split scheme with potentials v_j(x) = sum_h theta_{j,h} cos(2 pi h x / L_j)
(1D) and returns L = |<chi, phi_T>|^2.  Its backward runs the library's reverse
sweep (ls_adjoint): the factors are unitary, so phi_T is rebuilt step by step
while lambda = dL/d conj(phi) is pulled back; no trajectory is stored.

Checkpoints by drift.  Rebuilding phi backward in finite precision drifts from
the forward trajectory.  The forward pass measures that drift with the reverse
sweep itself: after ``probe`` steps it rebuilds phi_0 from a copy (ls_adjoint
with lambda = 0) and takes d = ||phi_0' - phi_0|| / ||phi_0||.  Assuming the
drift grows at most linearly in the number of reversed steps (rounding errors
that add up coherently; random ones grow more slowly), a segment of
L = drift_tol * probe / d steps keeps the rebuild drift below drift_tol, so
checkpoints are stored only every L steps (none if L >= nsteps).  The backward
pass replaces the rebuilt state by the stored one at each checkpoint and
records the drift it actually found there.  ``checkpoint_every`` forces a fixed
interval instead.

The loss derivative at the final time, lambda_T = <chi, phi_T> chi, is a scaled
copy of chi; every propagation and gradient accumulation runs in the library.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from ._binding import Context


def _cos_problem(base, theta1, theta2):
    def coeffs(th):
        hs, cs = [], []
        for h, t in enumerate(np.asarray(th, dtype=np.float64).reshape(-1), start=1):
            hs += [[h], [-h]]
            cs += [t / 2.0, t / 2.0]
        return np.array(hs, dtype=np.int64), np.array(cs, dtype=np.complex128)
    h1, c1 = coeffs(theta1)
    h2, c2 = coeffs(theta2)
    return base.with_potentials(c1, c2, h1, h2)


def _rebuild_drift(c, psi0, psi_k, k, tau, scheme, seed, step0):
    """||phi_0' - phi_0|| / ||phi_0|| where phi_0' is rebuilt from phi_k by the
    reverse sweep of k steps (the same kernels the backward pass runs)."""
    x = psi_k.clone()
    lam = torch.zeros_like(x)
    c.adjoint(x, lam, k, tau, scheme, seed=seed, step0=step0)
    return float(torch.linalg.vector_norm(x - psi0) / torch.linalg.vector_norm(psi0))


def checkpoint_plan(c, psi0, nsteps, tau, scheme, seed=0, drift_tol=1e-4, probe=50):
    """Checkpoint steps for a drift tolerance: probe the rebuild drift of the
    first min(probe, nsteps) steps and space checkpoints so that the linearly
    extrapolated drift of every segment stays below drift_tol.  Returns
    (sorted checkpoint steps, measured probe drift, probe length)."""
    P = max(1, min(int(probe), int(nsteps)))
    x = psi0.clone()
    c.step(x, P, tau, scheme, seed=seed, step0=0)
    d = _rebuild_drift(c, psi0, x, P, tau, scheme, seed, 0)
    rate = max(d, 1e-300) / P
    L = max(1, int(math.floor(drift_tol / rate)))
    L = max(L, 1)
    return list(range(L, nsteps, L)), d, P


class _OverlapLoss(torch.autograd.Function):
    @staticmethod
    def forward(actx, theta1, theta2, base, phi0, chi, tau, nsteps, scheme, dtype, checkpoint_every, drift_tol,
                probe, seed):
        prob = _cos_problem(base, theta1.detach().cpu().numpy(), theta2.detach().cpu().numpy())
        c = Context(prob, dtype)
        psi = c.from_dense(phi0) if isinstance(phi0, np.ndarray) else phi0.clone()
        chi_t = c.from_dense(chi) if isinstance(chi, np.ndarray) else chi
        probe_drift = None
        if checkpoint_every:
            marks = list(range(int(checkpoint_every), nsteps, int(checkpoint_every)))
        elif drift_tol:
            marks, probe_drift, _ = checkpoint_plan(c, psi, nsteps, tau, scheme, seed, drift_tol, probe)
        else:
            marks = []
        ckpts = {}
        done = 0
        for m in marks + [nsteps]:
            c.step(psi, m - done, tau, scheme, seed=seed, step0=done)
            done = m
            if m < nsteps:
                ckpts[m] = psi.clone()
        ov = c.observables(psi, chi_t)["overlap"]
        actx.c, actx.psi, actx.chi, actx.ov = c, psi, chi_t, ov
        actx.tau, actx.n, actx.scheme, actx.ckpts, actx.seed = tau, nsteps, scheme, ckpts, seed
        actx.nth = (theta1.numel(), theta2.numel())
        actx.probe_drift = probe_drift
        return torch.tensor(abs(ov) ** 2, dtype=torch.float64)

    @staticmethod
    def backward(actx, gL):
        c = actx.c
        # the sweep runs on a copy: phi_T stays in the context, so a second
        # backward (retain_graph=True) starts from phi_T again
        psi = actx.psi.clone()
        lam = (actx.chi * complex(actx.ov)).contiguous()
        n1, n2 = actx.nth
        g1 = np.zeros(n1)
        g2 = np.zeros(n2)
        drift = []
        end = actx.n
        for start in reversed([0] + sorted(actx.ckpts)):
            seg = end - start
            _, _, gc1, gc2 = c.adjoint(psi, lam, seg, actx.tau, actx.scheme, seed=actx.seed, step0=start)
            # coefficients come in (+h, -h) pairs, each theta_h / 2
            g1 += 0.5 * (gc1[0::2, 0] + gc1[1::2, 0])
            g2 += 0.5 * (gc2[0::2, 0] + gc2[1::2, 0])
            if start in actx.ckpts:
                ref = actx.ckpts[start]
                drift.append(float(torch.linalg.vector_norm(psi - ref).item()))
                psi.copy_(ref)
            end = start
        actx.drift = drift
        s = float(gL)
        return (torch.tensor(s * g1, dtype=torch.float64), torch.tensor(s * g2, dtype=torch.float64),
                None, None, None, None, None, None, None, None, None, None, None)


def overlap_loss(theta1, theta2, base, phi0, chi, tau: float, nsteps: int, scheme: str = "strang",
                 dtype: str = "c64", checkpoint_every: int = 0, drift_tol: float = 1e-4, probe: int = 50,
                 seed: int = 0):
    """L = |<chi, phi_T>|^2 as a differentiable function of the cosine
    coefficients theta1 (layer 1) and theta2 (layer 2) (float64 CPU tensors).
    ``base``: a 1D workloads.Problem (its potentials are replaced); phi0, chi:
    dense (M2, M1) arrays or device tensors in the context layout.
    Checkpoints: every ``checkpoint_every`` steps if set, otherwise placed by
    the measured rebuild drift against ``drift_tol`` (0: none).  ``seed``
    fixes the samples of the stochastic schemes (lie_stoch, strang_stoch)."""
    return _OverlapLoss.apply(theta1, theta2, base, phi0, chi, tau, nsteps, scheme, dtype, checkpoint_every,
                              drift_tol, probe, seed)
