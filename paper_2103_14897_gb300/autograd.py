"""Gradients of a final overlap with respect to the layer potentials.

``overlap_loss(theta1, theta2, ...)`` evolves phi_0 by nsteps steps of the
layer-split scheme with potentials v_j(x) = sum_h theta_{j,h} cos(2 pi h x / L_j)
(1D) and returns L = |<chi, phi_T>|^2.  Its backward runs the library's reverse
sweep (ls_adjoint): the factors are unitary, so phi_T is rebuilt step by step
while lambda = dL/d conj(phi) is pulled back; no trajectory is stored.
Optional checkpoints (every ``checkpoint_every`` steps) replace the rebuilt
state by the stored forward state at segment boundaries, removing the
reconstruction drift where a long run needs it.

The loss derivative at the final time, lambda_T = <chi, phi_T> chi, is a scaled
copy of chi; every propagation and gradient accumulation runs in the library.
"""
from __future__ import annotations

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


class _OverlapLoss(torch.autograd.Function):
    @staticmethod
    def forward(actx, theta1, theta2, base, phi0, chi, tau, nsteps, scheme, dtype, checkpoint_every):
        prob = _cos_problem(base, theta1.detach().cpu().numpy(), theta2.detach().cpu().numpy())
        c = Context(prob, dtype)
        psi = c.from_dense(phi0) if isinstance(phi0, np.ndarray) else phi0.clone()
        chi_t = c.from_dense(chi) if isinstance(chi, np.ndarray) else chi
        ckpts = {}
        if checkpoint_every and checkpoint_every < nsteps:
            done = 0
            while done < nsteps:
                k = min(checkpoint_every, nsteps - done)
                c.step(psi, k, tau, scheme)
                done += k
                if done < nsteps:
                    ckpts[done] = psi.clone()
        else:
            c.step(psi, nsteps, tau, scheme)
        ov = c.observables(psi, chi_t)["overlap"]
        actx.c, actx.psi, actx.chi, actx.ov = c, psi, chi_t, ov
        actx.tau, actx.n, actx.scheme, actx.ckpts = tau, nsteps, scheme, ckpts
        actx.nth = (theta1.numel(), theta2.numel())
        return torch.tensor(abs(ov) ** 2, dtype=torch.float64)

    @staticmethod
    def backward(actx, gL):
        c, psi = actx.c, actx.psi
        lam = (actx.chi * complex(actx.ov)).contiguous()
        n1, n2 = actx.nth
        g1 = np.zeros(n1)
        g2 = np.zeros(n2)
        bounds = sorted(actx.ckpts) + [actx.n]
        drift = []
        end = actx.n
        for start in reversed([0] + sorted(actx.ckpts)):
            seg = end - start
            _, _, gc1, gc2 = c.adjoint(psi, lam, seg, actx.tau, actx.scheme)
            # coefficients come in (+h, -h) pairs, each theta_h / 2
            g1 += 0.5 * (gc1[0::2, 0] + gc1[1::2, 0])
            g2 += 0.5 * (gc2[0::2, 0] + gc2[1::2, 0])
            if start in actx.ckpts:
                ref = actx.ckpts[start]
                drift.append(float(torch.linalg.vector_norm(psi - ref).item()))
                psi.copy_(ref)
            end = start
        actx.drift = drift
        del bounds
        s = float(gL)
        return (torch.tensor(s * g1, dtype=torch.float64), torch.tensor(s * g2, dtype=torch.float64),
                None, None, None, None, None, None, None, None)


def overlap_loss(theta1, theta2, base, phi0, chi, tau: float, nsteps: int, scheme: str = "strang",
                 dtype: str = "c64", checkpoint_every: int = 0):
    """L = |<chi, phi_T>|^2 as a differentiable function of the cosine
    coefficients theta1 (layer 1) and theta2 (layer 2) (float64 CPU tensors).
    ``base``: a 1D workloads.Problem (its potentials are replaced); phi0, chi:
    dense (M2, M1) arrays or device tensors in the context layout."""
    return _OverlapLoss.apply(theta1, theta2, base, phi0, chi, tau, nsteps, scheme, dtype, checkpoint_every)
