"""Plain FP64 NumPy oracle of the Fourier layer-splitting schemes.

TEST INFRASTRUCTURE ONLY (never imported by the library).  Slow and direct:
dense DFT matrices with exact integer-mod arguments, one factor at a time, no
merging of adjacent factors, no blocking.  Each function names the passage of
the paper (arXiv 2103.14897) it follows.

Representation.  A problem (see ``workloads.Problem``) lifts the two layers to
the coefficient array phi[n, m] (Sec. 3): the row index is the linear layer-2
index n, the column index the linear layer-1 index m (for d = 2 the first
component is fastest).  The wavevector of phi[n, m] is k = B1 m + B2 n.

Readings of passages the paper leaves open:

* The lifted array is the full index box; the joint cutoff |k|^2/2 <= Ec of the
  index sets (Sec. 3) is a mask used for the initial state, the index-set query
  and an optional projection.
* The real-space grid of layer j has exactly as many points per dimension as the
  box (Algorithm 3 transforms the coefficient vector itself), so each potential
  sub-step is unitary (Theorem 4.6).
* Algorithm 3 transforms only along the layer-1 index; the layer-2 sub-step is
  taken symmetrically along the layer-2 index (Eq. (3.7): V^2 acts on n).
* The second-order scheme is Strang splitting over H = H1 + H2 with
  H_j = D/2 + V^j (Sec. 4.2 and Appendix A), each exp(-i s H_j) approximated by
  the symmetric product K(s/4) P_j(s) K(s/4).
* The stochastic variant (Algorithm 4 applied to the exponential sub-steps):
  each potential sub-step acts on a seeded random subset of p of the S slices,
  with duration scaled by S/p; the kinetic factors act on every element.
* Shared periodic index (Example 3 of Sec. 5: periodic in y, incommensurate in
  x): a problem with ``shared = 1`` lifts to three indices (m, n, p), p the
  y index common to both layers, stored as a 2D problem whose layer-1 box is
  (q1, 1) and whose layer-2 box is (q2, q3) with the second component p, so
  that k = B1 m + B2 (n, p) = (G1 m + G2 n, G3 p).  A layer-1 factor acts on
  the 2D slices (m, p) at fixed n, a layer-2 factor on (n, p) at fixed m; each
  layer potential is a function of (x, y) with harmonics (h_x, h_y).
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "box_indices", "wavevectors", "kinetic_energy_diag", "index_mask", "mask_count",
    "dft_matrix", "grid_potential", "apply_K", "apply_P", "scheme_factors", "yoshida_weights", "step",
    "toeplitz_potential", "apply_C", "apply_semi_implicit", "density_on_line",
    "splitmix64_next", "sample_slices", "observables", "gaussian_packet",
    "settle_noop", "adjoint", "overlap_loss", "SCHEMES", "coefficient_gradient", "use_fft",
    "TRANSFORM", "sample_count", "expanded_factors", "layer_grid", "layer_slices", "from_layer_slices",
    "n_slices",
]

SCHEMES = ("lie", "strang", "strang_kp", "lie_stoch", "strang_stoch", "yoshida4", "cn_strang",
           "semi_implicit", "random_batch")
MASK64 = (1 << 64) - 1


# --------------------------------------------------------------------------
# Index sets and wavevectors (Sec. 3, definition of the index sets and basis)
# --------------------------------------------------------------------------
def box_indices(lo: Sequence[int], q: Sequence[int]) -> np.ndarray:
    """Integer index vectors of a box in layout order (first component fastest).
    Returns an int64 array of shape (prod q, d)."""
    d = len(q)
    if d == 1:
        return (np.arange(q[0], dtype=np.int64) + lo[0]).reshape(-1, 1)
    i2, i1 = np.meshgrid(np.arange(q[1]), np.arange(q[0]), indexing="ij")
    return np.stack([i1.reshape(-1) + lo[0], i2.reshape(-1) + lo[1]], axis=1).astype(np.int64)


def wavevectors(prob) -> np.ndarray:
    """k(n, m) = B1 m + B2 n for the whole lifted box, shape (M2, M1, d).

    Operation order is fixed (no fused multiply-add in NumPy): for component i,
    u_i = fl(B1[i,0] m_0) + fl(B1[i,1] m_1) + fl(B2[i,0] n_0) + fl(B2[i,1] n_1),
    accumulated left to right."""
    m = box_indices(prob.lo1, prob.q1).astype(np.float64)
    n = box_indices(prob.lo2, prob.q2).astype(np.float64)
    d = prob.d
    B1 = np.asarray(prob.B1, dtype=np.float64)
    B2 = np.asarray(prob.B2, dtype=np.float64)
    out = np.empty((n.shape[0], m.shape[0], d))
    for i in range(d):
        acc = None
        for j in range(d):
            t = B1[i, j] * m[:, j]
            acc = t[None, :] * np.ones((n.shape[0], 1)) if acc is None else acc + t[None, :]
        for j in range(d):
            acc = acc + (B2[i, j] * n[:, j])[:, None]
        out[..., i] = acc
    return out


def kinetic_energy_diag(prob) -> np.ndarray:
    """Diagonal of D (Eq. (3.5)): |k|^2 / 2 as fl(0.5 * fl(sum_i fl(u_i u_i)))."""
    k = wavevectors(prob)
    acc = k[..., 0] * k[..., 0]
    for i in range(1, prob.d):
        acc = acc + k[..., i] * k[..., i]
    return 0.5 * acc


def index_mask(prob) -> np.ndarray:
    """Joint energy-cutoff mask |k|^2/2 <= Ec over the box (inclusive, as the
    index sets of Sec. 3 use <=), shape (M2, M1) of bool."""
    return kinetic_energy_diag(prob) <= prob.ecut


def mask_count(prob) -> int:
    return int(index_mask(prob).sum())


# --------------------------------------------------------------------------
# Transforms and layer potentials (Algorithm 3; Appendix B normalisation)
# --------------------------------------------------------------------------
def dft_matrix(q: int) -> np.ndarray:
    """W[i, p] = exp(+2 pi i ((i p) mod q) / q): coefficient index i to grid
    point p (the unnormalised inverse transform of Algorithm 3).  The integer
    reduction keeps the FP64 argument exact.  The forward transform is
    conj(W) / q, so that the pair preserves the norm as in Appendix B."""
    ip = np.outer(np.arange(q, dtype=np.int64), np.arange(q, dtype=np.int64)) % q
    return np.exp(2j * math.pi * ip / q)


def grid_potential(h: np.ndarray, c: np.ndarray, q: Sequence[int]) -> np.ndarray:
    """v(x_p) = Re sum_h vhat_h exp(i G_h . x_p) on the layer grid
    x_p = A (p / q) (Eq. (2.2)); G_h . x_p = 2 pi sum_i h_i p_i / q_i, evaluated
    per component with exact integer reduction.  Flattened in layout order."""
    h = np.asarray(h, dtype=np.int64).reshape(len(c), -1)
    P = box_indices([0] * len(q), q)
    acc = np.zeros(P.shape[0], dtype=np.complex128)
    for t in range(len(c)):
        ph = np.ones(P.shape[0], dtype=np.complex128)
        for i in range(len(q)):
            r = (h[t, i] * P[:, i]) % q[i]
            ph = ph * np.exp(2j * math.pi * r / q[i])
        acc += c[t] * ph
    return acc.real.copy()


# Transform backend: "dft" (dense matrices, the definition) or "fft" (NumPy's
# FFT as a library primitive for the same transform, used for large arrays;
# pinned against "dft" in the tests).
TRANSFORM = {"kind": "dft"}


def use_fft(on: bool = True) -> None:
    TRANSFORM["kind"] = "fft" if on else "dft"


def _axis_dft(x: np.ndarray, q: Sequence[int], inverse: bool) -> np.ndarray:
    """Apply the (separable) DFT of a layer along axis 1 of x (shape (R, prod q)).
    inverse=True: coefficients -> grid values, W (unnormalised).
    inverse=False: grid values -> coefficients, conj(W) / prod(q).
    For d = 2 the transform matrix is the Kronecker product W(q1) (x) W(q0);
    it is applied one factor at a time."""
    R = x.shape[0]
    if TRANSFORM["kind"] == "fft":
        M = int(np.prod(q))
        y = np.asarray(x).reshape((R,) + tuple(q[::-1]))
        axes = tuple(range(1, len(q) + 1))
        if inverse:
            return (np.fft.ifftn(y, axes=axes) * M).reshape(R, M)
        return (np.fft.fftn(y, axes=axes) / M).reshape(R, M)
    if len(q) == 1:
        W = dft_matrix(q[0])
        return x @ W if inverse else (x @ W.conj()) / q[0]
    y = x.reshape(R, q[1], q[0])
    W0, W1 = dft_matrix(q[0]), dft_matrix(q[1])
    if inverse:
        y = np.einsum("rba,ap->rbp", y, W0)
        y = np.einsum("rbp,bs->rsp", y, W1)
        return y.reshape(R, -1)
    y = np.einsum("rba,ap->rbp", y, W0.conj())
    y = np.einsum("rbp,bs->rsp", y, W1.conj())
    return y.reshape(R, -1) / (q[0] * q[1])


# --------------------------------------------------------------------------
# Slices of a layer (Sec. 3 Kronecker structure; Example 3's shared index)
# --------------------------------------------------------------------------
def _shared(prob) -> bool:
    return bool(getattr(prob, "shared", 0))


def layer_grid(prob, layer: int):
    """(harmonics, coefficients, grid extents) of layer j's potential.  With a
    shared index the grid is (q_j, q3): x on the layer's own cell, y on the
    common period."""
    h, c = (prob.v1_h, prob.v1_c) if layer == 1 else (prob.v2_h, prob.v2_c)
    if _shared(prob):
        q = (prob.q1[0], prob.q2[1]) if layer == 1 else (prob.q2[0], prob.q2[1])
    else:
        q = prob.q1 if layer == 1 else prob.q2
    return h, c, tuple(q)


def layer_slices(prob, phi: np.ndarray, layer: int) -> np.ndarray:
    """The slices of layer j as the rows of a (slices, slice length) array:
    without a shared index, rows of phi (layer 1) or columns (layer 2); with
    one, the (m, p) planes at fixed n (layer 1, m fastest) or the (n, p) planes
    at fixed m (layer 2, n fastest)."""
    if not _shared(prob):
        return phi if layer == 1 else phi.T
    q1, q2, q3 = prob.q1[0], prob.q2[0], prob.q2[1]
    Y = phi.reshape(q3, q2, q1)                       # [p, n, m]
    if layer == 1:
        return Y.transpose(1, 0, 2).reshape(q2, q3 * q1)
    return Y.transpose(2, 0, 1).reshape(q1, q3 * q2)


def from_layer_slices(prob, X: np.ndarray, layer: int) -> np.ndarray:
    """Inverse of layer_slices."""
    if not _shared(prob):
        return X if layer == 1 else X.T.copy()
    q1, q2, q3 = prob.q1[0], prob.q2[0], prob.q2[1]
    if layer == 1:
        Y = X.reshape(q2, q3, q1).transpose(1, 0, 2)
    else:
        Y = X.reshape(q1, q3, q2).transpose(1, 2, 0)
    return np.ascontiguousarray(Y).reshape(q3 * q2, q1)


def n_slices(prob, layer: int) -> int:
    if _shared(prob):
        return prob.q2[0] if layer == 1 else prob.q1[0]
    return prob.M2 if layer == 1 else prob.M1


# --------------------------------------------------------------------------
# The factors of the splitting (Eq. (4.8) sub-problems; Algorithm 3 steps)
# --------------------------------------------------------------------------
def apply_K(prob, phi: np.ndarray, s: float, _kin=None) -> np.ndarray:
    """K(s) = exp(-i s D): phi_mn *= exp(-i s |k|^2 / 2) (Algorithm 3, step 1)."""
    kin = kinetic_energy_diag(prob) if _kin is None else _kin
    return phi * np.exp(-1j * (s * kin))


def apply_P(prob, phi: np.ndarray, layer: int, s: float,
            slices: Optional[np.ndarray] = None, _v=None) -> np.ndarray:
    """P_j(s) = F_j diag(exp(-i s v_j(x_p))) F_j^{-1} along layer j's index for
    every slice (fixed index of the other layer) (Algorithm 3, steps 2-5).

    ``slices`` (optional): indices of the slices the factor acts on; the others
    are left unchanged (the stochastic variant)."""
    h, c, q = layer_grid(prob, layer)
    X = layer_slices(prob, phi, layer)
    v = grid_potential(h, c, q) if _v is None else _v
    T = np.exp(-1j * (s * v))
    if slices is None:
        rows = X
    else:
        rows = X[np.asarray(slices, dtype=np.int64)]
    psi = _axis_dft(rows, q, inverse=True)          # to layer j's real-space grid
    psi = psi * T[None, :]                          # pointwise exp(-i s v_j)
    out_rows = _axis_dft(psi, q, inverse=False)     # back to coefficients
    if slices is None:
        Y = out_rows
    else:
        Y = X.copy()
        Y[np.asarray(slices, dtype=np.int64)] = out_rows
    return from_layer_slices(prob, Y, layer)


def yoshida_weights() -> Tuple[float, float]:
    """Weights of the symmetric fourth-order composition S(w1 t) S(w0 t) S(w1 t)
    of a symmetric second-order step S (Yoshida 1990, the higher-order
    splittings cited in Sec. 4.2 and Appendix A): 2 w1 + w0 = 1 keeps the
    total time, 2 w1^3 + w0^3 = 0 cancels the third-order error, so
    w1 = 1 / (2 - 2^(1/3)) and w0 = -2^(1/3) w1."""
    c = 2.0 ** (1.0 / 3.0)
    w1 = 1.0 / (2.0 - c)
    return w1, -c * w1


def scheme_factors(scheme: str, tau: float) -> List[Tuple]:
    """Factor list of one time step, in application order (rightmost operator
    first).  ('K', s) or ('P', layer, s).

    lie        : P2(t) P1(t) K(t)                     (Algorithm 3 order)
    strang     : L1(t/2) L2(t) L1(t/2), L_j(s) = K(s/4) P_j(s) K(s/4)
                 (Appendix A Strang over H = H1 + H2, H_j = D/2 + V^j)
    strang_kp  : K(t/2) P2(t) P1(t) K(t/2)             (kinetic/potential Strang)
    yoshida4   : strang(w1 t) strang(w0 t) strang(w1 t)  (fourth order, see
                 yoshida_weights)
    cn_strang  : C1(t/2) C2(t) C1(t/2), the Crank-Nicolson factors of Eq. (tsCN)
                 (see apply_C)
    semi_implicit, random_batch : one explicit-potential / implicit-kinetic
                 step (Algorithms 1 and 4, see apply_semi_implicit)
    *_stoch    : same factor list, potential factors act on sampled slices."""
    base = scheme.replace("_stoch", "")
    t = tau
    L = lambda j, s: [("K", s / 4), ("P", j, s), ("K", s / 4)]
    strang = lambda h: L(1, h / 2) + L(2, h) + L(1, h / 2)
    if base == "lie":
        return [("K", t), ("P", 1, t), ("P", 2, t)]
    if base == "strang":
        return strang(t)
    if base == "yoshida4":
        w1, w0 = yoshida_weights()
        return strang(w1 * t) + strang(w0 * t) + strang(w1 * t)
    if base == "cn_strang":
        return [("C", 1, t / 2), ("C", 2, t), ("C", 1, t / 2)]
    if base in ("semi_implicit", "random_batch"):
        return [("S", t)]
    if base == "strang_kp":
        return [("K", t / 2), ("P", 1, t), ("P", 2, t), ("K", t / 2)]
    raise ValueError(f"unknown scheme {scheme}")


# --------------------------------------------------------------------------
# Crank-Nicolson layer splitting (Sec. 4.2.1, Eq. (tsCN)); 1D boxes
# --------------------------------------------------------------------------
def toeplitz_potential(h, c, q: int) -> np.ndarray:
    """The plane-wave matrix of a layer potential on its 1D index box (Sec. 3,
    the matrices V^1, V^2 below Eq. (3.5)): V[m, m'] = vhat(m - m'), zero
    where m - m' carries no coefficient; no wrap across the box ends."""
    V = np.zeros((q, q), dtype=np.complex128)
    for hh, cc in zip(np.asarray(h, dtype=np.int64).reshape(-1), c):
        for m in range(q):
            if 0 <= m - hh < q:
                V[m, m - hh] += cc
    return V


def apply_C(prob, phi: np.ndarray, layer: int, s: float, _kin=None) -> np.ndarray:
    """One Crank-Nicolson factor of duration s for H_j = D/2 + V^j (Eq. (tsCN)):
    every slice x (fixed index of the other layer) becomes the solution y of
    (I + i s A/2) y = (I - i s A/2) x, A = diag(|k|^2/4) + V^j the slice's block.
    With s = tau/2 this is (4I + i tau H_1)^{-1} (4I - i tau H_1) of the first
    and third lines of Eq. (tsCN); with s = tau, (2I + i tau H_2)^{-1}
    (2I - i tau H_2) of the second.  Dense solves (np.linalg.solve)."""
    if prob.d != 1:
        raise ValueError("the Crank-Nicolson splitting is implemented for 1D boxes")
    kin = kinetic_energy_diag(prob) if _kin is None else _kin
    if layer == 1:
        V = toeplitz_potential(prob.v1_h, prob.v1_c, prob.q1[0])
        X, dk = phi, kin
    else:
        V = toeplitz_potential(prob.v2_h, prob.v2_c, prob.q2[0])
        X, dk = phi.T, kin.T
    eye = np.eye(X.shape[1])
    out = np.empty_like(X)
    for r in range(X.shape[0]):
        A = np.diag(dk[r] / 2.0) + V
        out[r] = np.linalg.solve(eye + 0.5j * s * A, (eye - 0.5j * s * A) @ X[r])
    return out if layer == 1 else np.ascontiguousarray(out.T)


# --------------------------------------------------------------------------
# Semi-implicit step and its random batch form (Sec. 4.1 Algorithm 1,
# Sec. 4.3 Algorithm 4); 1D boxes
# --------------------------------------------------------------------------
def apply_semi_implicit(prob, phi: np.ndarray, tau: float, rows=None, cols=None, _kin=None) -> np.ndarray:
    """phi <- (I + i tau D)^{-1} (phi - Psi_1 - Psi_2), Psi_1 = i tau V^1 phi
    slice by slice along m (every row n), Psi_2 = i tau V^2 phi along n (every
    column m); V^j the plane-wave potential matrices (Algorithm 1).
    rows / cols given (Algorithm 4): Psi_1 only on the rows n in rows, scaled by
    M2 / len(rows); Psi_2 only on the columns m in cols, scaled by M1 / len(cols)."""
    if prob.d != 1:
        raise ValueError("the semi-implicit step is implemented for 1D boxes")
    kin = kinetic_energy_diag(prob) if _kin is None else _kin
    V1 = toeplitz_potential(prob.v1_h, prob.v1_c, prob.q1[0])
    V2 = toeplitz_potential(prob.v2_h, prob.v2_c, prob.q2[0])
    psi1 = 1j * tau * (phi @ V1.T)            # row n: V1 @ phi[n, :]
    psi2 = 1j * tau * (V2 @ phi)              # column m: V2 @ phi[:, m]
    if rows is not None:
        w = np.zeros(prob.M2)
        w[np.asarray(rows)] = prob.M2 / len(rows)
        psi1 = psi1 * w[:, None]
    if cols is not None:
        w = np.zeros(prob.M1)
        w[np.asarray(cols)] = prob.M1 / len(cols)
        psi2 = psi2 * w[None, :]
    return (phi - psi1 - psi2) / (1.0 + 1j * tau * kin)


# --------------------------------------------------------------------------
# Real-space wave function on a line (Sec. 3 expansion; the localisation
# plots of Sec. 5)
# --------------------------------------------------------------------------
def density_on_line(prob, phi: np.ndarray, x) -> np.ndarray:
    """psi(x_j) = sum_{m,n} phi[n, m] exp(i k_mn . x_j), the plane-wave
    expansion of the wave function (Sec. 3), evaluated point by point; the
    phase k . x is formed in FP64 from k of wavevectors().  x: (npts,) for 1D
    boxes, (npts, 2) for 2D boxes."""
    k = wavevectors(prob)
    x = np.asarray(x, dtype=np.float64).reshape(-1, prob.d)
    out = np.empty(len(x), dtype=np.complex128)
    for j, xj in enumerate(x):
        out[j] = np.sum(phi * np.exp(1j * (k @ xj)))
    return out


# --------------------------------------------------------------------------
# Seeded slice sampling for the stochastic variant (Algorithm 4)
# --------------------------------------------------------------------------
def splitmix64_next(state: int) -> Tuple[int, int]:
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014).  Returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def sample_count(S: int, frac_den: int = 8) -> int:
    return max(1, S // frac_den)


def sample_slices(S: int, p: int, seed: int, g: int) -> np.ndarray:
    """p distinct slice indices out of S for global sub-step counter g.

    Stream state = seed XOR (g * 0xD1B54A32D192ED03 mod 2^64); a partial
    Fisher-Yates shuffle of 0..S-1 takes swap partner i + (r_i mod (S - i)) for
    the i-th SplitMix64 output r_i; the first p entries, sorted ascending."""
    state = (seed ^ ((g * 0xD1B54A32D192ED03) & MASK64)) & MASK64
    arr = list(range(S))
    for i in range(p):
        state, r = splitmix64_next(state)
        j = i + (r % (S - i))
        arr[i], arr[j] = arr[j], arr[i]
    return np.array(sorted(arr[:p]), dtype=np.int64)


# --------------------------------------------------------------------------
# Time stepping (Algorithm 3 and its Strang / stochastic variants)
# --------------------------------------------------------------------------
def _n_pfactors(scheme: str) -> int:
    return sum(1 for f in scheme_factors(scheme, 1.0) if f[0] == "P")


def expanded_factors(prob, scheme: str, tau: float, nsteps: int, seed: int = 0,
                     step0: int = 0, frac_den: int = 8) -> List[Tuple]:
    """Every factor of nsteps steps in application order.  Potential factors
    carry (layer, duration, slices-or-None)."""
    stoch = scheme.endswith("_stoch")
    base = scheme_factors(scheme, tau)
    npf = _n_pfactors(scheme)
    out = []
    for k in range(nsteps):
        pi = 0
        for f in base:
            if f[0] == "K":
                out.append(("K", f[1]))
                continue
            if f[0] == "C":
                out.append(f)
                continue
            if f[0] == "S":
                rows = cols = None
                if scheme == "random_batch":
                    g = (step0 + k) * 2
                    rows = sample_slices(prob.M2, sample_count(prob.M2, frac_den), seed, g)
                    cols = sample_slices(prob.M1, sample_count(prob.M1, frac_den), seed, g + 1)
                out.append(("S", f[1], rows, cols))
                continue
            layer, s = f[1], f[2]
            if stoch:
                S = n_slices(prob, layer)
                p = sample_count(S, frac_den)
                g = (step0 + k) * npf + pi
                sl = sample_slices(S, p, seed, g)
                out.append(("P", layer, s * S / p, sl))
            else:
                out.append(("P", layer, s, None))
            pi += 1
    return out


def step(prob, phi: np.ndarray, tau: float, scheme: str = "strang", nsteps: int = 1,
         seed: int = 0, step0: int = 0, frac_den: int = 8, project: bool = False) -> np.ndarray:
    """Advance phi (shape (M2, M1), complex128) by nsteps steps of tau.
    project=True zeroes coefficients outside the joint cutoff after each step."""
    if scheme not in SCHEMES:
        raise ValueError(scheme)
    phi = np.array(phi, dtype=np.complex128, copy=True)
    kin = kinetic_energy_diag(prob)
    mask = index_mask(prob) if project else None
    v1 = grid_potential(*layer_grid(prob, 1))
    v2 = grid_potential(*layer_grid(prob, 2))
    per = len(scheme_factors(scheme, tau))
    fl = expanded_factors(prob, scheme, tau, nsteps, seed, step0, frac_den)
    for i, f in enumerate(fl):
        if f[0] == "K":
            phi = apply_K(prob, phi, f[1], kin)
        elif f[0] == "C":
            phi = apply_C(prob, phi, f[1], f[2], kin)
        elif f[0] == "S":
            phi = apply_semi_implicit(prob, phi, f[1], f[2], f[3], kin)
        else:
            phi = apply_P(prob, phi, f[1], f[2], f[3], v1 if f[1] == 1 else v2)
        if project and (i + 1) % per == 0:
            phi = np.where(mask, phi, 0)
    return phi


def settle_noop(phi):
    return phi


# --------------------------------------------------------------------------
# Initial state and observables (Sec. 5 initial state; Eq. (2.4)-(2.5))
# --------------------------------------------------------------------------
def gaussian_packet(prob, x0, w: float, k0) -> np.ndarray:
    """phi = exp(-w^2 |k - k0|^2 / 2) exp(-i k . x0) on the joint mask,
    normalised to unit l2 norm.  With x0 = 0, k0 = 0 this is the paper's
    exp(-gamma |k|^2) initial state with gamma = w^2 / 2 (Sec. 5)."""
    k = wavevectors(prob)
    x0 = np.asarray(x0, dtype=np.float64).reshape(prob.d)
    k0 = np.asarray(k0, dtype=np.float64).reshape(prob.d)
    dk2 = np.sum((k - k0) ** 2, axis=-1)
    kx = np.sum(k * x0, axis=-1)
    phi = np.exp(-0.5 * w * w * dk2) * np.exp(-1j * kx)
    phi = np.where(index_mask(prob), phi, 0)
    return phi / np.linalg.norm(phi)


def observables(prob, phi: np.ndarray, chi: Optional[np.ndarray] = None) -> Dict:
    """Averaged mass and energy (Eq. (2.4)-(2.5)) in the lifted basis, using the
    orthonormality of the lifted plane waves (Eq. (3.2)):

      norm   = sum |phi|^2
      ekin   = sum |k|^2/2 |phi|^2
      epot_j = sum over layer-j slices of (1/M_j) sum_p v_j(x_p) |psi(x_p)|^2,
               psi the slice on layer j's grid (the pseudo-spectral V^j)
      kmean  = sum k |phi|^2
      overlap = sum conj(chi) phi."""
    a2 = np.abs(phi) ** 2
    out = {"norm": float(a2.sum()),
           "ekin": float((kinetic_energy_diag(prob) * a2).sum())}
    epot = []
    for layer in (1, 2):
        h, c, q = layer_grid(prob, layer)
        v = grid_potential(h, c, q)
        psi = _axis_dft(layer_slices(prob, phi, layer), q, inverse=True)
        epot.append(float((np.abs(psi) ** 2 * v[None, :]).sum() / int(np.prod(q))))
    out["epot1"], out["epot2"] = epot
    out["energy"] = out["ekin"] + out["epot1"] + out["epot2"]
    k = wavevectors(prob)
    out["kmean"] = [float((k[..., i] * a2).sum()) for i in range(prob.d)]
    out["overlap"] = complex(np.vdot(chi, phi)) if chi is not None else 0j
    return out


# --------------------------------------------------------------------------
# Adjoint (reverse mode through the unitary factors)
# --------------------------------------------------------------------------
def overlap_loss(chi: np.ndarray, phi: np.ndarray) -> Tuple[float, np.ndarray]:
    """L = |<chi, phi>|^2 and its Wirtinger gradient lambda = dL/d conj(phi) =
    <chi, phi> chi, so that dL = 2 Re <lambda, d phi>."""
    c = np.vdot(chi, phi)
    return float(abs(c) ** 2), c * chi


def adjoint(prob, phi0: np.ndarray, tau: float, scheme: str, nsteps: int,
            lam_T_fn, seed: int = 0, step0: int = 0, frac_den: int = 8):
    """Gradient of a real loss L(phi_T) with respect to the grid potentials
    v_1(x_p), v_2(x_p).  Stores the whole trajectory (plain and memory hungry).

    For a factor phi_out = F^H diag(exp(-i s v)) F phi_in with the unitary
    transform F = W/sqrt(M):  dL/dv_p = 2 s Im(conj(mu_p) psi_p), where
    psi = F phi_out and mu = F lambda_out; lambda_in = U^H lambda_out.

    Returns (loss, phi_T, g1, g2)."""
    kin = kinetic_energy_diag(prob)
    v1 = grid_potential(*layer_grid(prob, 1))
    v2 = grid_potential(*layer_grid(prob, 2))
    fl = expanded_factors(prob, scheme, tau, nsteps, seed, step0, frac_den)
    traj = [np.array(phi0, dtype=np.complex128)]
    phi = traj[0]
    for f in fl:
        if f[0] == "K":
            phi = apply_K(prob, phi, f[1], kin)
        else:
            phi = apply_P(prob, phi, f[1], f[2], f[3], v1 if f[1] == 1 else v2)
        traj.append(phi)
    loss, lam = lam_T_fn(phi)
    g = {j: np.zeros(int(np.prod(layer_grid(prob, j)[2]))) for j in (1, 2)}
    for idx in range(len(fl) - 1, -1, -1):
        f = fl[idx]
        out = traj[idx + 1]
        if f[0] == "K":
            lam = apply_K(prob, lam, -f[1], kin)
            continue
        layer, s, sl = f[1], f[2], f[3]
        q = layer_grid(prob, layer)[2]
        M = int(np.prod(q))
        X_out = layer_slices(prob, out, layer)
        X_lam = layer_slices(prob, lam, layer)
        if sl is not None:
            X_out, X_lam = X_out[sl], X_lam[sl]
        psi = _axis_dft(X_out, q, inverse=True) / math.sqrt(M)
        mu = _axis_dft(X_lam, q, inverse=True) / math.sqrt(M)
        g[layer] += 2.0 * s * np.imag(np.conj(mu) * psi).sum(axis=0)
        lam = apply_P(prob, lam, layer, -s, sl, v1 if layer == 1 else v2)
    return loss, phi, g[1], g[2]


def coefficient_gradient(g: np.ndarray, h: np.ndarray, q: Sequence[int]) -> np.ndarray:
    """Chain rule from grid gradients to coefficient gradients: with
    v_p = Re sum_h c_h e^{2 pi i h.p/q}, dv_p/dRe(c_h) = cos(.), dv_p/dIm(c_h) = -sin(.).
    Returns an array (nh, 2) of (dL/dRe c_h, dL/dIm c_h)."""
    h = np.asarray(h, dtype=np.int64).reshape(-1, len(q))
    P = box_indices([0] * len(q), q)
    out = np.zeros((h.shape[0], 2))
    for t in range(h.shape[0]):
        ph = np.zeros(P.shape[0])
        for i in range(len(q)):
            ph = ph + ((h[t, i] * P[:, i]) % q[i]) / q[i]
        out[t, 0] = float(np.sum(g * np.cos(2 * math.pi * ph)))
        out[t, 1] = float(np.sum(g * -np.sin(2 * math.pi * ph)))
    return out
