"""Seeded synthetic inputs for the layer-split stepper and its oracle.

This module only *describes* problems: lattices, index boxes, the Fourier
coefficients of the layer potentials, time steps and seeds.  It performs none of
the stepping arithmetic, so both the CUDA library (through its Python binding)
and the CPU oracle can take the same problem objects without sharing code.

Model (paper Sec. 2-3): two periodic layers with reciprocal lattices
B_j = 2*pi*A_j^{-T}; the lifted plane-wave coefficient phi[m, n] belongs to the
wavevector k = B1 m + B2 n (Eq. (3.3)); layer potentials are Fourier series
v_j(x) = sum_h vhat_j(h) exp(i G_jh . x) (Eq. (2.2)).

Workloads (the paper has no dataset; its examples are analytic potentials):

* ``bilayer_1d``: periods L1 = 1, L2 = (sqrt5-1)/2, v_j = a_j cos(2 pi x / L_j).
* ``twisted_2d``: two unit square lattices, the second rotated by theta;
  each potential is a sum of periodic Gaussian wells.
* ``bilayer_1d_adjoint``: v_j = sum_{h=1..8} theta_{j,h} cos(2 pi h x / L_j).
* ``batch_1d``: many independent 1D bilayers with uneven boxes.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

GOLDEN = (math.sqrt(5.0) - 1.0) / 2.0


@dataclasses.dataclass
class Problem:
    """One lifted two-layer problem.

    d          -- physical dimension (1 or 2)
    B1, B2     -- (d, d) reciprocal-lattice matrices; k = B1 @ m + B2 @ n
    lo1, q1    -- layer-1 index box: m_i in [lo1[i], lo1[i] + q1[i])
    lo2, q2    -- layer-2 index box
    ecut       -- energy cutoff Ec of the joint mask |k|^2/2 <= Ec
    v1_h, v1_c -- integer reciprocal indices (nv1, d) and complex coefficients
    v2_h, v2_c -- same for layer 2
    """

    d: int
    B1: np.ndarray
    B2: np.ndarray
    lo1: tuple
    q1: tuple
    lo2: tuple
    q2: tuple
    ecut: float
    v1_h: np.ndarray
    v1_c: np.ndarray
    v2_h: np.ndarray
    v2_c: np.ndarray
    name: str = ""
    shared: int = 0   # 1: the second layer-2 component is an index p common to both layers

    @property
    def M1(self) -> int:
        return int(np.prod(self.q1))

    @property
    def M2(self) -> int:
        return int(np.prod(self.q2))

    @property
    def dof(self) -> int:
        return self.M1 * self.M2

    def with_potentials(self, v1_c=None, v2_c=None, v1_h=None, v2_h=None) -> "Problem":
        p = dataclasses.replace(self)
        if v1_h is not None:
            p.v1_h = np.asarray(v1_h, dtype=np.int64).reshape(-1, self.d)
        if v2_h is not None:
            p.v2_h = np.asarray(v2_h, dtype=np.int64).reshape(-1, self.d)
        if v1_c is not None:
            p.v1_c = np.asarray(v1_c, dtype=np.complex128).reshape(-1)
        if v2_c is not None:
            p.v2_c = np.asarray(v2_c, dtype=np.complex128).reshape(-1)
        return p


def _cos_coeffs(amp: float, harmonics: Sequence[int] = (1,)):
    """cos(2 pi h x / L) = (e^{+i G_h x} + e^{-i G_h x}) / 2."""
    hs, cs = [], []
    for h, a in zip(harmonics, np.broadcast_to(amp, (len(harmonics),))):
        hs += [[h], [-h]]
        cs += [a / 2.0, a / 2.0]
    return np.array(hs, dtype=np.int64).reshape(-1, 1), np.array(cs, dtype=np.complex128)


def _box1(n_half: int):
    """Odd box -N..N (length 2N+1); even length 2N is -N..N-1."""
    return (-n_half,), (2 * n_half + 1,)


def bilayer_1d(n1: int, n2: Optional[int] = None, a1: float = 1.0, a2: float = 0.8,
               L1: float = 1.0, L2: float = GOLDEN, ecut: Optional[float] = None,
               name: str = "") -> Problem:
    """1D incommensurate bilayer with v_j = a_j cos(2 pi x / L_j).

    Box |m| <= n1, |n| <= n2.  Default cutoff follows Ec = 200 (n1/32)^2, the
    rule that keeps the 65x65, Ec = 200 strip geometry at larger boxes."""
    n2 = n1 if n2 is None else n2
    if ecut is None:
        ecut = 200.0 * (n1 / 32.0) ** 2
    lo1, q1 = _box1(n1)
    lo2, q2 = _box1(n2)
    h1, c1 = _cos_coeffs(a1)
    h2, c2 = _cos_coeffs(a2)
    return Problem(1, np.array([[2 * math.pi / L1]]), np.array([[2 * math.pi / L2]]),
                   lo1, q1, lo2, q2, float(ecut), h1, c1, h2, c2, name)


def config_small_1d() -> Problem:
    """65x65 lifted box, L2 = (sqrt5-1)/2, a = (1.0, 0.8), Ec = 200."""
    return bilayer_1d(32, 32, 1.0, 0.8, ecut=200.0, name="bilayer1d-65x65")


def config_scale_1d(seed: int = 2) -> Problem:
    """2049x2049 lifted box, a_j ~ U(0.5, 2) drawn from ``seed``."""
    rng = np.random.default_rng(seed)
    a1, a2 = rng.uniform(0.5, 2.0, size=2)
    return bilayer_1d(1024, 1024, float(a1), float(a2), name="bilayer1d-2049x2049")


def rotation(theta: float) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, -s], [s, c]])


def gaussian_wells_coeffs(seed: int, n_wells: int = 3, sigma: float = 0.15,
                          hmax: int = 8, depth=(1.0, 3.0)):
    """Fourier coefficients of v(x) = -sum_g d_g sum_R exp(-|x - c_g - R|^2 / (2 sigma^2))
    on a unit square lattice, in fractional coordinates (so they hold for any
    orthogonal A_j).  vhat_h = -sum_g d_g 2 pi sigma^2 exp(-sigma^2 |G_h|^2/2) e^{-i G_h.c_g}
    with G_h = 2 pi h and |Gamma| = 1; truncated to |h_i| <= hmax."""
    rng = np.random.default_rng(seed)
    d_g = rng.uniform(depth[0], depth[1], size=n_wells)
    c_g = rng.uniform(0.0, 1.0, size=(n_wells, 2))
    hs, cs = [], []
    for h1 in range(-hmax, hmax + 1):
        for h2 in range(-hmax, hmax + 1):
            G2 = (2 * math.pi) ** 2 * (h1 * h1 + h2 * h2)
            val = 0j
            for g in range(n_wells):
                ph = 2 * math.pi * (h1 * c_g[g, 0] + h2 * c_g[g, 1])
                val += -d_g[g] * 2 * math.pi * sigma ** 2 * math.exp(-sigma ** 2 * G2 / 2) \
                    * complex(math.cos(ph), -math.sin(ph))
            hs.append([h1, h2])
            cs.append(val)
    return np.array(hs, dtype=np.int64), np.array(cs, dtype=np.complex128)


def twisted_2d(q: int = 64, theta_deg: float = 5.0, ecut: float = 200.0,
               seeds=(31, 32), hmax: int = 8, name: str = "") -> Problem:
    """Two unit square lattices, layer 2 rotated by theta: B1 = 2 pi I,
    B2 = 2 pi R(theta) (A2 = R(theta) is orthogonal so A2^{-T} = R(theta))."""
    lo = -(q // 2)
    h1, c1 = gaussian_wells_coeffs(seeds[0], hmax=hmax)
    h2, c2 = gaussian_wells_coeffs(seeds[1], hmax=hmax)
    B1 = 2 * math.pi * np.eye(2)
    B2 = 2 * math.pi * rotation(math.radians(theta_deg))
    return Problem(2, B1, B2, (lo, lo), (q, q), (lo, lo), (q, q), float(ecut),
                   h1, c1, h2, c2, name or f"twisted2d-{q}^4")


def config_adjoint_1d(seed: int = 5, n_half: int = 256, n_params: int = 8):
    """513x513 box; v_j = sum_{h=1..8} theta_{j,h} cos(2 pi h x / L_j) with
    theta ~ N(0, 0.5) drawn from ``seed``.  Returns (problem, theta1, theta2)."""
    rng = np.random.default_rng(seed)
    th = rng.normal(0.0, 0.5, size=(2, n_params))
    p = bilayer_1d(n_half, n_half, name=f"bilayer1d-adjoint-{2 * n_half + 1}")
    hs = list(range(1, n_params + 1))
    h1, c1 = _cos_coeffs(th[0], hs)
    h2, c2 = _cos_coeffs(th[1], hs)
    return p.with_potentials(c1, c2, h1, h2), th[0].copy(), th[1].copy()


def example3(n1: int = 8, n2: int = 8, n3: int = 4, s1: float = 1.0, s2: float = 2.0,
             beta: float = GOLDEN, ecut: float = 100.0, name: str = "") -> Problem:
    """Example 3 of Sec. 5: a 2D system periodic in y and incommensurate in x,
    H = -Laplacian/2 + s1 cos^2(beta x) cos^2(pi y / 2) + s2 cos^2(x) cos^2(pi y / 2).
    Layer j is periodic in x with period pi / beta_j (beta_1 = beta, beta_2 = 1),
    so G_j = 2 beta_j; both share the y period 2, G3 = pi.  With cos^2 = (1 + cos)/2
    the coefficients of s_j cos^2(beta_j x) cos^2(pi y / 2) on the harmonics
    (h_x, h_y) are s_j/4 (0, 0), s_j/8 (+-1, 0) and (0, +-1), s_j/16 (+-1, +-1).
    Three-index lift (m, n, p): stored as a 2D problem with the shared index p
    as the second layer-2 component; box m in [-n1, n1), n in [-n2, n2),
    p in [-n3, n3) (even lengths)."""
    def coeffs(s):
        hs, cs = [], []
        for hx in (-1, 0, 1):
            for hy in (-1, 0, 1):
                hs.append([hx, hy])
                cs.append(s / 4.0 * (0.5 if hx else 1.0) * (0.5 if hy else 1.0))
        return np.array(hs, dtype=np.int64), np.array(cs, dtype=np.complex128)
    h1, c1 = coeffs(s1)
    h2, c2 = coeffs(s2)
    B1 = np.array([[2.0 * beta, 0.0], [0.0, 0.0]])
    B2 = np.array([[2.0, 0.0], [0.0, math.pi]])
    return Problem(2, B1, B2, (-n1, 0), (2 * n1, 1), (-n2, -n3), (2 * n2, 2 * n3), float(ecut), h1, c1, h2, c2,
                   name or f"example3-{2 * n1}x{2 * n2}x{2 * n3}", shared=1)


def trilayer_1d(n1: int = 8, n2: int = 8, n3: int = 4, a1: float = 1.0, a2: float = 0.8, a3: float = 0.6,
                L1: float = 1.0, L2: float = GOLDEN, L3: float = math.sqrt(2.0) / 2.0, ecut: float = 1e9,
                name: str = "") -> Problem:
    """Three incommensurate 1D layers, v_j = a_j cos(2 pi x / L_j), lifted to
    three indices (m, n, p) with k = b1 m + b2 n + b3 p, b_j = 2 pi / L_j.
    V1 acts along m, V2 along n, V3 along p, and V1, V3 act on different
    indices, so exp(-i s (V1 + V3)) = exp(-i s V1) exp(-i s V3) exactly.  The
    problem is stored as a shared-index problem: layer "1" on the (m, p) planes
    carries V1 on the first harmonic component and V3 on the second, layer "2"
    on the (n, p) planes carries V2; the wavevector is the 2-vector (k, 0), so
    B1 = [[b1, 0], [0, 0]] and B2 = [[b2, b3], [0, 0]].  Boxes m in [-n1, n1),
    n in [-n2, n2), p in [-n3, n3) (even lengths)."""
    b1, b2, b3 = (2.0 * math.pi / L for L in (L1, L2, L3))
    h1 = np.array([[1, 0], [-1, 0], [0, 1], [0, -1]], dtype=np.int64)
    c1 = np.array([a1 / 2, a1 / 2, a3 / 2, a3 / 2], dtype=np.complex128)
    h2 = np.array([[1, 0], [-1, 0]], dtype=np.int64)
    c2 = np.array([a2 / 2, a2 / 2], dtype=np.complex128)
    B1 = np.array([[b1, 0.0], [0.0, 0.0]])
    B2 = np.array([[b2, b3], [0.0, 0.0]])
    return Problem(2, B1, B2, (-n1, 0), (2 * n1, 1), (-n2, -n3), (2 * n2, 2 * n3), float(ecut), h1, c1, h2, c2,
                   name or f"trilayer1d-{2 * n1}x{2 * n2}x{2 * n3}", shared=1)


def cos_series_coeffs(theta: np.ndarray):
    """Coefficient list of sum_{h>=1} theta_h cos(2 pi h x / L)."""
    hs = list(range(1, len(theta) + 1))
    return _cos_coeffs(np.asarray(theta, dtype=np.float64), hs)


def batch_1d(count: int = 256, seed: int = 4, nmin: int = 16, nmax: int = 512) -> List[Problem]:
    """Independent 1D bilayers: L2 ~ U(0.3, 0.9), N1, N2 ~ U{nmin..nmax},
    a_j ~ U(0.5, 2), drawn from ``seed``."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        L2 = float(rng.uniform(0.3, 0.9))
        n1, n2 = (int(x) for x in rng.integers(nmin, nmax + 1, size=2))
        a1, a2 = (float(x) for x in rng.uniform(0.5, 2.0, size=2))
        out.append(bilayer_1d(n1, n2, a1, a2, L2=L2, name=f"batch{i}"))
    return out


def random_state(shape, seed: int, decay: Optional[np.ndarray] = None) -> np.ndarray:
    """Seeded complex128 array with N(0,1) real and imaginary parts, optionally
    multiplied by a decay envelope; normalised to unit l2 norm."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    if decay is not None:
        z = z * decay
    return z / np.linalg.norm(z)
