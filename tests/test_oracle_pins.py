"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formulas: each compares it with an
independent construction (dense Hamiltonians built from Fourier coefficients,
closed forms, a supercell solve, a textbook split-step per Bloch slice,
library FFTs, high-precision arithmetic, published generator values).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def small_1d(n1=4, n2=3, a1=3.0, a2=2.0, L1=5.0, ratio=W.GOLDEN):
    return W.bilayer_1d(n1, n2, a1, a2, L1=L1, L2=L1 * ratio, ecut=1e9)


def circulant_from_coeffs(h, c, q):
    """C[m, m'] = sum_{h = m - m' mod q} vhat_h, built straight from the Fourier
    coefficients (the Galerkin V^j of Eq. (3.6) with periodic wrap)."""
    C = np.zeros((q, q), dtype=np.complex128)
    for hh, cc in zip(np.asarray(h).reshape(-1), c):
        for m in range(q):
            C[m, (m - hh) % q] += cc
    return C


def dense_H_1d(prob):
    """H = D + I (x) C1 + C2 (x) I (Eq. (3.4)-(3.7)) with [n][m] ordering."""
    m = np.arange(prob.q1[0]) + prob.lo1[0]
    n = np.arange(prob.q2[0]) + prob.lo2[0]
    b1, b2 = prob.B1[0, 0], prob.B2[0, 0]
    k = b1 * m[None, :] + b2 * n[:, None]
    D = np.diag(0.5 * (k ** 2).reshape(-1))
    C1 = circulant_from_coeffs(prob.v1_h, prob.v1_c, prob.q1[0])
    C2 = circulant_from_coeffs(prob.v2_h, prob.v2_c, prob.q2[0])
    return D + np.kron(np.eye(prob.q2[0]), C1) + np.kron(C2, np.eye(prob.q1[0]))


def expm_herm(H, t):
    w, V = np.linalg.eigh(H)
    return (V * np.exp(-1j * t * w)) @ V.conj().T


def rand_state(prob, seed=0):
    return W.random_state((prob.M2, prob.M1), seed)


# ---------------------------------------------------------------- transforms
def test_dft_matrix_against_numpy_fft_and_unitarity():
    for q in (1, 2, 7, 64, 65, 129):
        Wm = O.dft_matrix(q)
        x = np.random.default_rng(q).standard_normal(q) + 0j
        # W maps coefficients to grid values: q * ifft (positive exponent).
        np.testing.assert_allclose(x @ Wm, q * np.fft.ifft(x), atol=1e-11 * q)
        # Appendix B normalisation: forward = conj(W)/q inverts it exactly.
        np.testing.assert_allclose(Wm.conj() @ Wm / q, np.eye(q), atol=1e-12)


def test_grid_potential_closed_form_cos():
    h, c = W._cos_coeffs(1.7)
    q = 65
    v = O.grid_potential(h, c, (q,))
    np.testing.assert_allclose(v, 1.7 * np.cos(2 * np.pi * np.arange(q) / q), atol=1e-14)


def test_2d_separable_transform_equals_kronecker_matrix():
    q = (4, 3)
    x = np.random.default_rng(1).standard_normal((5, 12)) + 1j
    K2 = np.kron(O.dft_matrix(q[1]), O.dft_matrix(q[0]))
    np.testing.assert_allclose(O.lsplit._axis_dft(x, q, True), x @ K2, atol=1e-12)
    np.testing.assert_allclose(O.lsplit._axis_dft(x @ K2, q, False), x, atol=1e-12)


# ---------------------------------------------------------------- closed forms
UNITARY_EXP = [s for s in O.SCHEMES if s not in ("cn_strang", "semi_implicit", "random_batch")]


@pytest.mark.parametrize("scheme", UNITARY_EXP)
def test_free_particle_exact_phase(scheme):
    """V = 0: every exponential scheme is exact, phi(T) = exp(-i T |k|^2 / 2)
    phi0 (the Crank-Nicolson split has its own closed form, below)."""
    p = W.bilayer_1d(6, 5, 0.0, 0.0, ecut=1e9)
    phi0 = rand_state(p, 3)
    tau, n = 0.013, 7
    out = O.step(p, phi0, tau, scheme, n, seed=5)
    m = np.arange(-6, 7)
    nn = np.arange(-5, 6)
    k = 2 * np.pi * m[None, :] + 2 * np.pi / W.GOLDEN * nn[:, None]
    np.testing.assert_allclose(out, np.exp(-0.5j * n * tau * k ** 2) * phi0, atol=1e-12)


def test_free_particle_large_k_argument():
    """Large tau|k|^2 (reduction of the phase argument): 2049-box kinetic extremes."""
    p = W.bilayer_1d(1024, 2, 0.0, 0.0, ecut=1e12)
    phi0 = rand_state(p, 4)
    out = O.step(p, phi0, 5e-4, "strang", 1)
    m = np.arange(-1024, 1025)
    nn = np.arange(-2, 3)
    k = 2 * np.pi * m[None, :] + 2 * np.pi / W.GOLDEN * nn[:, None]
    np.testing.assert_allclose(out, np.exp(-0.5j * 5e-4 * k ** 2) * phi0, atol=1e-10)


def test_constant_potential_is_global_phase():
    """v_j = const c_j: each P_j(s) = exp(-i s c_j) I (checks the 1/M of the
    forward transform and the sign of the exponent)."""
    p = W.bilayer_1d(5, 4, 0.0, 0.0, ecut=1e9).with_potentials(
        v1_h=[[0]], v1_c=[0.7], v2_h=[[0]], v2_c=[-0.3])
    phi0 = rand_state(p, 5)
    for scheme in ("lie", "strang", "strang_kp"):
        out = O.step(p, phi0, 0.02, scheme, 3)
        free = O.step(W.bilayer_1d(5, 4, 0.0, 0.0, ecut=1e9), phi0, 0.02, scheme, 3)
        np.testing.assert_allclose(out, np.exp(-1j * 0.06 * (0.7 - 0.3)) * free, atol=1e-13)


# ---------------------------------------------------------------- conservation
@pytest.mark.parametrize("scheme", [s for s in O.SCHEMES if s not in ("semi_implicit", "random_batch")])
def test_mass_conservation(scheme):
    """Theorem 4.6: the Fourier splitting conserves sum |phi|^2 exactly."""
    p = W.bilayer_1d(8, 7, 1.3, 0.9, ecut=1e9)
    phi0 = rand_state(p, 6)
    out = O.step(p, phi0, 0.01, scheme, 20, seed=11)
    assert abs(np.linalg.norm(out) - 1.0) < 1e-13


def test_layer_factors_commute():
    """Kronecker structure (Eq. (3.7)): P1(s) P2(t) = P2(t) P1(s)."""
    p = W.bilayer_1d(6, 5, 1.3, 0.9, ecut=1e9)
    x = rand_state(p, 7)
    a = O.apply_P(p, O.apply_P(p, x, 1, 0.3), 2, 0.2)
    b = O.apply_P(p, O.apply_P(p, x, 2, 0.2), 1, 0.3)
    np.testing.assert_allclose(a, b, atol=1e-13)


def test_yoshida_weights_conditions():
    """The composition keeps the total time (2 w1 + w0 = 1) and cancels the
    third-order term (2 w1^3 + w0^3 = 0); the middle step runs backward."""
    w1, w0 = O.yoshida_weights()
    assert abs(2 * w1 + w0 - 1) < 1e-15
    assert abs(2 * w1 ** 3 + w0 ** 3) < 1e-14
    assert w0 < 0 < w1
    f = O.scheme_factors("yoshida4", 0.3)
    assert abs(sum(x[1] for x in f if x[0] == "K") - 0.3) < 1e-15
    assert abs(sum(x[2] for x in f if x[0] == "P" and x[1] == 2) - 0.3) < 1e-15


def test_yoshida_time_reversible():
    p = W.bilayer_1d(6, 5, 1.3, 0.9, ecut=1e9)
    x = rand_state(p, 8)
    y = O.step(p, O.step(p, x, 0.01, "yoshida4", 3), -0.01, "yoshida4", 3)
    np.testing.assert_allclose(y, x, atol=1e-13)


def test_strang_time_reversible():
    p = W.bilayer_1d(6, 5, 1.3, 0.9, ecut=1e9)
    x = rand_state(p, 8)
    y = O.step(p, O.step(p, x, 0.01, "strang", 5), -0.01, "strang", 5)
    np.testing.assert_allclose(y, x, atol=1e-13)


# ---------------------------------------------------------------- dense exponential
def _errors(prob, scheme, T, ns, phi0, exact):
    return [np.linalg.norm(O.step(prob, phi0, T / n, scheme, n) - exact) for n in ns]


@pytest.mark.parametrize("scheme,order", [("lie", 1), ("strang", 2), ("strang_kp", 2), ("yoshida4", 4)])
def test_convergence_order_against_dense_exponential(scheme, order):
    """Theorem 4.5 (order 1 for the Lie form of Algorithm 3), Strang order 2
    (Appendix A) and order 4 for the Yoshida composition of Strang steps (the
    higher-order splittings of Sec. 4.2 and Appendix A), against exp(-i T H)
    of the dense lifted H from coefficients."""
    p = small_1d()
    H = dense_H_1d(p)
    phi0 = rand_state(p, 9)
    T = 0.2
    exact = (expm_herm(H, T) @ phi0.reshape(-1)).reshape(phi0.shape)
    ns = [16, 32, 64, 128]
    err = _errors(p, scheme, T, ns, phi0, exact)
    slope = np.polyfit(np.log([T / n for n in ns]), np.log(err), 1)[0]
    assert abs(slope - order) < 0.1, (scheme, slope, err)
    assert err[-1] < {1: 1e-2, 2: 1e-4, 4: 1e-7}[order]


def test_one_step_equals_dense_factor_product():
    """One step equals the product of exact dense exponentials of D, V^1, V^2
    (Eq. (4.8) sub-problems) in the order Algorithm 3 fixes (K, then V^1, then
    V^2) for the Lie form, and in the Strang compositions of Appendix A."""
    p = small_1d()
    M1, M2 = p.q1[0], p.q2[0]
    H = dense_H_1d(p)
    Dm = np.diag(np.diag(H).real - np.diag(np.kron(np.eye(M2), circulant_from_coeffs(p.v1_h, p.v1_c, M1))).real
                 - np.diag(np.kron(circulant_from_coeffs(p.v2_h, p.v2_c, M2), np.eye(M1))).real)
    V1 = np.kron(np.eye(M2), circulant_from_coeffs(p.v1_h, p.v1_c, M1))
    V2 = np.kron(circulant_from_coeffs(p.v2_h, p.v2_c, M2), np.eye(M1))
    E = lambda A, t: expm_herm(A, t)
    t = 0.03
    ref = {
        "lie": E(V2, t) @ E(V1, t) @ E(Dm, t),
        "strang": (E(Dm, t / 8) @ E(V1, t / 2) @ E(Dm, t / 8)) @ (E(Dm, t / 4) @ E(V2, t) @ E(Dm, t / 4))
                  @ (E(Dm, t / 8) @ E(V1, t / 2) @ E(Dm, t / 8)),
        "strang_kp": E(Dm, t / 2) @ E(V2, t) @ E(V1, t) @ E(Dm, t / 2),
    }
    x = rand_state(p, 30)
    for scheme, U in ref.items():
        out = O.step(p, x, t, scheme, 1)
        np.testing.assert_allclose(out.reshape(-1), U @ x.reshape(-1), atol=1e-12, err_msg=scheme)


def test_stochastic_converges_in_mean_structure():
    """Full sampling (p = S) reproduces the deterministic scheme exactly."""
    p = W.bilayer_1d(6, 5, 1.3, 0.9, ecut=1e9)
    x = rand_state(p, 10)
    for base in ("lie", "strang"):
        a = O.step(p, x, 0.01, base + "_stoch", 4, seed=3, frac_den=1)
        b = O.step(p, x, 0.01, base, 4)
        np.testing.assert_allclose(a, b, atol=1e-14)


def test_stochastic_sampled_factor_matches_dense():
    """One stochastic potential factor equals the dense exp(-i s S/p C1) on the
    sampled rows and the identity elsewhere."""
    p = W.bilayer_1d(6, 5, 1.3, 0.9, ecut=1e9)
    x = rand_state(p, 12)
    sl = np.array([1, 4, 7])
    y = O.apply_P(p, x, 1, 0.37, sl)
    C1 = circulant_from_coeffs(p.v1_h, p.v1_c, p.q1[0])
    U = expm_herm(C1, 0.37)
    ref = x.copy()
    ref[sl] = (U @ x[sl].T).T
    np.testing.assert_allclose(y, ref, atol=1e-13)


def _dense_stochastic_steps(p, x, tau, scheme, nsteps, seed, step0, frac_den):
    """Dense stand-in for the stochastic schemes: every potential factor of
    duration s is exp(-i s (S/p) C_j) (C_j the circulant built from the Fourier
    coefficients) on the p sampled slices and the identity on the others
    (Algorithm 4: the sampled part is amplified by |I|/p), the kinetic factors
    exp(-i s |k|^2/2) act on every element; Strang or Lie order."""
    m = np.arange(p.q1[0]) + p.lo1[0]
    n = np.arange(p.q2[0]) + p.lo2[0]
    k = p.B1[0, 0] * m[None, :] + p.B2[0, 0] * n[:, None]
    kin = 0.5 * k ** 2
    C = {1: circulant_from_coeffs(p.v1_h, p.v1_c, p.q1[0]), 2: circulant_from_coeffs(p.v2_h, p.v2_c, p.q2[0])}
    if scheme == "strang_stoch":
        seq = []
        for j, s in ((1, tau / 2), (2, tau), (1, tau / 2)):
            seq += [("K", s / 4), ("P", j, s), ("K", s / 4)]
    else:
        seq = [("K", tau), ("P", 1, tau), ("P", 2, tau)]
    y = np.array(x, dtype=np.complex128)
    for st in range(nsteps):
        pi = 0
        for f in seq:
            if f[0] == "K":
                y = y * np.exp(-1j * f[1] * kin)
                continue
            j, s = f[1], f[2]
            S = p.M2 if j == 1 else p.M1
            cnt = max(1, S // frac_den)
            sl = O.sample_slices(S, cnt, seed, (step0 + st) * (3 if scheme == "strang_stoch" else 2) + pi)
            U = expm_herm(C[j], s * S / cnt)
            if j == 1:
                y[sl] = (U @ y[sl].T).T
            else:
                y[:, sl] = U @ y[:, sl]
            pi += 1
    return y


@pytest.mark.parametrize("scheme", ["strang_stoch", "lie_stoch"])
def test_stochastic_steps_match_dense_sampled_factors(scheme):
    """p < S (frac_den = 3, so S/p = 11/3 and 13/4): the oracle's stochastic
    steps equal the dense construction above, which fixes the duration scale
    S/p of the sampled factors and the sub-step numbering of the samples."""
    p = W.bilayer_1d(6, 5, 1.3, 0.9, ecut=1e9)
    x = rand_state(p, 31)
    for nsteps, step0 in ((1, 0), (2, 3)):
        got = O.step(p, x, 0.02, scheme, nsteps, seed=9, step0=step0, frac_den=3)
        ref = _dense_stochastic_steps(p, x, 0.02, scheme, nsteps, 9, step0, 3)
        np.testing.assert_allclose(got, ref, atol=1e-12)


# ---------------------------------------------------------------- physics pins
def test_commensurate_fiber_sum_matches_supercell():
    """L2 = 2/3: k = pi (2m + 3n).  The fiber sum c_j = sum_{2m+3n=j} phi_mn of
    the lifted Strang solution equals a period-2 supercell split-step solve
    with the same factor sequence (textbook FFT split step)."""
    a1, a2 = 1.1, 0.7
    N = 14
    p = W.bilayer_1d(N, N, a1, a2, L1=1.0, L2=2.0 / 3.0, ecut=1e9)
    m = np.arange(-N, N + 1)
    n = np.arange(-N, N + 1)
    phi0 = np.exp(-0.35 * (m[None, :] ** 2 + n[:, None] ** 2)) * (1 + 0.3j * m[None, :])
    tau, nsteps = 0.01, 10
    lifted = O.step(p, phi0, tau, "strang", nsteps)
    J = 256
    j = np.fft.fftfreq(J, 1.0 / J).astype(int)          # plane waves e^{i pi j x}
    c = np.zeros(J, dtype=np.complex128)
    for ii, mm in enumerate(m):
        for jj, nn in enumerate(n):
            c[(2 * mm + 3 * nn) % J] += phi0[jj, ii]
    x = 2.0 * np.arange(J) / J
    v1 = a1 * np.cos(2 * np.pi * x)
    v2 = a2 * np.cos(2 * np.pi * x / (2.0 / 3.0))
    kin = 0.5 * (np.pi * j) ** 2

    def K(c, s):
        return c * np.exp(-1j * s * kin)

    def P(c, v, s):
        return np.fft.fft(np.fft.ifft(c) * np.exp(-1j * s * v))

    for _ in range(nsteps):
        for s, v in ((tau / 2, v1), (tau, v2), (tau / 2, v1)):
            c = K(P(K(c, s / 4), v, s), s / 4)
    cl = np.zeros(J, dtype=np.complex128)
    for ii, mm in enumerate(m):
        for jj, nn in enumerate(n):
            cl[(2 * mm + 3 * nn) % J] += lifted[jj, ii]
    np.testing.assert_allclose(cl, c, atol=1e-10)


def test_single_layer_reduces_to_bloch_split_step():
    """a2 = 0: each layer-1 slice n is a periodic problem at quasi-momentum
    kappa = B2 n, advanced by the textbook split-step Fourier method."""
    p = W.bilayer_1d(10, 4, 1.5, 0.0, ecut=1e9)
    x = rand_state(p, 13)
    tau, nsteps = 0.004, 6
    out = O.step(p, x, tau, "strang", nsteps)
    b1, b2 = 2 * np.pi, 2 * np.pi / W.GOLDEN
    Q = 21
    mm = np.arange(-10, 11)
    grid = np.arange(Q) / Q
    v = 1.5 * np.cos(2 * np.pi * grid)
    for r, nn in enumerate(range(-4, 5)):
        u = x[r].copy()
        kin = 0.5 * (b1 * mm + b2 * nn) ** 2
        # fft ordering: slice index i <-> m = i - 10; a shift is a real-space
        # modulation that commutes with the potential multiplication.
        for _ in range(nsteps):
            for s, pot in ((tau / 2, True), (tau, False), (tau / 2, True)):
                u = u * np.exp(-1j * s / 4 * kin)
                if pot:
                    u = np.fft.fft(np.fft.ifft(u) * np.exp(-1j * s * v))
                u = u * np.exp(-1j * s / 4 * kin)
        np.testing.assert_allclose(out[r], u, atol=1e-12)


# ---------------------------------------------------------------- observables
def test_observables_against_dense_quadratic_forms():
    p = W.bilayer_1d(5, 4, 1.3, 0.9, ecut=1e9)
    x = rand_state(p, 14)
    H = dense_H_1d(p)
    o = O.observables(p, x, chi=rand_state(p, 15))
    v = x.reshape(-1)
    assert abs(o["norm"] - 1.0) < 1e-14
    assert abs(o["energy"] - np.vdot(v, H @ v).real) < 1e-10
    m = np.arange(-5, 6)
    nn = np.arange(-4, 5)
    k = 2 * np.pi * m[None, :] + 2 * np.pi / W.GOLDEN * nn[:, None]
    assert abs(o["kmean"][0] - float((k * np.abs(x) ** 2).sum())) < 1e-11
    assert abs(o["overlap"] - np.vdot(rand_state(p, 15), x)) < 1e-14


def test_strang_energy_error_second_order():
    """Energy is not conserved exactly by the splitting, but its error after a
    fixed time shrinks like tau^2 (Strang, Appendix A)."""
    p = W.bilayer_1d(8, 8, 1.0, 0.8, ecut=200.0 * (8 / 32) ** 2 * 16)
    x = O.gaussian_packet(p, [0.0], 2.0, [1.0])
    e0 = O.observables(p, x)["energy"]
    d = [abs(O.observables(p, O.step(p, x, 0.1 / n, "strang", n))["energy"] - e0)
         for n in (50, 100)]
    assert d[0] < 1e-3 and 3.0 < d[0] / d[1] < 5.0, d


# ---------------------------------------------------------------- initial state
def test_gaussian_packet_reduces_to_paper_initial_state():
    """x0 = 0, k0 = 0: phi = exp(-gamma |k|^2) with gamma = w^2/2 (Sec. 5)."""
    p = W.config_small_1d()
    w = 2.0
    phi = O.gaussian_packet(p, [0.0], w, [0.0])
    m = np.arange(-32, 33)
    nn = np.arange(-32, 33)
    k = 2 * np.pi * m[None, :] + 2 * np.pi / W.GOLDEN * nn[:, None]
    ref = np.exp(-(w * w / 2) * k ** 2) * (0.5 * k ** 2 <= 200.0)
    np.testing.assert_allclose(phi, ref / np.linalg.norm(ref), atol=1e-15)


def test_gaussian_packet_position_and_momentum():
    """The packet in real space, through its plane-wave expansion (Sec. 3):
    every amplitude exp(-w^2 |k - k0|^2 / 2) is positive, so |psi(x)| <= sum |phi|
    with equality exactly at x = x0 (triangle inequality); moving the centre is
    a translation, psi_{x0}(x) = psi_0(x - x0); and the phase of psi advances at
    the mean momentum, close to k0, around x0."""
    p = W.config_small_1d()
    for x0, k0 in ((0.7, 1.0), (-1.3, -2.0)):
        phi = O.lsplit.gaussian_packet(p, [x0], 2.0, [k0])
        top = float(np.abs(phi).sum())
        xs = x0 + np.linspace(-3.0, 3.0, 61)
        d = np.abs(O.lsplit.density_on_line(p, phi, xs))
        assert abs(d[30] - top) < 1e-12 * top
        assert np.all(np.delete(d, 30) < top * (1 - 1e-6))
        np.testing.assert_allclose(O.lsplit.density_on_line(p, phi, xs),
                                   O.lsplit.density_on_line(p, O.lsplit.gaussian_packet(p, [0.0], 2.0, [k0]), xs - x0),
                                   atol=1e-10)
        e = O.lsplit.density_on_line(p, phi, [x0 - 1e-3, x0 + 1e-3])
        slope = float(np.angle(e[1] / e[0])) / 2e-3
        assert abs(slope - k0) < 0.03 * max(1.0, abs(k0)), (slope, k0)
    # 2D: the same peak and translation identities in the plane
    q = W.twisted_2d(q=8, ecut=30.0)
    x0 = np.array([0.1, -0.2])
    phi = O.lsplit.gaussian_packet(q, x0, 2.0, [1.0, 0.0])
    rng = np.random.default_rng(3)
    pts = np.concatenate([x0[None, :], x0 + rng.uniform(-2, 2, size=(40, 2))])
    d = np.abs(O.lsplit.density_on_line(q, phi, pts))
    assert abs(d[0] - np.abs(phi).sum()) < 1e-12 * d[0] and np.all(d[1:] < d[0])
    np.testing.assert_allclose(O.lsplit.density_on_line(q, phi, pts),
                               O.lsplit.density_on_line(q, O.lsplit.gaussian_packet(q, [0.0, 0.0], 2.0, [1.0, 0.0]), pts - x0),
                               atol=1e-10)


# ---------------------------------------------------------------- index set
def _exact_mask_mp(prob, idx):
    import mpmath as mp
    mp.mp.dps = 60
    b1 = 2 * mp.pi / mp.mpf(1)
    b2 = 2 * mp.pi / ((mp.sqrt(5) - 1) / 2)
    out, margin = [], mp.inf
    for (n, m) in idx:
        e = (b1 * m + b2 * n) ** 2 / 2
        out.append(e <= prob.ecut)
        margin = min(margin, abs(e - prob.ecut) / prob.ecut)
    return np.array(out), float(margin)


@pytest.mark.parametrize("cfg", ["small", "scale"])
def test_index_mask_matches_exact_predicate(cfg):
    """The FP64 joint-cutoff mask equals the exact real predicate with the true
    lattice L2 = (sqrt5 - 1)/2, with a certified relative margin (Sec. 3)."""
    pytest.importorskip("mpmath")
    p = W.config_small_1d() if cfg == "small" else W.config_scale_1d()
    mask = O.index_mask(p)
    e = O.kinetic_energy_diag(p)
    near = np.argwhere(np.abs(e - p.ecut) < 2e-3 * p.ecut)
    rows = near[:, 0] + p.lo2[0]
    cols = near[:, 1] + p.lo1[0]
    ex, margin = _exact_mask_mp(p, list(zip(rows, cols)))
    assert np.array_equal(ex, mask[near[:, 0], near[:, 1]])
    assert margin > 1e-9
    if cfg == "small":
        # Every element of the box, not just the near-boundary ones.
        allidx = [(n, m) for n in range(-32, 33) for m in range(-32, 33)]
        ex_all, _ = _exact_mask_mp(p, allidx)
        assert np.array_equal(ex_all.reshape(65, 65), mask)


# ---------------------------------------------------------------- sampling
def test_splitmix64_known_answers():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            vals = [int(t) for t in line.split()]
            s = vals[0]
            for want in vals[1:]:
                s, r = O.splitmix64_next(s)
                assert r == want


def test_sample_slices_properties():
    for S, p, seed, g in [(2049, 256, 7, 0), (2049, 256, 7, 1), (65, 8, 1, 5), (10, 10, 0, 0)]:
        s = O.sample_slices(S, p, seed, g)
        assert len(s) == p and len(set(s.tolist())) == p
        assert np.all(np.diff(s) > 0) and s[0] >= 0 and s[-1] < S
    assert not np.array_equal(O.sample_slices(2049, 256, 7, 0), O.sample_slices(2049, 256, 7, 1))
    # Uniformity: each slice is chosen with probability p/S.
    cnt = np.zeros(40)
    for g in range(4000):
        cnt[O.sample_slices(40, 5, 3, g)] += 1
    assert np.all(np.abs(cnt / 4000 - 5 / 40) < 0.03)


# ---------------------------------------------------------------- adjoint
def test_adjoint_matches_central_differences():
    th1 = np.array([0.6, -0.3, 0.2])
    th2 = np.array([0.4, 0.25])
    base = W.bilayer_1d(6, 5, 0.0, 0.0, ecut=1e9)

    def prob(t1, t2):
        h1, c1 = W.cos_series_coeffs(t1)
        h2, c2 = W.cos_series_coeffs(t2)
        return base.with_potentials(c1, c2, h1, h2)

    phi0 = O.gaussian_packet(base, [0.0], 0.8, [1.0])
    chi = O.gaussian_packet(base, [0.3], 0.8, [1.2])
    tau, n = 0.02, 6
    lossfn = lambda phi: O.overlap_loss(chi, phi)
    for scheme in ("strang", "lie"):
        L, _, g1, g2 = O.adjoint(prob(th1, th2), phi0, tau, scheme, n, lossfn)
        cg1 = O.coefficient_gradient(g1, np.array([[h] for h in (1, -1, 2, -2, 3, -3)]), (13,))
        # d/dtheta_h of theta_h cos = chain through the +h and -h halves (each /2).
        grad = [0.5 * (cg1[2 * i, 0] + cg1[2 * i + 1, 0]) for i in range(3)]
        h = 1e-4
        for i in range(3):
            tp, tm = th1.copy(), th1.copy()
            tp[i] += h
            tm[i] -= h
            Lp = lossfn(O.step(prob(tp, th2), phi0, tau, scheme, n))[0]
            Lm = lossfn(O.step(prob(tm, th2), phi0, tau, scheme, n))[0]
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - grad[i]) < 1e-7 * max(1.0, abs(fd)) + 1e-9, (scheme, i, fd, grad[i])
        # Layer 2, grid gradient direct: perturb v2 by a single cosine mode.
        for i in range(2):
            tp, tm = th2.copy(), th2.copy()
            tp[i] += h
            tm[i] -= h
            fd = (lossfn(O.step(prob(th1, tp), phi0, tau, scheme, n))[0]
                  - lossfn(O.step(prob(th1, tm), phi0, tau, scheme, n))[0]) / (2 * h)
            q = 11
            an = float(np.sum(g2 * np.cos(2 * np.pi * (i + 1) * np.arange(q) / q)))
            assert abs(fd - an) < 1e-7 * max(1.0, abs(fd)) + 1e-9


def test_adjoint_dot_product():
    """<U x, y> = <x, U^H y> with U^H applied as the reverse sweep (-tau)."""
    p = W.bilayer_1d(6, 5, 1.2, 0.7, ecut=1e9)
    x, y = rand_state(p, 20), rand_state(p, 21)
    Ux = O.step(p, x, 0.01, "strang", 4)
    UHy = O.step(p, y, -0.01, "strang", 4)   # symmetric scheme: U^H = U(-tau)
    assert abs(np.vdot(Ux, y) - np.vdot(x, UHy)) < 1e-13


# ---------------------------------------------------------------- 2D
def _dense_H_2d(prob):
    m = O.box_indices(prob.lo1, prob.q1).astype(float)
    n = O.box_indices(prob.lo2, prob.q2).astype(float)
    k = (m @ prob.B1.T)[None, :, :] + (n @ prob.B2.T)[:, None, :]
    D = np.diag(0.5 * (k ** 2).sum(-1).reshape(-1))

    def circ2(h, c, q):
        M = q[0] * q[1]
        C = np.zeros((M, M), dtype=np.complex128)
        for (h0, h1), cc in zip(h, c):
            for i1 in range(q[1]):
                for i0 in range(q[0]):
                    j0, j1 = (i0 - h0) % q[0], (i1 - h1) % q[1]
                    C[i1 * q[0] + i0, j1 * q[0] + j0] += cc
        return C

    C1 = circ2(prob.v1_h, prob.v1_c, prob.q1)
    C2 = circ2(prob.v2_h, prob.v2_c, prob.q2)
    return D + np.kron(np.eye(prob.M2), C1) + np.kron(C2, np.eye(prob.M1))


def test_2d_order_against_dense_exponential():
    p = W.twisted_2d(q=4, theta_deg=5.0, hmax=1)
    p.B1 = p.B1 / 4.0
    p.B2 = p.B2 / 4.0
    H = _dense_H_2d(p)
    phi0 = W.random_state((p.M2, p.M1), 22)
    T = 0.2
    exact = (expm_herm(H, T) @ phi0.reshape(-1)).reshape(phi0.shape)
    ns = [16, 32, 64]
    err = _errors(p, "strang", T, ns, phi0, exact)
    slope = np.polyfit(np.log([T / n for n in ns]), np.log(err), 1)[0]
    assert abs(slope - 2) < 0.15, (slope, err)


def test_2d_free_particle_and_mass():
    p = W.twisted_2d(q=4, hmax=1)
    phi0 = W.random_state((p.M2, p.M1), 23)
    z = p.with_potentials(v1_c=np.zeros(len(p.v1_c)), v2_c=np.zeros(len(p.v2_c)))
    out = O.step(z, phi0, 0.003, "strang", 3)
    m = O.box_indices(p.lo1, p.q1).astype(float)
    n = O.box_indices(p.lo2, p.q2).astype(float)
    k = (m @ p.B1.T)[None, :, :] + (n @ p.B2.T)[:, None, :]
    np.testing.assert_allclose(out, np.exp(-0.5j * 0.009 * (k ** 2).sum(-1)) * phi0, atol=1e-12)
    out = O.step(p, phi0, 0.003, "strang", 3)
    assert abs(np.linalg.norm(out) - 1) < 1e-13


def test_fft_backend_equals_dense_definition():
    """The NumPy-FFT backend (used for full-size parity) computes the same
    transforms as the dense DFT matrices of the definition."""
    for p in (W.bilayer_1d(16, 13, 1.1, 0.6, ecut=1e9), W.twisted_2d(q=4, hmax=1)):
        x = W.random_state((p.M2, p.M1), 40)
        ref = O.step(p, x, 0.01, "strang", 3)
        ob = O.observables(p, x)
        try:
            O.use_fft(True)
            got = O.step(p, x, 0.01, "strang", 3)
            og = O.observables(p, x)
        finally:
            O.use_fft(False)
        np.testing.assert_allclose(got, ref, atol=1e-13)
        assert abs(og["energy"] - ob["energy"]) < 1e-12


# ---------------------------------------------------------------- Crank-Nicolson layer splitting
def galerkin_by_quadrature(h, c, q, L=1.0, npts=256):
    """V[m, m'] = (1/L) int_0^L v(x) e^{-i G_m x} e^{i G_m' x} dx with
    v(x) = sum_h vhat_h e^{i 2 pi h x / L}, by the trapezoidal rule on npts
    points (exact for these trigonometric polynomials): the plane-wave matrix of
    Sec. 3 computed from the potential function, not from its index formula."""
    x = np.arange(npts) * L / npts
    v = np.zeros(npts, dtype=np.complex128)
    for hh, cc in zip(np.asarray(h).reshape(-1), c):
        v += cc * np.exp(2j * np.pi * hh * x / L)
    G = 2 * np.pi * np.arange(q) / L
    E = np.exp(1j * np.outer(G, x))              # e^{i G_m x}
    return (E.conj() * v) @ E.T / npts


def dense_H_1d_galerkin(prob):
    m = np.arange(prob.q1[0]) + prob.lo1[0]
    n = np.arange(prob.q2[0]) + prob.lo2[0]
    k = prob.B1[0, 0] * m[None, :] + prob.B2[0, 0] * n[:, None]
    D = np.diag(0.5 * (k ** 2).reshape(-1))
    V1 = galerkin_by_quadrature(prob.v1_h, prob.v1_c, prob.q1[0])
    V2 = galerkin_by_quadrature(prob.v2_h, prob.v2_c, prob.q2[0])
    return D + np.kron(np.eye(prob.q2[0]), V1) + np.kron(V2, np.eye(prob.q1[0]))


def test_toeplitz_potential_matches_quadrature():
    """Orientation and values of the plane-wave potential matrix, with complex
    (non-symmetric) coefficients so that a transposition would show."""
    h = np.array([[1], [-1], [2], [-2], [0]])
    c = np.array([0.3 + 0.2j, 0.3 - 0.2j, -0.1j, 0.1j, 0.25])
    for q in (1, 2, 5, 9):
        np.testing.assert_allclose(O.lsplit.toeplitz_potential(h, c, q), galerkin_by_quadrature(h, c, q), atol=1e-13)


def test_cn_mass_conservation():
    """Theorem 4.4 (mass conservation of Eq. (tsCN)): every factor is a
    Cayley transform of a Hermitian block, so the norm is kept to rounding."""
    p = W.bilayer_1d(6, 5, 1.3, 0.9, ecut=1e9)
    x = rand_state(p, 21)
    y = O.step(p, x, 0.05, "cn_strang", 20)
    assert abs(np.linalg.norm(y) - np.linalg.norm(x)) < 1e-13


def test_cn_free_particle_cayley_phases():
    """V = 0: each element is multiplied per step by C(tau/2) C(tau) C(tau/2)
    with C(s) = (1 - i s kin/4) / (1 + i s kin/4) (H_j = D/2, kin = |k|^2/2)."""
    p = W.bilayer_1d(8, 6, 0.0, 0.0, ecut=1e9)
    x = rand_state(p, 22)
    tau, n = 0.03, 4
    kin = O.kinetic_energy_diag(p)
    C = lambda s: (1 - 0.25j * s * kin) / (1 + 0.25j * s * kin)
    np.testing.assert_allclose(O.step(p, x, tau, "cn_strang", n), x * (C(tau / 2) ** 2 * C(tau)) ** n, atol=1e-13)


def test_cn_second_order_against_dense_galerkin_exponential():
    """Theorem 4.3 (second order of Eq. (tsCN)) against exp(-i T H) with the
    plane-wave potential matrices built by quadrature."""
    p = small_1d()
    H = dense_H_1d_galerkin(p)
    phi0 = rand_state(p, 9)
    T = 0.2
    exact = (expm_herm(H, T) @ phi0.reshape(-1)).reshape(phi0.shape)
    ns = [16, 32, 64, 128]
    err = _errors(p, "cn_strang", T, ns, phi0, exact)
    slope = np.polyfit(np.log([T / n for n in ns]), np.log(err), 1)[0]
    assert abs(slope - 2) < 0.1, (slope, err)
    assert err[-1] < 1e-3


def test_cn_time_reversible():
    p = W.bilayer_1d(6, 5, 1.3, 0.9, ecut=1e9)
    x = rand_state(p, 23)
    y = O.step(p, O.step(p, x, 0.02, "cn_strang", 4), -0.02, "cn_strang", 4)
    np.testing.assert_allclose(y, x, atol=1e-13)


# ---------------------------------------------------------------- semi-implicit step and random batch
def complex_potential_1d():
    """Small 1D box whose potentials have complex (Hermitian-paired)
    coefficients, so that a transposed plane-wave matrix would show."""
    p = W.bilayer_1d(4, 3, 0.0, 0.0, ecut=1e9)
    return p.with_potentials(v1_h=[[1], [-1], [2], [-2]], v1_c=[0.4 + 0.3j, 0.4 - 0.3j, 0.1j, -0.1j],
                             v2_h=[[1], [-1]], v2_c=[0.2 - 0.5j, 0.2 + 0.5j])


def test_semi_implicit_step_matches_dense_formula():
    """Algorithm 1 is phi' = (I + i tau D)^{-1} (I - i tau (V^1 + V^2)) phi with
    the Kronecker V^1 = I (x) Vc^1, V^2 = Vc^2 (x) I of Sec. 3; the matrices here
    come from quadrature of the potentials."""
    p = complex_potential_1d()
    H = dense_H_1d_galerkin(p)
    D = np.diag(np.diag(H)).real
    x = rand_state(p, 31)
    tau = 0.07
    want = np.linalg.solve(np.eye(len(H)) + 1j * tau * D, (np.eye(len(H)) - 1j * tau * (H - D)) @ x.reshape(-1))
    np.testing.assert_allclose(O.step(p, x, tau, "semi_implicit", 1).reshape(-1), want, atol=1e-13)


def test_semi_implicit_free_particle_closed_form():
    p = W.bilayer_1d(6, 5, 0.0, 0.0, ecut=1e9)
    x = rand_state(p, 32)
    kin = O.kinetic_energy_diag(p)
    np.testing.assert_allclose(O.step(p, x, 0.02, "semi_implicit", 3), x / (1 + 0.02j * kin) ** 3, atol=1e-13)


def test_semi_implicit_first_order_against_dense_galerkin_exponential():
    """Theorem 4.1 (first order of the semi-implicit method); a small box so
    that tau |k|^2 is small and the steps are in the asymptotic range."""
    p = small_1d(n1=2, n2=2)
    H = dense_H_1d_galerkin(p)
    phi0 = rand_state(p, 9)
    T = 0.05
    exact = (expm_herm(H, T) @ phi0.reshape(-1)).reshape(phi0.shape)
    ns = [64, 128, 256, 512]
    err = _errors(p, "semi_implicit", T, ns, phi0, exact)
    slope = np.polyfit(np.log([T / n for n in ns]), np.log(err), 1)[0]
    assert abs(slope - 1) < 0.1, (slope, err)


def test_random_batch_full_sample_is_semi_implicit():
    """Algorithm 4 with p = |I_j| (frac_den = 1) takes every row and column
    with weight 1: Algorithm 1."""
    p = complex_potential_1d()
    x = rand_state(p, 33)
    a = O.step(p, x, 0.03, "random_batch", 3, seed=9, frac_den=1)
    np.testing.assert_allclose(a, O.step(p, x, 0.03, "semi_implicit", 3), atol=1e-14)


def test_random_batch_is_unbiased():
    """E[Psi_j] over the sampled sets equals the full Psi_j (each slice is in
    the sample with probability p/S and carries the weight S/p), so the mean
    one-step result over seeds approaches Algorithm 1's step."""
    p = complex_potential_1d()
    x = rand_state(p, 34)
    tau = 0.05
    ref = O.step(p, x, tau, "semi_implicit", 1)
    n = 3000
    mean = sum(O.step(p, x, tau, "random_batch", 1, seed=s, frac_den=3) for s in range(n)) / n
    one = O.step(p, x, tau, "random_batch", 1, seed=0, frac_den=3)
    spread = np.linalg.norm(one - ref)
    assert spread > 1e-3                       # a single draw differs
    assert np.linalg.norm(mean - ref) < 5 * spread / np.sqrt(n)


# ---------------------------------------------------------------- real-space wave function on a line
def test_density_single_plane_wave():
    """One coefficient: psi(x) = phi_mn exp(i (B1 m + B2 n) x) exactly."""
    p = W.bilayer_1d(5, 4, 1.0, 1.0, ecut=1e9)
    phi = np.zeros((p.M2, p.M1), dtype=np.complex128)
    phi[1, 7] = 0.3 - 0.4j
    m, n = 7 + p.lo1[0], 1 + p.lo2[0]
    x = np.array([-3.7, 0.0, 0.25, 11.0])
    k = p.B1[0, 0] * m + p.B2[0, 0] * n
    np.testing.assert_allclose(O.lsplit.density_on_line(p, phi, x), (0.3 - 0.4j) * np.exp(1j * k * x), atol=1e-13)


def test_density_real_for_conjugate_symmetric_state():
    """phi(-m, -n) = conj(phi(m, n)) (a real wave function) gives a real psi(x)."""
    p = W.bilayer_1d(5, 4, 1.0, 1.0, ecut=1e9)
    a = rand_state(p, 41)
    phi = 0.5 * (a + np.conj(a[::-1, ::-1]))       # the boxes are symmetric about 0
    vals = O.lsplit.density_on_line(p, phi, np.linspace(-5, 5, 17))
    assert np.abs(vals.imag).max() < 1e-12 * np.abs(vals).max()


def test_density_periodic_for_commensurate_layers():
    """L2 = 2 L1 / 3: every k_mn is a multiple of 2 pi / (2 L1), so psi has
    period 2 L1."""
    p = W.bilayer_1d(4, 3, 1.0, 1.0, L1=1.0, L2=2.0 / 3.0, ecut=1e9)
    phi = rand_state(p, 42)
    x = np.array([0.1, 0.37, 1.3])
    np.testing.assert_allclose(O.lsplit.density_on_line(p, phi, x + 2.0), O.lsplit.density_on_line(p, phi, x), atol=1e-11)


def test_density_2d_single_plane_wave():
    """2D box: one coefficient gives phi_mn exp(i (B1 m + B2 n) . x)."""
    p = W.twisted_2d(q=4, hmax=1)
    phi = np.zeros((p.M2, p.M1), dtype=np.complex128)
    phi[5, 9] = 0.7 + 0.1j
    m = np.array([9 % 4, 9 // 4]) + np.array(p.lo1)
    n = np.array([5 % 4, 5 // 4]) + np.array(p.lo2)
    k = p.B1 @ m + p.B2 @ n
    x = np.array([[0.3, -1.2], [4.0, 2.5]])
    np.testing.assert_allclose(O.lsplit.density_on_line(p, phi, x), (0.7 + 0.1j) * np.exp(1j * (x @ k)), atol=1e-13)


# ---------------------------------------------------------------- shared periodic index (Example 3)
def _example3_dense(p):
    """Dense D, V1, V2 of a three-index problem (Example 3 of Sec. 5) built from
    the index ranges and Fourier coefficients: phi[n + q2 p][m] flattened row
    major; V1 couples (m, p) at fixed n, V2 couples (n, p) at fixed m, each
    with periodic wrap in both of its indices."""
    q1, q2, q3 = p.q1[0], p.q2[0], p.q2[1]
    G1, G2, G3 = p.B1[0, 0], p.B2[0, 0], p.B2[1, 1]
    m = np.arange(q1) + p.lo1[0]
    n = np.arange(q2) + p.lo2[0]
    pp = np.arange(q3) + p.lo2[1]
    N = q1 * q2 * q3
    idx = lambda mi, ni, pi: (ni + q2 * pi) * q1 + mi
    kin = np.zeros(N)
    V1 = np.zeros((N, N), dtype=np.complex128)
    V2 = np.zeros((N, N), dtype=np.complex128)
    for pi in range(q3):
        for ni in range(q2):
            for mi in range(q1):
                kin[idx(mi, ni, pi)] = 0.5 * ((G1 * m[mi] + G2 * n[ni]) ** 2 + (G3 * pp[pi]) ** 2)
                for (hx, hy), c in zip(p.v1_h, p.v1_c):
                    V1[idx(mi, ni, pi), idx((mi - hx) % q1, ni, (pi - hy) % q3)] += c
                for (hx, hy), c in zip(p.v2_h, p.v2_c):
                    V2[idx(mi, ni, pi), idx(mi, (ni - hx) % q2, (pi - hy) % q3)] += c
    return kin, V1, V2


def test_example3_free_particle_exact_phase():
    """V = 0 on the three-index lift: every scheme is the exact phase with
    k = (G1 m + G2 n, G3 p) (Example 3's wavevectors, formed from the ranges)."""
    p = W.example3(3, 2, 2)
    z = p.with_potentials(v1_c=np.zeros(len(p.v1_c)), v2_c=np.zeros(len(p.v2_c)))
    kin, _, _ = _example3_dense(z)
    x = W.random_state((p.M2, p.M1), 41)
    for scheme in ("strang", "lie", "strang_stoch"):
        out = O.step(z, x, 0.013, scheme, 3, seed=2)
        np.testing.assert_allclose(out.reshape(-1), np.exp(-1j * 0.039 * kin) * x.reshape(-1), atol=1e-12)


def test_example3_y_independent_reduces_to_1d_planes():
    """Potentials without y dependence: each plane p of the three-index lift is
    an independent 1D bilayer (the 1D oracle) times the phase of its extra
    kinetic energy (G3 p)^2 / 2."""
    p = W.example3(4, 3, 2)
    keep = lambda h, c: (h[h[:, 1] == 0], c[h[:, 1] == 0])
    h1, c1 = keep(np.asarray(p.v1_h), np.asarray(p.v1_c))
    h2, c2 = keep(np.asarray(p.v2_h), np.asarray(p.v2_c))
    p = p.with_potentials(v1_c=c1, v2_c=c2, v1_h=h1, v2_h=h2)
    x = W.random_state((p.M2, p.M1), 42)
    tau, n = 0.02, 4
    out = O.step(p, x, tau, "strang", n)
    q1, q2, q3 = p.q1[0], p.q2[0], p.q2[1]
    G1, G2, G3 = p.B1[0, 0], p.B2[0, 0], p.B2[1, 1]
    one = W.Problem(1, np.array([[G1]]), np.array([[G2]]), (p.lo1[0],), (q1,), (p.lo2[0],), (q2,), 1e9,
                    h1[:, :1], c1, h2[:, :1], c2)
    for pi in range(q3):
        y = p.lo2[1] + pi
        rows = slice(pi * q2, (pi + 1) * q2)
        ref = O.step(one, x[rows], tau, "strang", n) * np.exp(-0.5j * n * tau * (G3 * y) ** 2)
        np.testing.assert_allclose(out[rows], ref, atol=1e-12)


def test_example3_one_step_and_order_against_dense():
    """One step of the three-index lift equals the dense factor product
    (Strang order of Appendix A, V1 on (m, p) and V2 on (n, p)); Strang
    converges to the dense exponential of H = D + V1 + V2 with slope 2; the
    energy is the dense quadratic form."""
    p = W.example3(2, 2, 2, s1=3.0, s2=2.0)
    p.B1 = p.B1 / 3.0
    p.B2 = p.B2 / 3.0
    kin, V1, V2 = _example3_dense(p)
    D = np.diag(kin)
    E = lambda A, t: expm_herm(A, t)
    x = W.random_state((p.M2, p.M1), 43)
    t = 0.05
    U = (E(D, t / 8) @ E(V1, t / 2) @ E(D, t / 8)) @ (E(D, t / 4) @ E(V2, t) @ E(D, t / 4)) \
        @ (E(D, t / 8) @ E(V1, t / 2) @ E(D, t / 8))
    np.testing.assert_allclose(O.step(p, x, t, "strang", 1).reshape(-1), U @ x.reshape(-1), atol=1e-12)
    H = D + V1 + V2
    T = 0.4
    exact = E(H, T) @ x.reshape(-1)
    ns = [8, 16, 32]
    err = [np.linalg.norm(O.step(p, x, T / k, "strang", k).reshape(-1) - exact) for k in ns]
    slope = np.polyfit(np.log([T / k for k in ns]), np.log(err), 1)[0]
    assert abs(slope - 2) < 0.15, (slope, err)
    v = x.reshape(-1)
    assert abs(O.observables(p, x)["energy"] - np.vdot(v, H @ v).real) < 1e-10


# ---------------------------------------------------------------- three layers
def _trilayer_dense(n, a, L):
    """Dense D, V1, V2, V3 of three 1D layers lifted to (m, n, p), built from
    the layer periods and cosine amplitudes alone: k = sum_j (2 pi / L_j) i_j,
    V_j = (a_j / 2)(S_j + S_j^-1) with S_j the periodic shift along index j
    (the pseudo-spectral matrix of a_j cos(2 pi x / L_j), Eq. (3.6) with wrap);
    phi[n + q2 p][m] flattened row major."""
    q = [2 * x for x in n]
    idx = lambda i, j, k: (j + q[1] * k) * q[0] + i
    N = q[0] * q[1] * q[2]
    rng = [np.arange(qq) - qq // 2 for qq in q]
    b = [2 * np.pi / x for x in L]
    kin = np.zeros(N)
    V = [np.zeros((N, N)) for _ in range(3)]
    for k in range(q[2]):
        for j in range(q[1]):
            for i in range(q[0]):
                r = idx(i, j, k)
                kin[r] = 0.5 * (b[0] * rng[0][i] + b[1] * rng[1][j] + b[2] * rng[2][k]) ** 2
                for s_ in (1, -1):
                    V[0][r, idx((i + s_) % q[0], j, k)] += a[0] / 2
                    V[1][r, idx(i, (j + s_) % q[1], k)] += a[1] / 2
                    V[2][r, idx(i, j, (k + s_) % q[2])] += a[2] / 2
    return kin, V


def test_trilayer_free_particle_exact_phase():
    """V = 0 for three layers: every scheme is the exact phase with
    k = b1 m + b2 n + b3 p (the trilayer mapping's wavevector)."""
    n, L = (3, 2, 2), (1.0, W.GOLDEN, np.sqrt(2) / 2)
    p = W.trilayer_1d(*n, 0.0, 0.0, 0.0, *L)
    kin, _ = _trilayer_dense(n, (0, 0, 0), L)
    x = W.random_state((p.M2, p.M1), 61)
    for scheme in ("lie", "strang", "strang_kp", "yoshida4"):
        got = O.step(p, x, 0.01, scheme, 3).reshape(-1)
        np.testing.assert_allclose(got, np.exp(-1j * 0.03 * kin) * x.reshape(-1), atol=1e-12)


def test_trilayer_one_step_and_order_against_dense():
    """One Strang step of the trilayer mapping equals the dense product with
    the commuting layers 1 and 3 as one factor, exp(-i s (V1 + V3)) =
    exp(-i s V1) exp(-i s V3); Strang converges to the dense exponential of
    H = D + V1 + V2 + V3 with slope 2; the energy is the dense quadratic form."""
    n, a, L = (2, 2, 2), (1.3, 0.9, 0.7), (1.0, W.GOLDEN, np.sqrt(2) / 2)
    p = W.trilayer_1d(*n, *a, *L)
    kin, (V1, V2, V3) = _trilayer_dense(n, a, L)
    D = np.diag(kin) / 9.0
    p.B1 = p.B1 / 3.0
    p.B2 = p.B2 / 3.0
    E = lambda A, t: expm_herm(A, t)
    np.testing.assert_allclose(E(V1, 0.3) @ E(V3, 0.3), E(V1 + V3, 0.3), atol=1e-12)
    x = W.random_state((p.M2, p.M1), 62)
    t = 0.05
    U = (E(D, t / 8) @ E(V1 + V3, t / 2) @ E(D, t / 8)) @ (E(D, t / 4) @ E(V2, t) @ E(D, t / 4)) \
        @ (E(D, t / 8) @ E(V1 + V3, t / 2) @ E(D, t / 8))
    np.testing.assert_allclose(O.step(p, x, t, "strang", 1).reshape(-1), U @ x.reshape(-1), atol=1e-12)
    H = D + V1 + V2 + V3
    T = 0.4
    exact = E(H, T) @ x.reshape(-1)
    ns = [16, 32, 64]
    err = [np.linalg.norm(O.step(p, x, T / k, "strang", k).reshape(-1) - exact) for k in ns]
    slope = np.polyfit(np.log([T / k for k in ns]), np.log(err), 1)[0]
    assert abs(slope - 2) < 0.15, (slope, err)
    v = x.reshape(-1)
    assert abs(O.observables(p, x)["energy"] - np.vdot(v, H @ v).real) < 1e-10
