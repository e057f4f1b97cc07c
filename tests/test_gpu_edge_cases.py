"""Edge and degenerate cases of the CUDA path: single-plane-wave layers, the
longest 1D slices, rectangular 2D slices, zero steps and zero time step,
the zero state, and time reversal of the symmetric Strang step at the full
2049 x 2049 size (a property that holds at any size)."""
import dataclasses

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests._parity import rel

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "c128": 1e-11}


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_14897_gb300 import build as B
    B.build()
    import paper_2103_14897_gb300 as P
    P.load_library()
    return P




def run_vs_oracle(P, p, dtype, scheme, n=2, tau=5e-3, seed=0, fft=False):
    ctx = P.Context(p, dtype)
    x = W.random_state((p.M2, p.M1), 11)
    psi = ctx.from_dense(x)
    ctx.step(psi, n, tau, scheme, seed=seed)
    O.use_fft(fft)
    try:
        ref = O.step(p, x, tau, scheme, n, seed=seed)
    finally:
        O.use_fft(False)
    return rel(ctx.to_dense(psi), ref)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("scheme", ["strang", "lie", "strang_stoch"])
def test_single_plane_wave_layer(P, dtype, scheme):
    """A layer box of one index: its slices have one element and its factor is
    a plain multiplication by exp(-i s v(x_0)) (Sec. 3 with a one-point grid)."""
    for p in [W.bilayer_1d(16, 0, 1.3, 0.9, ecut=1e9), W.bilayer_1d(0, 16, 1.3, 0.9, ecut=1e9)]:
        assert run_vs_oracle(P, p, dtype, scheme, seed=2) < TOL[dtype] * 3, p.name


def test_largest_1d_box_one_step(P):
    """4097 x 4097 lifted box (16.8 M DOF, 134 MB complex64): both layers on
    the general pass with transforms of 8192, one Strang step against the
    oracle's FFT backend."""
    p = W.bilayer_1d(2048, 2048, 1.0, 0.8, ecut=1e9)
    ctx = P.Context(p, "c64")
    x = W.random_state((p.M2, p.M1), 19)
    psi = ctx.from_dense(x)
    ctx.step(psi, 1, 5e-4, "strang")
    O.use_fft(True)
    try:
        ref = O.step(p, x, 5e-4, "strang", 1)
    finally:
        O.use_fft(False)
    assert rel(ctx.to_dense(psi), ref) < TOL["c64"] * 3


@pytest.mark.parametrize("dtype", ["c64"])
def test_longest_1d_slices(P, dtype):
    """The largest accepted complex64 1D slices: q = 4097 (transform length
    8192 on the general pass) and the power of two 8192.  (complex128 stops at
    transform length 4096; ls_create rejects longer slices.)"""
    pow2 = W.Problem(1, np.array([[2 * np.pi]]), np.array([[2 * np.pi / W.GOLDEN]]), (-4096,), (8192,),
                     (-1,), (3,), 1e9, np.array([[1], [-1]]), np.array([0.6, 0.6], dtype=complex),
                     np.array([[2], [-2]]), np.array([0.3j, -0.3j]), "pow2-8192x3")
    for p in [W.bilayer_1d(2048, 2, 1.0, 0.7, ecut=1e9), pow2]:
        for scheme in ("strang", "lie"):
            assert run_vs_oracle(P, p, dtype, scheme, tau=1e-3, fft=True) < TOL[dtype] * 3, (p.name, scheme)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("scheme", ["strang", "lie", "strang_kp", "lie_stoch"])
def test_rectangular_2d_slices(P, dtype, scheme):
    base = W.twisted_2d(q=8, hmax=2)
    p = dataclasses.replace(base, lo1=(-16, -4), q1=(32, 8), lo2=(-2, -8), q2=(4, 16), name="rect-32x8-4x16")
    assert run_vs_oracle(P, p, dtype, scheme, seed=4) < TOL[dtype] * 3


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_zero_steps_and_zero_tau_are_identity(P, dtype):
    for p in [W.config_small_1d(), W.twisted_2d(q=8, hmax=2)]:
        ctx = P.Context(p, dtype)
        x = W.random_state((p.M2, p.M1), 12)
        psi = ctx.from_dense(x)
        ctx.step(psi, 0, 1e-3, "strang")
        ctx.step(psi, 3, 0.0, "strang")
        ctx.step(psi, 3, 0.0, "lie_stoch", seed=5)
        got = ctx.to_dense(psi)
        want = x.astype(np.complex64).astype(np.complex128) if dtype == "c64" else x
        assert np.array_equal(got, want), p.name


def test_zero_state_stays_zero(P):
    for p in [W.config_scale_1d(), W.twisted_2d(q=16, hmax=3)]:
        ctx = P.Context(p, "c64")
        psi = ctx.empty()
        psi.zero_()
        ctx.step(psi, 3, 1e-3, "strang")
        ctx.step(psi, 2, 1e-3, "strang_stoch", seed=3)
        assert float(psi.abs().max()) == 0.0
        assert ctx.observables(psi)["norm"] == 0.0


@pytest.mark.parametrize("dtype,tol", [("c64", 1e-5), ("c128", 1e-11)])
def test_strang_time_reversal_full_size(P, dtype, tol):
    """The Strang step is symmetric, so S(-tau) S(tau) = I: 20 steps forward
    and 20 back at the full 2049 x 2049 size return the initial state
    (the same launch configuration as the bench, fused multi-step calls)."""
    p = W.config_scale_1d()
    ctx = P.Context(p, dtype)
    import torch
    psi = ctx.from_dense(W.random_state((p.M2, p.M1), 13))
    x = psi.clone()
    ctx.step(psi, 20, 5e-4, "strang")
    moved = float(torch.linalg.vector_norm(psi - x) / torch.linalg.vector_norm(x))
    ctx.step(psi, 20, -5e-4, "strang")
    err = float(torch.linalg.vector_norm(psi - x) / torch.linalg.vector_norm(x))
    assert moved > 0.1, moved
    assert err < tol, err


@pytest.mark.parametrize("dtype,tol", [("c64", 2e-6), ("c128", 1e-12)])
def test_cn_and_semi_implicit_free_particle_closed_forms(P, dtype, tol):
    """V = 0, checked against closed forms rather than the oracle: the
    Crank-Nicolson split multiplies each element per step by
    C(tau/2)^2 C(tau), C(s) = (1 - i s kin/4)/(1 + i s kin/4) (no Jacobi sweep
    is needed); the semi-implicit step divides by (1 + i tau kin)."""
    p = W.bilayer_1d(300, 200, 0.0, 0.0, ecut=1e9)
    kin = O.kinetic_energy_diag(p)
    x = W.random_state((p.M2, p.M1), 21)
    tau, n = 2e-4, 3
    ctx = P.Context(p, dtype)
    psi = ctx.from_dense(x)
    ctx.step(psi, n, tau, "cn_strang")
    C = lambda s: (1 - 0.25j * s * kin) / (1 + 0.25j * s * kin)
    assert rel(ctx.to_dense(psi), x * (C(tau / 2) ** 2 * C(tau)) ** n) < tol
    psi = ctx.from_dense(x)
    ctx.step(psi, n, tau, "semi_implicit")
    assert rel(ctx.to_dense(psi), x / (1 + 1j * tau * kin) ** n) < tol
