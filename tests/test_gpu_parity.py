"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (the arithmetic is complex64 with FP64-derived tables and exact
fixed-point kinetic phases, or complex128):
  * complex64: rel-L2 <= 1e-5 after one step, <= 1e-4 after 1000 steps,
    | ||psi|| - 1 | <= 1e-5;
  * complex128: rel-L2 <= 1e-11;
  * integer work (index set, slice samples): bit-exact.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests._parity import rel

pytestmark = pytest.mark.gpu

TOL1 = {"c64": 1e-5, "c128": 1e-11}


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




def problems_1d():
    return [
        W.bilayer_1d(8, 8, 1.3, 0.9, ecut=1e9),          # q = 17 (Bluestein 32)
        W.bilayer_1d(16, 5, 1.3, 0.9, ecut=1e9),         # q = 33 x 11
        W.config_small_1d(),                              # 65 x 65
        W.bilayer_1d(64, 40, 0.7, 1.9, ecut=1e9).with_potentials(  # even lengths 128 x 81
            v1_h=[[1], [-1], [3], [-3]], v1_c=[0.5, 0.5, 0.2 + 0.1j, 0.2 - 0.1j]),
        W.Problem(1, np.array([[2 * np.pi]]), np.array([[2 * np.pi / W.GOLDEN]]), (-32,), (64,),
                  (-16,), (32,), 1e9, np.array([[1], [-1]]), np.array([0.6, 0.6], dtype=complex),
                  np.array([[2], [-2]]), np.array([0.3j, -0.3j]), "pow2-64x32"),
        W.bilayer_1d(256, 12, 1.0, 1.4, ecut=1e9),       # q = 513 (Bluestein 1024)
    ]


def problems_2d():
    return [W.twisted_2d(q=8, hmax=2), W.twisted_2d(q=16, hmax=3)]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_index_set_bit_exact(P, dtype):
    for p in [W.config_small_1d(), W.config_scale_1d(), W.twisted_2d(q=16, ecut=50.0),
              W.bilayer_1d(40, 33, ecut=731.25, L2=0.37)]:
        ctx = P.Context(p, dtype)
        mask, cnt = ctx.index_set()
        ref = O.index_mask(p)
        assert cnt == int(ref.sum())
        assert np.array_equal(mask, ref)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_gaussian_initial_state(P, dtype):
    for p, x0, k0 in [(W.config_small_1d(), [0.0], [1.0]), (W.config_small_1d(), [0.3], [-2.0]),
                      (W.twisted_2d(q=8, ecut=30.0), [0.1, -0.2], [1.0, 0.0])]:
        ctx = P.Context(p, dtype)
        psi = ctx.empty()
        ctx.init_gaussian(psi, x0, 2.0, k0)
        got = ctx.to_dense(psi)
        ref = O.gaussian_packet(p, x0, 2.0, k0)
        assert rel(got, ref) < TOL1[dtype]
        assert np.all(got[~O.index_mask(p)] == 0)


@pytest.mark.parametrize("form", ["compact", "convolution", "bluestein"])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("scheme", ["lie", "strang", "strang_kp"])
def test_step_parity_1d(P, dtype, scheme, form, monkeypatch):
    """Every form of the potential factor on 1D slices: the compact kernel
    (the taps of P - I above the working precision; the default where they
    qualify), the cyclic convolution through one power-of-two transform pair,
    and the chirp-z (Bluestein) transform to the real-space grid and back
    (powers of two: the radix transforms)."""
    if form != "compact":
        monkeypatch.setenv("LSPLIT_NO_STENCIL", "1")
    if form == "bluestein":
        monkeypatch.setenv("LSPLIT_TRANSFORM", "bluestein")
    for p in problems_1d() + [W.bilayer_1d(1024, 20, 1.1, 0.7, ecut=1e9)]:
        ctx = P.Context(p, dtype)
        x = W.random_state((p.M2, p.M1), 1)
        psi = ctx.from_dense(x)
        for n, tau in [(1, 1e-3), (3, 2e-2)]:
            psi = ctx.from_dense(x)
            ctx.step(psi, n, tau, scheme)
            got = ctx.to_dense(psi)
            ref = O.step(p, x, tau, scheme, n)
            # the FP64 oracle's own phase error grows with tau |k|^2 / 2
            th = tau * float(O.kinetic_energy_diag(p).max()) * n
            tol = TOL1[dtype] * (1 if n == 1 else 3) + (4e-16 * th if dtype == "c128" else 0.0)
            assert rel(got, ref) < tol, (p.name, n, rel(got, ref))
            assert np.all(psi[:, p.M1:].cpu().numpy() == 0)   # padding untouched


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("scheme", ["lie", "strang", "strang_kp"])
def test_step_parity_2d(P, dtype, scheme):
    for p in problems_2d():
        ctx = P.Context(p, dtype)
        x = W.random_state((p.M2, p.M1), 2)
        psi = ctx.from_dense(x)
        ctx.step(psi, 2, 5e-3, scheme)
        ref = O.step(p, x, 5e-3, scheme, 2)
        assert rel(ctx.to_dense(psi), ref) < TOL1[dtype] * 3, p.name


def problems_64x64_slices():
    """Boxes whose layer-1 (or layer-2) slices are 64 x 64, the shape of the
    dedicated 2D pass, next to a small box on the other layer so the oracle
    stays quick; every mode kept (large cutoff) and the default cutoff."""
    import dataclasses
    base = W.twisted_2d(q=64, hmax=3)
    return [
        dataclasses.replace(base, lo2=(-4, -4), q2=(8, 8), ecut=1e9, name="64x64-slices-layer1"),
        dataclasses.replace(base, lo1=(-4, -4), q1=(8, 8), ecut=1e9, name="64x64-slices-layer2"),
        dataclasses.replace(base, lo2=(-3, -2), q2=(8, 4), name="64x64-slices-cutoff"),
    ]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("scheme", ["lie", "strang", "strang_kp", "lie_stoch", "strang_stoch"])
def test_step_parity_64x64_slices(P, dtype, scheme):
    for p in problems_64x64_slices():
        ctx = P.Context(p, dtype)
        x = W.random_state((p.M2, p.M1), 5)
        psi = ctx.from_dense(x)
        ctx.step(psi, 3, 5e-3, scheme, seed=3, step0=2)
        ref = O.step(p, x, 5e-3, scheme, 3, seed=3, step0=2)
        assert rel(ctx.to_dense(psi), ref) < TOL1[dtype] * 3, (p.name, rel(ctx.to_dense(psi), ref))


def problems_strided_4096():
    """Layer-2 columns of transform length 4096 (the two-column pass of the
    strided layer): convolution form with an odd column count (the last CTA
    holds one column), a shorter odd length, and the plain power-of-two form."""
    return [
        W.bilayer_1d(8, 1024, 1.3, 0.9, ecut=1e9),       # 17 columns of q = 2049
        W.bilayer_1d(9, 600, 0.8, 1.1),                  # 19 columns of q = 1201, default cutoff
        W.Problem(1, np.array([[2 * np.pi]]), np.array([[2 * np.pi / W.GOLDEN]]), (-8,), (16,),
                  (-2048,), (4096,), 1e9, np.array([[1], [-1]]), np.array([0.6, 0.6], dtype=complex),
                  np.array([[3], [-3]]), np.array([0.2 + 0.1j, 0.2 - 0.1j]), "pow2-16x4096"),
    ]


@pytest.mark.parametrize("scheme", ["lie", "strang", "strang_kp"])
def test_step_parity_strided_4096(P, scheme, monkeypatch):
    monkeypatch.setenv("LSPLIT_NO_STENCIL", "1")   # the transform form of this pass
    O.use_fft(True)
    try:
        for p in problems_strided_4096():
            ctx = P.Context(p, "c64")
            x = W.random_state((p.M2, p.M1), 6)
            psi = ctx.from_dense(x)
            ctx.step(psi, 3, 2e-3, scheme)
            ref = O.step(p, x, 2e-3, scheme, 3)
            assert rel(ctx.to_dense(psi), ref) < TOL1["c64"] * 3, (p.name, rel(ctx.to_dense(psi), ref))
    finally:
        O.use_fft(False)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_step_parity_yoshida4(P, dtype):
    """Fourth-order composition: every pass carries its own kinetic unit (the
    three sub-step durations are incommensurate); general, fast, pair and
    64 x 64 passes."""
    probs = problems_1d() + problems_2d() + problems_64x64_slices()[:1]
    if dtype == "c64":
        probs.append(problems_strided_4096()[0])
    O.use_fft(True)
    try:
        for p in probs:
            ctx = P.Context(p, dtype)
            x = W.random_state((p.M2, p.M1), 14)
            psi = ctx.from_dense(x)
            ctx.step(psi, 3, 5e-3, "yoshida4")
            ref = O.step(p, x, 5e-3, "yoshida4", 3)
            assert rel(ctx.to_dense(psi), ref) < TOL1[dtype] * 5, (p.name, rel(ctx.to_dense(psi), ref))
    finally:
        O.use_fft(False)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_step_parity_cn_strang(P, dtype):
    """Crank-Nicolson layer splitting (Eq. (tsCN)): Jacobi-swept banded
    factors against the oracle's dense per-slice solves; potentials with one,
    two and three harmonics, odd and even lengths, rows and columns on tiles."""
    for p in problems_1d():
        ctx = P.Context(p, dtype)
        x = W.random_state((p.M2, p.M1), 15)
        psi = ctx.from_dense(x)
        ctx.step(psi, 3, 5e-3, "cn_strang")
        ref = O.step(p, x, 5e-3, "cn_strang", 3)
        assert rel(ctx.to_dense(psi), ref) < TOL1[dtype] * 3, (p.name, rel(ctx.to_dense(psi), ref))


def test_cn_strang_full_size_properties(P):
    """2049 x 2049: the factors are Cayley transforms, so the norm is kept and
    C(-s) C(s) = I makes 10 steps back undo 10 steps forward."""
    import torch
    p = W.config_scale_1d()
    ctx = P.Context(p, "c64")
    psi = ctx.from_dense(W.random_state((p.M2, p.M1), 16))
    x = psi.clone()
    n0 = float(torch.linalg.vector_norm(x))
    ctx.step(psi, 10, 5e-4, "cn_strang")
    moved = float(torch.linalg.vector_norm(psi - x)) / n0
    assert abs(float(torch.linalg.vector_norm(psi)) / n0 - 1) < 1e-5
    ctx.step(psi, 10, -5e-4, "cn_strang")
    assert moved > 0.1
    assert float(torch.linalg.vector_norm(psi - x)) / n0 < 1e-5


def test_cn_strang_1000_steps(P):
    """The accuracy gate of the FP32 path over a long run, for the
    Crank-Nicolson splitting: rel-L2 <= 1e-4 after 1000 steps and
    | ||psi|| - 1 | <= 1e-5 (65 x 65 box, random state)."""
    p = W.config_small_1d()
    ctx = P.Context(p, "c64")
    x = W.random_state((p.M2, p.M1), 3)
    psi = ctx.from_dense(x)
    ctx.step(psi, 1000, 1e-3, "cn_strang")
    ref = O.step(p, x, 1e-3, "cn_strang", 1000)
    got = ctx.to_dense(psi)
    assert rel(got, ref) < 1e-4
    assert abs(np.linalg.norm(got) / np.linalg.norm(x) - 1) < 1e-5


def test_cn_strang_rejects_unsupported(P):
    p2 = W.twisted_2d(q=8, hmax=2)
    ctx = P.Context(p2, "c64")
    with pytest.raises(P.LsplitError) as e:
        ctx.step(ctx.empty(), 1, 1e-3, "cn_strang")
    assert e.value.code == P.LS_ERR_INVALID
    p = W.config_small_1d()
    ctx = P.Context(p, "c64")
    with pytest.raises(P.LsplitError):
        ctx.step(ctx.empty(), 1, 10.0, "cn_strang")        # tau sum |vhat| >= 1
    wide = p.with_potentials(v1_h=[[9], [-9]], v1_c=[0.1, 0.1])
    ctx = P.Context(wide, "c64")
    with pytest.raises(P.LsplitError):
        ctx.step(ctx.empty(), 1, 1e-3, "cn_strang")        # band wider than 8


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("scheme", ["semi_implicit", "random_batch"])
def test_step_parity_semi_implicit(P, dtype, scheme):
    """Algorithms 1 and 4: out-of-place stencil steps (odd and even step
    counts, so that both the copy back and the plain ping-pong end are
    covered), sampled rows and columns bit-identical to the oracle's."""
    for p in problems_1d():
        ctx = P.Context(p, dtype)
        x = W.random_state((p.M2, p.M1), 17)
        for n in (3, 4):
            psi = ctx.from_dense(x)
            ctx.step(psi, n, 2e-3, scheme, seed=7, step0=2)
            ref = O.step(p, x, 2e-3, scheme, n, seed=7, step0=2)
            assert rel(ctx.to_dense(psi), ref) < TOL1[dtype] * 3, (p.name, n, rel(ctx.to_dense(psi), ref))
            assert np.all(psi[:, p.M1:].cpu().numpy() == 0)   # padding untouched
    with pytest.raises(P.LsplitError):
        c2 = P.Context(W.twisted_2d(q=8, hmax=2), dtype)
        c2.step(c2.empty(), 1, 1e-3, scheme)


def test_density_tensor_core_matches_cuda_cores(P, monkeypatch):
    """The complex64 contraction of ls_density in split TF32 on the tensor cores
    against the FP32 CUDA-core form and the oracle: 1000 points (16 CTA rows of
    64 with a ragged last one) on boxes of 65 x 65 and 513 x 25 (ragged m slabs
    and n tiles).  Tolerance: the complex64 density gate, 1e-5; the dropped
    lo*lo term is 2^-22 relative per product, and a random full-spectrum
    state's sums cancel (|psi(x)| is far below the sum of the term moduli),
    which raises the relative error of the result to about 1e-6."""
    x = np.linspace(-30.0, 30.0, 1000)
    for p in [W.config_small_1d(), W.bilayer_1d(256, 12, 1.0, 1.4, ecut=1e9)]:
        ctx = P.Context(p, "c64")
        phi = W.random_state((p.M2, p.M1), 19)
        psi = ctx.from_dense(phi)
        monkeypatch.delenv("LSPLIT_DENSITY_SIMT", raising=False)
        tc = ctx.density(psi, x)
        monkeypatch.setenv("LSPLIT_DENSITY_SIMT", "1")
        simt = ctx.density(psi, x)
        ref = O.density_on_line(p, phi, x)
        assert rel(tc, simt) < 1e-5, (p.name, rel(tc, simt))
        assert rel(tc, ref) < 1e-5, (p.name, rel(tc, ref))


@pytest.mark.parametrize("dtype,tol", [("c64", 1e-5), ("c128", 1e-11)])
def test_density_on_line_parity(P, dtype, tol):
    """psi(x) from the plane-wave expansion: exact fixed-point phase tables,
    tiled contraction over m, FP64 sum over n; small 1D boxes with many points
    (several 64 x 64 tiles and ragged edges), the 2049 x 2049 box at a few
    points, large |x|, and 2D boxes at points in the plane."""
    x = np.concatenate([np.linspace(-20.0, 20.0, 301), [1234.5, -987.25]])
    for p in [W.config_small_1d(), W.bilayer_1d(256, 12, 1.0, 1.4, ecut=1e9), problems_1d()[4]]:
        ctx = P.Context(p, dtype)
        phi = W.random_state((p.M2, p.M1), 18)
        got = ctx.density(ctx.from_dense(phi), x)
        ref = O.density_on_line(p, phi, x)
        # the FP64 oracle forms k.x in floating point: its own phase error
        # grows with max |k| |x| (the library's phases are exact fixed point)
        th = float(np.abs(O.wavevectors(p)).max() * np.abs(x).max())
        assert rel(got, ref) < tol + (4e-16 * th if dtype == "c128" else 0.0), (p.name, rel(got, ref))
    p = W.config_scale_1d()
    ctx = P.Context(p, dtype)
    psi = ctx.empty()
    ctx.init_gaussian(psi, [0.0], 2.0, [1.0])
    xs = np.array([-3.0, 0.0, 0.5, 2.25, 40.0])
    got = ctx.density(psi, xs)
    ref = O.density_on_line(p, ctx.to_dense(psi), xs)
    assert rel(got, ref) < tol * 10, rel(got, ref)
    # 2D boxes: points in the plane
    rng = np.random.default_rng(22)
    x2 = np.concatenate([rng.uniform(-6, 6, size=(129, 2)), [[150.0, -80.5]]])
    for p in [W.twisted_2d(q=8, hmax=2), W.twisted_2d(q=16, hmax=3)]:
        ctx = P.Context(p, dtype)
        phi = W.random_state((p.M2, p.M1), 23)
        got = ctx.density(ctx.from_dense(phi), x2)
        ref = O.density_on_line(p, phi, x2)
        assert rel(got, ref) < tol, (p.name, rel(got, ref))


def test_large_kinetic_phase_free_particle(P):
    """V = 0 at the 2049-box extremes: every element must be the exact phase
    exp(-i T |k|^2/2) (argument reduction of |theta| up to ~1e4 rad)."""
    p = W.bilayer_1d(1024, 1024, 0.0, 0.0, ecut=1e12)
    ctx = P.Context(p, "c64")
    x = W.random_state((p.M2, p.M1), 3)
    psi = ctx.from_dense(x)
    ctx.step(psi, 4, 5e-4, "strang")
    kin = O.kinetic_energy_diag(p)
    ref = x * np.exp(-1j * (4 * 5e-4) * kin)
    assert rel(ctx.to_dense(psi), ref) < 2e-6


def test_observables_parity(P):
    for p in [W.config_small_1d(), W.bilayer_1d(16, 5, 1.3, 0.9, ecut=1e9), W.twisted_2d(q=8, hmax=2)]:
        for dtype, tol in (("c64", 1e-6), ("c128", 1e-12)):
            ctx = P.Context(p, dtype)
            x = W.random_state((p.M2, p.M1), 4)
            chi = W.random_state((p.M2, p.M1), 5)
            o = ctx.observables(ctx.from_dense(x), ctx.from_dense(chi))
            r = O.observables(p, x.astype(np.complex64).astype(np.complex128) if dtype == "c64" else x,
                              chi.astype(np.complex64).astype(np.complex128) if dtype == "c64" else chi)
            scale = max(1.0, abs(r["energy"]))
            for k in ("norm", "ekin", "epot1", "epot2", "energy"):
                assert abs(o[k] - r[k]) < tol * max(1.0, abs(r[k])) * 10, (p.name, dtype, k, o[k], r[k])
            for i in range(p.d):
                assert abs(o["kmean"][i] - r["kmean"][i]) < tol * scale * 10
            assert abs(o["overlap"] - r["overlap"]) < tol * 10


def test_stochastic_samples_bit_exact(P):
    for p in [W.config_small_1d(), W.config_scale_1d(), W.bilayer_1d(16, 5, ecut=1e9)]:
        ctx = P.Context(p, "c64")
        for layer in (1, 2):
            S = p.M2 if layer == 1 else p.M1
            got = ctx.samples(layer, seed=7, g0=11, count=5)
            for i in range(5):
                ref = O.sample_slices(S, O.sample_count(S), 7, 11 + i)
                assert np.array_equal(got[i], ref)


@pytest.mark.parametrize("form", ["compact", "fft"])
@pytest.mark.parametrize("scheme", ["lie_stoch", "strang_stoch"])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_stochastic_step_parity(P, scheme, dtype, form, monkeypatch):
    if form == "fft":
        monkeypatch.setenv("LSPLIT_NO_STENCIL", "1")
    for p in [W.bilayer_1d(16, 20, 1.3, 0.9, ecut=1e9), W.config_small_1d(), W.twisted_2d(q=8, hmax=2)]:
        ctx = P.Context(p, dtype)
        x = W.random_state((p.M2, p.M1), 6)
        psi = ctx.from_dense(x)
        ctx.step(psi, 3, 1e-2, scheme, seed=5, step0=2)
        ref = O.step(p, x, 1e-2, scheme, 3, seed=5, step0=2)
        assert rel(ctx.to_dense(psi), ref) < TOL1[dtype] * 3, (p.name, rel(ctx.to_dense(psi), ref))
        # second call continues the sample sequence
        ctx.step(psi, 2, 1e-2, scheme, seed=5, step0=5)
        ref = O.step(p, ref, 1e-2, scheme, 2, seed=5, step0=5)
        assert rel(ctx.to_dense(psi), ref) < TOL1[dtype] * 5


def long_slice_boxes():
    """Rows (then columns) of length 2049: the layer-1 fast pass and the
    strided layer-2 passes of transform length 4096, next to a short other
    layer so the oracle stays quick."""
    return [W.bilayer_1d(1024, 16, 1.3, 0.9, ecut=1e9, name="2049x33"),
            W.bilayer_1d(16, 1024, 0.9, 1.3, ecut=1e9, name="33x2049")]


@pytest.mark.parametrize("form", ["compact", "fft"])
@pytest.mark.parametrize("scheme", ["lie_stoch", "strang_stoch"])
def test_stochastic_long_slices(P, scheme, form, monkeypatch):
    """The stochastic schemes where the sampled slices are 2049 long, so the
    lazy kinetic phases run inside the fast 1D passes (the sampled-slice path
    of the 2049 x 2049 workload): 3 steps, then 2 more continuing the sample
    sequence, against the oracle.  Both the compact-kernel form and the
    transform (fast pass) form."""
    if form == "fft":
        monkeypatch.setenv("LSPLIT_NO_STENCIL", "1")
    O.use_fft(True)
    try:
        for p in long_slice_boxes():
            ctx = P.Context(p, "c64")
            x = W.random_state((p.M2, p.M1), 24)
            psi = ctx.from_dense(x)
            ctx.step(psi, 3, 5e-4, scheme, seed=11, step0=4)
            ref = O.step(p, x, 5e-4, scheme, 3, seed=11, step0=4)
            assert rel(ctx.to_dense(psi), ref) < TOL1["c64"] * 3, (p.name, rel(ctx.to_dense(psi), ref))
            ctx.step(psi, 2, 5e-4, scheme, seed=11, step0=7)
            ref = O.step(p, ref, 5e-4, scheme, 2, seed=11, step0=7)
            assert rel(ctx.to_dense(psi), ref) < TOL1["c64"] * 5, (p.name, rel(ctx.to_dense(psi), ref))
    finally:
        O.use_fft(False)


@pytest.mark.parametrize("form", ["compact", "fft"])
def test_long_run_1000_steps_long_slices(P, form, monkeypatch):
    """The 1000-step gate through the headline kernels: 1000 Strang steps of
    tau = 5e-4 on boxes whose rows or columns are 2049 long (fused layer-1
    fast pass, two-column strided pass), random full-spectrum state:
    rel-L2 <= 1e-4 and | ||psi|| - 1 | <= 1e-5 against the oracle; the
    compact-kernel form and the transform form."""
    if form == "fft":
        monkeypatch.setenv("LSPLIT_NO_STENCIL", "1")
    O.use_fft(True)
    try:
        for p in long_slice_boxes():
            ctx = P.Context(p, "c64")
            x = W.random_state((p.M2, p.M1), 25)
            psi = ctx.from_dense(x)
            ctx.step(psi, 1000, 5e-4, "strang")
            ref = O.step(p, x, 5e-4, "strang", 1000)
            got = ctx.to_dense(psi)
            print(p.name, "1000-step rel", rel(got, ref), "norm-1", np.linalg.norm(got) - 1)
            assert rel(got, ref) < 1e-4, (p.name, rel(got, ref))
            assert abs(np.linalg.norm(got) - 1) < 1e-5
    finally:
        O.use_fft(False)


@pytest.mark.parametrize("scheme", ["lie", "strang", "strang_kp"])
def test_interaction_frame_matches_physical_frame(P, scheme, monkeypatch):
    """Deterministic complex64 calls whose factors all take the compact-kernel
    form run in the interaction frame (kinetic factors folded into the taps,
    applied once at the call's end); LSPLIT_NO_IP=1 applies them per pass.
    Same operator: both agree with each other to rounding and with the oracle,
    on odd, even and 2049-long slices (wrapped neighbours at both ends), for
    one call of 1 and of 7 steps."""
    O.use_fft(True)
    try:
        for p in problems_1d()[1:] + long_slice_boxes():
            x = W.random_state((p.M2, p.M1), 27)
            for n, tau in [(1, 1e-3), (7, 5e-4)]:
                got = {}
                for frame in ("interaction", "physical"):
                    if frame == "physical":
                        monkeypatch.setenv("LSPLIT_NO_IP", "1")
                    else:
                        monkeypatch.delenv("LSPLIT_NO_IP", raising=False)
                    ctx = P.Context(p, "c64")
                    psi = ctx.from_dense(x)
                    ctx.step(psi, n, tau, scheme)
                    got[frame] = ctx.to_dense(psi)
                ref = O.step(p, x, tau, scheme, n)
                assert rel(got["interaction"], got["physical"]) < 2e-6, (p.name, n)
                assert rel(got["interaction"], ref) < TOL1["c64"] * (1 if n == 1 else 3), (p.name, n)
    finally:
        O.use_fft(False)


def test_project_each_step_mode(P):
    """mask_mode "project": every step ends with the projection onto the joint
    cutoff of Sec. 3 (the oracle's project=True); members keep the scheme's
    values and everything outside the cutoff is zero after each call."""
    cases = [(W.config_small_1d(), ["lie", "strang", "strang_kp", "strang_stoch", "yoshida4", "cn_strang",
                                    "semi_implicit"]),
             (W.bilayer_1d(300, 5, 1.1, 0.7), ["strang", "lie_stoch"]),
             (W.twisted_2d(q=8, hmax=2, ecut=30.0), ["strang", "strang_stoch"])]
    for p, schemes in cases:
        mask = O.index_mask(p)
        assert 0 < mask.sum() < mask.size
        for dtype in ("c64", "c128"):
            ctx = P.Context(p, dtype, mask_mode="project")
            x = W.random_state((p.M2, p.M1), 26)
            for scheme in schemes:
                psi = ctx.from_dense(x)
                ctx.step(psi, 3, 2e-3, scheme, seed=4, step0=1)
                ref = O.step(p, x, 2e-3, scheme, 3, seed=4, step0=1, project=True)
                got = ctx.to_dense(psi)
                assert np.all(got[~mask] == 0), (p.name, scheme)
                assert rel(got, ref) < TOL1[dtype] * 3, (p.name, scheme, dtype, rel(got, ref))
            # the projection is not unitary: no reverse sweep
            with pytest.raises(P.LsplitError) as e:
                ctx.adjoint(ctx.empty(), ctx.empty(), 1, 1e-3, "strang")
            assert e.value.code == P.LS_ERR_INVALID


def test_full_sampling_equals_deterministic(P):
    p = W.bilayer_1d(16, 20, 1.3, 0.9, ecut=1e9)
    c1 = P.Context(p, "c128", frac_den=1)
    x = W.random_state((p.M2, p.M1), 7)
    a = c1.from_dense(x)
    b = c1.from_dense(x)
    c1.step(a, 3, 1e-2, "strang_stoch", seed=1)
    c1.step(b, 3, 1e-2, "strang")
    assert rel(c1.to_dense(a), c1.to_dense(b)) < 1e-13


def test_full_size_one_step_c64(P):
    """2049 x 2049 box (seeded U(0.5, 2) amplitudes), one Strang step of
    tau = 5e-4 from the Gaussian packet, against the oracle (FFT backend)."""
    p = W.config_scale_1d()
    ctx = P.Context(p, "c64")
    psi = ctx.empty()
    ctx.init_gaussian(psi, [0.0], 2.0, [1.0])
    x = O.gaussian_packet(p, [0.0], 2.0, [1.0])
    ctx.step(psi, 1, 5e-4, "strang")
    O.use_fft(True)
    try:
        ref = O.step(p, x, 5e-4, "strang", 1)
    finally:
        O.use_fft(False)
    got = ctx.to_dense(psi)
    assert rel(got, ref) < 1e-5
    assert abs(np.linalg.norm(got) - 1) < 1e-5


def test_full_size_random_state_c64(P):
    """Same box with a dense random state (every element significant)."""
    p = W.config_scale_1d()
    ctx = P.Context(p, "c64")
    x = W.random_state((p.M2, p.M1), 8)
    psi = ctx.from_dense(x)
    ctx.step(psi, 2, 5e-4, "strang")
    O.use_fft(True)
    try:
        ref = O.step(p, x, 5e-4, "strang", 2)
    finally:
        O.use_fft(False)
    assert rel(ctx.to_dense(psi), ref) < 2e-5


def test_long_run_1000_steps(P):
    """65 x 65, tau = 1e-3, 1000 Strang steps in complex64: rel-L2 <= 1e-4 and
    norm drift <= 1e-5 against the FP64 oracle."""
    p = W.config_small_1d()
    ctx = P.Context(p, "c64")
    x = O.gaussian_packet(p, [0.0], 2.0, [1.0])
    psi = ctx.from_dense(x)
    ctx.step(psi, 1000, 1e-3, "strang")
    ref = O.step(p, x, 1e-3, "strang", 1000)
    got = ctx.to_dense(psi)
    print("1000-step rel-L2", rel(got, ref), "norm-1", np.linalg.norm(got) - 1)
    assert rel(got, ref) < 1e-4
    assert abs(np.linalg.norm(got) - 1) < 1e-5


@pytest.mark.parametrize("calls", [1, 100])
def test_packet_1000_steps_long_rows(P, calls):
    """The Gaussian packet on a 2049 x 65 box (seeded U(0.5, 2) amplitudes as
    the 2049^2 workload): every row holds one dominant element whose
    neighbours are many orders smaller, the case where rounding in the
    interaction frame could repeat from pass to pass.  1000 Strang steps of
    tau = 5e-4 as one call or as 100 calls of 10: rel-L2 <= 1e-4 and
    | ||psi|| - 1 | <= 1e-5 against the oracle."""
    base = W.config_scale_1d()
    p = W.bilayer_1d(1024, 32, base.v1_c[0].real * 2, base.v2_c[0].real * 2, ecut=base.ecut, name="2049x65")
    O.use_fft(True)
    try:
        ctx = P.Context(p, "c64")
        x = O.gaussian_packet(p, [0.0], 2.0, [1.0])
        psi = ctx.from_dense(x)
        for _ in range(calls):
            ctx.step(psi, 1000 // calls, 5e-4, "strang")
        ref = O.step(p, x, 5e-4, "strang", 1000)
        got = ctx.to_dense(psi)
        print(p.name, calls, "calls: 1000-step rel-L2", rel(got, ref), "norm-1", np.linalg.norm(got) - 1)
        assert rel(got, ref) < 1e-4
        assert abs(np.linalg.norm(got) - 1) < 1e-5
    finally:
        O.use_fft(False)


def test_fast_and_generic_paths_agree(P, monkeypatch):
    """The compact-kernel pass, the register-resident fast pass and the
    generic pass compute the same step (each is also checked against the
    oracle above)."""
    for p in [W.config_scale_1d(), W.bilayer_1d(128, 200, 1.1, 0.6, ecut=1e9)]:
        x = W.random_state((p.M2, p.M1), 9)
        c = P.Context(p, "c64")
        monkeypatch.setenv("LSPLIT_NO_STENCIL", "1")
        a = P.Context(p, "c64")
        monkeypatch.setenv("LSPLIT_NO_FAST", "1")
        b = P.Context(p, "c64")
        monkeypatch.delenv("LSPLIT_NO_FAST")
        monkeypatch.delenv("LSPLIT_NO_STENCIL")
        pc = c.from_dense(x)
        c.step(pc, 3, 5e-4, "strang")
        pa, pb = a.from_dense(x), b.from_dense(x)
        a.step(pa, 3, 5e-4, "strang")
        b.step(pb, 3, 5e-4, "strang")
        assert rel(a.to_dense(pa), b.to_dense(pb)) < 3e-6
        assert rel(c.to_dense(pc), b.to_dense(pb)) < 3e-6


def test_fused_strang_passes_match_unfused(P, monkeypatch):
    """Adjacent layer-1 factors of consecutive Strang steps fused into one pass
    give the same state as separate passes (and the oracle); transform forms
    (the compact-kernel form has no fused pass)."""
    monkeypatch.setenv("LSPLIT_NO_STENCIL", "1")
    import dataclasses
    rect = dataclasses.replace(W.twisted_2d(q=64, hmax=3), lo2=(-4, -2), q2=(8, 4), ecut=1e9, name="64x64-fused")
    for p in [W.config_scale_1d(), W.bilayer_1d(256, 40, 1.4, 0.6, ecut=1e9), rect]:
        x = W.random_state((p.M2, p.M1), 12)
        a = P.Context(p, "c64")
        monkeypatch.setenv("LSPLIT_NO_FUSE", "1")
        pb = a.from_dense(x)
        a.step(pb, 5, 5e-4, "strang")
        monkeypatch.delenv("LSPLIT_NO_FUSE")
        b = P.Context(p, "c64")
        pa = b.from_dense(x)
        b.step(pa, 5, 5e-4, "strang")
        assert rel(b.to_dense(pa), a.to_dense(pb)) < 3e-6
        if p.M1 < 1000 or p.d == 2:
            O.use_fft(True)
            try:
                assert rel(b.to_dense(pa), O.step(p, x, 5e-4, "strang", 5)) < 3e-5
            finally:
                O.use_fft(False)


def test_fp64_config_small_100_steps(P):
    """65 x 65 in complex128, 100 Strang steps of 1e-3 (the small FP64 workload)."""
    p = W.config_small_1d()
    ctx = P.Context(p, "c128")
    psi = ctx.empty()
    ctx.init_gaussian(psi, [0.0], 2.0, [1.0])
    ctx.step(psi, 100, 1e-3, "strang")
    ref = O.step(p, O.gaussian_packet(p, [0.0], 2.0, [1.0]), 1e-3, "strang", 100)
    assert rel(ctx.to_dense(psi), ref) < 1e-11


def test_twisted_64_slices_one_step(P):
    """64^4 lifted box (twisted squares, 3 Gaussian wells per layer): one
    Strang step, compared on sampled output rows computed by the oracle... the
    step mixes all rows, so the oracle runs the full step with its FFT backend."""
    p = W.twisted_2d(q=64)
    ctx = P.Context(p, "c64")
    psi = ctx.empty()
    ctx.init_gaussian(psi, [0.0, 0.0], 2.0, [1.0, 0.0])
    x = ctx.to_dense(psi)
    ctx.step(psi, 1, 1e-3, "strang")
    O.use_fft(True)
    try:
        ref = O.step(p, x, 1e-3, "strang", 1)
    finally:
        O.use_fft(False)
    assert rel(ctx.to_dense(psi), ref) < 1e-5


@pytest.mark.parametrize("scheme", ["strang", "lie", "strang_kp", "yoshida4"])
def test_tensor_core_64x64_pass_parity(P, scheme, monkeypatch):
    """The layer pass of contiguous 64 x 64 slices with the DFTs as split-BF16
    matrix products on the tensor cores (fused Strang factors included):
    against the oracle on small other layers, within the complex64 tolerance."""
    monkeypatch.setenv("LSPLIT_TC2D", "1")
    import dataclasses
    base = W.twisted_2d(q=64, hmax=3)
    for p in [dataclasses.replace(base, lo2=(-4, -4), q2=(8, 8), ecut=1e9, name="tc-64x64-8x8"),
              dataclasses.replace(base, lo2=(-3, -2), q2=(8, 4), name="tc-64x64-cutoff")]:
        ctx = P.Context(p, "c64")
        x = W.random_state((p.M2, p.M1), 31)
        psi = ctx.from_dense(x)
        ctx.step(psi, 4, 1e-3, scheme)
        O.use_fft(True)
        try:
            ref = O.step(p, x, 1e-3, scheme, 4)
        finally:
            O.use_fft(False)
        assert rel(ctx.to_dense(psi), ref) < TOL1["c64"] * 3, (p.name, scheme, rel(ctx.to_dense(psi), ref))


def test_tensor_core_64x64_full_size_and_100_steps(P, monkeypatch):
    """64^4 twisted bilayer with the tensor-core layer pass: one Strang step
    from the packet against the oracle, and 100 steps of a random state on a
    64 x 64 x 8 x 8 box (rel-L2 and norm gates of the FP32 path)."""
    monkeypatch.setenv("LSPLIT_TC2D", "1")
    import dataclasses
    p = W.twisted_2d(q=64)
    ctx = P.Context(p, "c64")
    psi = ctx.empty()
    ctx.init_gaussian(psi, [0.0, 0.0], 2.0, [1.0, 0.0])
    x = ctx.to_dense(psi)
    ctx.step(psi, 1, 1e-3, "strang")
    O.use_fft(True)
    try:
        assert rel(ctx.to_dense(psi), O.step(p, x, 1e-3, "strang", 1)) < 1e-5
        q = dataclasses.replace(p, lo2=(-4, -4), q2=(8, 8), ecut=1e9, name="tc-100")
        c2 = P.Context(q, "c64")
        y = W.random_state((q.M2, q.M1), 32)
        py = c2.from_dense(y)
        c2.step(py, 100, 1e-3, "strang")
        got = c2.to_dense(py)
        assert rel(got, O.step(q, y, 1e-3, "strang", 100)) < 1e-4
        assert abs(np.linalg.norm(got) - 1) < 1e-5
    finally:
        O.use_fft(False)


def test_adjoint_parity(P):
    th1 = np.array([0.6, -0.3, 0.2])
    th2 = np.array([0.4, 0.25])
    base = W.bilayer_1d(16, 12, 0.0, 0.0, ecut=1e9)
    h1, c1 = W.cos_series_coeffs(th1)
    h2, c2 = W.cos_series_coeffs(th2)
    p = base.with_potentials(c1, c2, h1, h2)
    phi0 = O.gaussian_packet(p, [0.0], 0.8, [1.0])
    chi = O.gaussian_packet(p, [0.3], 0.8, [1.2])
    for scheme in ("strang", "lie", "strang_kp", "yoshida4", "lie_stoch", "strang_stoch"):
        L, phiT, g1, g2 = O.adjoint(p, phi0, 0.02, scheme, 6, lambda f: O.overlap_loss(chi, f), seed=5, step0=2)
        for dtype, tol in (("c64", 2e-5), ("c128", 1e-10)):
            ctx = P.Context(p, dtype)
            psi = ctx.from_dense(phiT)
            lam = ctx.from_dense(O.overlap_loss(chi, phiT)[1])
            gg1, gg2, gc1, gc2 = ctx.adjoint(psi, lam, 6, 0.02, scheme, seed=5, step0=2)
            sc = max(np.abs(g1).max(), np.abs(g2).max())
            assert np.abs(gg1 - g1).max() < tol * sc * 10, (scheme, dtype)
            assert np.abs(gg2 - g2).max() < tol * sc * 10, (scheme, dtype)
            assert rel(ctx.to_dense(psi), phi0) < tol * 10
            cg = O.coefficient_gradient(g1, h1, p.q1)
            assert np.abs(gc1 - cg).max() < tol * max(1, np.abs(cg).max()) * 10


def test_adjoint_round_trip_fast_and_64x64_passes(P):
    """Forward on the GPU through the fast 1D passes (slices of length 513)
    and the dedicated 64 x 64 passes, then the reverse sweep: the rebuilt state
    is the initial one and the gradients match the oracle's adjoint, for the
    fourth-order scheme (one kinetic unit per pass) and Strang."""
    import dataclasses
    th1 = np.array([0.5, -0.2])
    th2 = np.array([0.3, 0.15])
    h1, c1 = W.cos_series_coeffs(th1)
    h2, c2 = W.cos_series_coeffs(th2)
    p1 = W.bilayer_1d(256, 12, 0.0, 0.0, ecut=1e9).with_potentials(c1, c2, h1, h2)
    p2 = dataclasses.replace(W.twisted_2d(q=64, hmax=2), lo2=(-4, -4), q2=(8, 8), ecut=1e9, name="64x64-adj")
    O.use_fft(True)
    try:
        for p, n, tau in ((p1, 3, 5e-3), (p2, 2, 2e-3)):
            phi0 = W.random_state((p.M2, p.M1), 27)
            chi = W.random_state((p.M2, p.M1), 28)
            for scheme in ("yoshida4", "strang"):
                L, phiT, g1, g2 = O.adjoint(p, phi0, tau, scheme, n, lambda f: O.overlap_loss(chi, f))
                ctx = P.Context(p, "c64")
                psi = ctx.from_dense(phi0)
                ctx.step(psi, n, tau, scheme)
                assert rel(ctx.to_dense(psi), phiT) < 5e-5, (p.name, scheme)
                lam = ctx.from_dense(O.overlap_loss(chi, ctx.to_dense(psi))[1])
                gg1, gg2, _, _ = ctx.adjoint(psi, lam, n, tau, scheme)
                assert rel(ctx.to_dense(psi), phi0) < 1e-4, (p.name, scheme)
                sc = max(np.abs(g1).max(), np.abs(g2).max())
                assert np.abs(gg1 - g1).max() < 1e-3 * sc, (p.name, scheme)
                assert np.abs(gg2 - g2).max() < 1e-3 * sc, (p.name, scheme)
                # a later call on the context uses the call's own kinetic unit
                x = W.random_state((p.M2, p.M1), 29)
                y = ctx.from_dense(x)
                ctx.step(y, 1, tau, "strang_kp")
                assert rel(ctx.to_dense(y), O.step(p, x, tau, "strang_kp", 1)) < 1e-5
    finally:
        O.use_fft(False)


def test_error_codes(P):
    p = W.config_small_1d()
    ctx = P.Context(p, "c64")
    psi = ctx.empty()
    with pytest.raises(P.LsplitError) as e:
        ctx.step(psi, -1, 1e-3, "strang")
    assert e.value.code == P.LS_ERR_INVALID
    with pytest.raises(P.LsplitError):
        ctx.step(psi, 1, float("nan"), "strang")
    with pytest.raises(P.LsplitError):
        ctx.adjoint(psi, psi, 1, 1e-3, "cn_strang")
    with pytest.raises(P.LsplitError):
        ctx.adjoint(psi, psi, 1, 1e-3, "semi_implicit")


def example3_problems():
    """Example 3's three-index lift (periodic in y, incommensurate in x): the
    paper's potentials s1 cos^2(beta x) cos^2(pi y/2) + s2 cos^2(x) cos^2(pi y/2)
    with s = (1, 2) and (0.16, 8), boxes with a 2D (m, p) and (n, p) slice of
    several shapes, the cutoff Ec = 100 and every mode kept."""
    import dataclasses
    return [W.example3(8, 4, 4), W.example3(4, 8, 2, s1=0.16, s2=8.0),
            dataclasses.replace(W.example3(16, 2, 8), ecut=1e9, name="example3-32x4x16")]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("scheme", ["lie", "strang", "strang_kp", "yoshida4", "lie_stoch", "strang_stoch"])
def test_example3_three_index_parity(P, dtype, scheme):
    """Three-index lift on the GPU: layer factors over the (m, p) and (n, p)
    planes (2D slices sharing the y index), kinetic phases of
    |(G1 m + G2 n, G3 p)|^2 / 2, lazy phases of the stochastic schemes keyed
    by the other layer's x index; against the oracle."""
    for p in example3_problems():
        ctx = P.Context(p, dtype)
        x = W.random_state((p.M2, p.M1), 33)
        psi = ctx.from_dense(x)
        ctx.step(psi, 3, 5e-3, scheme, seed=2, step0=1)
        ref = O.step(p, x, 5e-3, scheme, 3, seed=2, step0=1)
        assert rel(ctx.to_dense(psi), ref) < TOL1[dtype] * 5, (p.name, scheme, rel(ctx.to_dense(psi), ref))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("scheme", ["lie", "strang", "strang_kp", "yoshida4", "strang_stoch"])
def test_trilayer_parity(P, dtype, scheme):
    """Three incommensurate 1D layers (workloads.trilayer_1d): layers 1 and 3
    act on different lifted indices and commute, so their factors run together
    on the (m, p) planes and layer 2 on the (n, p) planes; kinetic phases of
    (b1 m + b2 n + b3 p)^2 / 2.  16 x 16 x 8 and 64 x 64 x 64 boxes (the
    dedicated 64 x 64 passes), against the oracle."""
    O.use_fft(True)
    try:
        for p in (W.trilayer_1d(8, 8, 4), W.trilayer_1d(32, 32, 32, 1.4, 0.9, 1.1, ecut=400.0)):
            ctx = P.Context(p, dtype)
            x = W.random_state((p.M2, p.M1), 34)
            psi = ctx.from_dense(x)
            ctx.step(psi, 3, 2e-3, scheme, seed=3, step0=1)
            ref = O.step(p, x, 2e-3, scheme, 3, seed=3, step0=1)
            assert rel(ctx.to_dense(psi), ref) < TOL1[dtype] * 5, (p.name, scheme, rel(ctx.to_dense(psi), ref))
    finally:
        O.use_fft(False)


def test_example3_state_observables_and_adjoint(P):
    """Example 3: the packet initial state on the joint cutoff, observables
    (energy with both layer potentials on their (x, y) grids), the mass after
    200 Strang steps, the density at points of the plane, and the reverse
    sweep's gradients against the oracle's adjoint."""
    p = W.example3(8, 4, 4)
    for dtype, tol in (("c64", 1e-5), ("c128", 1e-11)):
        ctx = P.Context(p, dtype)
        psi = ctx.empty()
        ctx.init_gaussian(psi, [0.2, -0.3], 2.0, [1.0, 0.5])
        x = O.gaussian_packet(p, [0.2, -0.3], 2.0, [1.0, 0.5])
        assert rel(ctx.to_dense(psi), x) < tol
        o, r = ctx.observables(psi), O.observables(p, ctx.to_dense(psi))
        for k in ("norm", "ekin", "epot1", "epot2", "energy"):
            assert abs(o[k] - r[k]) < tol * 10 * max(1.0, abs(r[k])), (dtype, k, o[k], r[k])
        pts = np.array([[0.1, 0.2], [1.3, -0.7], [-2.5, 0.4]])
        assert rel(ctx.density(psi, pts), O.density_on_line(p, ctx.to_dense(psi), pts)) < tol
        ctx.step(psi, 200, 1e-3, "strang")
        got = ctx.to_dense(psi)
        assert rel(got, O.step(p, x, 1e-3, "strang", 200)) < (1e-4 if dtype == "c64" else 1e-10)
        assert abs(np.linalg.norm(got) - 1) < (1e-5 if dtype == "c64" else 1e-12)
        chi = O.gaussian_packet(p, [0.0, 0.0], 1.5, [0.5, 0.0])
        L, phiT, g1, g2 = O.adjoint(p, x, 1e-2, "strang", 4, lambda f: O.overlap_loss(chi, f))
        psi = ctx.from_dense(phiT)
        lam = ctx.from_dense(O.overlap_loss(chi, phiT)[1])
        gg1, gg2, _, _ = ctx.adjoint(psi, lam, 4, 1e-2, "strang")
        sc = max(np.abs(g1).max(), np.abs(g2).max())
        assert np.abs(gg1 - g1).max() < tol * 100 * sc and np.abs(gg2 - g2).max() < tol * 100 * sc, dtype
        assert rel(ctx.to_dense(psi), x) < tol * 10
