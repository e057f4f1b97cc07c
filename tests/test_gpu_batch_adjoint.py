"""Batched persistent runner and the autograd wrapper of the reverse sweep,
against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests._parity import rel

pytestmark = pytest.mark.gpu


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




def uneven_batch():
    # uneven boxes of the batched workload's kind (odd lengths, L2/L1 drawn,
    # cos potentials), small enough for the oracle
    return W.batch_1d(count=7, seed=4, nmin=3, nmax=40) + [W.bilayer_1d(64, 3, 1.0, 0.7, ecut=1e9)]


@pytest.mark.parametrize("form", ["compact", "fft"])
@pytest.mark.parametrize("dtype,tol", [("c64", 1e-5), ("c128", 1e-11)])
@pytest.mark.parametrize("scheme", ["strang", "lie", "strang_kp"])
def test_batched_runner_parity(P, dtype, tol, scheme, form, monkeypatch):
    if form == "fft":
        monkeypatch.setenv("LSPLIT_NO_STENCIL", "1")
    probs = uneven_batch()
    b = P.Batch(probs, dtype)
    psi = b.empty()
    xs = [W.random_state((p.M2, p.M1), 40 + i) for i, p in enumerate(probs)]
    for i, x in enumerate(xs):
        b.set_dense(psi, i, x)
    b.step(psi, 3, 1e-2, scheme)
    for i, p in enumerate(probs):
        ref = O.step(p, xs[i], 1e-2, scheme, 3)
        assert rel(b.get_dense(psi, i), ref) < tol * 3, (i, p.name, rel(b.get_dense(psi, i), ref))
    # single step (the "only step" units) and a second call continuing
    b.step(psi, 1, 1e-2, scheme)
    for i, p in enumerate(probs):
        ref = O.step(p, O.step(p, xs[i], 1e-2, scheme, 3), 1e-2, scheme, 1)
        assert rel(b.get_dense(psi, i), ref) < tol * 4


def test_batched_full_workload_sampled(P):
    """The 256-instance workload the bench times (67.4 M DOF, box half-widths
    16..512), Gaussian packets, Strang tau = 1e-3 through the tuned compact-only
    kernel in the interaction frame: after one call of 10 steps, sampled
    instances (first, middle, last, largest) against the oracle (rel-L2 <=
    3e-5); after 1000 steps (100 calls), the three smallest instances against
    the oracle (rel-L2 <= 1e-4) and every instance's norm within 1e-5."""
    probs = W.batch_1d(count=256, seed=4)
    b = P.Batch(probs, "c64")
    psi = b.empty()
    b.init_gaussian(psi, [0.0], 2.0, [1.0])
    dof = [p.M1 * p.M2 for p in probs]
    big = int(np.argmax(dof))
    small = [int(i) for i in np.argsort(dof)[:3]]
    sample = sorted({0, 128, 255, big})
    x0 = {i: b.get_dense(psi, i) for i in sample + small}
    O.use_fft(True)
    try:
        b.step(psi, 10, 1e-3, "strang")
        for i in sample:
            ref = O.step(probs[i], x0[i], 1e-3, "strang", 10)
            assert rel(b.get_dense(psi, i), ref) < 3e-5, (i, rel(b.get_dense(psi, i), ref))
        for _ in range(99):
            b.step(psi, 10, 1e-3, "strang")
        for i in small:
            ref = O.step(probs[i], x0[i], 1e-3, "strang", 1000)
            got = b.get_dense(psi, i)
            print(probs[i].name, "1000-step rel-L2", rel(got, ref))
            assert rel(got, ref) < 1e-4, (i, rel(got, ref))
    finally:
        O.use_fft(False)
    norms = np.array([o["norm"] for o in b.observables(psi)])
    assert np.abs(norms - 1).max() < 1e-5, np.abs(norms - 1).max()


@pytest.mark.parametrize("scheme", ["strang", "lie", "strang_kp"])
def test_batched_interaction_frame_long_call(P, scheme):
    """Deterministic complex64 calls of the compact-only kernel run in the
    interaction frame: one call of 300 steps (Lambda raised to the 300th power,
    the exact K(T) once at the end) on Gaussian packets, then a second call of
    1 step, against the oracle: rel-L2 <= 1e-4 and the norm within 1e-5."""
    probs = uneven_batch()
    b = P.Batch(probs, "c64")
    psi = b.empty()
    xs = [O.gaussian_packet(p, [0.0], 2.0, [1.0]) for p in probs]
    for i, x in enumerate(xs):
        b.set_dense(psi, i, x)
    b.step(psi, 300, 1e-3, scheme)
    b.step(psi, 1, 1e-3, scheme)
    for i, p in enumerate(probs):
        ref = O.step(p, xs[i], 1e-3, scheme, 301)
        got = b.get_dense(psi, i)
        assert rel(got, ref) < 1e-4, (i, p.name, rel(got, ref))
        assert abs(np.linalg.norm(got) - 1) < 1e-5


@pytest.mark.parametrize("form", ["compact", "fft"])
@pytest.mark.parametrize("dtype,tol", [("c64", 1e-5), ("c128", 1e-11)])
@pytest.mark.parametrize("scheme", ["strang_stoch", "lie_stoch"])
def test_batched_runner_stochastic_parity(P, dtype, tol, scheme, form, monkeypatch):
    if form == "fft":
        monkeypatch.setenv("LSPLIT_NO_STENCIL", "1")
    """Stochastic schemes inside the persistent launch: instance i samples with
    seed + i; lists drawn on the device; lazy kinetic phases and a settle phase."""
    probs = uneven_batch()
    b = P.Batch(probs, dtype)
    psi = b.empty()
    xs = [W.random_state((p.M2, p.M1), 60 + i) for i, p in enumerate(probs)]
    for i, x in enumerate(xs):
        b.set_dense(psi, i, x)
    b.step(psi, 3, 1e-2, scheme, seed=9, step0=4)
    refs = [O.step(p, xs[i], 1e-2, scheme, 3, seed=9 + i, step0=4) for i, p in enumerate(probs)]
    for i, p in enumerate(probs):
        assert rel(b.get_dense(psi, i), refs[i]) < tol * 3, (i, p.name, rel(b.get_dense(psi, i), refs[i]))
    b.step(psi, 2, 1e-2, scheme, seed=9, step0=7)
    for i, p in enumerate(probs):
        ref = O.step(p, refs[i], 1e-2, scheme, 2, seed=9 + i, step0=7)
        assert rel(b.get_dense(psi, i), ref) < tol * 5


@pytest.mark.parametrize("scheme", ["strang", "lie", "strang_stoch"])
@pytest.mark.parametrize("form", ["compact", "fft"])
def test_batched_fast_tiles_parity(P, scheme, form, monkeypatch):
    """Lengths 129..1001 (transforms of 256..2048 points): every slice runs on
    the compact-kernel tiles, or (transform form) most on the register-resident
    fast tiles inside the persistent launch."""
    if form == "fft":
        monkeypatch.setenv("LSPLIT_NO_STENCIL", "1")
    probs = W.batch_1d(count=5, seed=8, nmin=64, nmax=500)
    b = P.Batch(probs, "c64")
    psi = b.empty()
    xs = [W.random_state((p.M2, p.M1), 70 + i) for i, p in enumerate(probs)]
    for i, x in enumerate(xs):
        b.set_dense(psi, i, x)
    b.step(psi, 3, 1e-3, scheme, seed=5, step0=1)
    O.use_fft(True)
    try:
        for i, p in enumerate(probs):
            ref = O.step(p, xs[i], 1e-3, scheme, 3, seed=5 + i, step0=1)
            assert rel(b.get_dense(psi, i), ref) < 3e-5, (i, p.name, rel(b.get_dense(psi, i), ref))
    finally:
        O.use_fft(False)


@pytest.mark.parametrize("cfg", ["256,3", "256,4", "128,6", "128,8", "128,6,2", "256,3,4"])
def test_batched_compact_configurations_parity(P, cfg, monkeypatch):
    """Every launch configuration of the compact-kernel batched kernel (threads
    per CTA, CTAs per SM and the tile widths they imply) against the oracle,
    deterministic and stochastic."""
    monkeypatch.setenv("LSPLIT_STENCIL_CFG", cfg)
    probs = uneven_batch()
    b = P.Batch(probs, "c64")
    want = [int(v) for v in cfg.split(",")] + [1]
    assert (b.config()["threads"], b.config()["ctas_per_sm"], b.config()["tiles_per_item"]) == tuple(want[:3])
    xs = [W.random_state((p.M2, p.M1), 90 + i) for i, p in enumerate(probs)]
    for scheme in ("strang", "strang_stoch"):
        psi = b.empty()
        for i, x in enumerate(xs):
            b.set_dense(psi, i, x)
        b.step(psi, 3, 1e-2, scheme, seed=4, step0=1)
        for i, p in enumerate(probs):
            ref = O.step(p, xs[i], 1e-2, scheme, 3, seed=4 + i, step0=1)
            assert rel(b.get_dense(psi, i), ref) < 3e-5, (cfg, scheme, i, rel(b.get_dense(psi, i), ref))


def test_batched_autotuner_never_slower_than_default(P, monkeypatch):
    """The autotuner times the compact-kernel configurations and the transform
    forms on the first call and keeps the fastest: on the batched workload's
    length classes (half-widths 16..512) the tuned launch is not slower than
    the untuned default configuration (256 threads, 3 CTAs per SM), and both
    give the same states."""
    import torch
    monkeypatch.delenv("LSPLIT_TUNE", raising=False)
    monkeypatch.delenv("LSPLIT_STENCIL_CFG", raising=False)
    probs = W.batch_1d(count=48, seed=4)
    bt = P.Batch(probs, "c64")
    pt = bt.empty()
    bt.init_gaussian(pt, [0.0], 2.0, [1.0])
    bt.step(pt, 4, 1e-3, "strang")
    cfg = bt.config()
    assert cfg["tuned"] and len(cfg["tune_ms"]) == 8, cfg
    assert min(cfg["tune_ms"]) > 0
    monkeypatch.setenv("LSPLIT_STENCIL_CFG", "256,3")
    bd = P.Batch(probs, "c64")
    pd = bd.empty()
    bd.init_gaussian(pd, [0.0], 2.0, [1.0])
    bd.step(pd, 4, 1e-3, "strang")
    assert not bd.config()["tuned"]
    assert rel(bt.get_dense(pt, 5), bd.get_dense(pd, 5)) < 3e-6

    def timed(b, psi):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        b.step(psi, 4, 1e-3, "strang")
        ev[0].record()
        for _ in range(5):
            b.step(psi, 4, 1e-3, "strang")
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1])
    t_tuned = min(timed(bt, pt) for _ in range(2))
    t_default = min(timed(bd, pd) for _ in range(2))
    print("tuned", cfg, t_tuned, "default", t_default)
    assert t_tuned <= 1.05 * t_default, (cfg, t_tuned, t_default)


def test_batched_fused_walk_matches_unfused(P, monkeypatch):
    """Deterministic Strang in the persistent launch fuses adjacent layer-1
    factors of consecutive steps (fused tiles for the convolution-form
    instances, back-to-back factors for the others); the state is the same
    as with the plain walk."""
    import torch
    probs = W.batch_1d(count=6, seed=12, nmin=40, nmax=400)
    outs = []
    for flag in (None, "1"):
        if flag:
            monkeypatch.setenv("LSPLIT_NO_FUSE", flag)
        else:
            monkeypatch.delenv("LSPLIT_NO_FUSE", raising=False)
        b = P.Batch(probs, "c64")
        psi = b.empty()
        b.init_gaussian(psi, [0.0], 2.0, [1.0])
        b.step(psi, 5, 1e-3, "strang")
        outs.append(psi)
    assert float(torch.linalg.vector_norm(outs[0] - outs[1])) <= 1e-6 * float(torch.linalg.vector_norm(outs[1]))


def test_batched_matches_single_contexts(P):
    """The same instances stepped one context at a time agree with the batch."""
    probs = W.batch_1d(count=5, seed=11, nmin=8, nmax=300)
    b = P.Batch(probs, "c64")
    psi = b.empty()
    b.init_gaussian(psi, [0.0], 2.0, [1.0])
    b.step(psi, 10, 1e-3, "strang")
    obs = b.observables(psi)
    for i, p in enumerate(probs):
        c = P.Context(p, "c64")
        x = c.empty()
        c.init_gaussian(x, [0.0], 2.0, [1.0])
        c.step(x, 10, 1e-3, "strang")
        assert rel(b.get_dense(psi, i), c.to_dense(x)) < 2e-6
        assert abs(obs[i]["norm"] - 1) < 1e-5


def test_batched_wait_timeout_is_reported_and_recoverable(P):
    """A dependency that nothing satisfies makes the bounded wait expire: the
    call returns LS_ERR_TIMEOUT and the batch works again afterwards."""
    probs = W.batch_1d(count=3, seed=2, nmin=4, nmax=20)
    b = P.Batch(probs, "c64")
    psi = b.empty()
    b.debug(True, 0.2)
    with pytest.raises(P.LsplitError) as e:
        b.step(psi, 2, 1e-2, "strang")
    assert e.value.code == P.LS_ERR_TIMEOUT
    b.debug(False, 1.0)
    xs = [W.random_state((p.M2, p.M1), 50 + i) for i, p in enumerate(probs)]
    for i, x in enumerate(xs):
        b.set_dense(psi, i, x)
    b.step(psi, 2, 1e-2, "strang")
    for i, p in enumerate(probs):
        assert rel(b.get_dense(psi, i), O.step(p, xs[i], 1e-2, "strang", 2)) < 3e-5


def test_autograd_overlap_gradient_matches_oracle(P):
    import torch
    from paper_2103_14897_gb300.autograd import overlap_loss
    base = W.bilayer_1d(20, 16, 0.0, 0.0, ecut=1e9)
    th1 = np.array([0.6, -0.3, 0.2, 0.1])
    th2 = np.array([0.4, 0.25, -0.1])
    phi0 = O.gaussian_packet(base, [0.0], 0.8, [1.0])
    chi = O.gaussian_packet(base, [0.3], 0.8, [1.2])
    h1, c1 = W.cos_series_coeffs(th1)
    h2, c2 = W.cos_series_coeffs(th2)
    prob = base.with_potentials(c1, c2, h1, h2)
    Lref, _, g1, g2 = O.adjoint(prob, phi0, 0.02, "strang", 8, lambda f: O.overlap_loss(chi, f))
    cg1 = O.coefficient_gradient(g1, h1, prob.q1)
    cg2 = O.coefficient_gradient(g2, h2, prob.q2)
    ref1 = 0.5 * (cg1[0::2, 0] + cg1[1::2, 0])
    ref2 = 0.5 * (cg2[0::2, 0] + cg2[1::2, 0])
    for dtype, tol in (("c64", 1e-5), ("c128", 1e-10)):
        for ck in (0, 3):
            t1 = torch.tensor(th1, requires_grad=True)
            t2 = torch.tensor(th2, requires_grad=True)
            L = overlap_loss(t1, t2, base, phi0, chi, 0.02, 8, "strang", dtype, checkpoint_every=ck)
            L.backward()
            assert abs(float(L.detach()) - Lref) < tol * 10
            sc = max(np.abs(ref1).max(), np.abs(ref2).max())
            assert np.abs(t1.grad.numpy() - ref1).max() < tol * sc * 20, (dtype, ck)
            assert np.abs(t2.grad.numpy() - ref2).max() < tol * sc * 20, (dtype, ck)


def test_autograd_backward_twice_and_stochastic(P):
    """A second backward (retain_graph=True) gives the same gradients as the
    first; the stochastic schemes differentiate with the forward call's
    samples (Algorithm 4), against the oracle's adjoint with the same seed."""
    import torch
    from paper_2103_14897_gb300.autograd import overlap_loss
    base = W.bilayer_1d(20, 16, 0.0, 0.0, ecut=1e9)
    th1 = np.array([0.6, -0.3, 0.2])
    th2 = np.array([0.4, 0.25])
    phi0 = O.gaussian_packet(base, [0.0], 0.8, [1.0])
    chi = O.gaussian_packet(base, [0.3], 0.8, [1.2])
    h1, c1 = W.cos_series_coeffs(th1)
    h2, c2 = W.cos_series_coeffs(th2)
    prob = base.with_potentials(c1, c2, h1, h2)
    for scheme, ck in (("strang", 3), ("strang", 0), ("strang_stoch", 4), ("lie_stoch", 0)):
        Lref, _, g1, g2 = O.adjoint(prob, phi0, 0.02, scheme, 9, lambda f: O.overlap_loss(chi, f), seed=6)
        cg1 = O.coefficient_gradient(g1, h1, prob.q1)
        cg2 = O.coefficient_gradient(g2, h2, prob.q2)
        ref1 = 0.5 * (cg1[0::2, 0] + cg1[1::2, 0])
        ref2 = 0.5 * (cg2[0::2, 0] + cg2[1::2, 0])
        sc = max(np.abs(ref1).max(), np.abs(ref2).max())
        t1 = torch.tensor(th1, requires_grad=True)
        t2 = torch.tensor(th2, requires_grad=True)
        L = overlap_loss(t1, t2, base, phi0, chi, 0.02, 9, scheme, "c64", checkpoint_every=ck, seed=6)
        assert abs(float(L.detach()) - Lref) < 1e-4
        a1, a2 = torch.autograd.grad(L, (t1, t2), retain_graph=True)
        b1, b2 = torch.autograd.grad(L, (t1, t2))
        assert np.abs(a1.numpy() - ref1).max() < 2e-4 * sc, (scheme, ck)
        assert np.abs(a2.numpy() - ref2).max() < 2e-4 * sc, (scheme, ck)
        # same sweep from phi_T again (the gradient's atomic accumulation
        # order is not fixed, so agreement is to rounding, not bitwise)
        np.testing.assert_allclose(b1.numpy(), a1.numpy(), rtol=1e-9, atol=1e-12 * sc)
        np.testing.assert_allclose(b2.numpy(), a2.numpy(), rtol=1e-9, atol=1e-12 * sc)


def test_autograd_reduced_box_500_steps_against_oracle(P):
    """The adjoint workload's potentials (8 cosine coefficients per layer,
    N(0, 0.5), seed 5) and 500 steps of tau = 1e-3 on a reduced 65 x 65 box:
    the FP32 reverse sweep with drift-placed checkpoints against the oracle's
    trajectory-storing FP64 adjoint."""
    import torch
    from paper_2103_14897_gb300.autograd import overlap_loss
    _, th1, th2 = W.config_adjoint_1d()
    base = W.bilayer_1d(32, 32, 0.0, 0.0)
    h1, c1 = W.cos_series_coeffs(th1)
    h2, c2 = W.cos_series_coeffs(th2)
    prob = base.with_potentials(c1, c2, h1, h2)
    phi0 = O.gaussian_packet(base, [0.0], 2.0, [1.0])
    chi = O.gaussian_packet(base, [0.5], 2.0, [1.2])
    Lref, _, g1, g2 = O.adjoint(prob, phi0, 1e-3, "strang", 500, lambda f: O.overlap_loss(chi, f))
    cg1 = O.coefficient_gradient(g1, h1, prob.q1)
    cg2 = O.coefficient_gradient(g2, h2, prob.q2)
    ref = np.concatenate([0.5 * (cg1[0::2, 0] + cg1[1::2, 0]), 0.5 * (cg2[0::2, 0] + cg2[1::2, 0])])
    t1 = torch.tensor(th1, requires_grad=True)
    t2 = torch.tensor(th2, requires_grad=True)
    L = overlap_loss(t1, t2, base, phi0, chi, 1e-3, 500, "strang", "c64", drift_tol=1e-5)
    L.backward()
    got = np.concatenate([t1.grad.numpy(), t2.grad.numpy()])
    assert abs(float(L.detach()) - Lref) < 1e-4 * max(1.0, Lref)
    assert np.abs(got - ref).max() < 1e-3 * np.abs(ref).max(), (got, ref)


def test_autograd_adjoint_workload_central_differences(P):
    """513 x 513 box, 8 cosine coefficients per layer (N(0, 0.5), seed 5),
    overlap loss after 500 steps of tau = 1e-3: the FP32 reverse-sweep gradient
    against central differences (h = 1e-4) of the FP64 GPU forward."""
    import torch
    from paper_2103_14897_gb300.autograd import overlap_loss
    prob, th1, th2 = W.config_adjoint_1d()
    base = prob
    phi0 = O.gaussian_packet(base, [0.0], 2.0, [1.0])
    chi = O.gaussian_packet(base, [0.5], 2.0, [1.2])
    from paper_2103_14897_gb300.autograd import checkpoint_plan
    # drift-placed checkpoints against the fixed policy (every 100 steps)
    grads = {}
    for name, kw in (("fixed", {"checkpoint_every": 100}), ("drift", {"drift_tol": 1e-4})):
        t1 = torch.tensor(th1, requires_grad=True)
        t2 = torch.tensor(th2, requires_grad=True)
        L = overlap_loss(t1, t2, base, phi0, chi, 1e-3, 500, "strang", "c64", **kw)
        L.backward()
        grads[name] = (t1.grad.numpy().copy(), t2.grad.numpy().copy())
    c = P.Context(prob, "c64")
    marks, d, probe = checkpoint_plan(c, c.from_dense(phi0), 500, 1e-3, "strang", drift_tol=1e-4)
    print("drift-placed checkpoints", marks, "probe drift", d, "over", probe, "steps")
    assert len(marks) < 4
    h = 1e-4

    def f(a, b):
        return float(overlap_loss(torch.tensor(a), torch.tensor(b), base, phi0, chi, 1e-3, 500, "strang", "c128"))
    fd1, fd2 = [], []
    for i in (0, 3, 7):
        a, b = th1.copy(), th1.copy()
        a[i] += h
        b[i] -= h
        fd1.append((f(a, th2) - f(b, th2)) / (2 * h))
    for i in (1, 6):
        a, b = th2.copy(), th2.copy()
        a[i] += h
        b[i] -= h
        fd2.append((f(th1, a) - f(th1, b)) / (2 * h))
    scale = max(np.abs(fd1).max(), np.abs(fd2).max(), 1e-6)
    for name, (a1, a2) in grads.items():
        got1 = a1[[0, 3, 7]]
        got2 = a2[[1, 6]]
        assert np.abs(got1 - fd1).max() < 1e-3 * scale + 1e-7, (name, got1, fd1)
        assert np.abs(got2 - fd2).max() < 1e-3 * scale + 1e-7, (name, got2, fd2)
