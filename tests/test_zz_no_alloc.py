"""ls_mass_noalloc: the mass without any allocation inside the library.

Callers that cannot allocate device memory (hosts whose device memory all
comes from their own pool, loops that must not touch the allocator) use this
entry point; its scratch is a fixed device array.  Checked
against the context-based ls_observables() on two calls in a row, within the
observables tolerance of the parity tests.  Collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,tol", [("c64", 1e-5), ("c128", 1e-11)])
def test_mass_noalloc_matches_observables(dtype, tol):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_14897_gb300 import build as B
    B.build()
    import paper_2103_14897_gb300 as P
    from paper_2103_14897_gb300._binding import mass_noalloc
    for p in [W.config_small_1d(), W.bilayer_1d(300, 700, 1.0, 0.5, ecut=1e9)]:
        ctx = P.Context(p, dtype)
        x = W.random_state((p.M2, p.M1), 17) * 1.7
        psi = ctx.from_dense(x)
        ref = ctx.observables(psi)["norm"]
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        for k in range(2):
            mass_noalloc(psi, dtype, ctx.rows, ctx.M1, ctx.pitch, out[k:k + 1])
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= tol * abs(ref)), (got, ref)
    # sizes beyond the fixed scratch are refused
    big = torch.zeros((65537, 16), dtype=torch.complex64, device="cuda")
    with pytest.raises(P.LsplitError) as e:
        mass_noalloc(big, "c64", 65537, 16, 16, out[:1])
    assert e.value.code == P.LS_ERR_INVALID
