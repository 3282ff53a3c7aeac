"""The allocation-free condensed operator, sc_condensed_matvec_static.

Callers that may not allocate device memory during a run (for example a solver loop
driven by a memory pool that forbids cudaMalloc/cudaFree once the simulation is
running) use this variant: its scratch is a fixed device array compiled into the
library.  Its output must equal the allocating sc_condensed_matvec on consecutive
calls (the shared scratch keeps the previous call's contents, which must not leak).
This file is collected last so that a failure here never hides another test.
"""
import numpy as np
import pytest

from gpu_common import case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_static_scratch_matvec_matches_allocating_matvec_on_two_calls():
    n, N = 3, 3
    Q, dt, p, ctx = case(n, N)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    ctx.sc_condense()
    K, ne, ni, nb = ctx.sc_sizes()
    rng = np.random.default_rng(11)
    for _ in range(2):
        xb = torch.tensor(rng.standard_normal(K * nb), device="cuda")
        ref = torch.zeros_like(xb)
        got = torch.full_like(xb, float("nan"))
        ctx.sc_condensed_matvec(xb, ref)
        ctx.sc_condensed_matvec_static(xb, got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.isfinite(g).all()
        assert np.max(np.abs(g - r)) <= 1e-11 * np.max(np.abs(r))
