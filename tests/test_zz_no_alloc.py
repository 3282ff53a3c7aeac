"""The allocation-free condensed operator, sc_condensed_matvec_static.

Callers that may not allocate device memory during a run (for example a solver loop
driven by a memory pool that forbids cudaMalloc/cudaFree once the simulation is
running) use this variant: its scratch is a fixed device array compiled into the
library.  Its output must equal the allocating sc_condensed_matvec, and the oracle's
dense condensed matrix S, on consecutive calls (the shared scratch keeps the previous
call's contents, which must not leak); device memory must not change across its calls;
and a mesh beyond the array's size must be refused with a clear error.
This file is collected last so that a failure here never hides another test.
"""
import numpy as np
import pytest

import oracle as O
from gpu_common import TWO_PI, case, gpu_context

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _system(n, N, **cfg):
    Q, dt, p, ctx = case(n, N, **cfg)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    ctx.sc_condense()
    return Q, p, ctx


def _oracle_S(p, Q, n, N):
    """Dense S of the oracle in the condensed order (element-major, boundary nodes in
    natural order, 5 variables) -- the same order as the library's boundary vectors."""
    return O.condensed_operator(O.jacobian(p, Q), n, N).dense_S()


@pytest.mark.parametrize("mixed", [False, True])
def test_static_scratch_matvec_matches_allocating_matvec_and_oracle_on_two_calls(mixed):
    from paper_1911_02366_gb300 import sc
    n, N = 3, 3
    cfg = dict(precision=sc.SC_PREC_MIXED) if mixed else {}
    Q, p, ctx = _system(n, N, **cfg)
    K, ne, ni, nb = ctx.sc_sizes()
    S = _oracle_S(p, Q, n, N)
    rng = np.random.default_rng(11)
    xs = [torch.tensor(rng.standard_normal(K * nb), device="cuda") for _ in range(2)]
    refs = [torch.zeros_like(x) for x in xs]
    gots = [torch.full_like(x, float("nan")) for x in xs]
    ctx.sc_condensed_matvec_static(xs[0], gots[0])  # first call: may load device code
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for x, r, g in zip(xs, refs, gots):
        ctx.sc_condensed_matvec(x, r)
        ctx.sc_condensed_matvec_static(x, g)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "device memory changed across the calls"
    for x, r, g in zip(xs, refs, gots):
        r, g, xn = r.cpu().numpy(), g.cpu().numpy(), x.cpu().numpy()
        assert np.isfinite(g).all()
        # same operator passes, same arithmetic
        assert np.max(np.abs(g - r)) <= 1e-12 * np.max(np.abs(r))
        y = S @ xn
        tol = 1e-4 if mixed else 1e-11  # FP32 blocks on the mixed arm
        assert np.max(np.abs(g - y)) <= tol * np.max(np.abs(y))


def test_static_scratch_matvec_refuses_a_mesh_beyond_its_array():
    from paper_1911_02366_gb300 import sc
    # FP64 arm at N = 4: 20^3 elements x 135 interior dofs = 1,080,000 doubles > 1,048,576
    ctx = gpu_context()
    ctx.sc_set_mesh(20, TWO_PI, 4)
    K, ne, ni, nb = ctx.sc_sizes()
    assert K * ni > (8 << 20) // 8
    x = torch.zeros(K * nb, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(sc.SCError) as ei:
        ctx.sc_condensed_matvec_static(x, y)
    assert ei.value.status == sc.SC_ERR_ARG
    assert "static buffer" in str(ei.value)
