"""Spectrum estimate of the global and the condensed matrices (Sec. 4, Fig.
ConditionNumber) through the C ABI against the oracle's dense eigenvalues."""
import numpy as np
import pytest

import oracle as O
import oracle.spectrum as SP
from gpu_common import case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,N,cfl", [(2, 2, 10.0), (2, 3, 10.0)])
def test_spectrum_estimate_matches_oracle_dense_eigenvalues(n, N, cfl):
    Q, dt, p, ctx = case(n, N, cfl=cfl, gmres_restart=60, gmres_max_iters=4000)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    ctx.sc_condense()
    ref = SP.condition_estimates(O.jacobian(p, Q), n, N)
    for which in ("A", "S"):
        got = ctx.sc_spectrum_estimate(which, m_max=60, m_min=60, inv_tol=1e-13)
        lmax, lmin, ratio = ref[which]
        assert abs(abs(got["lam_max"]) - abs(lmax)) <= 1e-6 * abs(lmax), (which, got, ref[which])
        assert abs(abs(got["lam_min"]) - abs(lmin)) <= 1e-6 * abs(lmin), (which, got, ref[which])
        assert abs(got["cond"] - ratio) <= 2e-6 * ratio, (which, got, ref[which])
        assert got["inner_iters"] > 0


def test_spectrum_estimate_needs_the_fp64_arm_and_a_condensed_system():
    from paper_1911_02366_gb300 import sc
    Q, dt, p, ctx = case(2, 2, gmres_restart=30)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    with pytest.raises(sc.SCError) as ei:
        ctx.sc_spectrum_estimate("S")
    assert ei.value.status == sc.SC_ERR_STATE
    ctx.sc_condense()
    with pytest.raises(sc.SCError) as ei:
        ctx.sc_spectrum_estimate("S", m_max=31)
    assert ei.value.status == sc.SC_ERR_ARG
