"""Pins of the spectrum oracle (oracle/spectrum.py): the condition-number estimate of
Sec. 4 (Fig. ConditionNumber) in the limit where the mass matrix dominates."""
import numpy as np
import pytest

import oracle as O
import oracle.spectrum as SP
import sc_inputs as I


def _limit(N, dt, n=2):
    Q, _ = I.tgv_state(n, N, cfl=10.0, seed=0)
    p = O.Params(n=n, N=N, dt=dt)
    return p, SP.condition_estimates(O.jacobian(p, Q), n, N)


@pytest.mark.parametrize("N", [2, 3])
def test_small_time_step_reduces_the_estimates_to_gauss_lobatto_weight_ratios(N):
    """As dt -> 0 the backward-Euler term M/dt dominates A (M = J w_i w_j w_k, diagonal):
    |lambda_max| -> J w_max^3 / dt, |lambda_min| -> J w_min^3 / dt, so the ratio of A tends
    to (w_max / w_min)^3.  The condensed S = A_bb - A_bi A_ii^-1 A_ib tends to M_bb / dt, whose
    nodes all carry at least one end weight w_min: its ratio tends to (w_max / w_min)^2.
    Closed forms: N = 2 has w = 1/3, 4/3, 1/3 (ratios 64 and 16); N = 3 has w = 1/6, 5/6
    (ratios 125 and 25)."""
    dt = 1e-9
    p, est = _limit(N, dt)
    wmax, wmin = {2: (4 / 3, 1 / 3), 3: (5 / 6, 1 / 6)}[N]
    J = (p.L / p.n / 2.0) ** 3
    lmax_A, lmin_A, rA = est["A"]
    lmax_S, lmin_S, rS = est["S"]
    assert abs(abs(lmax_A) - J * wmax ** 3 / dt) <= 1e-5 * J * wmax ** 3 / dt
    assert abs(abs(lmin_A) - J * wmin ** 3 / dt) <= 1e-5 * J * wmin ** 3 / dt
    assert abs(rA - (wmax / wmin) ** 3) <= 1e-4 * (wmax / wmin) ** 3
    assert abs(abs(lmax_S) - J * wmax ** 2 * wmin / dt) <= 1e-5 * J * wmax ** 2 * wmin / dt
    assert abs(rS - (wmax / wmin) ** 2) <= 1e-4 * (wmax / wmin) ** 2


def test_extremes_are_the_largest_and_smallest_moduli():
    # a similarity transform of a known spectrum, including a complex pair
    rng = np.random.default_rng(1)
    D = np.zeros((6, 6))
    D[0, 0], D[1, 1] = 7.0, -0.25
    D[2:4, 2:4] = [[1.0, 2.0], [-2.0, 1.0]]  # 1 +- 2i
    D[4, 4], D[5, 5] = 3.0, -6.5
    T = rng.standard_normal((6, 6)) + 6 * np.eye(6)
    lmax, lmin, r = SP.extreme_eigenvalues(T @ D @ np.linalg.inv(T))
    assert abs(lmax - 7.0) < 1e-10 and abs(lmin + 0.25) < 1e-10 and abs(r - 28.0) < 1e-9
