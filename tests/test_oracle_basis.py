"""Pins of the oracle's Gauss-Lobatto basis (App. C) against closed forms."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _ev(s):
    return eval(s, {"sqrt": math.sqrt})


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_gl_matches_closed_forms(N):
    g = json.load(open(os.path.join(GOLD, "gauss_lobatto.json")))["rules"][str(N)]
    xi, w, _ = O.gl(N)
    np.testing.assert_allclose(xi, [_ev(s) for s in g["nodes"]], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [_ev(s) for s in g["weights"]], rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_gl_quadrature_exact_to_degree_2N_minus_1(N):
    # The GL rule integrates polynomials up to degree 2N-1 exactly and no further
    # (the accuracy statement of Sec. 1).
    xi, w, _ = O.gl(N)
    for k in range(0, 2 * N):
        exact = (1 - (-1) ** (k + 1)) / (k + 1)
        assert abs(np.sum(w * xi ** k) - exact) < 1e-14
    k = 2 * N
    exact = 2.0 / (k + 1)
    assert abs(np.sum(w * xi ** k) - exact) > 1e-6


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6])
def test_derivative_matrix_exact_on_polynomials(N):
    xi, _, D = O.gl(N)
    for k in range(0, N + 1):
        d = D @ xi ** k
        ref = k * xi ** (k - 1) if k > 0 else np.zeros_like(xi)
        np.testing.assert_allclose(d, ref, atol=1e-12)


@pytest.mark.parametrize("N", [2, 4, 6])
def test_lagrange_discrete_orthogonality_and_derivative(N):
    xi, _, _ = O.gl(N)
    for i in range(N + 1):
        for j in range(N + 1):
            v, _ = O.lagrange(N, i, xi[j])
            assert v == (1.0 if i == j else 0.0)
        # derivative against a central difference of the value at off-node points
        for x in (-0.77, 0.13, 0.91):
            h = 1e-6
            vp, _ = O.lagrange(N, i, x + h)
            vm, _ = O.lagrange(N, i, x - h)
            _, d = O.lagrange(N, i, x)
            assert abs(d - (vp - vm) / (2 * h)) < 1e-7 * max(1.0, abs(d))


@pytest.mark.parametrize("N", [2, 3, 5])
def test_summation_by_parts(N):
    # W D + (W D)^T = diag(-1, 0, ..., 0, 1): the SBP property of the GL-DGSEM.
    _, w, D = O.gl(N)
    Q = np.diag(w) @ D
    B = np.zeros((N + 1, N + 1)); B[0, 0] = -1; B[N, N] = 1
    np.testing.assert_allclose(Q + Q.T, B, atol=1e-13)
