"""The seeded input generator shared by both sides of every parity check."""
import numpy as np

import sc_inputs as I


def test_splitmix64_reference_value():
    # splitmix64 with state 0 returns 0xE220A8397B1DCDAF (Steele, Lea & Flood 2014).
    assert int(I.splitmix64(0, np.array([0]))[0]) == 0xE220A8397B1DCDAF


def test_uniform_range_and_determinism():
    u = I.uniform_pm1(7, np.arange(100000, dtype=np.uint64))
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01
    np.testing.assert_array_equal(u[123:456], I.uniform_pm1(7, np.arange(123, 456, dtype=np.uint64)))


def test_tgv_state_is_isothermal_and_divergence_free_sampled():
    Q, dt = I.tgv_state(2, 3, eps=0.0)
    rho = Q[..., 0]
    u = Q[..., 1] / rho
    assert np.all(rho > 0) and dt > 0
    xyz = I.node_coordinates(2, 3)
    np.testing.assert_allclose(u, np.sin(xyz[..., 0]) * np.cos(xyz[..., 1]) * np.cos(xyz[..., 2]), atol=1e-14)


def test_lobatto_points_are_symmetric():
    for N in range(1, 8):
        x = I.lobatto_points(N)
        np.testing.assert_allclose(x, -x[::-1], atol=0)
        assert x[0] == -1.0 and x[-1] == 1.0


def test_mixed_order_inputs_reduce_to_the_uniform_ones():
    # one order everywhere: same nodes, same state, same perturbation counters, same dt
    n, N = 3, 3
    orders = np.full(n ** 3, N)
    np.testing.assert_array_equal(I.node_coordinates_mixed(n, orders), I.node_coordinates(n, N).reshape(-1, 3))
    Qm, dtm = I.tgv_state_mixed(n, orders, seed=4)
    Q, dt = I.tgv_state(n, N, seed=4)
    np.testing.assert_array_equal(Qm, Q.reshape(-1, 5))
    assert dtm == dt
    np.testing.assert_array_equal(I.uniform_state_mixed(n, orders), I.uniform_state(n, N).reshape(-1, 5))


def test_mixed_order_coordinates_follow_each_elements_order():
    n = 2
    orders = np.array([2, 3, 4, 5, 6, 2, 3, 4])
    xyz = I.node_coordinates_mixed(n, orders)
    assert xyz.shape == (sum((N + 1) ** 3 for N in orders), 3)
    off = 0
    for e, N in enumerate(orders):
        blk = xyz[off:off + (N + 1) ** 3]
        np.testing.assert_array_equal(blk, I.node_coordinates(n, int(N))[e])
        off += (N + 1) ** 3
