"""Pins of the oracle's overrelaxation step (Sec. 2.2: the alternative to the
exact SU(2) update in the heatbath figure).

The reflection of an SU(2) subgroup is fixed by what it must do, not by its
formula: the subgroup block of U A keeps its real trace and has its quaternion
part conjugated (w_hat -> w_hat^+), reflecting twice with the same staple is
the identity, the link stays in SU(3), and a sweep leaves the Wilson action
unchanged while moving the links by O(1).  A dropped dagger, a product on the
wrong side or a wrong subgroup embedding fails at least one of these.
"""
import numpy as np

from paper_1209_5942_gb300 import inputs

SUBGROUPS = [(0, 1), (1, 2), (0, 2)]


def _quaternion(W, p, q):
    """(q0, q1, q2, q3) of the real-quaternion part of block (p, q) of W,
    block = [[q0 + i q3, q2 + i q1], [-q2 + i q1, q0 - i q3]] + i (another one)."""
    a, b, c, d = W[p, p], W[p, q], W[q, p], W[q, q]
    return np.array([0.5 * (a + d).real, 0.5 * (b + c).imag, 0.5 * (b - c).real, 0.5 * (a - d).imag])


def _link_and_staple(oracle, seed):
    L = (2, 4, 2, 4)
    U = inputs.random_gauge(L, "near", seed=seed, eps=0.9)
    i, mu = 9, 2
    return U, L, i, mu, U[i, mu].copy(), oracle.staple(U, L, i, mu)


def test_reflection_conjugates_the_quaternion_part(oracle):
    for seed in (61, 62, 63):
        _, _, _, _, u, A = _link_and_staple(oracle, seed)
        for g, (p, q) in enumerate(SUBGROUPS):
            u2, skipped = oracle.overrelax_link(u, A, 1 << g)
            assert skipped == 0
            q_old = _quaternion(u @ A, p, q)
            q_new = _quaternion(u2 @ A, p, q)
            assert np.max(np.abs(q_new - q_old * np.array([1, -1, -1, -1]))) < 1e-13
            # the link really moves (the block was not already real)
            assert np.max(np.abs(u2 - u)) > 1e-3
            # rows outside the subgroup are untouched
            r = 3 - p - q
            assert np.array_equal(u2[r], u[r])


def test_reflection_twice_is_identity(oracle):
    _, _, _, _, u, A = _link_and_staple(oracle, 64)
    for g in range(3):
        u1, _ = oracle.overrelax_link(u, A, 1 << g)
        u2, _ = oracle.overrelax_link(u1, A, 1 << g)
        assert np.max(np.abs(u2 - u)) < 1e-14


def test_link_update_keeps_local_action_and_su3(oracle):
    for seed in (65, 66):
        _, _, _, _, u, A = _link_and_staple(oracle, seed)
        u2, skipped = oracle.overrelax_link(u, A, 7)
        assert skipped == 0
        assert abs(np.trace(u2 @ A).real - np.trace(u @ A).real) < 1e-13 * np.abs(A).max()
        assert np.max(np.abs(u2 @ u2.conj().T - np.eye(3))) < 1e-14
        assert abs(np.linalg.det(u2) - 1) < 1e-14


def test_real_block_is_a_fixed_point(oracle):
    """A staple that makes U A = 1 has w_hat = 1 in every subgroup: v = 1."""
    u = inputs.haar_su3(1, 67)[0]
    A = u.conj().T
    u2, skipped = oracle.overrelax_link(u, A, 7)
    assert skipped == 0
    assert np.max(np.abs(u2 - u)) < 1e-15


def test_sweep_is_microcanonical_and_moves_links(oracle):
    L = (4, 4, 4, 4)
    beta = 5.7
    U = inputs.random_gauge(L, "haar", seed=68)
    for s in range(3):  # a rough field near equilibrium, from the oracle's heatbath
        U, _ = oracle.heatbath_sweep(U, L, beta, 11, s)
    S0 = oracle.gauge_action(U, L, beta)
    U1, skipped = oracle.overrelax_sweep(U, L)
    assert skipped == 0
    assert abs(oracle.gauge_action(U1, L, beta) - S0) < 1e-12 * S0
    assert np.max(np.abs(U1 - U)) > 0.3
    eye = np.eye(3)
    assert np.max(np.abs(U1 @ np.conj(np.transpose(U1, (0, 1, 3, 2))) - eye)) < 1e-13
    # a second sweep is not the inverse of the first (the subgroups do not commute)
    U2, _ = oracle.overrelax_sweep(U1, L)
    assert np.max(np.abs(U2 - U)) > 1e-3
    assert abs(oracle.gauge_action(U2, L, beta) - S0) < 1e-12 * S0
