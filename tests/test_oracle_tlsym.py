"""Pins of the oracle's tree-level Symanzik gauge action (Sec. 2.1, eq.
"S_tlsym") and of the 2MN integrator on two time scales (Sec. 2.2; Sec. 5.3
"separate time scales for the gauge and fermion parts") against closed forms,
invariants, finite differences and exactly solvable motion."""
import numpy as np
import pytest
import scipy.linalg

from paper_1209_5942_gb300 import inputs

C1 = -1.0 / 12.0


def _abelian_flux_field(L, n_flux):
    """U_x(x, y, z, t) = diag(e^{i a y}, e^{-i a y}, 1) with a = 2 pi n / Ly,
    all other links 1: every x-y plaquette is D(-a), every other one is 1."""
    V = inputs.volume(L)
    U = inputs.random_gauge(L, "cold")
    a = 2 * np.pi * n_flux / L[1]
    for i in range(V):
        y = (i // L[0]) % L[1]
        U[i, 0] = np.diag([np.exp(1j * a * y), np.exp(-1j * a * y), 1.0])
    return U, a


def test_wilson_limit(oracle):
    """c1 = 0 is the Wilson plaquette action and its force."""
    L = (4, 2, 4, 2)
    U = inputs.random_gauge(L, "near", seed=301, eps=0.5)
    assert abs(oracle.gauge_action_sym(U, L, 5.3, 0.0) - oracle.gauge_action(U, L, 5.3)) < 1e-10
    F = oracle.gauge_dSdw_sym(U, L, 5.3, 0.0)
    assert np.max(np.abs(F - oracle.gauge_dSdw(U, L, 5.3))) < 1e-13


def test_cold_start_and_gauge_invariance(oracle):
    L = (2, 4, 2, 4)
    V = inputs.volume(L)
    Uc = inputs.random_gauge(L, "cold")
    assert oracle.gauge_action_sym(Uc, L, 3.9, C1) == 0.0
    assert np.all(oracle.gauge_dSdw_sym(Uc, L, 3.9, C1) == 0.0)
    U = inputs.random_gauge(L, "haar", seed=302)
    G = inputs.haar_su3(V, 303)
    from tests.test_oracle_dirac import _gauge_transform
    Ug = _gauge_transform(U, G, L)
    s0, s1 = oracle.gauge_action_sym(U, L, 3.9, C1), oracle.gauge_action_sym(Ug, L, 3.9, C1)
    assert abs(s0 - s1) < 1e-11 * abs(s0)


@pytest.mark.parametrize("L,n", [((4, 4, 2, 2), 1), ((2, 6, 2, 4), 2)])
def test_rectangles_in_a_constant_abelian_field(oracle, L, n):
    """Constant flux a through every x-y plaquette: Re Tr P_xy = 1 + 2 cos a and
    both 2x1 loops of the x-y plane (R_xy, R_yx) enclose 2a, so
    sum (3 - Re Tr R) = 2 V (2 - 2 cos 2a); all other loops are trivial.  A 1x1
    or 3x1 loop in place of the rectangle would give cos a or cos 3a."""
    V = inputs.volume(L)
    U, a = _abelian_flux_field(L, n)
    assert abs(oracle.rectangle_sum(U, L) - 2 * V * (2 - 2 * np.cos(2 * a))) < 1e-10 * V
    beta = 3.9
    expect = beta / 3 * ((1 - 8 * C1) * V * (2 - 2 * np.cos(a)) + C1 * 2 * V * (2 - 2 * np.cos(2 * a)))
    assert abs(oracle.gauge_action_sym(U, L, beta, C1) - expect) < 1e-10 * abs(expect)


def _rotate_link(U, i, mu, a, h, oracle):
    Ud = U.copy()
    Ud[i, mu] = scipy.linalg.expm(1j * h * oracle.generator(a)) @ U[i, mu]
    return Ud


def test_tlsym_force_finite_difference(oracle):
    """Central differences of S_tlsym on single links (one on each boundary
    wrap) agree with the loop-by-loop derivative."""
    L = (4, 2, 4, 4)
    V = inputs.volume(L)
    beta = 3.9
    U = inputs.random_gauge(L, "near", seed=304, eps=0.6)
    F = oracle.gauge_dSdw_sym(U, L, beta, C1)
    h = 1e-5
    for (i, mu) in [(0, 0), (3, 0), (7, 1), (V - 1, 3), (37, 2)]:
        for a in range(8):
            sp = oracle.gauge_action_sym(_rotate_link(U, i, mu, a, h, oracle), L, beta, C1)
            sm = oracle.gauge_action_sym(_rotate_link(U, i, mu, a, -h, oracle), L, beta, C1)
            fd = (sp - sm) / (2 * h)
            assert abs(fd - F[mu, i, a]) < 1e-7 * max(1.0, abs(fd)), (i, mu, a, fd, F[mu, i, a])


def test_2mn_free_motion_is_exact(oracle):
    """beta = 0, no fermions: P is constant and U(tau) = exp(i tau P) U(0)
    exactly, so the nested steps must add up to tau on every scale."""
    L = (2, 2, 2, 4)
    V = inputs.volume(L)
    U0 = inputs.random_gauge(L, "haar", seed=305)
    P0 = oracle.momenta(L, seed=306, traj=0)
    U1, P1, dH, _ = oracle.hmc_md_2mn(U0, P0, None, L, 0.0, 0.16, 0.1, nf=0, nsteps_f=3, nsteps_g=4,
                                      tau=0.7)
    assert np.array_equal(P1, P0)
    T = [oracle.generator(a) for a in range(8)]
    for i in range(V):
        for mu in range(4):
            H = sum(P0[mu, i, a] * T[a] for a in range(8))
            assert np.max(np.abs(U1[i, mu] - scipy.linalg.expm(1j * 0.7 * H) @ U0[i, mu])) < 1e-12
    assert abs(dH) < 1e-12


def test_2mn_nested_without_fermions_is_single_scale(oracle):
    """With no fermion force the outer scale only splits time: n_f = 1 outer
    step with n_g inner steps is 2 n_g plain 2MN steps; compare with n_f = 2,
    n_g = n_g / 2, which must give the same field up to rounding."""
    L = (2, 2, 2, 4)
    U0 = inputs.random_gauge(L, "near", seed=307, eps=0.4)
    P0 = oracle.momenta(L, seed=308, traj=0)
    Ua, Pa, da, _ = oracle.hmc_md_2mn(U0, P0, None, L, 3.9, 0.16, 0.1, nf=0, nsteps_f=1, nsteps_g=4, tau=0.5)
    Ub, Pb, db, _ = oracle.hmc_md_2mn(U0, P0, None, L, 3.9, 0.16, 0.1, nf=0, nsteps_f=2, nsteps_g=2, tau=0.5)
    assert np.max(np.abs(Ua - Ub)) < 1e-12
    assert np.max(np.abs(Pa - Pb)) < 1e-11
    assert abs(da - db) < 1e-10


def test_2mn_reversible_and_second_order(oracle):
    """Reversibility, and dH ~ eps^2: halving both step sizes divides |dH| by
    about 4."""
    L = (2, 2, 2, 4)
    beta, kappa, mu = 3.9, 0.14, 0.1 / 0.28
    U0 = inputs.random_gauge(L, "near", seed=309, eps=0.3)
    ev = ~oracle.parity_mask(L)
    eta = inputs.gaussian_spinor(L, 310) * ev[:, None, None]
    phi = oracle.apply_Mhat(U0, eta, L, kappa, mu, dagger=True)
    P0 = oracle.momenta(L, seed=311, traj=0)
    kw = dict(c1=C1, tau=0.6, tol=1e-14)
    U1, P1, dH, _ = oracle.hmc_md_2mn(U0, P0, phi, L, beta, kappa, mu, nsteps_f=4, nsteps_g=2, **kw)
    U2, P2, dH2, _ = oracle.hmc_md_2mn(U1, -P1, phi, L, beta, kappa, mu, nsteps_f=4, nsteps_g=2, **kw)
    assert np.max(np.abs(U2 - U0)) < 1e-10
    assert np.max(np.abs(P2 + P0)) < 1e-9
    assert abs(dH + dH2) < 1e-9
    d = []
    for nf_, ng in ((4, 2), (8, 4)):
        _, _, x, _ = oracle.hmc_md_2mn(U0, P0, phi, L, beta, kappa, mu, nsteps_f=nf_, nsteps_g=ng, **kw)
        d.append(abs(x))
    assert 3.0 < d[0] / d[1] < 5.3, d
