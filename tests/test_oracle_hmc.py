"""Pins of the oracle's fermion force, random numbers, heatbath and HMC.

* fermion force (Sec. 2.2, dD^-1 = -D^-1 dD D^-1): central finite differences
  of S_pf = phi^+ (Mhat^+ Mhat)^-1 phi on single links, including links that
  cross the antiperiodic time boundary; same for the unpreconditioned form;
* Philox4x32-10: published known-answer vectors (tests/golden);
* SU(2) sampler (Creutz below b = 1.5, Kennedy-Pendleton above): Kolmogorov-Smirnov test against the exact CDF of
  sqrt(1 - x^2) exp(b x) obtained by quadrature;
* heatbath (Sec. 2.2): SU(3) strong-coupling expansion of the plaquette,
  <P> = beta/18 + beta^2/216 + O(beta^3);
* HMC (Sec. 2.2): reversibility, dH ~ eps^2, S_pf(phi = Mhat^+ eta) = eta^+ eta.
"""
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

from paper_1209_5942_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rot(U, i, mu, a, h, oracle):
    Ud = U.copy()
    Ud[i, mu] = scipy.linalg.expm(1j * h * oracle.generator(a)) @ U[i, mu]
    return Ud


@pytest.mark.parametrize("eo", [True, False])
def test_fermion_force_finite_difference(oracle, eo):
    L = (2, 2, 2, 4)
    V = inputs.volume(L)
    kappa, mu = 0.14, 0.1
    U = inputs.random_gauge(L, "near", seed=101, eps=0.4)
    phi = inputs.gaussian_spinor(L, 102)
    if eo:
        phi = phi * (~oracle.parity_mask(L))[:, None, None]
    S0, X = oracle.pseudofermion_action(U, phi, L, kappa, mu, eo=eo, tol=1e-14)
    F = oracle.fermion_dSdw(U, X, L, kappa, mu, eo=eo)
    c = inputs.site_coords(L)
    # links: interior, and forward links from t = Lt-1 (cross the boundary)
    tb = [i for i in range(V) if c[i, 3] == L[3] - 1]
    links = [(0, 0), (3, 1), (6, 2), (9, 3), (tb[0], 3), (tb[3], 3), (tb[2], 0)]
    h = 1e-5
    worst = 0.0
    for (i, m) in links:
        for a in range(8):
            sp, _ = oracle.pseudofermion_action(_rot(U, i, m, a, h, oracle), phi, L, kappa, mu,
                                                eo=eo, tol=1e-14)
            sm, _ = oracle.pseudofermion_action(_rot(U, i, m, a, -h, oracle), phi, L, kappa, mu,
                                                eo=eo, tol=1e-14)
            fd = (sp - sm) / (2 * h)
            worst = max(worst, abs(fd - F[m, i, a]) / max(1.0, abs(fd)))
    assert worst < 1e-6, worst


def test_philox_known_answers(oracle):
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(v, 16) for v in line.split()]
            got = oracle.philox4x32_10(w[0:4], w[4:6])
            assert list(got) == w[6:10]
            n += 1
    assert n == 3


def test_uniform_and_gaussian_moments(oracle):
    L = (4, 4, 4, 4)
    P = oracle.momenta(L, seed=123, traj=0)
    assert abs(P.mean()) < 0.02 and abs(P.var() - 1) < 0.03
    eta = oracle.gaussian_spinor(L, seed=123, traj=0)
    assert abs(eta.real.var() - 0.5) < 0.02 and abs(eta.imag.var() - 0.5) < 0.02
    u = np.array([oracle.philox_uniform2(k, 1, 2, 3, 99) for k in range(2000)]).ravel()
    assert u.min() > 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.02


@pytest.mark.parametrize("b", [0.01, 0.3, 1.4, 1.5, 6.0, 40.0])
def test_su2_sampler_distribution(oracle, b):
    x = np.sort(oracle.su2_y0_samples(b, seed=7, n=20000))
    assert x.min() >= -1 and x.max() <= 1
    f = lambda s: np.sqrt(max(0.0, 1 - s * s)) * np.exp(b * s)
    Z = scipy.integrate.quad(f, -1, 1)[0]
    grid = np.linspace(-1, 1, 2001)
    cdf = np.concatenate([[0], np.cumsum([scipy.integrate.quad(f, grid[k], grid[k + 1])[0]
                                          for k in range(2000)])]) / Z
    F = np.interp(x, grid, cdf)
    n = len(x)
    D = np.max(np.maximum(np.arange(1, n + 1) / n - F, F - np.arange(0, n) / n))
    assert D < 1.63 / np.sqrt(n), D  # 1 % level of the Kolmogorov distribution


def test_heatbath_strong_coupling(oracle):
    L = (4, 4, 4, 4)
    beta = 0.3
    U = inputs.random_gauge(L, "cold")
    for s in range(10):
        U, fails = oracle.heatbath_sweep(U, L, beta, 2024, s)
    vals = []
    for s in range(10, 70):
        U, fails = oracle.heatbath_sweep(U, L, beta, 2024, s)
        assert fails == 0
        vals.append(oracle.plaquette(U, L))
    vals = np.array(vals)
    expect = beta / 18 + beta ** 2 / 216
    err = vals.std() / np.sqrt(len(vals))
    assert abs(vals.mean() - expect) < 4 * err + 2e-4, (vals.mean(), expect, err)
    # links stay in SU(3)
    eye = np.eye(3)
    assert np.max(np.abs(U @ np.conj(np.transpose(U, (0, 1, 3, 2))) - eye)) < 1e-12
    assert np.max(np.abs(np.linalg.det(U) - 1)) < 1e-12


def test_heatbath_beta_zero_is_haar(oracle):
    """beta = 0: the heatbath samples the Haar measure, so <P> = 0 and every link
    stays in SU(3) (the degenerate b = 0 case of the SU(2) update)."""
    L = (4, 4, 4, 4)
    U = inputs.random_gauge(L, "cold")
    vals = []
    for s in range(20):
        U, fails = oracle.heatbath_sweep(U, L, 0.0, 31, s)
        assert fails == 0
        vals.append(oracle.plaquette(U, L))
    vals = np.array(vals[2:])
    assert abs(vals.mean()) < 4 * (1 / np.sqrt(18 * 6 * 256)) / np.sqrt(len(vals)) + 1e-3
    assert np.all(np.isfinite(U))
    assert np.max(np.abs(np.linalg.det(U) - 1)) < 1e-12


def test_heatbath_weak_coupling_orders(oracle):
    """At large beta the heatbath drives a Haar start towards plaquette ~ 1 - c/beta."""
    L = (4, 4, 4, 4)
    U = inputs.random_gauge(L, "haar", seed=5)
    for s in range(30):
        U, _ = oracle.heatbath_sweep(U, L, 20.0, 77, s)
    P = oracle.plaquette(U, L)
    # leading weak-coupling value 1 - 4/(3 beta) * (1 - small corrections)
    assert 0.85 < P < 0.97, P


def test_hmc_reversibility_and_scaling(oracle):
    L = (2, 2, 2, 4)
    beta, kappa, mu = 5.6, 0.14, 0.05 / 0.28
    U0 = inputs.random_gauge(L, "near", seed=201, eps=0.3)
    ev = ~oracle.parity_mask(L)
    eta = inputs.gaussian_spinor(L, 202) * ev[:, None, None]
    phi = oracle.apply_Mhat(U0, eta, L, kappa, mu, dagger=True)
    S, _ = oracle.pseudofermion_action(U0, phi, L, kappa, mu, eo=True, tol=1e-14)
    assert abs(S - np.vdot(eta, eta).real) < 1e-10 * S
    P0 = oracle.momenta(L, seed=203, traj=0)
    U1, P1, dH, _ = oracle.hmc_md(U0, P0, phi, L, beta, kappa, mu, nsteps=8, tau=0.5, tol=1e-14)
    U2, P2, dH2, _ = oracle.hmc_md(U1, -P1, phi, L, beta, kappa, mu, nsteps=8, tau=0.5, tol=1e-14)
    assert np.max(np.abs(U2 - U0)) < 1e-10
    assert np.max(np.abs(P2 + P0)) < 1e-9
    assert abs(dH + dH2) < 1e-9
    dHs = []
    for n in (8, 16):
        _, _, d, _ = oracle.hmc_md(U0, P0, phi, L, beta, kappa, mu, nsteps=n, tau=0.5, tol=1e-14)
        dHs.append(abs(d))
    ratio = dHs[0] / dHs[1]
    assert 3.0 < ratio < 5.3, (dHs, ratio)


def test_hasenbusch_ratio_pins(oracle):
    """Mass preconditioning with a heavier twisted mass mu2: with mu2 = mu the
    ratio action is phi^+ phi exactly and its force vanishes (the two terms
    cancel); the heatbath source gives S2 = eta^+ eta; central differences of
    S2 on single links (one across the time boundary) match the force."""
    import scipy.linalg
    L = (2, 4, 2, 4)
    V = inputs.volume(L)
    kappa, mu, mu2 = 0.14, 0.05, 0.3
    U = inputs.random_gauge(L, "near", seed=401, eps=0.4)
    ev = ~oracle.parity_mask(L)
    phi = inputs.gaussian_spinor(L, 402) * ev[:, None, None]
    S_same, X_same = oracle.hasenbusch_action(U, phi, L, kappa, mu, mu, tol=1e-14)
    assert abs(S_same - np.vdot(phi, phi).real) < 1e-10 * S_same
    F_same = oracle.hasenbusch_dSdw(U, phi, X_same, L, kappa, mu, mu)
    assert np.max(np.abs(F_same)) < 1e-9
    eta = inputs.gaussian_spinor(L, 403) * ev[:, None, None]
    phi2 = oracle.hasenbusch_source(U, eta, L, kappa, mu, mu2, tol=1e-14)
    S2, _ = oracle.hasenbusch_action(U, phi2, L, kappa, mu, mu2, tol=1e-14)
    assert abs(S2 - np.vdot(eta, eta).real) < 1e-9 * S2
    S, X = oracle.hasenbusch_action(U, phi, L, kappa, mu, mu2, tol=1e-14)
    F = oracle.hasenbusch_dSdw(U, phi, X, L, kappa, mu, mu2)
    h = 1e-5
    for (i, m) in [(0, 0), (9, 3), (V - 1, 3), (14, 1)]:
        for a in (0, 3, 7):
            Up, Um = U.copy(), U.copy()
            T = oracle.generator(a)
            Up[i, m] = scipy.linalg.expm(1j * h * T) @ U[i, m]
            Um[i, m] = scipy.linalg.expm(-1j * h * T) @ U[i, m]
            sp, _ = oracle.hasenbusch_action(Up, phi, L, kappa, mu, mu2, tol=1e-14)
            sm, _ = oracle.hasenbusch_action(Um, phi, L, kappa, mu, mu2, tol=1e-14)
            fd = (sp - sm) / (2 * h)
            assert abs(fd - F[m, i, a]) < 1e-6 * max(1.0, abs(fd)), (i, m, a, fd, F[m, i, a])


def test_mass_preconditioned_2mn_pins(oracle):
    """The three-scale mass-preconditioned trajectory of the oracle:
    (1) with mu2 = mu the ratio action is eta2^+ eta2 and its force vanishes,
        so the outer scale only splits the time: the trajectory equals the
        pinned two-scale 2MN of the W pseudofermion with 2 nsteps nsteps_mid
        fermion steps (same links, same dH);
    (2) H0 = K + S_g + eta1^+ eta1 + eta2^+ eta2 (both sources so drawn);
    (3) reversible: flipping the final momenta and integrating again gives
        back the start links;
    (4) second order: dH falls ~4x when all step counts double."""
    L = (2, 4, 2, 4)
    beta, kappa, mu, mu2, c1 = 3.9, 0.14, 0.05, 0.25, oracle.TLSYM_C1
    U = inputs.random_gauge(L, "near", seed=411, eps=0.3)
    ev = ~oracle.parity_mask(L)
    eta1 = inputs.gaussian_spinor(L, 412) * ev[:, None, None]
    eta2 = inputs.gaussian_spinor(L, 413) * ev[:, None, None]
    P0 = inputs.gaussian_algebra(L, 414)
    tau = 0.5
    # (1) reduction to the two-scale integrator at mu2 = mu (the middle scale then
    #     carries the twisted mass mu itself)
    Ua, Pa, dHa, _, _ = oracle.hmc_md_2mn_hasenbusch(U, P0, eta1, eta2, L, beta, kappa, mu, mu, c1=c1,
                                                  nsteps=2, nsteps_mid=2, nsteps_g=2, tau=tau)
    phi = oracle.apply_Mhat(U, eta1, L, kappa, mu, dagger=True)
    Ub, Pb, dHb, _ = oracle.hmc_md_2mn(U, P0, phi, L, beta, kappa, mu, c1=c1, nf=1, nsteps_f=8,
                                       nsteps_g=2, tau=tau, tol=1e-13)
    assert np.max(np.abs(Ua - Ub)) < 1e-10
    assert np.max(np.abs(Pa - Pb)) < 1e-8
    assert abs(dHa - dHb) < 1e-8
    # (2) start Hamiltonian
    U1, P1, dH, (H0, H1), phis = oracle.hmc_md_2mn_hasenbusch(U, P0, eta1, eta2, L, beta, kappa, mu, mu2, c1=c1,
                                                        nsteps=2, nsteps_mid=2, nsteps_g=2, tau=tau)
    H0_expect = (0.5 * np.sum(P0 ** 2) + oracle.gauge_action_sym(U, L, beta, c1)
                 + np.vdot(eta1, eta1).real + np.vdot(eta2, eta2).real)
    assert abs(H0 - H0_expect) < 1e-9 * abs(H0_expect)
    # (3) reversibility, with the pseudofermion fields of the forward trip
    assert np.max(np.abs(U1 - U)) > 1e-3
    Ur, Pr, dHr, _, _ = oracle.hmc_md_2mn_hasenbusch(U1, -P1, None, None, L, beta, kappa, mu, mu2, c1=c1,
                                                     nsteps=2, nsteps_mid=2, nsteps_g=2, tau=tau, phis=phis)
    assert np.max(np.abs(Ur - U)) < 1e-10
    assert np.max(np.abs(Pr + P0)) < 1e-8
    assert abs(dHr + dH) < 1e-8
    # (4) second order
    _, _, dH2, _, _ = oracle.hmc_md_2mn_hasenbusch(U, P0, eta1, eta2, L, beta, kappa, mu, mu2, c1=c1,
                                                nsteps=4, nsteps_mid=2, nsteps_g=2, tau=tau)
    assert abs(dH) < 1.0
    assert 3.0 < dH / dH2 < 5.3, (dH, dH2)
