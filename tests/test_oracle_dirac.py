"""Pins of the oracle's Dirac operator against what the paper and mathematics fix.

Sec. 2.1, eq. D_tm: M = (1 + 2 i kappa mu g5) - kappa H.  Each test below is
chosen so that a plausible mistake in the oracle (a dropped term, a wrong
sign, a transposed link, a wrong boundary factor, a wrong gamma basis) fails:

* Clifford algebra and gamma_5 of the chiral basis;
* free field (U = 1): plane waves are eigenvectors with the closed-form
  momentum-space matrix m(p) + i a g5 + 2 i kappa sum_mu g_mu sin p_mu,
  including the antiperiodic time momenta;
* adjointness <chi, M psi> = <M^+ chi, psi>;
* gamma_5-hermiticity M(mu)^+ = g5 M(-mu) g5;
* gauge covariance M[U^G] G psi = G M[U] psi;
* the twisted-mass identity M(mu)^+ M(mu) = M(0)^+ M(0) + (2 kappa mu)^2
  (the paper's det D_tm = det(D_W^2 + 4 kappa^2 mu^2));
* brute force on 2^4: the dense matrix's LU solve equals the CG solution,
  and the even-odd solve with reconstruction equals both.
"""
import numpy as np
import pytest

from paper_1209_5942_gb300 import inputs

L44 = (4, 4, 4, 4)
LASYM = (2, 4, 6, 8)


def test_gamma_clifford(oracle):
    g = [oracle.gamma(m) for m in range(4)]
    one = np.eye(4)
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T, atol=0)
        for n in range(4):
            ac = g[m] @ g[n] + g[n] @ g[m]
            assert np.allclose(ac, 2 * one * (m == n), atol=1e-15)
    g5 = oracle.gamma(4)
    # reading: chiral basis with gamma_5 = g_x g_y g_z g_t = diag(1, 1, -1, -1)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]), atol=1e-15)
    assert np.allclose(g[0] @ g[1] @ g[2] @ g[3], g5, atol=1e-15)
    for m in range(4):
        assert np.allclose(g5 @ g[m] + g[m] @ g5, 0, atol=1e-15)


def _plane_wave(L, n):
    """e^{i p x} with p_k = 2 pi n_k / L_k (space), p_t = (2 n_t + 1) pi / L_t."""
    c = inputs.site_coords(L)
    p = np.array([2 * np.pi * n[0] / L[0], 2 * np.pi * n[1] / L[1], 2 * np.pi * n[2] / L[2],
                  (2 * n[3] + 1) * np.pi / L[3]])
    return np.exp(1j * (c @ p)), p


@pytest.mark.parametrize("L", [L44, LASYM])
@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 1, 0), (1, 2, 3, 1), (3, 1, 2, 2)])
def test_free_field_closed_form(oracle, L, n):
    kappa, mu = 0.13, 0.37
    a = 2 * kappa * mu
    U = inputs.random_gauge(L, "cold")
    phase, p = _plane_wave(L, n)
    g = [oracle.gamma(m) for m in range(4)]
    g5 = oracle.gamma(4)
    u = inputs.rng(7).standard_normal((4, 3)) + 1j * inputs.rng(8).standard_normal((4, 3))
    psi = phase[:, None, None] * u[None]
    m_p = 1 - 2 * kappa * np.sum(np.cos(p))
    Mp = m_p * np.eye(4) + 1j * a * g5 + 2j * kappa * sum(g[k] * np.sin(p[k]) for k in range(4))
    expect = phase[:, None, None] * (Mp @ u)[None]
    got = oracle.apply_M(U, psi, L, kappa, mu)
    assert np.max(np.abs(got - expect)) < 1e-13
    # M^+ M is diagonal: m(p)^2 + a^2 + 4 kappa^2 sum sin^2 p
    MdM = oracle.apply_M(U, got, L, kappa, mu, dagger=True)
    lam = m_p ** 2 + a ** 2 + 4 * kappa ** 2 * np.sum(np.sin(p) ** 2)
    assert np.max(np.abs(MdM - lam * psi)) < 1e-13


def test_free_field_periodic_time_differs(oracle):
    """With periodic fermions in time the antiperiodic plane wave is NOT an eigenvector:
    pins that the boundary factor is applied exactly on hops across t = Lt-1 <-> 0."""
    L = L44
    kappa, mu = 0.13, 0.0
    U = inputs.random_gauge(L, "cold")
    phase, p = _plane_wave(L, (0, 0, 0, 0))
    psi = np.zeros((inputs.volume(L), 4, 3), np.complex128)
    psi[:, 0, 0] = phase
    out_ap = oracle.apply_M(U, psi, L, kappa, mu, antiperiodic_t=True)
    out_p = oracle.apply_M(U, psi, L, kappa, mu, antiperiodic_t=False)
    c = inputs.site_coords(L)
    edge = (c[:, 3] == 0) | (c[:, 3] == L[3] - 1)
    diff = np.abs(out_ap - out_p).max(axis=(1, 2))
    assert np.all(diff[~edge] < 1e-14) and np.all(diff[edge] > 1e-3)


@pytest.mark.parametrize("L", [L44, LASYM])
def test_adjoint(oracle, L):
    kappa, mu = 0.15, 0.0333
    U = inputs.random_gauge(L, "haar", seed=11)
    psi = inputs.gaussian_spinor(L, 12)
    chi = inputs.gaussian_spinor(L, 13)
    lhs = np.vdot(chi, oracle.apply_M(U, psi, L, kappa, mu))
    rhs = np.vdot(oracle.apply_M(U, chi, L, kappa, mu, dagger=True), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    lhs = np.vdot(chi, oracle.apply_Mhat(U, psi, L, kappa, mu))
    rhs = np.vdot(oracle.apply_Mhat(U, chi, L, kappa, mu, dagger=True), psi)
    ev = ~oracle.parity_mask(L)
    lhs = np.vdot(chi[ev], oracle.apply_Mhat(U, psi * ev[:, None, None], L, kappa, mu)[ev])
    rhs = np.vdot(oracle.apply_Mhat(U, chi * ev[:, None, None], L, kappa, mu, dagger=True)[ev],
                  psi[ev])
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_gamma5_hermiticity(oracle):
    L = LASYM
    kappa, mu = 0.15, 0.0333
    U = inputs.random_gauge(L, "haar", seed=21)
    psi = inputs.gaussian_spinor(L, 22)
    g5 = np.array([1, 1, -1, -1])[None, :, None]
    lhs = oracle.apply_M(U, psi, L, kappa, mu, dagger=True)
    rhs = g5 * oracle.apply_M(U, g5 * psi, L, kappa, -mu)
    assert np.max(np.abs(lhs - rhs)) < 1e-14
    lhs = oracle.apply_Mhat(U, psi, L, kappa, mu, dagger=True)
    rhs = g5 * oracle.apply_Mhat(U, g5 * psi, L, kappa, -mu)
    assert np.max(np.abs(lhs - rhs)) < 1e-14


def _gauge_transform(U, G, L):
    V = inputs.volume(L)
    c = inputs.site_coords(L)
    Ug = np.empty_like(U)
    for mu in range(4):
        cn = c.copy()
        cn[:, mu] = (cn[:, mu] + 1) % L[mu]
        j = cn[:, 0] + L[0] * (cn[:, 1] + L[1] * (cn[:, 2] + L[2] * cn[:, 3]))
        Ug[:, mu] = G @ U[:, mu] @ np.conj(np.transpose(G[j], (0, 2, 1)))
    assert Ug.shape == (V, 4, 3, 3)
    return Ug


def test_gauge_covariance(oracle):
    L = LASYM
    kappa, mu = 0.15, 0.0333
    U = inputs.random_gauge(L, "haar", seed=31)
    G = inputs.haar_su3(inputs.volume(L), 32)
    psi = inputs.gaussian_spinor(L, 33)
    Ug = _gauge_transform(U, G, L)
    Gpsi = np.einsum("vab,vsb->vsa", G, psi)
    lhs = oracle.apply_M(Ug, Gpsi, L, kappa, mu)
    rhs = np.einsum("vab,vsb->vsa", G, oracle.apply_M(U, psi, L, kappa, mu))
    assert np.max(np.abs(lhs - rhs)) < 1e-13
    lhs = oracle.apply_Mhat(Ug, Gpsi, L, kappa, mu)
    rhs = np.einsum("vab,vsb->vsa", G, oracle.apply_Mhat(U, psi, L, kappa, mu))
    assert np.max(np.abs(lhs - rhs)) < 1e-13


def test_twisted_mass_identity(oracle):
    L = L44
    kappa, mu = 0.15, 0.21
    a = 2 * kappa * mu
    U = inputs.random_gauge(L, "haar", seed=41)
    psi = inputs.gaussian_spinor(L, 42)
    lhs = oracle.apply_M(U, oracle.apply_M(U, psi, L, kappa, mu), L, kappa, mu, dagger=True)
    rhs = oracle.apply_M(U, oracle.apply_M(U, psi, L, kappa, 0.0), L, kappa, 0.0, dagger=True)
    assert np.max(np.abs(lhs - rhs - a * a * psi)) < 1e-13


def _dense(oracle, U, L, kappa, mu, dagger=False):
    V = inputs.volume(L)
    N = 12 * V
    D = np.zeros((N, N), np.complex128)
    for k in range(N):
        e = np.zeros(N, np.complex128)
        e[k] = 1
        D[:, k] = oracle.apply_M(U, e.reshape(V, 4, 3), L, kappa, mu, dagger).reshape(-1)
    return D


def test_dense_2x4_bruteforce(oracle):
    L = (2, 2, 2, 2)
    kappa, mu = 0.15, 0.01 / 0.3
    U = inputs.random_gauge(L, "haar", seed=51)
    D = _dense(oracle, U, L, kappa, mu)
    Dd = _dense(oracle, U, L, kappa, mu, dagger=True)
    assert np.max(np.abs(Dd - D.conj().T)) < 1e-15
    # det identity of Sec. 2.1: det(M^+ M) = det(D_W^+ D_W + a^2)
    a = 2 * kappa * mu
    DW = _dense(oracle, U, L, kappa, 0.0)
    ev1 = np.linalg.eigvalsh(D.conj().T @ D)
    ev2 = np.linalg.eigvalsh(DW.conj().T @ DW) + a * a
    assert np.max(np.abs(ev1 - ev2)) < 1e-12
    assert ev1.min() >= a * a * (1 - 1e-9)
    b = inputs.gaussian_spinor(L, 52)
    x_lu = np.linalg.solve(D, b.reshape(-1)).reshape(b.shape)
    x_cg = oracle.solve(U, b, L, kappa, mu, tol=1e-13)
    assert np.max(np.abs(x_cg - x_lu)) < 1e-9 * np.max(np.abs(x_lu))
    # even-odd: CG on Mhat^+ Mhat, then reconstruct the odd sites
    bhat = oracle.eo_prepare(U, b, L, kappa, mu)
    rhs = oracle.apply_Mhat(U, bhat, L, kappa, mu, dagger=True)
    xe, it, res = oracle.cg(U, rhs, L, kappa, mu, tol=1e-14, eo=True)
    assert it > 0
    x = oracle.eo_reconstruct(U, b, xe, L, kappa, mu)
    assert np.max(np.abs(x - x_lu)) < 1e-9 * np.max(np.abs(x_lu))


def test_eo_schur_consistency_4x4(oracle):
    L = L44
    kappa, mu = 0.15, 0.01 / 0.3
    U = inputs.random_gauge(L, "near", seed=61, eps=0.3)
    x = inputs.gaussian_spinor(L, 62)
    b = oracle.apply_M(U, x, L, kappa, mu)
    # the Schur complement maps the even part of the true solution onto bhat
    bhat = oracle.eo_prepare(U, b, L, kappa, mu)
    ev = ~oracle.parity_mask(L)
    xe = x * ev[:, None, None]
    assert np.max(np.abs(oracle.apply_Mhat(U, xe, L, kappa, mu)[ev] - bhat[ev])) < 1e-13
    # reconstruction recovers the odd part exactly
    xr = oracle.eo_reconstruct(U, b, xe, L, kappa, mu)
    assert np.max(np.abs(xr - x)) < 1e-13


def test_cg_true_residual(oracle):
    L = L44
    kappa, mu = 0.15, 0.01 / 0.3
    U = inputs.random_gauge(L, "haar", seed=71)
    b = inputs.gaussian_spinor(L, 72)
    x, it, res = oracle.cg(U, b, L, kappa, mu, tol=1e-11)
    assert it > 0 and res <= 1e-11
    r = b - oracle.apply_M(U, x, L, kappa, mu)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-11


def test_cg_fixed_iters_matches_cg_and_its_residual(oracle):
    """The oracle's fixed-iteration CG (used only to time the CPU baseline)
    is the even-odd CG on Mhat^+ Mhat x = Mhat^+ bhat: after N iterations its
    iterate equals or_cg(eo=1)'s after N iterations, its reported residual is
    the true normal-equation residual of that iterate, and with enough
    iterations the iterate solves Mhat x = bhat."""
    L = L44
    kappa, mu = 0.15, 0.01 / 0.3
    U = inputs.random_gauge(L, "haar", seed=73)
    b = inputs.gaussian_spinor(L, 74)
    bhat = oracle.eo_prepare(U, b, L, kappa, mu)
    ev = ~oracle.parity_mask(L)
    rhs = oracle.apply_Mhat(U, bhat, L, kappa, mu, dagger=True) * ev[:, None, None]
    for n in (1, 7, 25):
        xf, rf = oracle.cg_fixed_iters(U, bhat, L, kappa, mu, n)
        xc, it, rc = oracle.cg(U, rhs, L, kappa, mu, tol=0.0, max_iter=n, eo=True)
        assert it == -1  # ran all n iterations
        assert np.max(np.abs(xf - xc)) <= 1e-13 * np.max(np.abs(xc))
        assert abs(rf - rc) <= 1e-12 * rc
        r = rhs - oracle.apply_Mhat(U, oracle.apply_Mhat(U, xf, L, kappa, mu), L, kappa, mu, dagger=True)
        true = np.linalg.norm(r[ev]) / np.linalg.norm(rhs[ev])
        assert abs(true - rf) <= 1e-9 * max(rf, 1e-12)
    xf, rf = oracle.cg_fixed_iters(U, bhat, L, kappa, mu, 400)
    assert rf < 1e-12
    res = oracle.apply_Mhat(U, xf, L, kappa, mu) - bhat
    assert np.linalg.norm(res[ev]) <= 1e-10 * np.linalg.norm(bhat[ev])
