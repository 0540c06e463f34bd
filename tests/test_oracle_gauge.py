"""Pins of the oracle's gauge-side functions (Sec. 2.1 action, Sec. 2.2 forces,
Sec. 4.1 REC12) against closed forms, invariants, finite differences and
library routines."""
import numpy as np
import pytest
import scipy.linalg

from paper_1209_5942_gb300 import inputs

L44 = (4, 4, 4, 4)
LASYM = (2, 4, 6, 8)


def test_generators(oracle):
    T = [oracle.generator(a) for a in range(8)]
    for a in range(8):
        assert np.allclose(T[a], T[a].conj().T, atol=0)
        assert abs(np.trace(T[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(T[a] @ T[b]) - 0.5 * (a == b)) < 1e-15
    # f^{123} = 1: [T1, T2] = i T3
    assert np.allclose(T[0] @ T[1] - T[1] @ T[0], 1j * T[2], atol=1e-15)


def test_cold_start(oracle):
    U = inputs.random_gauge(L44, "cold")
    assert oracle.plaquette(U, L44) == 1.0
    assert oracle.gauge_action(U, L44, 5.7) == 0.0
    assert np.all(oracle.gauge_dSdw(U, L44, 5.7) == 0.0)


def test_single_link_plaquette_closed_form(oracle):
    """One link diag(e^{i th}, e^{-i th}, 1), all others 1: the six plaquettes
    through it each lose 2 - 2 cos th."""
    L = LASYM
    V = inputs.volume(L)
    th = 0.7
    U = inputs.random_gauge(L, "cold")
    U[5, 2] = np.diag([np.exp(1j * th), np.exp(-1j * th), 1.0])
    expect = 1 - 6 * (2 - 2 * np.cos(th)) / (18 * V)
    assert abs(oracle.plaquette(U, L) - expect) < 1e-15
    beta = 5.6
    assert abs(oracle.gauge_action(U, L, beta) - beta / 3 * 6 * (2 - 2 * np.cos(th))) < 1e-12


def test_plaquette_gauge_invariant_and_haar(oracle):
    L = LASYM
    V = inputs.volume(L)
    U = inputs.random_gauge(L, "haar", seed=3)
    G = inputs.haar_su3(V, 4)
    from tests.test_oracle_dirac import _gauge_transform
    Ug = _gauge_transform(U, G, L)
    assert abs(oracle.plaquette(U, L) - oracle.plaquette(Ug, L)) < 1e-14
    # Haar average of Re Tr/3 of a plaquette is 0 with variance 1/18 per plaquette
    assert abs(oracle.plaquette(U, L)) < 5 / np.sqrt(18 * 6 * V)


def test_staple_sum_counts_each_plaquette_four_times(oracle):
    L = (2, 2, 4, 4)
    V = inputs.volume(L)
    U = inputs.random_gauge(L, "near", seed=5, eps=0.5)
    tot = 0.0
    for i in range(V):
        for mu in range(4):
            tot += np.real(np.trace(U[i, mu] @ oracle.staple(U, L, i, mu)))
    assert abs(tot - 4 * 3 * 6 * V * oracle.plaquette(U, L)) < 1e-10


def _rotate_link(U, i, mu, a, h, oracle):
    Ud = U.copy()
    Ud[i, mu] = scipy.linalg.expm(1j * h * oracle.generator(a)) @ U[i, mu]
    return Ud


def test_gauge_force_finite_difference(oracle):
    L = (2, 4, 2, 4)
    beta = 5.6
    U = inputs.random_gauge(L, "near", seed=7, eps=0.6)
    F = oracle.gauge_dSdw(U, L, beta)
    h = 1e-5
    for (i, mu) in [(0, 0), (5, 3), (17, 1), (30, 2)]:
        for a in range(8):
            sp = oracle.gauge_action(_rotate_link(U, i, mu, a, h, oracle), L, beta)
            sm = oracle.gauge_action(_rotate_link(U, i, mu, a, -h, oracle), L, beta)
            fd = (sp - sm) / (2 * h)
            assert abs(fd - F[mu, i, a]) < 1e-7 * max(1.0, abs(fd)), (i, mu, a, fd, F[mu, i, a])


def test_expi_matches_library(oracle):
    p = inputs.rng(9).standard_normal(8) * 3.0
    for eps in (0.01, 0.3, 2.0):
        H = sum(p[a] * oracle.generator(a) for a in range(8))
        ref = scipy.linalg.expm(1j * eps * H)
        got = oracle.expi(p, eps)
        assert np.max(np.abs(got - ref)) < 1e-14


def test_rec12_and_reunitarize(oracle):
    W = inputs.haar_su3(64, 10)
    for w in W[:8]:
        assert np.max(np.abs(oracle.rec12_third_row(w) - w[2])) < 1e-15
    # reunitarisation leaves SU(3) matrices unchanged ...
    assert np.max(np.abs(oracle.reunitarize(W) - W)) < 1e-15
    # ... and projects perturbed matrices back to SU(3)
    P = W + 1e-3 * inputs.rng(11).standard_normal(W.shape)
    R = oracle.reunitarize(P)
    eye = np.eye(3)
    assert np.max(np.abs(R @ np.conj(np.transpose(R, (0, 2, 1))) - eye)) < 1e-14
    assert np.max(np.abs(np.linalg.det(R) - 1)) < 1e-14


def test_update_links_matches_library(oracle):
    L = (2, 2, 2, 2)
    V = inputs.volume(L)
    U = inputs.random_gauge(L, "haar", seed=12)
    P = inputs.gaussian_algebra(L, 13)
    eps = 0.05
    got = oracle.update_links(U, P, L, eps)
    T = np.stack([oracle.generator(a) for a in range(8)])
    for i in (0, 7, 15):
        for mu in range(4):
            H = np.einsum("a,aij->ij", P[mu, i], T)
            ref = scipy.linalg.expm(1j * eps * H) @ U[i, mu]
            assert np.max(np.abs(got[i, mu] - ref)) < 1e-14
    assert V == 16
