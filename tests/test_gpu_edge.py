"""Edge and degenerate cases of the GPU path, each against the oracle or an exact
property:

* the 2^4 lattice, where x + mu and x - mu are the same site in every direction;
* a zero right-hand side (x = 0 exactly), alone and inside a multi-RHS solve;
* a 32^3 x 64 lattice (the largest workload of the configs) on every site;
* beta = 0 heatbath (the b -> 0 limit of the SU(2) update: Haar measure);
* argument errors (non-finite kappa, bad parity, NULL stats) rejected before launch.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1209_5942_gb300 import inputs, lqcd
from tests.gpu_util import dev, eo_full_from_lexi, host, lexi_from_eo_full, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1209_5942_gb300 import build
    build.build()
    return lqcd.Context(0)


@pytest.mark.parametrize("prec", [lqcd.LQCD_F64, lqcd.LQCD_DF64, lqcd.LQCD_F32])
def test_two_site_extents(ctx, oracle, prec):
    L = (2, 2, 2, 2)
    kappa, mu = 0.15, 0.01 / 0.3
    U = inputs.random_gauge(L, "haar", seed=61)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    psi = inputs.gaussian_spinor(L, 62)
    for dagger in (False, True):
        ref = oracle.apply_M(U, psi, L, kappa, mu, dagger=dagger)
        _, _, fi = eo_full_from_lexi(ctx, L, psi, prec)
        od, osc = lqcd.alloc_field(L, lqcd.LQCD_FULL, prec)
        fo = lqcd.field(od, lqcd.LQCD_LAYOUT_EO, prec, 1, osc)
        (lqcd.lqcd_apply_Mdag if dagger else lqcd.lqcd_apply_M)(ctx, G, fi, fo, kappa, mu)
        tol = 2e-6 if prec == lqcd.LQCD_F32 else 1e-13
        assert relerr(lexi_from_eo_full(ctx, L, fo), ref) <= tol
    x = torch.zeros((16, 4, 3), dtype=torch.complex128, device="cuda")
    st = lqcd.lqcd_cg_solve(ctx, G, lqcd.field(dev(psi), lqcd.LQCD_LAYOUT_LEXI),
                            lqcd.field(x, lqcd.LQCD_LAYOUT_LEXI), kappa, mu, lqcd.cg_params(tol=1e-10))
    r = psi - oracle.apply_M(U, host(x), L, kappa, mu)
    assert st[0]["converged"] and np.linalg.norm(r) / np.linalg.norm(psi) <= 1e-10


@pytest.mark.parametrize("inner", [lqcd.LQCD_F64, lqcd.LQCD_F32])
def test_zero_right_hand_side(ctx, oracle, inner):
    L = (4, 4, 4, 4)
    kappa, mu = 0.15, 0.1
    U = inputs.random_gauge(L, "haar", seed=63)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    b = np.zeros((3, 256, 4, 3), np.complex128)
    b[1] = inputs.gaussian_spinor(L, 64)
    x = torch.full((3, 256, 4, 3), 7.0, dtype=torch.complex128, device="cuda")
    prm = lqcd.cg_params(tol=1e-10, inner_prec=inner)
    st = lqcd.lqcd_cg_solve(ctx, G, lqcd.field(dev(b), lqcd.LQCD_LAYOUT_LEXI, nrhs=3),
                            lqcd.field(x, lqcd.LQCD_LAYOUT_LEXI, nrhs=3), kappa, mu, prm)
    xh = host(x)
    assert np.all(xh[0] == 0) and np.all(xh[2] == 0)
    assert st[0]["true_resid"] == 0.0 and st[0]["converged"] == 1
    r = b[1] - oracle.apply_M(U, xh[1], L, kappa, mu)
    assert np.linalg.norm(r) / np.linalg.norm(b[1]) <= 1e-10


@pytest.mark.parametrize("prec", [lqcd.LQCD_F64, lqcd.LQCD_DF64, lqcd.LQCD_F32])
def test_degenerate_parameters(ctx, oracle, prec):
    """The method's degenerate points: kappa = 0 makes M the identity (no hop,
    no twisted term), mu = 0 the plain Wilson operator, and the solve of M x
    = b at kappa = 0 returns b itself."""
    L = (4, 4, 2, 6)
    U = inputs.random_gauge(L, "haar", seed=68)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    psi = inputs.gaussian_spinor(L, 69)
    tol = 2e-6 if prec == lqcd.LQCD_F32 else 1e-13
    for kappa, mu in ((0.0, 0.7), (0.14, 0.0)):
        ref = psi if kappa == 0.0 else oracle.apply_M(U, psi, L, kappa, mu)
        _, _, fi = eo_full_from_lexi(ctx, L, psi, prec)
        od, osc = lqcd.alloc_field(L, lqcd.LQCD_FULL, prec)
        fo = lqcd.field(od, lqcd.LQCD_LAYOUT_EO, prec, 1, osc)
        lqcd.lqcd_apply_M(ctx, G, fi, fo, kappa, mu)
        assert relerr(lexi_from_eo_full(ctx, L, fo), ref) <= tol, (kappa, mu)
    x = torch.zeros((inputs.volume(L), 4, 3), dtype=torch.complex128, device="cuda")
    st = lqcd.lqcd_cg_solve(ctx, G, lqcd.field(dev(psi), lqcd.LQCD_LAYOUT_LEXI),
                            lqcd.field(x, lqcd.LQCD_LAYOUT_LEXI), 0.0, 0.7,
                            lqcd.cg_params(tol=1e-10, outer_prec=prec if prec != lqcd.LQCD_F32 else lqcd.LQCD_DF64,
                                           inner_prec=prec))
    assert st[0]["converged"] == 1
    assert np.max(np.abs(host(x) - psi)) <= 1e-10 * np.max(np.abs(psi))


def test_largest_workload_lattice(ctx, oracle):
    """32^3 x 64 (2097152 sites): M on every site against the oracle, F64 and DF64."""
    L = (32, 32, 32, 64)
    kappa, mu = 0.157, 0.003 / 0.314
    U = inputs.random_gauge(L, "near", seed=65, eps=0.3)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    psi = inputs.gaussian_spinor(L, 66)
    ref = oracle.apply_M(U, psi, L, kappa, mu)
    for prec in (lqcd.LQCD_F64, lqcd.LQCD_DF64):
        _, _, fi = eo_full_from_lexi(ctx, L, psi, prec)
        od, osc = lqcd.alloc_field(L, lqcd.LQCD_FULL, prec)
        fo = lqcd.field(od, lqcd.LQCD_LAYOUT_EO, prec, 1, osc)
        lqcd.lqcd_apply_M(ctx, G, fi, fo, kappa, mu)
        assert relerr(lexi_from_eo_full(ctx, L, fo), ref) <= 1e-13


def test_heatbath_beta_zero(ctx, oracle):
    L = (4, 4, 4, 4)
    U = inputs.random_gauge(L, "haar", seed=67)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    lqcd.lqcd_heatbath_sweep(ctx, G, 0.0, 5, 0)
    Uo, fails = oracle.heatbath_sweep(U, L, 0.0, 5, 0)
    out = torch.zeros((256, 4, 3, 3), dtype=torch.complex128, device="cuda")
    lqcd.lqcd_gauge_export(ctx, G, out)
    got = host(out)
    assert np.all(np.isfinite(got))
    diff = np.abs(got - Uo).max(axis=(2, 3))
    assert np.sum(diff > 1e-9) <= 4 and np.median(diff) < 1e-13


def test_argument_errors(ctx):
    L = (4, 4, 4, 4)
    G = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "cold")), L)
    d, _ = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64)
    d2, _ = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64)
    f, f2 = lqcd.field(d), lqcd.field(d2)
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.lqcd_apply_M(ctx, G, f, f2, float("nan"), 0.1)
    assert e.value.status == lqcd.LQCD_ERR_NONFINITE
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.lqcd_apply_M(ctx, G, f, f2, 0.1, 0.1, parity=7)
    assert e.value.status == lqcd.LQCD_ERR_INVALID
    g = G.geom
    st = lqcd.lib().lqcd_cg_solve(ctx.handle, G.handle, f, f2, ctypes.byref(g), 0.1, 0.1,
                                  ctypes.byref(lqcd.cg_params()), None)
    assert st == lqcd.LQCD_ERR_INVALID
    with pytest.raises(lqcd.LqcdError) as e:  # geometry mismatch
        other = lqcd.geom((4, 4, 4, 8))
        ctx.check(lqcd.lib().lqcd_dslash(ctx.handle, G.handle, f, f2, ctypes.byref(other),
                                         lqcd.LQCD_EVEN, 0))
    assert e.value.status == lqcd.LQCD_ERR_INVALID
