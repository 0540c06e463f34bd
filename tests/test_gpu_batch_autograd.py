"""GPU tests of the batched solver over uneven lattices and of the autograd
wrapper of the fermion force.

Batched solve: every system's solution has a true residual <= 1e-10 against
the oracle's operator, and equals the solution of the unbatched solver bit for
bit (the batched kernels run the same per-site arithmetic and reduce over the
same 32-site groups in the same order).
"""
import numpy as np
import pytest
import torch

from paper_1209_5942_gb300 import inputs, lqcd
from tests.gpu_util import dev, eo_full_from_lexi, half_views, host, lexi_from_eo_full

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1209_5942_gb300 import build
    build.build()
    return lqcd.Context(0)


SHAPES = [(4, 4, 4, 4), (4, 4, 4, 8), (6, 4, 4, 4), (8, 8, 8, 8), (2, 4, 6, 8)]


def _systems(ctx, recon=18):
    out = []
    for k, L in enumerate(SHAPES):
        U = inputs.random_gauge(L, "near", seed=700 + k, eps=0.3)
        b = inputs.gaussian_spinor(L, 800 + k)
        G = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=recon)
        bd, _, fb = eo_full_from_lexi(ctx, L, b)
        xd, _ = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64)
        fx = lqcd.field(xd, lqcd.LQCD_LAYOUT_EO)
        kappa = 0.15 + 0.002 * k
        mu = (0.005 + 0.001 * k) / (2 * kappa)
        out.append(dict(L=L, U=U, b=b, G=G, fb=fb, fx=fx, xd=xd, kappa=kappa, mu=mu))
    return out


@pytest.mark.parametrize("outer,inner,recon,graph", [
    (lqcd.LQCD_F64, lqcd.LQCD_F64, 18, 1),
    (lqcd.LQCD_DF64, lqcd.LQCD_F32, 12, 1),
    (lqcd.LQCD_DF64, lqcd.LQCD_BF16S, 12, 0),
    (lqcd.LQCD_F64, lqcd.LQCD_F32, 18, 0),
])
def test_batched_solve_matches_oracle_and_unbatched(ctx, oracle, outer, inner, recon, graph):
    sysl = _systems(ctx, recon)
    prm = lqcd.cg_params(tol=1e-10, outer_prec=outer, inner_prec=inner, use_graph=graph,
                         sloppy_recon=recon)
    st = lqcd.lqcd_cg_solve_batch(ctx, [s["G"] for s in sysl], [s["fb"] for s in sysl],
                                  [s["fx"] for s in sysl], [s["kappa"] for s in sysl],
                                  [s["mu"] for s in sysl], prm)
    assert len(st) == len(sysl)
    for s, stat in zip(sysl, st):
        assert stat["converged"] == 1, stat
        x = lexi_from_eo_full(ctx, s["L"], s["fx"])
        r = s["b"] - oracle.apply_M(s["U"], x, s["L"], s["kappa"], s["mu"])
        assert np.linalg.norm(r) / np.linalg.norm(s["b"]) <= 1e-10
        # the unbatched solver gives the same bits
        xd2, _ = lqcd.alloc_field(s["L"], lqcd.LQCD_FULL, lqcd.LQCD_F64)
        fx2 = lqcd.field(xd2, lqcd.LQCD_LAYOUT_EO)
        st1 = lqcd.lqcd_cg_solve(ctx, s["G"], s["fb"], fx2, s["kappa"], s["mu"], prm)
        torch.cuda.synchronize()
        if inner == outer:  # no reliable updates: one shared iteration path
            assert st1[0]["iters"] == stat["iters"]
            assert torch.equal(xd2, s["xd"])
        else:
            assert np.linalg.norm(lexi_from_eo_full(ctx, s["L"], fx2) - x) <= 1e-8 * np.linalg.norm(x)


def test_fermion_action_autograd(ctx, oracle):
    from paper_1209_5942_gb300.autograd import FermionAction
    L = (4, 4, 2, 4)
    V = inputs.volume(L)
    kappa, mu = 0.14, 0.1
    U = inputs.random_gauge(L, "near", seed=901, eps=0.4)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    ev = ~oracle.parity_mask(L)
    phi = inputs.gaussian_spinor(L, 902) * ev[:, None, None]
    d, s, _ = eo_full_from_lexi(ctx, L, phi)
    fphi, _ = half_views(L, d, s, lqcd.LQCD_F64)
    prm = lqcd.cg_params(tol=1e-13, max_iter=50000)
    Sref, X = oracle.pseudofermion_action(U, phi, L, kappa, mu, eo=True, tol=1e-14)
    ref = oracle.fermion_dSdw(U, X, L, kappa, mu, eo=True)
    for recompute in (False, True):
        omega = torch.zeros((4, V, 8), dtype=torch.float64, device="cuda", requires_grad=True)
        S = FermionAction.apply(omega, G, fphi, kappa, mu, prm, recompute)
        (2.5 * S).backward()
        assert abs(S.item() - Sref) < 1e-10 * abs(Sref)
        g = host(omega.grad)
        assert np.max(np.abs(g - 2.5 * ref)) < 1e-9 * np.max(np.abs(ref))
    # omega != 0 is not the field the library evaluates: refused, not ignored
    omega = torch.zeros((4, V, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    with torch.no_grad():
        omega[1, 3, 2] = 1e-3
    with pytest.raises(ValueError):
        FermionAction.apply(omega, G, fphi, kappa, mu, prm, False)


def test_fermion_action_recompute_keeps_no_gradient(ctx, oracle):
    """With recompute=True the forward pass allocates no [4, V, 8] gradient
    (torch's peak memory over the forward pass stays far below its size)
    and the backward pass still gives the oracle's force."""
    from paper_1209_5942_gb300.autograd import FermionAction
    L = (8, 8, 8, 8)
    V = inputs.volume(L)
    kappa, mu = 0.13, 0.1
    U = inputs.random_gauge(L, "near", seed=903, eps=0.4)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    ev = ~oracle.parity_mask(L)
    phi = inputs.gaussian_spinor(L, 904) * ev[:, None, None]
    d, s, _ = eo_full_from_lexi(ctx, L, phi)
    fphi, _ = half_views(L, d, s, lqcd.LQCD_F64)
    prm = lqcd.cg_params(tol=1e-12, max_iter=50000)
    omega = torch.zeros((4, V, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    grad_bytes = omega.numel() * 8
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    m0 = torch.cuda.memory_allocated()
    S = FermionAction.apply(omega, G, fphi, kappa, mu, prm, True)
    torch.cuda.synchronize()
    assert torch.cuda.max_memory_allocated() - m0 < grad_bytes // 4
    S.backward()
    Sref, X = oracle.pseudofermion_action(U, phi, L, kappa, mu, eo=True, tol=1e-13)
    assert abs(S.item() - Sref) < 1e-9 * abs(Sref)
    ref = oracle.fermion_dSdw(U, X, L, kappa, mu, eo=True)
    assert np.max(np.abs(host(omega.grad) - ref)) < 1e-8 * np.max(np.abs(ref))
