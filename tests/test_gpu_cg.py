"""GPU parity of the even-odd CG solve (Sec. 2.1, eq. solvereq) against the oracle.

Every solution is checked with the oracle's own operator: the true residual
|b - M x| / |b| <= 1e-10 recomputed on the CPU, and (on small lattices) the
distance to the oracle's independent unpreconditioned CG solution.  Covers
plain FP64, float-float, mixed FP32 / BF16 / FP16 inner solves with reliable
updates, multi-RHS point sources, graph and non-graph execution, and the
non-convergence status.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1209_5942_gb300 import inputs, lqcd
from tests.gpu_util import dev, host, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1209_5942_gb300 import build
    build.build()
    return lqcd.Context(0)


def _solve(ctx, G, L, b, kappa, mu, nrhs=1, **kw):
    V = inputs.volume(L)
    shape = (V, 4, 3) if nrhs == 1 else (nrhs, V, 4, 3)
    x = torch.zeros(shape, dtype=torch.complex128, device="cuda")
    fb = lqcd.field(dev(b), lqcd.LQCD_LAYOUT_LEXI, nrhs=nrhs)
    fx = lqcd.field(x, lqcd.LQCD_LAYOUT_LEXI, nrhs=nrhs)
    allow = kw.pop("allow_noconv", False)
    st = lqcd.lqcd_cg_solve(ctx, G, fb, fx, kappa, mu, lqcd.cg_params(**kw), allow_noconv=allow)
    return host(x), st


def _true_resid(oracle, U, L, x, b, kappa, mu):
    r = b - oracle.apply_M(U, x, L, kappa, mu)
    return np.linalg.norm(r) / np.linalg.norm(b)


def test_config1_4x4_haar(ctx, oracle):
    """4^4, Haar links, kappa = 0.15, 2 kappa mu = 0.01, Gaussian source."""
    L = (4, 4, 4, 4)
    kappa, mu = 0.15, 0.01 / 0.3
    U = inputs.random_gauge(L, "haar", seed=1001)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    b = inputs.gaussian_spinor(L, 1002)
    x, st = _solve(ctx, G, L, b, kappa, mu, tol=1e-10)
    assert st[0]["converged"] == 1 and st[0]["true_resid"] <= 1e-10
    assert _true_resid(oracle, U, L, x, b, kappa, mu) <= 1e-10
    xr = oracle.solve(U, b, L, kappa, mu, tol=1e-13)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-7


@pytest.mark.parametrize("outer,inner,recon", [
    (lqcd.LQCD_F64, lqcd.LQCD_F64, 18),
    (lqcd.LQCD_DF64, lqcd.LQCD_DF64, 18),
    (lqcd.LQCD_DF64, lqcd.LQCD_DF64, 12),
    (lqcd.LQCD_F64, lqcd.LQCD_F32, 18),
    (lqcd.LQCD_F64, lqcd.LQCD_F32, 12),
    (lqcd.LQCD_DF64, lqcd.LQCD_F32, 12),
    (lqcd.LQCD_DF64, lqcd.LQCD_BF16S, 12),
    (lqcd.LQCD_DF64, lqcd.LQCD_F16S, 12),
])
@pytest.mark.parametrize("use_graph", [1, 0])
def test_solve_precisions(ctx, oracle, outer, inner, recon, use_graph):
    L = (6, 4, 4, 8)
    kappa, mu = 0.16, 0.005 / 0.32
    U = inputs.random_gauge(L, "near", seed=1101, eps=0.3)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=recon)
    b = inputs.gaussian_spinor(L, 1102)
    x, st = _solve(ctx, G, L, b, kappa, mu, tol=1e-10, outer_prec=outer, inner_prec=inner,
                   use_graph=use_graph, max_iter=20000)
    assert st[0]["converged"] == 1, st
    assert _true_resid(oracle, U, L, x, b, kappa, mu) <= 1e-10
    if inner != outer:
        assert st[0]["reliable_updates"] >= 1


def test_multi_rhs_point_sources(ctx, oracle):
    """12 unit point sources solved together; each solution checked alone."""
    L = (4, 4, 4, 8)
    kappa, mu = 0.157, 0.003 / 0.314
    U = inputs.random_gauge(L, "near", seed=1201, eps=0.4)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=12)
    b = inputs.point_sources(L)
    for inner in (lqcd.LQCD_DF64, lqcd.LQCD_F32):
        x, st = _solve(ctx, G, L, b, kappa, mu, nrhs=12, tol=1e-10, outer_prec=lqcd.LQCD_DF64,
                       inner_prec=inner)
        assert len(st) == 12
        for r in range(12):
            assert st[r]["converged"] == 1
            assert _true_resid(oracle, U, L, x[r], b[r], kappa, mu) <= 1e-10


@pytest.mark.parametrize("inner", [lqcd.LQCD_BF16S, lqcd.LQCD_F16S])
def test_multi_rhs_16bit_inner_any_launch(ctx, oracle, inner):
    """12 point sources with a 16-bit inner recursion, whose 12-RHS hops the
    tuner may run as the kernel with links staged in shared memory (reducing
    variants included): with the launch left to the tuner and with each
    staged-link candidate forced (the 12-RHS 16-bit candidate list puts them
    at 39-50), every solution reaches the oracle's true residual and the
    solutions are the same bits."""
    L = (4, 4, 4, 8)
    kappa, mu = 0.157, 0.003 / 0.314
    U = inputs.random_gauge(L, "near", seed=1211, eps=0.4)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=12)
    b = inputs.point_sources(L)
    ref = None
    for choice in (-1, 39, 41, 44, 47, 50):
        lqcd.lqcd_set_launch_choice(ctx, choice)
        try:
            x, st = _solve(ctx, G, L, b, kappa, mu, nrhs=12, tol=1e-10, outer_prec=lqcd.LQCD_DF64,
                           inner_prec=inner)
        finally:
            lqcd.lqcd_set_launch_choice(ctx, -1)
        assert all(s["converged"] == 1 for s in st), (choice, st)
        if ref is None:
            ref = x
            for r in range(12):
                assert _true_resid(oracle, U, L, x[r], b[r], kappa, mu) <= 1e-10
        else:
            assert np.array_equal(x, ref), choice


def test_multi_rhs_equals_single(ctx):
    """Batched right-hand sides give the single-RHS solutions bit for bit
    (same kernels, same reduction order per right-hand side)."""
    L = (4, 4, 4, 4)
    kappa, mu = 0.15, 0.01 / 0.3
    U = inputs.random_gauge(L, "haar", seed=1301)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    b = inputs.gaussian_spinor(L, 1302, nrhs=3)
    xm, stm = _solve(ctx, G, L, b, kappa, mu, nrhs=3, tol=1e-10)
    for r in range(3):
        xs, sts = _solve(ctx, G, L, b[r], kappa, mu, tol=1e-10)
        assert sts[0]["iters"] == stm[r]["iters"]
        assert np.array_equal(xs, xm[r])


def test_deterministic_iteration_count(ctx):
    L = (8, 8, 8, 8)
    kappa, mu = 0.16, 0.005 / 0.32
    U = inputs.random_gauge(L, "near", seed=1401, eps=0.3)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    b = inputs.gaussian_spinor(L, 1402)
    x1, s1 = _solve(ctx, G, L, b, kappa, mu, tol=1e-10)
    x2, s2 = _solve(ctx, G, L, b, kappa, mu, tol=1e-10)
    assert s1[0]["iters"] == s2[0]["iters"]
    assert np.array_equal(x1, x2)


def test_noconv_status(ctx):
    L = (4, 4, 4, 4)
    kappa, mu = 0.15, 0.01 / 0.3
    U = inputs.random_gauge(L, "haar", seed=1501)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    b = inputs.gaussian_spinor(L, 1502)
    with pytest.raises(lqcd.LqcdError) as e:
        _solve(ctx, G, L, b, kappa, mu, tol=1e-10, max_iter=5, max_restarts=0)
    assert e.value.status == lqcd.LQCD_ERR_NOCONV
    x, st = _solve(ctx, G, L, b, kappa, mu, tol=1e-10, max_iter=5, max_restarts=0,
                   allow_noconv=True)
    assert st[0]["converged"] == 0 and st[0]["iters"] >= 5 and st[0]["true_resid"] > 1e-10


def test_nonfinite_source_rejected(ctx):
    L = (4, 4, 4, 4)
    U = inputs.random_gauge(L, "haar", seed=1601)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    b = inputs.gaussian_spinor(L, 1602)
    b[17, 2, 1] = np.nan
    with pytest.raises(lqcd.LqcdError) as e:
        _solve(ctx, G, L, b, 0.15, 0.03, tol=1e-10)
    assert e.value.status == lqcd.LQCD_ERR_NONFINITE


def test_full_size_24x48_solve(ctx, oracle):
    """The 24^3 x 48 workload (near-identity links eps = 0.3, kappa = 0.16,
    2 kappa mu = 0.005): true residual recomputed by the oracle."""
    L = (24, 24, 24, 48)
    kappa, mu = 0.16, 0.005 / 0.32
    U = inputs.random_gauge(L, "near", seed=2001, eps=0.3)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=12)
    b = inputs.gaussian_spinor(L, 2002)
    for outer, inner in ((lqcd.LQCD_DF64, lqcd.LQCD_DF64), (lqcd.LQCD_DF64, lqcd.LQCD_F32)):
        x, st = _solve(ctx, G, L, b, kappa, mu, tol=1e-10, outer_prec=outer, inner_prec=inner)
        assert st[0]["converged"] == 1
        assert _true_resid(oracle, U, L, x, b, kappa, mu) <= 1e-10
    G.free()
    # the benchmark's own path: IEEE FP64 with 18-real links, and the mixed
    # solve with IEEE-FP64 reliable updates and an FP32 REC12 inner operator
    G18 = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=18)
    for outer, inner, recon in ((lqcd.LQCD_F64, lqcd.LQCD_F64, 18), (lqcd.LQCD_F64, lqcd.LQCD_F32, 12)):
        x, st = _solve(ctx, G18, L, b, kappa, mu, tol=1e-10, outer_prec=outer, inner_prec=inner,
                       sloppy_recon=recon)
        assert st[0]["converged"] == 1 and st[0]["true_resid"] <= 1e-10
        res = _true_resid(oracle, U, L, x, b, kappa, mu)
        assert res <= 1e-10
        # the library's own FP64 true residual agrees with the oracle's
        assert abs(res - st[0]["true_resid"]) < 1e-3 * res


@pytest.mark.parametrize("outer,inner,recon", [
    (lqcd.LQCD_F64, lqcd.LQCD_F64, 18),
    (lqcd.LQCD_DF64, lqcd.LQCD_DF64, 18),
    (lqcd.LQCD_DF64, lqcd.LQCD_F32, 12),
    (lqcd.LQCD_DF64, lqcd.LQCD_F16S, 12),
])
@pytest.mark.parametrize("L,kind,kappa", [((4, 4, 4, 4), "haar", 0.15), ((6, 4, 2, 10), "haar", 0.15),
                                          ((6, 4, 2, 10), "near", 0.12)])
def test_bicgstab_on_mhat(ctx, oracle, outer, inner, recon, L, kind, kappa):
    """BiCGStab on Mhat (the paper's other standard solver): the oracle's true
    residual <= 1e-10 and the oracle's own solution, in plain FP64, float-float
    and mixed precision with outer refinement.  BiCGStab needs the spectrum of
    Mhat away from the origin, so the fields are Haar links, or near-identity
    links below the free critical kappa 1/8."""
    mu = 0.01 / (2 * kappa)
    U = inputs.random_gauge(L, kind, seed=1101, eps=0.4)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    b = inputs.gaussian_spinor(L, 1102)
    x, st = _solve(ctx, G, L, b, kappa, mu, tol=1e-10, outer_prec=outer, inner_prec=inner,
                   sloppy_recon=recon, solver=lqcd.LQCD_SOLVER_BICGSTAB, max_restarts=8)
    assert st[0]["converged"] == 1 and st[0]["true_resid"] <= 1e-10
    assert _true_resid(oracle, U, L, x, b, kappa, mu) <= 1e-10
    xr = oracle.solve(U, b, L, kappa, mu, tol=1e-13)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-7


def test_bicgstab_rejects_several_rhs_and_batch(ctx):
    L = (4, 4, 4, 4)
    U = inputs.random_gauge(L, "near", seed=1103)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    b = inputs.gaussian_spinor(L, 1104, nrhs=2)
    with pytest.raises(lqcd.LqcdError) as e:
        _solve(ctx, G, L, b, 0.15, 0.1, nrhs=2, solver=lqcd.LQCD_SOLVER_BICGSTAB)
    assert e.value.status == lqcd.LQCD_ERR_UNSUPPORTED


def test_bicgstab_reports_divergence(ctx):
    """Near-free links beyond the free critical kappa (spectrum of Mhat around
    the origin): BiCGStab does not converge and says so; CG on Mhat^+ Mhat
    solves the same system."""
    L = (6, 4, 2, 10)
    kappa, mu = 0.16, 0.005 / 0.32
    U = inputs.random_gauge(L, "near", seed=1105, eps=0.3)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    b = inputs.gaussian_spinor(L, 1106)
    x, st = _solve(ctx, G, L, b, kappa, mu, tol=1e-10, solver=lqcd.LQCD_SOLVER_BICGSTAB, max_iter=2000,
                   allow_noconv=True)
    x2, st2 = _solve(ctx, G, L, b, kappa, mu, tol=1e-10)
    assert st2[0]["converged"] == 1
    if not st[0]["converged"]:
        assert st[0]["true_resid"] > 1e-10


@pytest.mark.parametrize("graph,check_every", [(1, 7), (0, 7), (1, 50)])
def test_work_counters_count_executed_iterations(ctx, check_every, graph):
    """The work counters credit the iterations the device ran, not the chunk
    of check_every iterations the host enqueued (after the halting reduction
    every kernel of a host-enqueued chunk returns at once).  A plain FP64 solve of n
    iterations runs 4 half hops per iteration except the last (2: it halts
    at the |s|^2 reduction), plus 2 for the first z = Mhat^+ s and 4 outside
    the CG (source, reconstruction, the two halves of the true residual):
    4 n + 4 half hops of Vh sites, whatever the chunking."""
    L = (8, 8, 8, 8)
    kappa, mu = 0.15, 0.01 / 0.3
    U = inputs.random_gauge(L, "near", seed=1301, eps=0.4)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    b = inputs.gaussian_spinor(L, 1302)
    lqcd.lib().lqcd_reset_counters(ctx.handle)
    _, st = _solve(ctx, G, L, b, kappa, mu, tol=1e-10, check_every=check_every, use_graph=graph)
    torch.cuda.synchronize()
    cnt = lqcd.lqcd_counters()
    lqcd.lib().lqcd_get_counters(ctx.handle, ctypes.byref(cnt))
    n = st[0]["iters"]
    assert st[0]["converged"] == 1 and st[0]["restarts"] == 0
    Vh = inputs.volume(L) // 2
    assert cnt.hop_sites == Vh * (4 * n + 4)
    # launches: every enqueued kernel.  The graph runs the iterations in a
    # device-side while loop that ends at the halt, so it launches 4 half hops
    # per iteration begun (plus 2 for the first z and the 4 outside the CG);
    # host-enqueued chunks also launch the halted iterations' kernels.
    if graph:
        assert cnt.hop_launches == 4 * n + 6
    else:
        assert cnt.hop_launches == 4 * (-(-n // check_every) * check_every) + 6
