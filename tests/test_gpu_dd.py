"""Domain decomposition of the half hop along t, and along z and t (the
paper's Sec. 6 outlook), on one GPU: the lattice is split into nt (or nz x
nt) domains held as separate library fields on their local geometry, each
half hop packs the spin-projected faces, moves them between the domains (the
device copies of LocalExchange stand in for NCCL; the kernels do not wait on
one another) and runs the domain hops.  The assembled result is compared
with the FP64 oracle's hop on the whole lattice, for both parities, H and
H^+, 18 and 12 real links, periodic and antiperiodic time, and with the
library's own single-domain hop; the decomposed CG likewise with the
oracle's solution."""
import numpy as np
import pytest
import torch

from paper_1209_5942_gb300 import dd, inputs, lqcd
from tests.gpu_util import dev, eo_full_from_lexi, half_views, host, relerr

pytestmark = pytest.mark.gpu

TOL = {lqcd.LQCD_F64: 1e-13, lqcd.LQCD_DF64: 1e-13, lqcd.LQCD_F32: 2e-6}


@pytest.fixture(scope="module")
def ctx():
    from paper_1209_5942_gb300 import build
    build.build()
    return lqcd.Context(0)


def _domain_hop(ctx, U, psi, L, nt, prec, recon, parity, dagger, antiper, nz=1):
    """Assembled lexicographic result of the domain-decomposed half hop."""
    slabs = dd.DomainGrid(L, nz, nt, antiper)
    Ll = slabs.local_L
    p = 0 if parity == lqcd.LQCD_EVEN else 1
    gauges, ins, outs, keep = [], [], [], []
    for d in range(slabs.ndomains):
        G = lqcd.lqcd_gauge_import(ctx, dev(U[slabs.block(d)]), Ll, recon=recon, antiperiodic_t=False)
        data, scale, _ = eo_full_from_lexi_local(ctx, Ll, psi[slabs.block(d)], prec)
        fe, fo = half_views(Ll, data, scale, prec)
        odata, oscale = lqcd.alloc_field(Ll, lqcd.LQCD_FULL, prec)
        oe, oo = half_views(Ll, odata, oscale, prec)
        gauges.append(G)
        ins.append(fo if p == 0 else fe)
        outs.append(oe if p == 0 else oo)
        keep.append((data, scale, odata, oscale))
    dd.dslash_local_domains(ctx, slabs, gauges, ins, outs, parity, dagger)
    torch.cuda.synchronize()
    res = np.zeros_like(psi)
    for d in range(slabs.ndomains):
        full = lqcd.field(keep[d][2], lqcd.LQCD_LAYOUT_EO, prec, 1, keep[d][3])
        V = slabs.local_volume
        o = torch.zeros((1, V, 4, 3), dtype=torch.complex128, device="cuda")
        lqcd.lqcd_spinor_unpack(ctx, Ll, full, o, antiperiodic_t=False)
        res[slabs.block(d)] = host(o)[0]
    return res


def eo_full_from_lexi_local(ctx, L, psi_lexi, prec):
    data, scale = lqcd.alloc_field(L, lqcd.LQCD_FULL, prec)
    f = lqcd.field(data, lqcd.LQCD_LAYOUT_EO, prec, 1, scale)
    lqcd.lqcd_spinor_pack(ctx, L, dev(np.ascontiguousarray(psi_lexi)), f, antiperiodic_t=False)
    torch.cuda.synchronize()
    return data, scale, f


@pytest.mark.parametrize("L,nt", [((4, 4, 4, 8), 1), ((4, 4, 4, 8), 2), ((4, 4, 4, 8), 4), ((6, 4, 2, 12), 3)])
@pytest.mark.parametrize("prec", [lqcd.LQCD_F64, lqcd.LQCD_DF64, lqcd.LQCD_F32])
def test_dd_hop_matches_oracle(ctx, oracle, L, nt, prec):
    U = inputs.random_gauge(L, "haar", seed=71)
    psi = inputs.gaussian_spinor(L, 72)
    odd = oracle.parity_mask(L)
    for recon in (18, 12):
        for antiper in (True, False):
            for parity in (lqcd.LQCD_EVEN, lqcd.LQCD_ODD):
                for dagger in (0, 1):
                    got = _domain_hop(ctx, U, psi, L, nt, prec, recon, parity, dagger, antiper)
                    src = psi * (odd if parity == lqcd.LQCD_EVEN else ~odd)[:, None, None]
                    ref = oracle.hop(U, src, L, antiperiodic_t=antiper, dagger=bool(dagger))
                    mask = ~odd if parity == lqcd.LQCD_EVEN else odd
                    err = relerr(got[mask], ref[mask])
                    assert err < TOL[prec], (recon, antiper, parity, dagger, err)


@pytest.mark.parametrize("L,nz,nt", [((4, 4, 4, 8), 2, 1), ((4, 4, 4, 8), 2, 2), ((4, 2, 8, 4), 4, 2),
                                     ((6, 4, 4, 12), 2, 3)])
@pytest.mark.parametrize("prec", [lqcd.LQCD_F64, lqcd.LQCD_DF64, lqcd.LQCD_F32])
def test_dd_hop_zt_matches_oracle(ctx, oracle, L, nz, nt, prec):
    """The lattice split along z and t: z faces (periodic, no sign) and t
    faces (the global antiperiodic sign) together give the oracle's hop."""
    U = inputs.random_gauge(L, "haar", seed=75)
    psi = inputs.gaussian_spinor(L, 76)
    odd = oracle.parity_mask(L)
    for recon in (18, 12):
        for antiper in (True, False):
            for parity in (lqcd.LQCD_EVEN, lqcd.LQCD_ODD):
                for dagger in (0, 1):
                    got = _domain_hop(ctx, U, psi, L, nt, prec, recon, parity, dagger, antiper, nz=nz)
                    src = psi * (odd if parity == lqcd.LQCD_EVEN else ~odd)[:, None, None]
                    ref = oracle.hop(U, src, L, antiperiodic_t=antiper, dagger=bool(dagger))
                    mask = ~odd if parity == lqcd.LQCD_EVEN else odd
                    err = relerr(got[mask], ref[mask])
                    assert err < TOL[prec], (recon, antiper, parity, dagger, err)


def test_dd_face_sizes_and_direction_checks(ctx):
    """Face bytes along z and t; a pack along x, y or an unknown direction is
    refused, as is a z face pair with one pointer missing."""
    Ll = (4, 6, 2, 4)
    assert lqcd.lqcd_dd_face_bytes_dir(Ll, 3, lqcd.LQCD_F64) == 2 * 6 * 2 * 6 * 16
    assert lqcd.lqcd_dd_face_bytes_dir(Ll, 2, lqcd.LQCD_F64) == 2 * 6 * 4 * 6 * 16
    assert lqcd.lqcd_dd_face_bytes_dir(Ll, 2, lqcd.LQCD_F32) == 2 * 6 * 4 * 6 * 8
    assert lqcd.lqcd_dd_face_bytes_dir(Ll, 1, lqcd.LQCD_F64) == 0
    assert lqcd.lqcd_dd_face_bytes(Ll, lqcd.LQCD_F64) == lqcd.lqcd_dd_face_bytes_dir(Ll, 3, lqcd.LQCD_F64)
    G = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(Ll, "cold")), Ll, antiperiodic_t=False)
    d64, _ = lqcd.alloc_field(Ll, lqcd.LQCD_EVEN, lqcd.LQCD_F64)
    o64, _ = lqcd.alloc_field(Ll, lqcd.LQCD_EVEN, lqcd.LQCD_F64)
    f, o = lqcd.field(d64, lqcd.LQCD_LAYOUT_EO), lqcd.field(o64, lqcd.LQCD_LAYOUT_EO)
    buf = torch.zeros(8192, dtype=torch.float64, device="cuda")
    for mu in (0, 1, 4):
        with pytest.raises(lqcd.LqcdError) as e:
            lqcd.lqcd_dd_pack_dir(ctx, G, f, mu, buf, buf[4096:], lqcd.LQCD_ODD)
        assert e.value.status == lqcd.LQCD_ERR_INVALID
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.lqcd_dd_dslash_zt(ctx, G, f, o, buf, buf[2048:], buf[4096:], None, lqcd.LQCD_ODD)
    assert e.value.status == lqcd.LQCD_ERR_INVALID


def test_dd_hop_matches_single_domain_library_hop(ctx, oracle):
    """nt = 2 against lqcd_dslash on the undivided lattice (F64)."""
    L = (4, 4, 2, 8)
    U = inputs.random_gauge(L, "near", seed=73, eps=0.5)
    psi = inputs.gaussian_spinor(L, 74)
    got = _domain_hop(ctx, U, psi, L, 2, lqcd.LQCD_F64, 18, lqcd.LQCD_ODD, 0, True)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    data, scale, _ = eo_full_from_lexi(ctx, L, psi)
    fe, fo = half_views(L, data, scale, lqcd.LQCD_F64)
    odata, oscale = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64)
    oe, oo = half_views(L, odata, oscale, lqcd.LQCD_F64)
    lqcd.lqcd_dslash(ctx, G, fe, oo, lqcd.LQCD_ODD, 0)
    V = inputs.volume(L)
    o = torch.zeros((1, V, 4, 3), dtype=torch.complex128, device="cuda")
    lqcd.lqcd_spinor_unpack(ctx, L, lqcd.field(odata, lqcd.LQCD_LAYOUT_EO), o)
    ref = host(o)[0]
    mask = oracle.parity_mask(L)
    assert relerr(got[mask], ref[mask]) < 1e-14


def test_dd_rejects_bad_input(ctx):
    L = (4, 4, 4, 4)
    G = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "cold")), L, antiperiodic_t=False)
    d, s = lqcd.alloc_field(L, lqcd.LQCD_EVEN, lqcd.LQCD_BF16S)
    f = lqcd.field(d, lqcd.LQCD_LAYOUT_EO, lqcd.LQCD_BF16S, 1, s)
    buf = torch.zeros(4096, dtype=torch.float64, device="cuda")
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.lqcd_dd_pack(ctx, G, f, buf, buf[2048:], lqcd.LQCD_EVEN)
    assert e.value.status == lqcd.LQCD_ERR_UNSUPPORTED
    d64, _ = lqcd.alloc_field(L, lqcd.LQCD_EVEN, lqcd.LQCD_F64)
    f64 = lqcd.field(d64, lqcd.LQCD_LAYOUT_EO)
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.lqcd_dd_pack(ctx, G, f64, buf, buf, lqcd.LQCD_EVEN)  # aliasing faces
    assert e.value.status == lqcd.LQCD_ERR_INVALID
    assert lqcd.lqcd_dd_face_bytes((4, 4, 4, 3), lqcd.LQCD_F64) == 0
    assert lqcd.lqcd_dd_face_bytes((4, 4, 4, 4), lqcd.LQCD_F64) == 2 * 4 * 4 * 6 * 16


# ---------------------------------------------------------------------------
# The domain-decomposed CG (lqcd_dd_cg_solve), FP64 and mixed precision
# ---------------------------------------------------------------------------

def _dd_solve(ctx, U, b, L, nt, kappa, mu, antiper=True, recon=18, hooks=None, nz=1, **kw):
    """Solve M x = b with the lattice split into nt (nz x nt) domains held in
    this process; hooks = (exchange, allreduce) factory or None (the library
    moves the faces).  Returns the assembled lexicographic x and the stats."""
    slabs = dd.DomainGrid(L, nz, nt, antiper)
    Ll = slabs.local_L
    gauges, bs, xs, keep = [], [], [], []
    for d in range(slabs.ndomains):
        G = lqcd.lqcd_gauge_import(ctx, dev(U[slabs.block(d)]), Ll, recon=recon, antiperiodic_t=False)
        bd, _, fb = eo_full_from_lexi_local(ctx, Ll, b[slabs.block(d)], lqcd.LQCD_F64)
        xd, _ = lqcd.alloc_field(Ll, lqcd.LQCD_FULL, lqcd.LQCD_F64)
        gauges.append(G)
        bs.append(fb)
        xs.append(lqcd.field(xd, lqcd.LQCD_LAYOUT_EO))
        keep.append((bd, xd))
    prm = lqcd.cg_params(**kw)
    if hooks is None:
        st = dd.cg_solve_local_domains(ctx, slabs, gauges, bs, xs, kappa, mu, prm)
    else:
        faces = [dd.domain_faces(slabs, lqcd.LQCD_F64) for _ in range(slabs.ndomains)]
        exchange, allreduce = hooks(slabs, faces)
        st = lqcd.lqcd_dd_cg_solve(ctx, gauges, bs, xs, faces, 0, nt, kappa, mu, prm, antiperiodic_t=antiper,
                                   exchange=exchange, allreduce=allreduce, nz=nz)
    torch.cuda.synchronize()
    x = np.zeros_like(b)
    for d in range(slabs.ndomains):
        o = torch.zeros((1, slabs.local_volume, 4, 3), dtype=torch.complex128, device="cuda")
        lqcd.lqcd_spinor_unpack(ctx, Ll, xs[d], o, antiperiodic_t=False)
        x[slabs.block(d)] = host(o)[0]
    return x, st


def _oracle_resid(oracle, U, L, x, b, kappa, mu, antiper=True):
    r = b - oracle.apply_M(U, x, L, kappa, mu, antiperiodic_t=antiper)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("L,nt", [((4, 4, 4, 8), 1), ((4, 4, 4, 8), 2), ((4, 4, 4, 8), 4), ((6, 4, 2, 12), 3)])
def test_dd_cg_matches_oracle(ctx, oracle, L, nt):
    """The decomposed solve reaches the oracle's true residual 1e-10 on the
    whole lattice and the oracle's own solution, for 18 and 12 real links and
    antiperiodic and periodic time."""
    kappa, mu = 0.15, 0.01 / 0.3
    U = inputs.random_gauge(L, "haar", seed=81)
    b = inputs.gaussian_spinor(L, 82)
    for recon, antiper in ((18, True), (12, True), (18, False)):
        x, st = _dd_solve(ctx, U, b, L, nt, kappa, mu, antiper=antiper, recon=recon, tol=1e-10)
        assert st["converged"] == 1 and st["true_resid"] <= 1e-10, (recon, antiper, st)
        assert _oracle_resid(oracle, U, L, x, b, kappa, mu, antiper) <= 1e-10
        xr = oracle.solve(U, b, L, kappa, mu, tol=1e-13, antiperiodic_t=antiper)
        assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-7, (recon, antiper)


def test_dd_cg_iterations_match_the_single_domain_solver(ctx, oracle):
    """Same recurrence as lqcd_cg_solve in plain FP64: the iteration counts
    agree (the norms are summed in another order, so the iterates differ by
    rounding only), near-identity links at kappa = 0.16 as in the bench
    workload."""
    L = (8, 4, 4, 8)
    kappa, mu = 0.16, 0.005 / 0.32
    U = inputs.random_gauge(L, "near", seed=83, eps=0.3)
    b = inputs.gaussian_spinor(L, 84)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    xg = torch.zeros((inputs.volume(L), 4, 3), dtype=torch.complex128, device="cuda")
    st1 = lqcd.lqcd_cg_solve(ctx, G, lqcd.field(dev(b), lqcd.LQCD_LAYOUT_LEXI),
                             lqcd.field(xg, lqcd.LQCD_LAYOUT_LEXI), kappa, mu, lqcd.cg_params(tol=1e-10))[0]
    for nt in (2, 4):
        x, st = _dd_solve(ctx, U, b, L, nt, kappa, mu, tol=1e-10)
        assert abs(st["iters"] - st1["iters"]) <= 1, (nt, st["iters"], st1["iters"])
        assert st["true_resid"] <= 1e-10
        assert relerr(x, host(xg)) < 1e-8


@pytest.mark.parametrize("nz,nt", [(1, 2), (2, 2)])
@pytest.mark.parametrize("inner", [lqcd.LQCD_F64, lqcd.LQCD_F32])
def test_dd_cg_with_caller_hooks_equals_library_moves(ctx, inner, nz, nt):
    """The same solve with the faces moved and the norms summed by the
    caller's hooks (as a multi-process job would, here device copies in one
    process, of the leading bytes the library names only) gives the same
    bits; every half hop calls the exchange hook and every norm the allreduce
    hook; a mixed solve asks for FP64 faces in its FP64 steps and for F32
    faces (half the bytes) in its inner ones; z faces only when z is split."""
    L = (4, 4, 4, 8)
    kappa, mu = 0.15, 0.01 / 0.3
    U = inputs.random_gauge(L, "haar", seed=85)
    b = inputs.gaussian_spinor(L, 86)
    calls = {"ex": 0, "ar": 0, "bytes": set()}

    def hooks(slabs, faces):
        def exchange(t_bytes, z_bytes):
            calls["ex"] += 1
            calls["bytes"].add((t_bytes, z_bytes))
            for k, mu in enumerate(slabs.dirs):
                nb = t_bytes if mu == dd.T_DIR else z_bytes
                lead = [[f.view(torch.uint8)[:nb] for f in fs[4 * k:4 * k + 4]] for fs in faces]
                dd.LocalExchange().exchange(slabs, [f[0] for f in lead], [f[1] for f in lead],
                                            [f[2] for f in lead], [f[3] for f in lead], mu=mu)
            torch.cuda.synchronize()

        def allreduce(vals):
            calls["ar"] += 1
            return vals
        return exchange, allreduce

    x0, st0 = _dd_solve(ctx, U, b, L, nt, kappa, mu, tol=1e-10, inner_prec=inner, nz=nz)
    x1, st1 = _dd_solve(ctx, U, b, L, nt, kappa, mu, hooks=hooks, tol=1e-10, inner_prec=inner, nz=nz)
    assert st0["iters"] == st1["iters"] and np.array_equal(x0, x1)
    assert calls["ex"] >= 4 * st1["iters"] and calls["ar"] >= 3 * st1["iters"]
    Ll = dd.DomainGrid(L, nz, nt).local_L
    t64 = lqcd.lqcd_dd_face_bytes_dir(Ll, 3, lqcd.LQCD_F64)
    z64 = lqcd.lqcd_dd_face_bytes_dir(Ll, 2, lqcd.LQCD_F64) if nz > 1 else 0
    assert calls["bytes"] == ({(t64, z64)} if inner == lqcd.LQCD_F64 else {(t64, z64), (t64 // 2, z64 // 2)})


@pytest.mark.parametrize("inner", [lqcd.LQCD_F64, lqcd.LQCD_F32])
@pytest.mark.parametrize("L,nz,nt", [((4, 4, 4, 8), 2, 1), ((4, 4, 4, 8), 2, 2), ((4, 2, 8, 8), 4, 2)])
def test_dd_cg_zt_matches_oracle(ctx, oracle, L, nz, nt, inner):
    """The decomposed solve on a z x t grid of domains reaches the oracle's
    true residual 1e-10 on the whole lattice and the oracle's solution, FP64
    and with an F32 inner solve, 18 and 12 real links, both time
    boundaries."""
    kappa, mu = 0.15, 0.01 / 0.3
    U = inputs.random_gauge(L, "haar", seed=89)
    b = inputs.gaussian_spinor(L, 90)
    for recon, antiper in ((18, True), (12, True), (18, False)):
        x, st = _dd_solve(ctx, U, b, L, nt, kappa, mu, antiper=antiper, recon=recon, tol=1e-10, nz=nz,
                          inner_prec=inner)
        assert st["converged"] == 1 and st["true_resid"] <= 1e-10, (recon, antiper, st)
        assert _oracle_resid(oracle, U, L, x, b, kappa, mu, antiper) <= 1e-10
        xr = oracle.solve(U, b, L, kappa, mu, tol=1e-13, antiperiodic_t=antiper)
        assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-7, (recon, antiper)


@pytest.mark.parametrize("inner", [lqcd.LQCD_F32, lqcd.LQCD_DF64])
@pytest.mark.parametrize("L,nt", [((4, 4, 4, 8), 1), ((4, 4, 4, 8), 2), ((4, 4, 4, 8), 4), ((6, 4, 2, 12), 3)])
def test_dd_mixed_cg_matches_oracle(ctx, oracle, L, nt, inner):
    """Mixed precision in the decomposed solve (defect correction with an F32
    or float-float inner CGLS): the oracle's true residual 1e-10 on the whole
    lattice and the oracle's own solution, for 18 and 12 real links, 12-real
    inner links under an 18-real field, and antiperiodic and periodic time;
    the F32 solve needs refinement cycles (each gains 1e-5 at most)."""
    kappa, mu = 0.15, 0.01 / 0.3
    U = inputs.random_gauge(L, "haar", seed=81)
    b = inputs.gaussian_spinor(L, 82)
    xr = {ap: oracle.solve(U, b, L, kappa, mu, tol=1e-13, antiperiodic_t=ap) for ap in (True, False)}
    for recon, sloppy, antiper in ((18, 0, True), (12, 0, True), (18, 12, True), (18, 0, False)):
        x, st = _dd_solve(ctx, U, b, L, nt, kappa, mu, antiper=antiper, recon=recon, tol=1e-10,
                          inner_prec=inner, sloppy_recon=sloppy)
        assert st["converged"] == 1 and st["true_resid"] <= 1e-10, (recon, sloppy, antiper, st)
        assert _oracle_resid(oracle, U, L, x, b, kappa, mu, antiper) <= 1e-10
        assert np.linalg.norm(x - xr[antiper]) / np.linalg.norm(xr[antiper]) < 1e-7, (recon, sloppy, antiper)
        if inner == lqcd.LQCD_F32:
            assert st["restarts"] >= 1, st


def test_dd_mixed_cg_iterations_near_the_fp64_solve(ctx):
    """On a bench-like field (near-identity links, kappa = 0.16) the F32 inner
    solve with defect correction takes at most 1.5 times the FP64 solve's
    iterations to the same tolerance, and the float-float one at most 1.1
    times; every solve reaches 1e-10."""
    L = (8, 4, 4, 8)
    kappa, mu = 0.16, 0.005 / 0.32
    U = inputs.random_gauge(L, "near", seed=83, eps=0.3)
    b = inputs.gaussian_spinor(L, 84)
    _, s64 = _dd_solve(ctx, U, b, L, 2, kappa, mu, tol=1e-10)
    for inner, bound in ((lqcd.LQCD_F32, 1.5), (lqcd.LQCD_DF64, 1.1)):
        _, st = _dd_solve(ctx, U, b, L, 2, kappa, mu, tol=1e-10, inner_prec=inner)
        assert st["true_resid"] <= 1e-10, (inner, st)
        assert st["iters"] <= bound * s64["iters"] + 2, (inner, st["iters"], s64["iters"])


def test_dd_cg_reports_hook_failures_and_bad_requests(ctx):
    L = (4, 4, 4, 8)
    U = inputs.random_gauge(L, "haar", seed=87)
    b = inputs.gaussian_spinor(L, 88)

    def failing(slabs, faces):
        def exchange(t_bytes, z_bytes):
            raise RuntimeError("peer lost")
        return exchange, None

    with pytest.raises(RuntimeError, match="peer lost"):
        _dd_solve(ctx, U, b, L, 2, 0.15, 0.1, hooks=failing, tol=1e-10)
    slabs = dd.TimeSlabs(L, 2)
    Ll = slabs.local_L
    G = lqcd.lqcd_gauge_import(ctx, dev(U[slabs.block(0)]), Ll, antiperiodic_t=False)
    bd, _, fb = eo_full_from_lexi_local(ctx, Ll, b[slabs.block(0)], lqcd.LQCD_F64)
    xd, _ = lqcd.alloc_field(Ll, lqcd.LQCD_FULL, lqcd.LQCD_F64)
    fx = lqcd.field(xd, lqcd.LQCD_LAYOUT_EO)
    faces = [dd.domain_faces(slabs, lqcd.LQCD_F64)]
    with pytest.raises(lqcd.LqcdError) as e:  # one of two domains, no hooks
        lqcd.lqcd_dd_cg_solve(ctx, [G], [fb], [fx], faces, 0, 2, 0.15, 0.1, lqcd.cg_params())
    assert e.value.status == lqcd.LQCD_ERR_INVALID
    for bad in (dict(inner_prec=lqcd.LQCD_BF16S), dict(outer_prec=lqcd.LQCD_DF64, inner_prec=lqcd.LQCD_F32),
                dict(solver=lqcd.LQCD_SOLVER_BICGSTAB)):
        with pytest.raises(lqcd.LqcdError) as e:  # 16-bit inner, float-float outer, BiCGStab: not offered
            lqcd.lqcd_dd_cg_solve(ctx, [G], [fb], [fx], faces, 0, 1, 0.15, 0.1, lqcd.cg_params(**bad))
        assert e.value.status == lqcd.LQCD_ERR_UNSUPPORTED, bad


def _dd_rank(rank, world, port, L, kappa, mu, inner, nz, q):
    """One rank of a two-process decomposed solve: its own CUDA context on the
    same GPU, gloo for the face exchange (through host copies) and the norm
    sums, so no kernel waits on the other process."""
    import os
    import torch.distributed as dist
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        torch.cuda.set_device(0)
        ctx = lqcd.Context(0)
        slabs = dd.DomainGrid(L, nz, world // nz)
        Ll = slabs.local_L
        U = inputs.random_gauge(L, "haar", seed=91)
        b = inputs.gaussian_spinor(L, 92)
        G = lqcd.lqcd_gauge_import(ctx, dev(U[slabs.block(rank)]), Ll, antiperiodic_t=False)
        _, _, fb = eo_full_from_lexi_local(ctx, Ll, b[slabs.block(rank)], lqcd.LQCD_F64)
        xd, _ = lqcd.alloc_field(Ll, lqcd.LQCD_FULL, lqcd.LQCD_F64)
        fx = lqcd.field(xd, lqcd.LQCD_LAYOUT_EO)
        st = dd.cg_solve_distributed(ctx, slabs, rank, G, fb, fx, kappa, mu,
                                     lqcd.cg_params(tol=1e-10, inner_prec=inner))
        torch.cuda.synchronize()
        o = torch.zeros((1, slabs.local_volume, 4, 3), dtype=torch.complex128, device="cuda")
        lqcd.lqcd_spinor_unpack(ctx, Ll, fx, o, antiperiodic_t=False)
        q.put((rank, host(o)[0], st))
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent
        q.put((rank, None, repr(e)))


@pytest.mark.parametrize("inner,nz", [(lqcd.LQCD_F64, 1), (lqcd.LQCD_F32, 1), (lqcd.LQCD_F64, 2)])
def test_dd_cg_two_processes_with_gloo(ctx, oracle, inner, nz):
    """The decomposed solve as a two-process job (one domain per rank, the
    solver's hooks from DistributedComm over gloo), split along t (FP64 and
    with an F32 inner solve) or along z: the assembled solution reaches the
    oracle's true residual 1e-10 on the whole lattice, and both ranks report
    the same iterations and residual."""
    import socket
    import torch.multiprocessing as mp
    s_ = socket.socket()
    s_.bind(("127.0.0.1", 0))
    port = s_.getsockname()[1]
    s_.close()
    L = (4, 4, 4, 8)
    kappa, mu = 0.15, 0.01 / 0.3
    mpc = mp.get_context("spawn")
    q = mpc.Queue()
    procs = [mpc.Process(target=_dd_rank, args=(r, 2, port, L, kappa, mu, inner, nz, q)) for r in range(2)]
    for p_ in procs:
        p_.start()
    got = {}
    try:
        for _ in range(2):
            r, x, st = q.get(timeout=300)
            assert x is not None, st
            got[r] = (x, st)
    finally:
        for p_ in procs:
            p_.join(timeout=60)
            if p_.is_alive():
                p_.kill()
    slabs = dd.DomainGrid(L, nz, 2 // nz)
    U = inputs.random_gauge(L, "haar", seed=91)
    b = inputs.gaussian_spinor(L, 92)
    x = np.zeros_like(b)
    for r in range(2):
        x[slabs.block(r)] = got[r][0]
    assert got[0][1]["iters"] == got[1][1]["iters"] and got[0][1]["true_resid"] == got[1][1]["true_resid"]
    assert got[0][1]["converged"] == 1 and got[0][1]["true_resid"] <= 1e-10
    assert _oracle_resid(oracle, U, L, x, b, kappa, mu) <= 1e-10
