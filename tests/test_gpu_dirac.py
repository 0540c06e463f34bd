"""GPU parity of the Dirac operator (Sec. 2.1, eq. D_tm) against the FP64 oracle.

Bar: FP64 (and float-float DF64) results within a max relative error of 1e-13
(max |y - y_ref| / max |y_ref| over all complex components); FP32 within 2e-6;
16-bit storage within a bound derived from its unit roundoff.  Sizes span
several thread blocks and ragged tails (Vh not a multiple of 128), asymmetric
extents, and the full 24^3 x 48 workload.
"""
import numpy as np
import pytest
import torch

from paper_1209_5942_gb300 import inputs, lqcd
from tests.gpu_util import (dev, eo_full_from_lexi, half_views, host, lexi_from_eo_full,
                            relerr)

pytestmark = pytest.mark.gpu

TOL = {lqcd.LQCD_F64: 1e-13, lqcd.LQCD_DF64: 1e-13, lqcd.LQCD_F32: 2e-6,
       lqcd.LQCD_BF16S: 2e-2, lqcd.LQCD_F16S: 3e-3}
SHAPES = [(4, 4, 4, 4), (2, 4, 6, 8), (6, 4, 2, 10), (8, 8, 8, 4)]


@pytest.fixture(scope="module")
def ctx():
    from paper_1209_5942_gb300 import build
    build.build()
    return lqcd.Context(0)


def _gauge(ctx, L, kind="haar", seed=1, recon=18, eps=0.3):
    U = inputs.random_gauge(L, kind, seed=seed, eps=eps)
    return U, lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=recon)


@pytest.mark.parametrize("L", SHAPES)
@pytest.mark.parametrize("prec", [lqcd.LQCD_F64, lqcd.LQCD_DF64, lqcd.LQCD_F32, lqcd.LQCD_BF16S,
                                  lqcd.LQCD_F16S])
def test_pack_roundtrip(ctx, oracle, L, prec):
    psi = inputs.gaussian_spinor(L, 5)
    _, _, f = eo_full_from_lexi(ctx, L, psi, prec)
    back = lexi_from_eo_full(ctx, L, f)
    bound = {lqcd.LQCD_F64: 0.0, lqcd.LQCD_DF64: 2 ** -46, lqcd.LQCD_F32: 2 ** -23,
             lqcd.LQCD_BF16S: 2 ** -8, lqcd.LQCD_F16S: 2 ** -11}[prec]
    assert relerr(back, psi) <= bound


@pytest.mark.parametrize("L", SHAPES)
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("recon", [18, 12])
def test_apply_M_full_lexi(ctx, oracle, L, dagger, recon):
    kappa, mu = 0.15, 0.01 / 0.3
    U, G = _gauge(ctx, L, recon=recon)
    psi = inputs.gaussian_spinor(L, 7)
    ref = oracle.apply_M(U, psi, L, kappa, mu, dagger=dagger)
    V = inputs.volume(L)
    out = torch.zeros((V, 4, 3), dtype=torch.complex128, device="cuda")
    fi = lqcd.field(dev(psi), lqcd.LQCD_LAYOUT_LEXI)
    fo = lqcd.field(out, lqcd.LQCD_LAYOUT_LEXI)
    fn = lqcd.lqcd_apply_Mdag if dagger else lqcd.lqcd_apply_M
    fn(ctx, G, fi, fo, kappa, mu, lqcd.LQCD_FULL)
    assert relerr(host(out), ref) <= 1e-13


@pytest.mark.parametrize("L", SHAPES)
@pytest.mark.parametrize("prec", [lqcd.LQCD_F64, lqcd.LQCD_DF64, lqcd.LQCD_F32])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_M_full_eo(ctx, oracle, L, prec, dagger):
    kappa, mu = 0.16, 0.005 / 0.32
    U, G = _gauge(ctx, L, kind="near", seed=3)
    psi = inputs.gaussian_spinor(L, 8)
    ref = oracle.apply_M(U, psi, L, kappa, mu, dagger=dagger)
    _, _, fi = eo_full_from_lexi(ctx, L, psi, prec)
    od, osc = lqcd.alloc_field(L, lqcd.LQCD_FULL, prec)
    fo = lqcd.field(od, lqcd.LQCD_LAYOUT_EO, prec, 1, osc)
    fn = lqcd.lqcd_apply_Mdag if dagger else lqcd.lqcd_apply_M
    fn(ctx, G, fi, fo, kappa, mu, lqcd.LQCD_FULL)
    assert relerr(lexi_from_eo_full(ctx, L, fo), ref) <= TOL[prec]


@pytest.mark.parametrize("L", SHAPES)
@pytest.mark.parametrize("prec", [lqcd.LQCD_F64, lqcd.LQCD_DF64, lqcd.LQCD_F32])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("recon", [18, 12])
def test_apply_Mhat_even(ctx, oracle, L, prec, dagger, recon):
    kappa, mu = 0.15, 0.01 / 0.3
    U, G = _gauge(ctx, L, recon=recon, seed=4)
    ev = ~oracle.parity_mask(L)
    psi = inputs.gaussian_spinor(L, 9) * ev[:, None, None]
    ref = oracle.apply_Mhat(U, psi, L, kappa, mu, dagger=dagger)
    di, si, _ = eo_full_from_lexi(ctx, L, psi, prec)
    fie, _ = half_views(L, di, si, prec)
    od, osc = lqcd.alloc_field(L, lqcd.LQCD_FULL, prec)
    foe, _ = half_views(L, od, osc, prec)
    fn = lqcd.lqcd_apply_Mdag if dagger else lqcd.lqcd_apply_M
    fn(ctx, G, fie, foe, kappa, mu, lqcd.LQCD_EVEN)
    got = lexi_from_eo_full(ctx, L, lqcd.field(od, lqcd.LQCD_LAYOUT_EO, prec, 1, osc))
    assert relerr(got, ref) <= TOL[prec]


@pytest.mark.parametrize("L", SHAPES)
@pytest.mark.parametrize("prec", [lqcd.LQCD_F64, lqcd.LQCD_DF64, lqcd.LQCD_F32, lqcd.LQCD_BF16S,
                                  lqcd.LQCD_F16S])
@pytest.mark.parametrize("out_parity", [lqcd.LQCD_EVEN, lqcd.LQCD_ODD])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("recon", [12, 18])
def test_dslash_half_hop(ctx, oracle, L, prec, out_parity, dagger, recon):
    if recon == 18 and prec in (lqcd.LQCD_BF16S, lqcd.LQCD_F16S):
        pytest.skip("16-bit links are stored in REC12 form only")
    U, G = _gauge(ctx, L, seed=6, recon=recon)
    odd = oracle.parity_mask(L)
    src_mask = odd if out_parity == lqcd.LQCD_EVEN else ~odd
    psi = inputs.gaussian_spinor(L, 10) * src_mask[:, None, None]
    ref = oracle.hop(U, psi, L, dagger=dagger) * (~src_mask)[:, None, None]
    di, si, _ = eo_full_from_lexi(ctx, L, psi, prec)
    fie, fio = half_views(L, di, si, prec)
    od, osc = lqcd.alloc_field(L, lqcd.LQCD_FULL, prec)
    foe, foo = half_views(L, od, osc, prec)
    if out_parity == lqcd.LQCD_EVEN:
        lqcd.lqcd_dslash(ctx, G, fio, foe, out_parity, dagger)
    else:
        lqcd.lqcd_dslash(ctx, G, fie, foo, out_parity, dagger)
    got = lexi_from_eo_full(ctx, L, lqcd.field(od, lqcd.LQCD_LAYOUT_EO, prec, 1, osc))
    assert relerr(got, ref) <= TOL[prec]


def test_multi_rhs_dslash_matches_single(ctx, oracle):
    """The multi-RHS launch (link loaded once per site for all RHS) gives the
    single-RHS result bit for bit in every precision."""
    L = (4, 4, 6, 8)
    U, G12 = _gauge(ctx, L, seed=12, recon=12)
    G18 = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=18)
    nrhs = 12
    for prec, G in ((lqcd.LQCD_F64, G12), (lqcd.LQCD_F32, G12), (lqcd.LQCD_BF16S, G12),
                    (lqcd.LQCD_DF64, G18), (lqcd.LQCD_DF64, G12)):
        psis = inputs.gaussian_spinor(L, 13, nrhs=nrhs)
        n_half, sb_half = lqcd.field_bytes(L, lqcd.LQCD_EVEN, prec, 1)
        din = torch.zeros(nrhs * n_half // 8, dtype=torch.float64, device="cuda")
        sin = torch.zeros(max(nrhs * sb_half // 4, 1), dtype=torch.float32, device="cuda")
        dout = torch.zeros_like(din)
        sout = torch.zeros_like(sin)
        # fill each rhs's odd half from a packed full field
        singles = []
        for r in range(nrhs):
            d, s, _ = eo_full_from_lexi(ctx, L, psis[r], prec)
            _, fo = half_views(L, d, s, prec)
            din.view(torch.uint8)[r * n_half:(r + 1) * n_half].copy_(
                d.view(torch.uint8)[n_half:2 * n_half])
            if sb_half:
                sin.view(torch.uint8)[r * sb_half:(r + 1) * sb_half].copy_(
                    s.view(torch.uint8)[sb_half:2 * sb_half])
            od, osc = lqcd.alloc_field(L, lqcd.LQCD_FULL, prec)
            foe, _ = half_views(L, od, osc, prec)
            lqcd.lqcd_dslash(ctx, G, fo, foe, lqcd.LQCD_EVEN, 0)
            singles.append((od.view(torch.uint8)[:n_half].clone(),
                            osc.view(torch.uint8)[:sb_half].clone() if sb_half else None))
        sc = sin if sb_half else None
        fi = lqcd.field(din, lqcd.LQCD_LAYOUT_EO, prec, nrhs, sc)
        fo = lqcd.field(dout, lqcd.LQCD_LAYOUT_EO, prec, nrhs, sout if sb_half else None)
        lqcd.lqcd_dslash(ctx, G, fi, fo, lqcd.LQCD_EVEN, 0)
        torch.cuda.synchronize()
        for r in range(nrhs):
            assert torch.equal(dout.view(torch.uint8)[r * n_half:(r + 1) * n_half], singles[r][0])
            if sb_half:
                assert torch.equal(sout.view(torch.uint8)[r * sb_half:(r + 1) * sb_half],
                                   singles[r][1])


@pytest.mark.parametrize("L", [(4, 4, 6, 8), (16, 8, 8, 4)])
@pytest.mark.parametrize("nrhs", [1, 5, 12])
def test_every_launch_shape_gives_the_same_bits(ctx, nrhs, L):
    """Every candidate the autotuner can pick (block shape, grid size, load
    order, RHS per thread) writes the same bits: the multi-RHS hop of each
    candidate equals the default launch in every precision, including ragged
    RHS groups (5 = 2 + 2 + 1, 4 + 1), on a small lattice and on one whose
    half volume (2048) fills whole blocks of every shape."""
    U, G12 = _gauge(ctx, L, seed=21, recon=12)
    G18 = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=18)
    for prec, G in ((lqcd.LQCD_F64, G18), (lqcd.LQCD_DF64, G18), (lqcd.LQCD_DF64, G12),
                    (lqcd.LQCD_F32, G12), (lqcd.LQCD_F32, G18), (lqcd.LQCD_BF16S, G12),
                    (lqcd.LQCD_F16S, G12)):
        psis = inputs.gaussian_spinor(L, 22, nrhs=nrhs)
        n_half, sb_half = lqcd.field_bytes(L, lqcd.LQCD_EVEN, prec, 1)
        din = torch.zeros(nrhs * n_half // 8, dtype=torch.float64, device="cuda")
        sin = torch.zeros(max(nrhs * sb_half // 4, 1), dtype=torch.float32, device="cuda")
        for r in range(nrhs):
            d, s, _ = eo_full_from_lexi(ctx, L, psis[r], prec)
            din.view(torch.uint8)[r * n_half:(r + 1) * n_half].copy_(d.view(torch.uint8)[n_half:2 * n_half])
            if sb_half:
                sin.view(torch.uint8)[r * sb_half:(r + 1) * sb_half].copy_(
                    s.view(torch.uint8)[sb_half:2 * sb_half])
        fi = lqcd.field(din, lqcd.LQCD_LAYOUT_EO, prec, nrhs, sin if sb_half else None)

        def run(choice):
            dout = torch.full_like(din, float("nan"))
            sout = torch.full_like(sin, float("nan"))
            fo = lqcd.field(dout, lqcd.LQCD_LAYOUT_EO, prec, nrhs, sout if sb_half else None)
            lqcd.lqcd_set_launch_choice(ctx, choice)
            try:
                lqcd.lqcd_dslash(ctx, G, fi, fo, lqcd.LQCD_EVEN, 1)
            finally:
                lqcd.lqcd_set_launch_choice(ctx, -1)
            torch.cuda.synchronize()
            return dout.view(torch.uint8).clone(), (sout.view(torch.uint8).clone() if sb_half else None)

        ref = run(-1)
        for choice in range(64):
            got = run(choice)
            assert torch.equal(got[0], ref[0]), (prec, choice)
            if sb_half:
                assert torch.equal(got[1], ref[1]), (prec, choice)


@pytest.mark.parametrize("L,choices", [((4, 4, 6, 8), (-1, 0, 7, 19, 33)),
                                       ((16, 8, 8, 4), (-1, 0, 7, 19, 33, 39))])
def test_cg_iterates_do_not_depend_on_launch_shape(ctx, L, choices):
    """A mixed-precision multi-RHS solve (reducing hops, per-warp partials)
    returns the same bits and iteration counts whatever launch the tuner
    picks."""
    U, G = _gauge(ctx, L, seed=23, recon=12)
    nrhs = 3
    b = dev(inputs.gaussian_spinor(L, 24, nrhs=nrhs))
    prm = lqcd.cg_params(tol=1e-10, outer_prec=lqcd.LQCD_DF64, inner_prec=lqcd.LQCD_F32,
                         sloppy_recon=12)
    outs = []
    for choice in choices:
        x = torch.zeros_like(b)
        lqcd.lqcd_set_launch_choice(ctx, choice)
        try:
            st = lqcd.lqcd_cg_solve(ctx, G, lqcd.field(b, lqcd.LQCD_LAYOUT_LEXI, nrhs=nrhs),
                                    lqcd.field(x, lqcd.LQCD_LAYOUT_LEXI, nrhs=nrhs), 0.15, 0.01 / 0.3, prm)
        finally:
            lqcd.lqcd_set_launch_choice(ctx, -1)
        torch.cuda.synchronize()
        outs.append((x.clone(), [s["iters"] for s in st]))
    for x, its in outs[1:]:
        assert its == outs[0][1]
        assert torch.equal(x, outs[0][0])


@pytest.mark.parametrize("nrhs", [1, 3])
def test_df64_pair_kernels_on_a_ragged_lattice(ctx, oracle, nrhs):
    """The float-float 18-real-link hop in scalar and in packed FP32x2
    arithmetic, the packed one also with shared-memory staging (every block
    shape and grid of the three) on a lattice whose half
    volume (144) ends in a partial block and a partial 32-site reduction
    group: the reducing hops of a DF64 CG give the same bits and iteration
    counts for every choice, and the solution meets the oracle's."""
    L = (6, 4, 2, 6)
    kappa, mu = 0.15, 0.01 / 0.3
    U = inputs.random_gauge(L, "near", seed=25, eps=0.4)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=18)
    bh = inputs.gaussian_spinor(L, 26, nrhs=nrhs)
    b = dev(bh)
    prm = lqcd.cg_params(tol=1e-10, outer_prec=lqcd.LQCD_DF64, inner_prec=lqcd.LQCD_DF64)
    outs = []
    for choice in [-1] + list(range(18)):
        x = torch.zeros_like(b)
        lqcd.lqcd_set_launch_choice(ctx, choice)
        try:
            st = lqcd.lqcd_cg_solve(ctx, G, lqcd.field(b, lqcd.LQCD_LAYOUT_LEXI, nrhs=nrhs),
                                    lqcd.field(x, lqcd.LQCD_LAYOUT_LEXI, nrhs=nrhs), kappa, mu, prm)
        finally:
            lqcd.lqcd_set_launch_choice(ctx, -1)
        torch.cuda.synchronize()
        outs.append((x.clone(), [s["iters"] for s in st]))
    for x, its in outs[1:]:
        assert its == outs[0][1]
        assert torch.equal(x, outs[0][0])
    x = host(outs[0][0])
    for r in range(nrhs):
        res = bh[r] - oracle.apply_M(U, x[r], L, kappa, mu)
        assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(bh[r])


@pytest.mark.parametrize("inner", [lqcd.LQCD_BF16S, lqcd.LQCD_F16S])
def test_16bit_kernels_on_a_ragged_lattice(ctx, oracle, inner):
    """The 16-bit hop in every launch form the tuner can pick (one site per
    thread in both load orders, two sites per thread in packed FP32x2 with
    direct loads or with cp.async-staged operands) inside a mixed DF64/16-bit
    CG on a lattice whose half volume (144) ends in a partial block of every
    form: every choice gives the same bits and iteration counts, and the
    solution meets the oracle's residual."""
    L = (6, 4, 2, 6)
    kappa, mu = 0.15, 0.01 / 0.3
    U = inputs.random_gauge(L, "near", seed=27, eps=0.4)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=12)
    bh = inputs.gaussian_spinor(L, 28, nrhs=1)
    b = dev(bh)
    prm = lqcd.cg_params(tol=1e-10, outer_prec=lqcd.LQCD_DF64, inner_prec=inner, sloppy_recon=12)
    outs = []
    for choice in [-1] + list(range(24)):
        x = torch.zeros_like(b)
        lqcd.lqcd_set_launch_choice(ctx, choice)
        try:
            st = lqcd.lqcd_cg_solve(ctx, G, lqcd.field(b, lqcd.LQCD_LAYOUT_LEXI, nrhs=1),
                                    lqcd.field(x, lqcd.LQCD_LAYOUT_LEXI, nrhs=1), kappa, mu, prm)
        finally:
            lqcd.lqcd_set_launch_choice(ctx, -1)
        torch.cuda.synchronize()
        outs.append((x.clone(), [s["iters"] for s in st]))
    for x, its in outs[1:]:
        assert its == outs[0][1]
        assert torch.equal(x, outs[0][0])
    x = host(outs[0][0])
    res = bh[0] - oracle.apply_M(U, x[0], L, kappa, mu)
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(bh[0])


def test_full_size_24x48_apply_M(ctx, oracle):
    """The 24^3 x 48 workload: M and Mhat on every site against the oracle."""
    L = (24, 24, 24, 48)
    kappa, mu = 0.16, 0.005 / 0.32
    U, G = _gauge(ctx, L, kind="near", seed=2, eps=0.3)
    psi = inputs.gaussian_spinor(L, 21)
    ref = oracle.apply_M(U, psi, L, kappa, mu)
    # DF64 with 18-real links: the tuned launch, then the scalar, packed and
    # packed + shared-memory-staged pair kernels (128-thread blocks, full grid)
    for prec, choice in ((lqcd.LQCD_F64, -1), (lqcd.LQCD_DF64, -1), (lqcd.LQCD_DF64, 1),
                         (lqcd.LQCD_DF64, 3), (lqcd.LQCD_DF64, 5)):
        _, _, fi = eo_full_from_lexi(ctx, L, psi, prec)
        od, osc = lqcd.alloc_field(L, lqcd.LQCD_FULL, prec)
        fo = lqcd.field(od, lqcd.LQCD_LAYOUT_EO, prec, 1, osc)
        lqcd.lqcd_set_launch_choice(ctx, choice)
        try:
            lqcd.lqcd_apply_M(ctx, G, fi, fo, kappa, mu, lqcd.LQCD_FULL)
        finally:
            lqcd.lqcd_set_launch_choice(ctx, -1)
        assert relerr(lexi_from_eo_full(ctx, L, fo), ref) <= 1e-13, (prec, choice)


def test_invalid_arguments_rejected(ctx):
    L = (4, 4, 4, 4)
    U, G = _gauge(ctx, L)
    d, s = lqcd.alloc_field(L, lqcd.LQCD_EVEN, lqcd.LQCD_F64)
    f = lqcd.field(d, lqcd.LQCD_LAYOUT_EO)
    with pytest.raises(lqcd.LqcdError) as e:  # aliasing
        lqcd.lqcd_dslash(ctx, G, f, f, lqcd.LQCD_EVEN, 0)
    assert e.value.status == lqcd.LQCD_ERR_INVALID
    bad = lqcd.field(d, lqcd.LQCD_LAYOUT_EO)
    bad.ptr = d.data_ptr() + 8  # misaligned
    d2, _ = lqcd.alloc_field(L, lqcd.LQCD_EVEN, lqcd.LQCD_F64)
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.lqcd_dslash(ctx, G, bad, lqcd.field(d2), lqcd.LQCD_EVEN, 0)
    assert e.value.status == lqcd.LQCD_ERR_INVALID
    # non-SU(3) links with REC12
    Ub = inputs.random_gauge(L, "haar", seed=3) * 1.01
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.lqcd_gauge_import(ctx, dev(Ub), L, recon=12)
    assert e.value.status == lqcd.LQCD_ERR_INVALID
    # odd extent
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge((4, 4, 4, 4), "cold")), (3, 4, 4, 4))
    assert e.value.status == lqcd.LQCD_ERR_INVALID
