"""Domain decomposition of the half hop along t (the paper's Sec. 6 outlook),
on one GPU: the lattice is split into nt domains held as separate library
fields on their local geometry, each half hop packs the spin-projected faces,
moves them between the domains (the device copies of LocalExchange stand in
for NCCL; the kernels do not wait on one another) and runs the domain hops.
The assembled result is compared with the FP64 oracle's hop on the whole
lattice, for both parities, H and H^+, 18 and 12 real links, periodic and
antiperiodic time, and with the library's own single-domain hop."""
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


def _domain_hop(ctx, U, psi, L, nt, prec, recon, parity, dagger, antiper):
    """Assembled lexicographic result of the domain-decomposed half hop."""
    slabs = dd.TimeSlabs(L, nt, antiper)
    Ll = slabs.local_L
    p = 0 if parity == lqcd.LQCD_EVEN else 1
    gauges, ins, outs, keep = [], [], [], []
    for d in range(nt):
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
    for d in range(nt):
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
