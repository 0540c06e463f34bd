"""The entry points of the C ABI that the operator, solver and HMC tests do not
reach directly: the momentum step, precision conversion of EO fields, the
context's stream, the autotuner's cache file and the peak microbenchmark.
Each is checked through the ABI against a plain computation of what its
declaration in include/lqcd.h states."""
import json
import os

import numpy as np
import pytest
import torch

from paper_1209_5942_gb300 import inputs, lqcd
from tests.gpu_util import dev, eo_full_from_lexi, half_views, host, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1209_5942_gb300 import build
    build.build()
    return lqcd.Context(0)


def test_momenta_update_is_p_minus_eps_f(ctx):
    """P <- P - eps dSdw on every component of [4][V][8]."""
    L = (4, 4, 2, 6)
    V = inputs.volume(L)
    rng = np.random.default_rng(7)
    P0 = rng.standard_normal((4, V, 8))
    F = rng.standard_normal((4, V, 8))
    P = torch.from_numpy(P0.copy()).cuda()
    lqcd.lqcd_momenta_update(ctx, L, P, torch.from_numpy(F).cuda(), 0.0625)
    torch.cuda.synchronize()
    # eps = 2^-4 makes eps F exact, so the fused and the two-step forms agree
    assert np.array_equal(host(P), P0 - 0.0625 * F)


@pytest.mark.parametrize("prec", [lqcd.LQCD_DF64, lqcd.LQCD_F32, lqcd.LQCD_BF16S, lqcd.LQCD_F16S])
def test_spinor_convert_round_trip(ctx, prec):
    """F64 -> prec -> F64 on a full EO field and on one half: float-float keeps
    the value to its 48 bits, F32 rounds each real to nearest, the 16-bit
    formats keep each site within its storage precision times the site scale
    (the largest |real| of the site); the other half of a half-field
    conversion is not touched."""
    L = (4, 4, 4, 6)
    psi = inputs.gaussian_spinor(L, 11)
    d64, _, f64 = eo_full_from_lexi(ctx, L, psi)
    dlo, slo = lqcd.alloc_field(L, lqcd.LQCD_FULL, prec)
    flo = lqcd.field(dlo, lqcd.LQCD_LAYOUT_EO, prec, 1, slo)
    lqcd.lqcd_spinor_convert(ctx, L, lqcd.LQCD_FULL, f64, flo)
    dback, _ = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64)
    fback = lqcd.field(dback, lqcd.LQCD_LAYOUT_EO)
    lqcd.lqcd_spinor_convert(ctx, L, lqcd.LQCD_FULL, flo, fback)
    torch.cuda.synchronize()
    a, b = host(d64).view(np.float64), host(dback).view(np.float64)
    if prec == lqcd.LQCD_DF64:
        assert np.max(np.abs(a - b) / np.maximum(np.abs(a), 1e-300)) < 2.0 ** -47
    elif prec == lqcd.LQCD_F32:
        assert np.array_equal(b, a.astype(np.float32).astype(np.float64))
    else:
        unit = 2.0 ** -8 if prec == lqcd.LQCD_BF16S else 2.0 ** -11
        assert relerr(b, a) < 2 * unit
    # a half field: only that parity is written
    dh, sh = lqcd.alloc_field(L, lqcd.LQCD_FULL, prec)
    fe64, fo64 = half_views(L, d64, None, lqcd.LQCD_F64)
    fe, fo = half_views(L, dh, sh, prec)
    lqcd.lqcd_spinor_convert(ctx, L, lqcd.LQCD_ODD, fo64, fo)
    torch.cuda.synchronize()
    n_half, sb_half = lqcd.field_bytes(L, lqcd.LQCD_EVEN, prec, 1)
    raw = dh.view(torch.uint8)
    assert int(raw[:n_half].count_nonzero()) == 0
    assert int(raw[n_half:2 * n_half].count_nonzero()) > 0


def test_set_stream_runs_the_library_on_that_stream(ctx):
    """After lqcd_set_stream the context's work is ordered on the given stream:
    M applied there, with the default stream idle, equals M on the default
    stream."""
    L = (4, 4, 4, 4)
    U = inputs.random_gauge(L, "haar", seed=13)
    c2 = lqcd.Context(0)
    G = lqcd.lqcd_gauge_import(c2, dev(U), L)
    psi = dev(inputs.gaussian_spinor(L, 14))
    ref = torch.zeros_like(psi)
    lqcd.lqcd_apply_M(c2, G, lqcd.field(psi, lqcd.LQCD_LAYOUT_LEXI), lqcd.field(ref, lqcd.LQCD_LAYOUT_LEXI),
                      0.15, 0.1)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    c2.set_stream(s)
    out = torch.zeros_like(psi)
    with torch.cuda.stream(s):
        lqcd.lqcd_apply_M(c2, G, lqcd.field(psi, lqcd.LQCD_LAYOUT_LEXI), lqcd.field(out, lqcd.LQCD_LAYOUT_LEXI),
                          0.15, 0.1)
    s.synchronize()
    assert torch.equal(out, ref)
    G.free()
    c2.close()


def test_autotune_cache_file_round_trip(ctx, tmp_path):
    """The tuner writes its choices to the cache file; a new context that loads
    the file reuses them (no new keys) and gets the same bits."""
    path = str(tmp_path / "tune.json")
    L = (8, 4, 4, 8)
    U = inputs.random_gauge(L, "haar", seed=15)
    psi = inputs.gaussian_spinor(L, 16)
    outs = []
    for _ in range(2):
        c = lqcd.Context(0)
        lqcd.lqcd_set_autotune(c, True, path)
        G = lqcd.lqcd_gauge_import(c, dev(U), L)
        d, sc, _ = eo_full_from_lexi(c, L, psi)
        fe, fo = half_views(L, d, sc, lqcd.LQCD_F64)
        od, osc = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64)
        oe, _ = half_views(L, od, osc, lqcd.LQCD_F64)
        lqcd.lqcd_dslash(c, G, fo, oe, lqcd.LQCD_EVEN, 0)
        torch.cuda.synchronize()
        outs.append(od.clone())
        G.free()
        c.close()
        keys = json.load(open(path))
        if len(outs) == 1:
            first = dict(keys)
    assert os.path.exists(path) and any(k.split("|")[1].startswith("hop") for k in first)
    assert keys == first
    assert torch.equal(outs[0], outs[1])


def test_measure_peaks_plausible(ctx):
    """The FP64 and packed-FP32 FMA microbenchmarks return rates of the order of
    the GPU's nominal ones (GB300: about 1.25 and 80 TFLOP/s)."""
    fp64, fp32 = lqcd.lqcd_measure_peaks(ctx)
    assert 0.3 < fp64 < 5.0, fp64
    assert 10.0 < fp32 < 400.0, fp32
    assert fp32 > 10 * fp64
