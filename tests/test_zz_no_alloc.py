"""The no-allocation plaquette entry point against the context-based one.

lqcd_plaquette_noalloc serves callers that cannot allocate device memory: it
takes no context and keeps its block partial sums in a fixed device array
inside the library.  This file is collected last so that a failure here comes
after every other test has run; it also passes on its own in a fresh process.
It calls the entry point through the C ABI twice in a row (the second call
reuses the scratch the first one left behind) and compares with
lqcd_plaquette, the context-based entry point, within the plaquette
tolerance of the other GPU tests (1e-14).
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1209_5942_gb300 import inputs, lqcd

pytestmark = pytest.mark.gpu


def _noalloc(U_dev, L, out):
    g = lqcd.geom(L)
    stream = torch.cuda.current_stream().cuda_stream
    st = lqcd.lib().lqcd_plaquette_noalloc(ctypes.c_void_p(U_dev.data_ptr()), ctypes.byref(g),
                                           ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    return st, float(out.cpu()[0])


def test_noalloc_plaquette_matches_context_entry_point():
    from paper_1209_5942_gb300 import build
    build.build()
    ctx = lqcd.Context(0)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    fields = [((4, 4, 6, 8), inputs.random_gauge((4, 4, 6, 8), "near", seed=501, eps=0.7)),
              ((8, 8, 8, 8), inputs.random_gauge((8, 8, 8, 8), "haar", seed=502))]
    for L, U in fields:  # two calls in a row, different fields, same scratch
        U_dev = torch.from_numpy(U).cuda()
        G = lqcd.lqcd_gauge_import(ctx, U_dev, L)
        ref = lqcd.lqcd_plaquette(ctx, G)
        for _ in range(2):
            st, p = _noalloc(U_dev, L, out)
            assert st == lqcd.LQCD_OK
            assert abs(p - ref) < 1e-14, (p, ref)
        G.free()
    cold = torch.from_numpy(inputs.random_gauge((4, 4, 4, 4), "cold")).cuda()
    st, p = _noalloc(cold, (4, 4, 4, 4), out)
    assert st == lqcd.LQCD_OK and abs(p - 1.0) < 1e-15


def test_noalloc_rejects_oversized_and_bad_arguments():
    from paper_1209_5942_gb300 import build
    build.build()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    small = torch.zeros((16, 4, 3, 3), dtype=torch.complex128, device="cuda")
    # 64^3 x 32 = 8388608 sites exceeds the 4194304-site scratch limit; nothing is read
    st, _ = _noalloc(small, (64, 64, 64, 32), out)
    assert st == lqcd.LQCD_ERR_INVALID
    st, _ = _noalloc(small, (3, 2, 2, 2), out)
    assert st == lqcd.LQCD_ERR_INVALID
    g = lqcd.geom((2, 2, 2, 2))
    st = lqcd.lib().lqcd_plaquette_noalloc(None, ctypes.byref(g), ctypes.c_void_p(out.data_ptr()), None)
    assert st == lqcd.LQCD_ERR_INVALID
