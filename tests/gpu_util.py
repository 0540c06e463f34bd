"""Helpers for the GPU parity tests (marshalling between numpy/oracle layouts
and the library's device fields).  No arithmetic of the method lives here."""
import numpy as np
import torch

from paper_1209_5942_gb300 import lqcd


def relerr(got, ref) -> float:
    """max_i |got_i - ref_i| / max_i |ref_i| over all complex components."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(got - ref)) / (den if den > 0 else 1.0))


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy()


def eo_full_from_lexi(ctx, L, psi_lexi, prec=lqcd.LQCD_F64, nrhs=1):
    """Pack lexicographic complex128 spinor(s) into a new EO full field."""
    data, scale = lqcd.alloc_field(L, lqcd.LQCD_FULL, prec, nrhs)
    f = lqcd.field(data, lqcd.LQCD_LAYOUT_EO, prec, nrhs, scale)
    src = dev(psi_lexi.astype(np.complex128))
    lqcd.lqcd_spinor_pack(ctx, L, src, f)
    torch.cuda.synchronize()
    return data, scale, f


def lexi_from_eo_full(ctx, L, f, nrhs=1):
    V = int(np.prod(L))
    out = torch.zeros((nrhs, V, 4, 3), dtype=torch.complex128, device="cuda")
    lqcd.lqcd_spinor_unpack(ctx, L, f, out)
    return host(out)[0] if nrhs == 1 else host(out)


def half_views(L, data, scale, prec, nrhs=1):
    """(even, odd) lqcd_field views into an EO full buffer (nrhs == 1 only)."""
    assert nrhs == 1
    n_half, sb_half = lqcd.field_bytes(L, lqcd.LQCD_EVEN, prec, 1)
    base = data.data_ptr()
    fe = lqcd.field(data, lqcd.LQCD_LAYOUT_EO, prec, 1, scale)
    fo = lqcd.field(data, lqcd.LQCD_LAYOUT_EO, prec, 1, scale)
    fo._keep = fe._keep
    fo.ptr = base + n_half
    if scale is not None:
        fo.scale = scale.data_ptr() + sb_half
    return fe, fo
