"""The caller-allocator hook of the C ABI (lqcd_set_allocator): with PyTorch's
caching allocator behind it, the library's workspace, gauge fields and their
derived copies come from torch's pool, are returned to it, and the results are
those of a context that allocates by itself."""
import pytest
import torch

from paper_1209_5942_gb300 import inputs, lqcd
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu


def _solve(ctx, L, U_d, b_d, kappa, mu):
    G = lqcd.lqcd_gauge_import(ctx, U_d, L)
    x = torch.zeros_like(b_d)
    prm = lqcd.cg_params(tol=1e-10, outer_prec=lqcd.LQCD_DF64, inner_prec=lqcd.LQCD_F32, sloppy_recon=12)
    st = lqcd.lqcd_cg_solve(ctx, G, lqcd.field(b_d, lqcd.LQCD_LAYOUT_LEXI), lqcd.field(x, lqcd.LQCD_LAYOUT_LEXI),
                            kappa, mu, prm)
    return G, x, st


def test_torch_caching_allocator_backs_the_library():
    from paper_1209_5942_gb300 import build
    build.build()
    L = (8, 8, 8, 8)
    V = inputs.volume(L)
    kappa, mu = 0.15, 0.01 / 0.3
    U_d = dev(inputs.random_gauge(L, "near", seed=1201, eps=0.4))
    b_d = dev(inputs.gaussian_spinor(L, 1202))
    ref_ctx = lqcd.Context(0)
    G0, x_ref, st_ref = _solve(ref_ctx, L, U_d, b_d, kappa, mu)
    G0.free()
    ref_ctx.close()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()

    ctx = lqcd.Context(0, torch_allocator=True)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() > base  # the workspace came from torch's pool
    G, x, st = _solve(ctx, L, U_d, b_d, kappa, mu)
    torch.cuda.synchronize()
    # master links (576 B per site) and the derived DF64 / F32 copies live in torch's pool
    assert torch.cuda.memory_allocated() >= base + 576 * V + V * 16 * 2  # + x itself
    assert st[0]["converged"] == 1 and st_ref[0]["converged"] == 1
    assert torch.equal(x, x_ref)  # same kernels, same bits
    del x
    G.free()
    ctx.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base  # everything went back


def test_allocator_pair_must_be_complete():
    ctx = lqcd.Context(0)
    ta = lqcd.TorchAllocator(0, torch.cuda.current_stream())
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.lqcd_set_allocator(ctx, ta.alloc_fn, None)
    assert e.value.status == lqcd.LQCD_ERR_INVALID
    lqcd.lqcd_set_allocator(ctx, None, None)  # back to the default
    ctx.close()


def test_context_pool_keeps_and_trims_memory():
    """The default allocator: the context's pool keeps freed memory mapped for
    the next import (its reserved bytes do not drop when a gauge field is
    freed), serves the re-import from it, and lqcd_trim_memory returns what
    no live allocation uses (a 16^4 field: 38 MB of links, more than one
    chunk of the pool beside the workspace)."""
    L = (16, 16, 16, 16)
    V = inputs.volume(L)
    U_d = dev(inputs.random_gauge(L, "near", seed=1203, eps=0.4))
    ctx = lqcd.Context(0)
    r0, u0 = lqcd.lqcd_memory_stats(ctx)
    assert u0 > 0 and r0 >= u0  # the workspace
    G = lqcd.lqcd_gauge_import(ctx, U_d, L)
    torch.cuda.synchronize()
    r1, u1 = lqcd.lqcd_memory_stats(ctx)
    assert u1 >= u0 + 576 * V and r1 >= u1  # FP64 master links
    G.free()
    torch.cuda.synchronize()
    r2, u2 = lqcd.lqcd_memory_stats(ctx)
    assert u2 == u0 and r2 == r1  # freed, still held
    G = lqcd.lqcd_gauge_import(ctx, U_d, L)
    torch.cuda.synchronize()
    assert lqcd.lqcd_memory_stats(ctx)[0] == r1  # served from the pool
    G.free()
    lqcd.lqcd_trim_memory(ctx)
    r3, u3 = lqcd.lqcd_memory_stats(ctx)
    assert u3 == u0 and r3 < r1
    ctx.close()
