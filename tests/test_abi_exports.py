"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/lqcd.h declares; the binding's ctypes signatures cover
them.  No compute call is made here."""
import ctypes
import os

from paper_1209_5942_gb300 import build, lqcd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = lqcd.declared_symbols()
    assert len(declared) >= 29, declared
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    bound = {name for name, _, _ in lqcd.SIGNATURES}
    assert set(declared) <= bound, sorted(set(declared) - bound)


def test_abi_version_and_host_side_calls():
    build.build()
    lib = lqcd.lib()
    assert lib.lqcd_abi_version() == 2
    # pure host-side helpers work without a GPU
    n, sb = lqcd.field_bytes((4, 4, 4, 8), lqcd.LQCD_FULL, lqcd.LQCD_F64)
    assert n == 4 * 4 * 4 * 8 * 192 and sb == 0
    n, sb = lqcd.field_bytes((4, 4, 4, 8), lqcd.LQCD_EVEN, lqcd.LQCD_BF16S, 3)
    assert n == 3 * 256 * 48 and sb == 3 * 256 * 4
    assert lqcd.field_bytes((3, 4, 4, 8), lqcd.LQCD_FULL, lqcd.LQCD_F64)[0] == 0
    # invalid handles are rejected before anything touches a device
    assert lib.lqcd_destroy(None) == lqcd.LQCD_ERR_INVALID
    assert lib.lqcd_last_error(None) == b"context is NULL"
    g = lqcd.geom((2, 2, 2, 2))
    assert lib.lqcd_plaquette_noalloc(None, ctypes.byref(g), None, None) == lqcd.LQCD_ERR_INVALID


def test_header_declares_the_paper_calls():
    names = set(lqcd.declared_symbols())
    for required in ("lqcd_apply_M", "lqcd_apply_Mdag", "lqcd_cg_solve", "lqcd_fermion_force",
                     "lqcd_heatbath_sweep", "lqcd_cg_solve_batch", "lqcd_plaquette"):
        assert required in names
