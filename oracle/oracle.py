"""Python access to the FP64 CPU oracle (``lqcd_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline
leg of ``bench.py`` import this module; the product package never does.

The C file is compiled with gcc (``-O2 -fopenmp -ffp-contract=off``) into
``oracle/_build/liboracle.so`` on first use or by :func:`build`.  All fields
are numpy ``complex128`` arrays in the lexicographic layouts described in the
C file:

* gauge  ``U[t, z, y, x, mu, a, b]`` (shape ``(V, 4, 3, 3)`` flattened by site)
* spinor ``psi[site, spin, colour]`` (shape ``(V, 4, 3)``)
* algebra fields ``P[mu, site, 8]`` (float64)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lqcd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle shared library; returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


def _declare(L):
    L.or_gamma.argtypes = [ctypes.c_int, _dp]
    L.or_generator.argtypes = [ctypes.c_int, _dp]
    L.or_parity.argtypes = [ctypes.c_long, _ip]
    L.or_parity.restype = ctypes.c_int
    L.or_hop.argtypes = [_dp, _dp, _dp, _ip, ctypes.c_int, ctypes.c_int]
    L.or_apply_M.argtypes = [_dp, _dp, _dp, _ip, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                             ctypes.c_int]
    L.or_apply_Mhat.argtypes = L.or_apply_M.argtypes
    L.or_eo_prepare.argtypes = [_dp, _dp, _dp, _ip, ctypes.c_int, ctypes.c_double,
                                ctypes.c_double]
    L.or_eo_reconstruct.argtypes = L.or_eo_prepare.argtypes
    L.or_cg.argtypes = [_dp, _dp, _dp, _ip, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                        ctypes.c_double, ctypes.c_int, ctypes.c_int, _dp]
    L.or_cg.restype = ctypes.c_int
    L.or_cg_fixed_iters.argtypes = [_dp, _dp, _dp, _ip, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int]
    L.or_cg_fixed_iters.restype = ctypes.c_double
    L.or_plaquette.argtypes = [_dp, _ip]
    L.or_plaquette.restype = ctypes.c_double
    L.or_gauge_action.argtypes = [_dp, _ip, ctypes.c_double]
    L.or_gauge_action.restype = ctypes.c_double
    L.or_staple.argtypes = [_dp, _ip, ctypes.c_long, ctypes.c_int, _dp]
    L.or_gauge_dSdw.argtypes = [_dp, _ip, ctypes.c_double, _dp]
    L.or_fermion_dSdw.argtypes = [_dp, _dp, _ip, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_int, _dp]
    L.or_fermion_dSdw_lr.argtypes = [_dp, _dp, _dp, _ip, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, _dp]
    L.or_pseudofermion_action.argtypes = [_dp, _dp, _dp, _ip, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_int]
    L.or_pseudofermion_action.restype = ctypes.c_double
    L.or_rec12_third_row.argtypes = [_dp, _dp]
    L.or_reunitarize.argtypes = [_dp, ctypes.c_long]
    L.or_expi.argtypes = [_dp, ctypes.c_double, _dp]
    L.or_update_links.argtypes = [_dp, _dp, _ip, ctypes.c_double]
    u32p = ctypes.POINTER(ctypes.c_uint32)
    L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.or_philox_uniform2.argtypes = [ctypes.c_uint32] * 4 + [ctypes.c_uint64, _dp]
    L.or_momenta.argtypes = [_dp, _ip, ctypes.c_uint64, ctypes.c_uint32]
    L.or_gaussian_spinor.argtypes = [_dp, _ip, ctypes.c_uint64, ctypes.c_uint32]
    L.or_su2_y0_samples.argtypes = [ctypes.c_double, ctypes.c_uint64, ctypes.c_int, _dp]
    L.or_heatbath_sweep.argtypes = [_dp, _ip, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32]
    L.or_heatbath_sweep.restype = ctypes.c_int
    L.or_overrelax_link.argtypes = [_dp, _dp, ctypes.c_int]
    L.or_overrelax_link.restype = ctypes.c_int
    L.or_overrelax_sweep.argtypes = [_dp, _ip]
    L.or_overrelax_sweep.restype = ctypes.c_int
    L.or_hmc_md.argtypes = [_dp, _dp, _dp, _ip, ctypes.c_double, ctypes.c_double,
                            ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                            ctypes.c_double, ctypes.c_int, _dp]
    L.or_hmc_md.restype = ctypes.c_double
    L.or_rectangle_sum.argtypes = [_dp, _ip]
    L.or_rectangle_sum.restype = ctypes.c_double
    L.or_gauge_action_sym.argtypes = [_dp, _ip, ctypes.c_double, ctypes.c_double]
    L.or_gauge_action_sym.restype = ctypes.c_double
    L.or_gauge_dSdw_sym.argtypes = [_dp, _ip, ctypes.c_double, ctypes.c_double, _dp]
    L.or_hmc_md_2mn.argtypes = [_dp, _dp, _dp, _ip, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp]
    L.or_hmc_md_2mn.restype = ctypes.c_double


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(_dp)


def _dims(L):
    arr = (ctypes.c_int * 4)(*[int(v) for v in L])
    return arr


def volume(L) -> int:
    return int(np.prod(L))


def _cplx(a, shape):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    assert a.size == int(np.prod(shape)), (a.shape, shape)
    return a


# ----------------------------------------------------------------------------
# Wrappers (each cites the section of the paper the C routine follows)
# ----------------------------------------------------------------------------

def gamma(mu: int) -> np.ndarray:
    """gamma_mu (mu=0..3) or gamma_5 (mu=4), chiral basis (Sec. 2.1)."""
    out = np.zeros((4, 4), np.complex128)
    lib().or_gamma(mu, _p(out))
    return out


def generator(a: int) -> np.ndarray:
    """T^a = lambda^a / 2 (a = 0..7)."""
    out = np.zeros((3, 3), np.complex128)
    lib().or_generator(a, _p(out))
    return out


def parity(i: int, L) -> int:
    return lib().or_parity(i, _dims(L))


def parity_mask(L) -> np.ndarray:
    """Boolean array over lexicographic sites: True on odd sites."""
    x = np.arange(L[0])
    y = np.arange(L[1])
    z = np.arange(L[2])
    t = np.arange(L[3])
    tt, zz, yy, xx = np.meshgrid(t, z, y, x, indexing="ij")
    return ((xx + yy + zz + tt) % 2 == 1).reshape(-1)


def hop(U, psi, L, antiperiodic_t=True, dagger=False):
    """Hopping term H (or H^+) of Sec. 2.1, eq. D_tm."""
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    psi = _cplx(psi, (V, 4, 3))
    out = np.empty((V, 4, 3), np.complex128)
    lib().or_hop(_p(U), _p(psi), _p(out), _dims(L), int(antiperiodic_t), int(dagger))
    return out


def apply_M(U, psi, L, kappa, mu, dagger=False, antiperiodic_t=True):
    """M = (1 + 2 i kappa mu g5) - kappa H (or M^+), Sec. 2.1 eq. D_tm."""
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    psi = _cplx(psi, (V, 4, 3))
    out = np.empty((V, 4, 3), np.complex128)
    lib().or_apply_M(_p(U), _p(psi), _p(out), _dims(L), int(antiperiodic_t), kappa, mu,
                     int(dagger))
    return out


def apply_Mhat(U, psi, L, kappa, mu, dagger=False, antiperiodic_t=True):
    """Even-site Schur complement A_e - kappa^2 H_eo A_o^-1 H_oe (or adjoint)."""
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    psi = _cplx(psi, (V, 4, 3))
    out = np.empty((V, 4, 3), np.complex128)
    lib().or_apply_Mhat(_p(U), _p(psi), _p(out), _dims(L), int(antiperiodic_t), kappa, mu,
                        int(dagger))
    return out


def eo_prepare(U, b, L, kappa, mu, antiperiodic_t=True):
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    b = _cplx(b, (V, 4, 3))
    out = np.empty((V, 4, 3), np.complex128)
    lib().or_eo_prepare(_p(U), _p(b), _p(out), _dims(L), int(antiperiodic_t), kappa, mu)
    return out


def eo_reconstruct(U, b, x_even, L, kappa, mu, antiperiodic_t=True):
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    b = _cplx(b, (V, 4, 3))
    x = np.array(_cplx(x_even, (V, 4, 3)), copy=True)
    lib().or_eo_reconstruct(_p(U), _p(b), _p(x), _dims(L), int(antiperiodic_t), kappa, mu)
    return x


def cg(U, b, L, kappa, mu, tol=1e-12, max_iter=100000, eo=False, antiperiodic_t=True):
    """Plain CG on the normal equations (Sec. 2.1, eq. solvereq).

    Returns (x, iterations, residual); iterations = -1 if not converged."""
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    b = _cplx(b, (V, 4, 3))
    x = np.zeros((V, 4, 3), np.complex128)
    res = ctypes.c_double(0)
    it = lib().or_cg(_p(U), _p(b), _p(x), _dims(L), int(antiperiodic_t), kappa, mu, tol,
                     max_iter, int(eo), ctypes.byref(res))
    return x, it, res.value


def cg_fixed_iters(U, bhat, L, kappa, mu, iters, antiperiodic_t=True):
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    bhat = _cplx(bhat, (V, 4, 3))
    x = np.zeros((V, 4, 3), np.complex128)
    r = lib().or_cg_fixed_iters(_p(U), _p(bhat), _p(x), _dims(L), int(antiperiodic_t), kappa, mu,
                                int(iters))
    return x, r


def solve(U, b, L, kappa, mu, tol=1e-12, max_iter=100000, antiperiodic_t=True):
    """Solution of M x = b by plain unpreconditioned CG on M^+ M."""
    x, it, res = cg(U, b, L, kappa, mu, tol, max_iter, eo=False, antiperiodic_t=antiperiodic_t)
    if it < 0:
        raise RuntimeError(f"oracle CG did not converge (residual {res})")
    return x


def plaquette(U, L) -> float:
    """(1/(6V)) sum (1/3) Re Tr U_munu (Sec. 2.1)."""
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    return lib().or_plaquette(_p(U), _dims(L))


def gauge_action(U, L, beta) -> float:
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    return lib().or_gauge_action(_p(U), _dims(L), beta)


def staple(U, L, i, mu) -> np.ndarray:
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    out = np.zeros((3, 3), np.complex128)
    lib().or_staple(_p(U), _dims(L), int(i), int(mu), _p(out))
    return out


def gauge_dSdw(U, L, beta) -> np.ndarray:
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    out = np.zeros((4, V, 8), np.float64)
    lib().or_gauge_dSdw(_p(U), _dims(L), beta, _p(out))
    return out


def fermion_dSdw(U, X, L, kappa, mu, eo=True, antiperiodic_t=True) -> np.ndarray:
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    X = _cplx(X, (V, 4, 3))
    out = np.zeros((4, V, 8), np.float64)
    lib().or_fermion_dSdw(_p(U), _p(X), _dims(L), int(antiperiodic_t), kappa, mu, int(eo),
                          _p(out))
    return out


def fermion_dSdw_lr(U, Y, X, L, kappa, mu, eo=True, antiperiodic_t=True) -> np.ndarray:
    """-2 Re[Y^+ dMhat(mu) X] / domega for given Y, X (Y = Mhat X: fermion_dSdw)."""
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    X = _cplx(X, (V, 4, 3))
    Y = _cplx(Y, (V, 4, 3))
    out = np.zeros((4, V, 8), np.float64)
    lib().or_fermion_dSdw_lr(_p(U), _p(Y), _p(X), _dims(L), int(antiperiodic_t), kappa, mu, int(eo),
                             _p(out))
    return out


def pseudofermion_action(U, phi, L, kappa, mu, eo=True, tol=1e-13, max_iter=100000,
                         antiperiodic_t=True):
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    phi = _cplx(phi, (V, 4, 3))
    X = np.zeros((V, 4, 3), np.complex128)
    s = lib().or_pseudofermion_action(_p(U), _p(phi), _p(X), _dims(L), int(antiperiodic_t),
                                      kappa, mu, int(eo), tol, max_iter)
    return s, X


def rec12_third_row(link) -> np.ndarray:
    link = np.ascontiguousarray(link, np.complex128).reshape(3, 3)
    out = np.zeros(3, np.complex128)
    lib().or_rec12_third_row(_p(link), _p(out))
    return out


def reunitarize(U) -> np.ndarray:
    U = np.array(U, dtype=np.complex128, copy=True, order="C")
    lib().or_reunitarize(_p(U), U.size // 9)
    return U


def expi(p8, eps) -> np.ndarray:
    p8 = np.ascontiguousarray(p8, np.float64)
    out = np.zeros((3, 3), np.complex128)
    lib().or_expi(_p(p8), eps, _p(out))
    return out


def update_links(U, P, L, eps) -> np.ndarray:
    V = volume(L)
    U = np.array(_cplx(U, (V, 4, 3, 3)), copy=True)
    P = np.ascontiguousarray(P, np.float64)
    lib().or_update_links(_p(U), _p(P), _dims(L), eps)
    return U


def philox4x32_10(ctr, key) -> np.ndarray:
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def philox_uniform2(c0, c1, c2, c3, seed):
    out = np.zeros(2, np.float64)
    lib().or_philox_uniform2(c0, c1, c2, c3, seed, _p(out))
    return out


def momenta(L, seed, traj) -> np.ndarray:
    V = volume(L)
    out = np.zeros((4, V, 8), np.float64)
    lib().or_momenta(_p(out), _dims(L), seed, traj)
    return out


def gaussian_spinor(L, seed, traj) -> np.ndarray:
    V = volume(L)
    out = np.zeros((V, 4, 3), np.complex128)
    lib().or_gaussian_spinor(_p(out), _dims(L), seed, traj)
    return out


def su2_y0_samples(b, seed, n) -> np.ndarray:
    """Samples of y0 ~ sqrt(1 - y0^2) exp(b y0) from the heatbath's SU(2) sampler."""
    out = np.zeros(n, np.float64)
    lib().or_su2_y0_samples(b, seed, n, _p(out))
    return out


def heatbath_sweep(U, L, beta, seed, sweep):
    """One Cabibbo-Marinari/Kennedy-Pendleton sweep (Sec. 2.2). Returns (U, failures)."""
    V = volume(L)
    U = np.array(_cplx(U, (V, 4, 3, 3)), copy=True)
    f = lib().or_heatbath_sweep(_p(U), _dims(L), beta, seed, sweep)
    return U, f


def overrelax_link(link, staple_sum, gmask=7):
    """Overrelaxation of one link (Sec. 2.2): the SU(2) subgroups in gmask
    (bits 0, 1, 2 = (0,1), (1,2), (0,2)) reflected, v = (w_hat^+)^2.
    Returns (link', skipped subgroups)."""
    u = np.array(_cplx(link, (3, 3)), copy=True)
    A = _cplx(staple_sum, (3, 3))
    n = lib().or_overrelax_link(_p(u), _p(A), int(gmask))
    return u, n


def overrelax_sweep(U, L):
    """One overrelaxation sweep in the heatbath's checkerboard order (Sec. 2.2).
    Returns (U, skipped subgroups)."""
    V = volume(L)
    U = np.array(_cplx(U, (V, 4, 3, 3)), copy=True)
    n = lib().or_overrelax_sweep(_p(U), _dims(L))
    return U, n


def hmc_md(U, P, phi, L, beta, kappa, mu, nf=1, nsteps=10, tau=1.0, tol=1e-12,
           max_iter=100000):
    """Leapfrog molecular dynamics (Sec. 2.2). Returns (U', P', dH, (H0, H1, Spf0))."""
    V = volume(L)
    U = np.array(_cplx(U, (V, 4, 3, 3)), copy=True)
    P = np.array(P, dtype=np.float64, copy=True, order="C")
    phi = _cplx(phi if phi is not None else np.zeros((V, 4, 3)), (V, 4, 3))
    h = np.zeros(3, np.float64)
    dH = lib().or_hmc_md(_p(U), _p(P), _p(phi), _dims(L), beta, kappa, mu, int(nf), int(nsteps),
                         tau, tol, int(max_iter), _p(h))
    return U, P, dH, tuple(h)


# -- tree-level Symanzik gauge action and the 2MN integrator (Sec. 2.1 eq.
# "S_tlsym", Sec. 2.2) -------------------------------------------------------

TLSYM_C1 = -1.0 / 12.0  # tree-level value (the printed +1/12 is read as -1/12)
OMELYAN_LAMBDA = 0.1931833275037836  # 2MN parameter (Omelyan, Mryglod, Folk 2003)


def rectangle_sum(U, L) -> float:
    """sum_{x, mu != nu} (3 - Re Tr R_munu(x)) over the 2x1 loops."""
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    return lib().or_rectangle_sum(_p(U), _dims(L))


def gauge_action_sym(U, L, beta, c1=TLSYM_C1) -> float:
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    return lib().or_gauge_action_sym(_p(U), _dims(L), beta, c1)


def gauge_dSdw_sym(U, L, beta, c1=TLSYM_C1) -> np.ndarray:
    V = volume(L)
    U = _cplx(U, (V, 4, 3, 3))
    out = np.zeros((4, V, 8), np.float64)
    lib().or_gauge_dSdw_sym(_p(U), _dims(L), beta, c1, _p(out))
    return out


def hmc_md_2mn(U, P, phi, L, beta, kappa, mu, c1=TLSYM_C1, nf=1, nsteps_f=10, nsteps_g=10,
               lam=OMELYAN_LAMBDA, tau=1.0, tol=1e-12, max_iter=100000):
    """Nested 2MN molecular dynamics.  Returns (U', P', dH, (H0, H1, Spf0))."""
    V = volume(L)
    U = np.array(_cplx(U, (V, 4, 3, 3)), copy=True)
    P = np.array(P, dtype=np.float64, copy=True, order="C")
    phi = _cplx(phi if phi is not None else np.zeros((V, 4, 3)), (V, 4, 3))
    h = np.zeros(3, np.float64)
    dH = lib().or_hmc_md_2mn(_p(U), _p(P), _p(phi), _dims(L), beta, c1, kappa, mu, int(nf),
                             int(nsteps_f), int(nsteps_g), lam, tau, tol, int(max_iter), _p(h))
    return U, P, dH, tuple(h)


# -- mass preconditioning (Hasenbusch) with a heavier twisted mass (Sec. 2.2:
# det D = det A det(D / A) with a second, heavier fermion matrix) -------------

def hasenbusch_action(U, phi2, L, kappa, mu, mu2, tol=1e-13):
    """S2 = phi2^+ W (Mhat^+ Mhat)^-1 W^+ phi2 with W = Mhat(mu2): the ratio
    det(Mhat^+ Mhat) / det(W^+ W).  Returns (S2, X), X = (Mhat^+ Mhat)^-1 W^+ phi2."""
    psi = apply_Mhat(U, phi2, L, kappa, mu2, dagger=True)
    return pseudofermion_action(U, psi, L, kappa, mu, eo=True, tol=tol)


def hasenbusch_dSdw(U, phi2, X, L, kappa, mu, mu2):
    """dS2/domega = -2 Re[Y^+ dMhat(mu) X] + 2 Re[phi2^+ dW X], Y = Mhat(mu) X."""
    return fermion_dSdw(U, X, L, kappa, mu, eo=True) + fermion_dSdw_lr(U, -np.asarray(phi2), X, L, kappa, mu2,
                                                                       eo=True)


def hasenbusch_source(U, eta, L, kappa, mu, mu2, tol=1e-13):
    """phi2 = W^-+ Mhat^+ eta (even sites), so that S2 = eta^+ eta:
    W^-+ = W (W^+ W)^-1."""
    rhs = apply_Mhat(U, eta, L, kappa, mu, dagger=True)
    _, Z = pseudofermion_action(U, rhs, L, kappa, mu2, eo=True, tol=tol)
    return apply_Mhat(U, Z, L, kappa, mu2, dagger=False)


def hmc_md_2mn_hasenbusch(U, P, eta1, eta2, L, beta, kappa, mu, mu2, c1=TLSYM_C1, nsteps=2,
                          nsteps_mid=2, nsteps_g=2, lam=OMELYAN_LAMBDA, tau=1.0, tol=1e-13, phis=None):
    """Molecular dynamics of mass-preconditioned HMC (Sec. 2.2: det D =
    det A det(D / A) with a heavier second fermion matrix A, and 2MN on
    multiple time scales), written from the pinned oracle routines above.

    Pseudofermions (reading G24): W = Mhat(mu2), phi1 = W^+ eta1 with
    S1 = phi1^+ (W^+ W)^-1 phi1, and phi2 = W^-+ Mhat^+ eta2 with the ratio
    S2 = phi2^+ W (Mhat^+ Mhat)^-1 W^+ phi2.  Three nested 2MN scales: the
    ratio force outside (nsteps steps over tau), the W force in the middle
    (nsteps_mid steps over each outer position update), the gauge force
    inside (nsteps_g steps over each middle position update), whose position
    update is U <- exp(i h P) U.  One 2MN step of size e for force F and
    position update Q:  P -= lam e F; Q(e/2); P -= (1 - 2 lam) e F; Q(e/2);
    P -= lam e F.  Every force is evaluated where the scheme needs it.
    phis = (phi1, phi2) replaces the sources drawn from (eta1, eta2) (for the
    reverse trajectory of a reversibility check).
    Returns (U', P', dH, (H0, H1), (phi1, phi2))."""
    V = volume(L)
    U = np.array(_cplx(U, (V, 4, 3, 3)), copy=True)
    P = np.array(P, dtype=np.float64, copy=True, order="C")
    if phis is None:
        phi1 = apply_Mhat(U, eta1, L, kappa, mu2, dagger=True)
        phi2 = hasenbusch_source(U, eta2, L, kappa, mu, mu2, tol=tol)
    else:
        phi1, phi2 = phis

    def hamiltonian(U, P):
        S1, _ = pseudofermion_action(U, phi1, L, kappa, mu2, eo=True, tol=tol)
        S2, _ = hasenbusch_action(U, phi2, L, kappa, mu, mu2, tol=tol)
        return 0.5 * float(np.sum(P * P)) + gauge_action_sym(U, L, beta, c1) + S1 + S2

    def force(level, U):
        if level == 0:
            _, X2 = hasenbusch_action(U, phi2, L, kappa, mu, mu2, tol=tol)
            return hasenbusch_dSdw(U, phi2, X2, L, kappa, mu, mu2)
        if level == 1:
            _, X1 = pseudofermion_action(U, phi1, L, kappa, mu2, eo=True, tol=tol)
            return fermion_dSdw(U, X1, L, kappa, mu2, eo=True)
        return gauge_dSdw_sym(U, L, beta, c1)

    steps = (nsteps, nsteps_mid, nsteps_g)

    def position(level, U, h):
        return integrate(level + 1, U, h) if level < 2 else update_links(U, P, L, h)

    def integrate(level, U, h):
        e = h / steps[level]
        for _ in range(steps[level]):
            P[...] -= lam * e * force(level, U)
            U = position(level, U, 0.5 * e)
            P[...] -= (1.0 - 2.0 * lam) * e * force(level, U)
            U = position(level, U, 0.5 * e)
            P[...] -= lam * e * force(level, U)
        return U

    H0 = hamiltonian(U, P)
    U = integrate(0, U, tau)
    H1 = hamiltonian(U, P)
    return U, P, H1 - H0, (H0, H1), (phi1, phi2)
