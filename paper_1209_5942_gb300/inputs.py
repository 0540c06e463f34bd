"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle calls.

This module holds no arithmetic of the method (no Dirac operator, no action,
no solver): it only draws random fields with numpy's PCG64 generator, in the
lexicographic layouts of the C ABI:

* gauge field  complex128 ``[V, 4, 3, 3]``, site ``i = x + Lx*(y + Ly*(z + Lz*t))``,
  direction ``mu = 0..3 = x, y, z, t``
* spinor field complex128 ``[V, 4, 3]`` (spin, colour)

Workload recipes (the paper's lattices are synthetic too):

* Haar-random SU(3) links: QR decomposition of a complex Gaussian matrix, phases
  of R's diagonal moved into Q, then the determinant's phase divided out.
* near-identity links ``exp(i eps H)`` with ``H = sum_a h_a lambda_a / 2``,
  ``h_a ~ N(0, 1)``, built through the eigen-decomposition of ``H``.
* Gaussian spinors with density ``exp(-|z|^2)`` per complex component.
* unit point sources ``delta_{x,0} delta_{spin,alpha} delta_{colour,c}``.
"""
from __future__ import annotations

import numpy as np


def volume(L) -> int:
    return int(np.prod(L))


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _project_det_one(Q: np.ndarray) -> np.ndarray:
    det = np.linalg.det(Q)
    ph = det / np.abs(det)
    return Q * (ph ** (-1.0 / 3.0))[..., None, None]


def haar_su3(n: int, seed: int) -> np.ndarray:
    """n Haar-distributed SU(3) matrices, shape (n, 3, 3)."""
    g = rng(seed)
    Z = (g.standard_normal((n, 3, 3)) + 1j * g.standard_normal((n, 3, 3))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    Q = Q * (d / np.abs(d))[..., None, :]
    return _project_det_one(Q)


def _gellmann() -> np.ndarray:
    lam = np.zeros((8, 3, 3), np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def near_identity_su3(n: int, eps: float, seed: int, chunk: int = 1 << 20) -> np.ndarray:
    """n matrices exp(i eps H), H = sum_a h_a lambda_a/2, h_a ~ N(0,1)."""
    g = rng(seed)
    T = _gellmann() / 2.0
    out = np.empty((n, 3, 3), np.complex128)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        h = g.standard_normal((m, 8))
        H = np.einsum("na,aij->nij", h, T)
        w, Vec = np.linalg.eigh(H)
        E = np.exp(1j * eps * w)
        M = np.einsum("nij,nj,nkj->nik", Vec, E, Vec.conj())
        out[s:s + m] = _project_det_one(M)
    return out


def random_gauge(L, kind: str = "haar", seed: int = 1, eps: float = 0.3) -> np.ndarray:
    """Gauge field [V, 4, 3, 3]: kind = 'haar', 'near' (exp(i eps H)) or 'cold'."""
    V = volume(L)
    if kind == "cold":
        U = np.zeros((V, 4, 3, 3), np.complex128)
        U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
        return U
    if kind == "haar":
        return haar_su3(4 * V, seed).reshape(V, 4, 3, 3)
    if kind == "near":
        return near_identity_su3(4 * V, eps, seed).reshape(V, 4, 3, 3)
    raise ValueError(kind)


def gaussian_spinor(L, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Spinor [V, 4, 3] (or [nrhs, V, 4, 3]) with re, im ~ N(0, 1/2)."""
    V = volume(L)
    g = rng(seed)
    shape = (V, 4, 3) if nrhs is None else (nrhs, V, 4, 3)
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)) * np.sqrt(0.5)


def point_sources(L, site: int = 0) -> np.ndarray:
    """The 12 unit point sources at one site, shape [12, V, 4, 3]."""
    V = volume(L)
    b = np.zeros((12, V, 4, 3), np.complex128)
    for k in range(12):
        b[k, site, k // 3, k % 3] = 1.0
    return b


def gaussian_algebra(L, seed: int) -> np.ndarray:
    """Real algebra field [4, V, 8] with N(0, 1) entries (e.g. momenta)."""
    return rng(seed).standard_normal((4, volume(L), 8))


def site_coords(L) -> np.ndarray:
    """(V, 4) integer coordinates (x, y, z, t) of the lexicographic sites."""
    V = volume(L)
    i = np.arange(V)
    x = i % L[0]
    y = (i // L[0]) % L[1]
    z = (i // (L[0] * L[1])) % L[2]
    t = i // (L[0] * L[1] * L[2])
    return np.stack([x, y, z, t], axis=1)
