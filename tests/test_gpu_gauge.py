"""GPU parity of the gauge-side kernels and the HMC pieces (Sec. 2.1 action,
Sec. 2.2 forces, heatbath, HMC) against the FP64 oracle.

The GPU and the oracle draw the same Philox4x32-10 streams, so momenta,
Gaussian spinors, heatbath sweeps and whole trajectories are compared value
by value; where a floating-point comparison decides an integer (a heatbath
rejection), both sides decide in FP64 and the rare flips caused by libm
rounding differences are counted and bounded.
"""
import numpy as np
import pytest
import scipy.linalg
import torch

from paper_1209_5942_gb300 import inputs, lqcd
from tests.gpu_util import dev, eo_full_from_lexi, half_views, host, lexi_from_eo_full, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1209_5942_gb300 import build
    build.build()
    return lqcd.Context(0)


def _export(ctx, G, L):
    V = inputs.volume(L)
    out = torch.zeros((V, 4, 3, 3), dtype=torch.complex128, device="cuda")
    lqcd.lqcd_gauge_export(ctx, G, out)
    return host(out)


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (2, 4, 6, 8), (6, 4, 2, 10)])
def test_gauge_roundtrip_and_plaquette(ctx, oracle, L):
    U = inputs.random_gauge(L, "near", seed=31, eps=0.6)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    assert np.array_equal(_export(ctx, G, L), U)
    assert abs(lqcd.lqcd_plaquette(ctx, G) - oracle.plaquette(U, L)) < 1e-14
    Gc = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "cold")), L)
    assert lqcd.lqcd_plaquette(ctx, Gc) == 1.0


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (2, 4, 6, 8)])
def test_gauge_force(ctx, oracle, L):
    beta = 5.6
    U = inputs.random_gauge(L, "near", seed=32, eps=0.5)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    F = torch.zeros((4, inputs.volume(L), 8), dtype=torch.float64, device="cuda")
    S = lqcd.lqcd_gauge_force(ctx, G, beta, F)
    ref = oracle.gauge_dSdw(U, L, beta)
    assert relerr(host(F), ref) < 1e-13
    assert abs(S - oracle.gauge_action(U, L, beta)) < 1e-10 * abs(S)


def test_momenta_and_eta_match_oracle_streams(ctx, oracle):
    L = (4, 4, 4, 8)
    V = inputs.volume(L)
    P = torch.zeros((4, V, 8), dtype=torch.float64, device="cuda")
    lqcd.lqcd_momenta_gaussian(ctx, L, P, 99, 7)
    assert relerr(host(P), oracle.momenta(L, 99, 7)) < 1e-13
    K = lqcd.lqcd_momenta_kinetic(ctx, L, P)
    assert abs(K - 0.5 * np.sum(oracle.momenta(L, 99, 7) ** 2)) < 1e-10 * K
    d, s = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F64)
    f = lqcd.field(d, lqcd.LQCD_LAYOUT_EO)
    lqcd.lqcd_spinor_gaussian(ctx, L, f, lqcd.LQCD_EVEN, 99, 7)
    eta = lexi_from_eo_full(ctx, L, f)
    ref = oracle.gaussian_spinor(L, 99, 7) * (~oracle.parity_mask(L))[:, None, None]
    assert relerr(eta, ref) < 1e-13


def test_gauge_update_matches_library_expm(ctx, oracle):
    L = (4, 4, 2, 4)
    V = inputs.volume(L)
    U = inputs.random_gauge(L, "haar", seed=33)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    P = inputs.gaussian_algebra(L, 34) * 3.0
    eps = 0.07
    lqcd.lqcd_gauge_update(ctx, G, dev(P), eps)
    got = _export(ctx, G, L)
    ref = oracle.update_links(U, P, L, eps)
    assert relerr(got, ref) < 1e-13
    T = np.stack([oracle.generator(a) for a in range(8)])
    H = np.einsum("a,aij->ij", P[2, 5], T)
    assert np.max(np.abs(got[5, 2] - scipy.linalg.expm(1j * eps * H) @ U[5, 2])) < 1e-13


@pytest.mark.parametrize("eps,scale", [(0.07, 3.0), (0.004, 1.0), (2.0, 1.0)])
def test_gauge_update_df64_matches_oracle(ctx, oracle, eps, scale):
    """U <- exp(i eps P) U in float-float against the oracle's FP64 update and
    scipy's expm, for a molecular-dynamics step size, a tiny one, and a large
    one that takes the scaling-and-squaring path; the result stays in SU(3)."""
    L = (4, 4, 2, 4)
    U = inputs.random_gauge(L, "haar", seed=33)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    P = inputs.gaussian_algebra(L, 34) * scale
    lqcd.lqcd_gauge_update_prec(ctx, G, dev(P), eps, lqcd.LQCD_DF64)
    got = _export(ctx, G, L)
    ref = oracle.update_links(U, P, L, eps)
    assert relerr(got, ref) < 1e-13
    T = np.stack([oracle.generator(a) for a in range(8)])
    H = np.einsum("a,aij->ij", P[1, 7], T)
    assert np.max(np.abs(got[7, 1] - scipy.linalg.expm(1j * eps * H) @ U[7, 1])) < 1e-13
    eye = np.eye(3)
    assert np.max(np.abs(got @ np.conj(np.transpose(got, (0, 1, 3, 2))) - eye)) < 1e-13
    assert np.max(np.abs(np.linalg.det(got) - 1)) < 1e-13
    with pytest.raises(lqcd.LqcdError):
        lqcd.lqcd_gauge_update_prec(ctx, G, dev(P), eps, lqcd.LQCD_F32)
    # the float-float copy the update writes next to the FP64 field is current:
    # a float-float hop on it equals the FP64 hop on the updated links
    lqcd.lqcd_gauge_update_prec(ctx, G, dev(P), eps, lqcd.LQCD_DF64)
    psi = inputs.gaussian_spinor(L, 35)
    outs = {}
    for prec in (lqcd.LQCD_F64, lqcd.LQCD_DF64):
        data, scale, _ = eo_full_from_lexi(ctx, L, psi, prec)
        fe, fo = half_views(L, data, scale, prec)
        od, osc = lqcd.alloc_field(L, lqcd.LQCD_FULL, prec)
        oe, oo = half_views(L, od, osc, prec)
        lqcd.lqcd_dslash(ctx, G, fo, oe, lqcd.LQCD_EVEN, 0)
        outs[prec] = lexi_from_eo_full(ctx, L, lqcd.field(od, lqcd.LQCD_LAYOUT_EO, prec, 1, osc))
    assert relerr(outs[lqcd.LQCD_DF64], outs[lqcd.LQCD_F64]) < 1e-13


@pytest.mark.parametrize("recon", [18, 12])
def test_heatbath_sweep_matches_oracle(ctx, oracle, recon):
    """Three FP64 sweeps link by link; with recon = 12 the sweep runs on the
    12-real FP64 copy, the third row rebuilt on every load (Sec. 4.1)."""
    L = (4, 4, 4, 4)
    U = inputs.random_gauge(L, "haar", seed=35)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=recon)
    Uo = U.copy()
    for sweep in range(3):
        lqcd.lqcd_heatbath_sweep(ctx, G, 5.7, 4242, sweep)
        Uo, fails = oracle.heatbath_sweep(Uo, L, 5.7, 4242, sweep)
        assert fails == 0
    got = _export(ctx, G, L)
    diff = np.abs(got - Uo).max(axis=(2, 3))
    flips = int(np.sum(diff > 1e-9))
    # links agree to rounding, except where libm rounding flipped a rejection
    assert flips <= max(2, diff.size // 500), flips
    assert np.median(diff) < 1e-13
    eye = np.eye(3)
    assert np.max(np.abs(got @ np.conj(np.transpose(got, (0, 1, 3, 2))) - eye)) < 1e-12


@pytest.mark.parametrize("recon", [18, 12])
def test_heatbath_df64_staples_match_oracle(ctx, oracle, recon):
    """The FP64-class sweep with its staples in float-float (prec = LQCD_DF64:
    twelve 3x3 products per link on the FP32 pipe, the SU(2) samplers and the
    update in IEEE FP64): three sweeps link by link against the oracle, as the
    FP64 sweep; the staples round at 2^-46 relative instead of 2^-53, so a
    rejection decision flips only where a uniform falls that close to its
    threshold."""
    L = (4, 4, 4, 4)
    U = inputs.random_gauge(L, "haar", seed=35)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=recon)
    Uo = U.copy()
    for sweep in range(3):
        lqcd.lqcd_heatbath_sweep(ctx, G, 5.7, 4242, sweep, prec=lqcd.LQCD_DF64)
        Uo, fails = oracle.heatbath_sweep(Uo, L, 5.7, 4242, sweep)
        assert fails == 0
    got = _export(ctx, G, L)
    diff = np.abs(got - Uo).max(axis=(2, 3))
    flips = int(np.sum(diff > 1e-9))
    assert flips <= max(2, diff.size // 500), flips
    assert np.median(diff) < 1e-12
    eye = np.eye(3)
    assert np.max(np.abs(got @ np.conj(np.transpose(got, (0, 1, 3, 2))) - eye)) < 1e-12


def test_heatbath_df64_equilibrium_plaquette(ctx):
    """The float-float-staple sweep and the FP64 sweep reach the same
    plaquette at beta = 5.7 (40 measured sweeps after 30)."""
    L = (8, 8, 8, 8)
    means = {}
    for prec in (lqcd.LQCD_F64, lqcd.LQCD_DF64):
        G = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "cold")), L)
        vals = []
        for s in range(70):
            lqcd.lqcd_heatbath_sweep(ctx, G, 5.7, 97, s, n_or=1, prec=prec)
            if s >= 30:
                vals.append(lqcd.lqcd_plaquette(ctx, G))
        means[prec] = np.mean(vals)
        G.free()
    assert abs(means[lqcd.LQCD_DF64] - means[lqcd.LQCD_F64]) < 4e-3, means


def test_heatbath_strong_coupling_gpu(ctx):
    """<P> = beta/18 + beta^2/216 at beta = 0.3 (SU(3) strong coupling)."""
    L = (8, 8, 8, 8)
    beta = 0.3
    G = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "cold")), L)
    vals = []
    for s in range(80):
        lqcd.lqcd_heatbath_sweep(ctx, G, beta, 77, s)
        if s >= 10:
            vals.append(lqcd.lqcd_plaquette(ctx, G))
    vals = np.array(vals)
    expect = beta / 18 + beta ** 2 / 216
    err = vals.std() / np.sqrt(len(vals))
    assert abs(vals.mean() - expect) < 4 * err + 2e-4


def test_overrelaxation_preserves_action(ctx):
    L = (4, 4, 4, 4)
    G = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "near", seed=36, eps=0.8)), L)
    F = torch.zeros((4, inputs.volume(L), 8), dtype=torch.float64, device="cuda")
    lqcd.lqcd_heatbath_sweep(ctx, G, 5.7, 1, 0)
    p0 = lqcd.lqcd_plaquette(ctx, G)
    # one heatbath sweep followed by overrelaxation: compare against heatbath alone
    G2 = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "cold")), L)
    lqcd.lqcd_gauge_copy(ctx, G, G2)
    lqcd.lqcd_heatbath_sweep(ctx, G, 5.7, 1, 1, n_or=0)
    lqcd.lqcd_heatbath_sweep(ctx, G2, 5.7, 1, 1, n_or=2)
    # overrelaxation is microcanonical: same action as the heatbath-only field ...
    S1 = lqcd.lqcd_gauge_force(ctx, G, 5.7, F)
    S2 = lqcd.lqcd_gauge_force(ctx, G2, 5.7, F)
    assert abs(S2 - S1) < 1e-8 * abs(S1)
    assert p0 > 0.3
    # ... but not the identity: the links moved by O(1)
    assert np.abs(_export(ctx, G, L) - _export(ctx, G2, L)).max() > 0.3


@pytest.mark.parametrize("prec,recon,tol", [(lqcd.LQCD_F64, 18, 1e-12), (lqcd.LQCD_F64, 12, 1e-12),
                                            (lqcd.LQCD_DF64, 18, 1e-11), (lqcd.LQCD_DF64, 12, 1e-11),
                                            (lqcd.LQCD_F32, 18, 5e-5), (lqcd.LQCD_F32, 12, 5e-5)])
def test_overrelax_sweep_matches_oracle(ctx, oracle, prec, recon, tol):
    """One overrelaxation sweep (Sec. 2.2) from a rough field made by the
    oracle's heatbath, link by link against the oracle's sweep.  FP64: 1e-12.
    FP64 with float-float staples: the staple rounds at 2^-46 instead of
    2^-53 relative (2^7 larger), and the reflection divides the subgroup block
    by its norm: 1e-11.
    FP32: staples, reflection and update in binary32 (unit roundoff 2^-24
    ~ 6e-8; a staple entry sums 6 triple products, ~20 roundings, and three
    subgroups compound), written back and reunitarised in FP64: 5e-5 ~ 800 u."""
    L = (4, 4, 4, 4)
    U = inputs.random_gauge(L, "haar", seed=38)
    for s in range(3):
        U, _ = oracle.heatbath_sweep(U, L, 5.7, 21, s)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=recon)
    lqcd.lqcd_overrelax_sweep(ctx, G, 1, prec)
    got = _export(ctx, G, L)
    ref, skipped = oracle.overrelax_sweep(U, L)
    assert skipped == 0
    err = np.abs(got - ref).max()
    assert err < tol, err
    assert np.abs(ref - U).max() > 0.3  # the sweep is not close to the identity
    # two passes against two oracle sweeps
    lqcd.lqcd_overrelax_sweep(ctx, G, 1, prec)
    ref2, _ = oracle.overrelax_sweep(ref, L)
    assert np.abs(_export(ctx, G, L) - ref2).max() < 2 * tol


def test_overrelax_rejects_bad_arguments(ctx):
    L = (4, 4, 4, 4)
    G = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "cold")), L)
    for n_or, prec in [(0, lqcd.LQCD_F64), (65, lqcd.LQCD_F64), (1, lqcd.LQCD_BF16S)]:
        with pytest.raises(lqcd.LqcdError):
            lqcd.lqcd_overrelax_sweep(ctx, G, n_or, prec)


def _even_half_field(ctx, L, psi_even):
    d, s, _ = eo_full_from_lexi(ctx, L, psi_even)
    fe, _ = half_views(L, d, s, lqcd.LQCD_F64)
    return d, fe


@pytest.mark.parametrize("outer,inner,recon", [(lqcd.LQCD_F64, lqcd.LQCD_F64, 18),
                                               (lqcd.LQCD_DF64, lqcd.LQCD_F32, 18),
                                               (lqcd.LQCD_F64, lqcd.LQCD_F64, 12)])
def test_fermion_force_vs_oracle(ctx, oracle, outer, inner, recon):
    """The adjoint force kernel against the oracle's, with 18-real links and
    with REC12 links (third row rebuilt inside the force kernel)."""
    L = (4, 4, 2, 4)
    V = inputs.volume(L)
    kappa, mu = 0.14, 0.1
    U = inputs.random_gauge(L, "near", seed=37, eps=0.4)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=recon)
    ev = ~oracle.parity_mask(L)
    phi = inputs.gaussian_spinor(L, 38) * ev[:, None, None]
    keep, fphi = _even_half_field(ctx, L, phi)
    F = torch.zeros((4, V, 8), dtype=torch.float64, device="cuda")
    prm = lqcd.cg_params(tol=1e-13, outer_prec=outer, inner_prec=inner, max_iter=50000)
    S, st = lqcd.lqcd_fermion_force(ctx, G, fphi, F, kappa, mu, prm)
    Sref, X = oracle.pseudofermion_action(U, phi, L, kappa, mu, eo=True, tol=1e-14)
    ref = oracle.fermion_dSdw(U, X, L, kappa, mu, eo=True)
    assert abs(S - Sref) < 1e-10 * abs(Sref)
    assert relerr(host(F), ref) < 1e-9


@pytest.mark.parametrize("recon", [18, 12])
def test_fermion_force_at_equal_X(ctx, oracle, recon):
    """The force kernel alone at the oracle's X = (Mhat^+ Mhat)^-1 phi, handed
    in through X_cache (reserved = 1: no solve runs), against the oracle's
    force from the same X to 1e-12; then the store path: with reserved = 0 the
    call solves, stores X and sets reserved, and the next call reuses it."""
    L = (4, 4, 2, 4)
    V = inputs.volume(L)
    kappa, mu = 0.14, 0.1
    U = inputs.random_gauge(L, "near", seed=37, eps=0.4)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=recon)
    ev = ~oracle.parity_mask(L)
    phi = inputs.gaussian_spinor(L, 38) * ev[:, None, None]
    Sref, X = oracle.pseudofermion_action(U, phi, L, kappa, mu, eo=True, tol=1e-14)
    ref = oracle.fermion_dSdw(U, X, L, kappa, mu, eo=True)
    keep, fphi = _even_half_field(ctx, L, phi)
    keepx, fx = _even_half_field(ctx, L, X * ev[:, None, None])
    fx.reserved = 1
    F = torch.zeros((4, V, 8), dtype=torch.float64, device="cuda")
    prm = lqcd.cg_params(tol=1e-13, max_iter=50000)
    S, st = lqcd.lqcd_fermion_force(ctx, G, fphi, F, kappa, mu, prm, X_cache=fx)
    assert st["iters"] == 0
    assert relerr(host(F), ref) < 1e-12
    assert abs(S - np.vdot(phi, X).real) < 1e-12 * abs(S)
    # store path
    keepy, fy = _even_half_field(ctx, L, np.zeros_like(phi))
    F1 = torch.zeros_like(F)
    S1, st1 = lqcd.lqcd_fermion_force(ctx, G, fphi, F1, kappa, mu, prm, X_cache=fy)
    assert st1["iters"] > 0 and fy.reserved == 1
    F2 = torch.zeros_like(F)
    S2, st2 = lqcd.lqcd_fermion_force(ctx, G, fphi, F2, kappa, mu, prm, X_cache=fy)
    assert st2["iters"] == 0 and S2 == S1
    assert torch.equal(F1, F2)
    assert relerr(host(F2), ref) < 1e-9


def test_fermion_force_finite_difference_gpu(ctx, oracle):
    """Central differences of the GPU action S = phi^+ (Mhat^+ Mhat)^-1 phi on single
    links (one crossing the time boundary) agree with the GPU force to 1e-6."""
    L = (4, 4, 2, 4)
    V = inputs.volume(L)
    kappa, mu = 0.14, 0.1
    U = inputs.random_gauge(L, "near", seed=39, eps=0.4)
    ev = ~oracle.parity_mask(L)
    phi = inputs.gaussian_spinor(L, 40) * ev[:, None, None]
    keep, fphi = _even_half_field(ctx, L, phi)
    prm = lqcd.cg_params(tol=1e-14, max_iter=50000)
    F = torch.zeros((4, V, 8), dtype=torch.float64, device="cuda")
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    lqcd.lqcd_fermion_force(ctx, G, fphi, F, kappa, mu, prm)
    Fh = host(F)
    c = inputs.site_coords(L)
    tb = int(np.nonzero(c[:, 3] == L[3] - 1)[0][1])
    h = 1e-5
    worst = 0.0
    for (i, m) in [(0, 0), (9, 1), (tb, 3)]:
        for a in range(8):
            vals = []
            for sgn in (1, -1):
                Ud = U.copy()
                Ud[i, m] = scipy.linalg.expm(1j * sgn * h * oracle.generator(a)) @ U[i, m]
                Gd = lqcd.lqcd_gauge_import(ctx, dev(Ud), L)
                S, _ = lqcd.lqcd_fermion_force(ctx, Gd, fphi, F, kappa, mu, prm)
                vals.append(S)
                Gd.free()
            fd = (vals[0] - vals[1]) / (2 * h)
            worst = max(worst, abs(fd - Fh[m, i, a]) / max(1.0, abs(fd)))
    assert worst < 1e-6, worst


def test_hmc_trajectory_matches_oracle(ctx, oracle):
    """One leapfrog trajectory from the same links with the same Philox momenta
    and pseudofermion: dH and the final links agree with the oracle."""
    L = (4, 4, 2, 4)
    beta, kappa, mu = 5.6, 0.14, 0.05 / 0.28
    U = inputs.random_gauge(L, "near", seed=41, eps=0.3)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    seed, traj = 1234, 3
    prm = lqcd.hmc_params(beta, kappa, mu, tau=0.5, nsteps=8, nf=1, seed=seed, traj=traj,
                          cg=lqcd.cg_params(tol=1e-13, max_iter=50000))
    st = lqcd.lqcd_hmc_trajectory(ctx, G, prm)
    P0 = oracle.momenta(L, seed, traj)
    eta = oracle.gaussian_spinor(L, seed, traj) * (~oracle.parity_mask(L))[:, None, None]
    phi = oracle.apply_Mhat(U, eta, L, kappa, mu, dagger=True)
    U1, P1, dH, (H0, H1, Sf0) = oracle.hmc_md(U, P0, phi, L, beta, kappa, mu, nf=1, nsteps=8,
                                              tau=0.5, tol=1e-13)
    assert abs(st["H0"] - H0) < 1e-9 * abs(H0)
    assert abs(st["dH"] - dH) < 1e-7 * max(1.0, abs(dH))
    if st["accepted"]:
        assert relerr(_export(ctx, G, L), U1) < 1e-10
    else:
        assert np.array_equal(_export(ctx, G, L), U)


def test_pure_gauge_hmc_matches_oracle_and_scales(ctx, oracle):
    """Pure-gauge trajectory (nf = 0): dH equals the oracle's for the same
    Philox momenta, and halving the step size divides dH by about 4."""
    L = (4, 4, 4, 4)
    U = inputs.random_gauge(L, "near", seed=42, eps=0.3)
    dHs = {}
    for n in (20, 40):
        G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
        st = lqcd.lqcd_hmc_trajectory(ctx, G, lqcd.hmc_params(5.6, 0.0, 0.0, tau=1.0, nsteps=n,
                                                              nf=0, seed=9, traj=0))
        dHs[n] = st["dH"]
        G.free()
    _, _, dH_ref, _ = oracle.hmc_md(U, oracle.momenta(L, 9, 0), None, L, 5.6, 0.0, 0.0, nf=0,
                                    nsteps=20, tau=1.0)
    assert abs(dHs[20] - dH_ref) < 1e-8 * max(1.0, abs(dH_ref))
    assert 3.0 < dHs[20] / dHs[40] < 5.3


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (2, 4, 6, 8)])
@pytest.mark.parametrize("prec", [lqcd.LQCD_F64, lqcd.LQCD_DF64])
@pytest.mark.parametrize("c1", [lqcd.TLSYM_C1, 0.0])
def test_tlsym_gauge_force_and_action(ctx, oracle, L, prec, c1):
    """Tree-level Symanzik action (c1 = -1/12, Sec. 2.1 eq. S_tlsym) and the
    Wilson action (c1 = 0), in FP64 and in float-float: the GPU staples
    against the oracle's loop-by-loop derivative, and the action against the
    oracle's plaquette + rectangle sums."""
    beta = 3.9
    U = inputs.random_gauge(L, "near", seed=43, eps=0.5)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    F = torch.zeros((4, inputs.volume(L), 8), dtype=torch.float64, device="cuda")
    S = lqcd.lqcd_gauge_force(ctx, G, beta, F, c1=c1, prec=prec)
    assert relerr(host(F), oracle.gauge_dSdw_sym(U, L, beta, c1)) < 1e-13
    Sref = oracle.gauge_action_sym(U, L, beta, c1)
    assert abs(S - Sref) < 1e-11 * abs(Sref)


@pytest.mark.parametrize("force_prec", [lqcd.LQCD_F64, lqcd.LQCD_DF64])
def test_hmc_2mn_tlsym_trajectory_matches_oracle(ctx, oracle, force_prec):
    """One trajectory of the paper's HMC setup kind (Sec. 5.3): tlSym gauge
    action, 2MN on separate fermion and gauge time scales, from the same links
    and Philox streams as the oracle; dH and the final links agree."""
    L = (4, 4, 2, 4)
    beta, kappa, mu, c1 = 3.9, 0.14, 0.1 / 0.28, lqcd.TLSYM_C1
    U = inputs.random_gauge(L, "near", seed=44, eps=0.3)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    seed, traj = 77, 5
    prm = lqcd.hmc_params(beta, kappa, mu, tau=0.5, nsteps=3, nf=1, seed=seed, traj=traj,
                          cg=lqcd.cg_params(tol=1e-13, max_iter=50000), integrator=lqcd.LQCD_2MN,
                          c1=c1, nsteps_gauge=2, force_prec=force_prec)
    st = lqcd.lqcd_hmc_trajectory(ctx, G, prm)
    P0 = oracle.momenta(L, seed, traj)
    eta = oracle.gaussian_spinor(L, seed, traj) * (~oracle.parity_mask(L))[:, None, None]
    phi = oracle.apply_Mhat(U, eta, L, kappa, mu, dagger=True)
    U1, P1, dH, (H0, H1, Sf0) = oracle.hmc_md_2mn(U, P0, phi, L, beta, kappa, mu, c1=c1, nf=1,
                                                  nsteps_f=3, nsteps_g=2, tau=0.5, tol=1e-13)
    assert abs(st["H0"] - H0) < 1e-9 * abs(H0)
    assert abs(st["dH"] - dH) < 1e-7 * max(1.0, abs(dH))
    if st["accepted"]:
        assert relerr(_export(ctx, G, L), U1) < 1e-10
    else:
        assert np.array_equal(_export(ctx, G, L), U)


def test_hmc_2mn_pure_gauge_scaling(ctx, oracle):
    """Pure-gauge 2MN (tlSym): dH equals the oracle's and is second order."""
    L = (4, 4, 4, 4)
    U = inputs.random_gauge(L, "near", seed=45, eps=0.3)
    c1 = lqcd.TLSYM_C1
    dHs = {}
    for ng in (2, 4):
        G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
        prm = lqcd.hmc_params(3.9, 0.0, 0.0, tau=1.0, nsteps=2, nf=0, seed=10, traj=0,
                              integrator=lqcd.LQCD_2MN, c1=c1, nsteps_gauge=ng)
        dHs[ng] = lqcd.lqcd_hmc_trajectory(ctx, G, prm)["dH"]
        G.free()
    _, _, dH_ref, _ = oracle.hmc_md_2mn(U, oracle.momenta(L, 10, 0), None, L, 3.9, 0.0, 0.0, c1=c1, nf=0,
                                        nsteps_f=2, nsteps_g=2, tau=1.0)
    assert abs(dHs[2] - dH_ref) < 1e-8 * max(1.0, abs(dH_ref))
    assert 3.0 < dHs[2] / dHs[4] < 5.3, dHs


@pytest.mark.parametrize("recon", [18, 12])
def test_f32_heatbath_strong_coupling(ctx, recon):
    """The single-precision heatbath (Sec. 5.1 measures the FP32 kernels), with
    18-real and REC12 links: <P> = beta/18 + beta^2/216 at beta = 0.3."""
    L = (8, 8, 8, 8)
    beta = 0.3
    G = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "cold")), L, recon=recon)
    vals = []
    for s in range(80):
        lqcd.lqcd_heatbath_sweep(ctx, G, beta, 78, s, prec=lqcd.LQCD_F32)
        if s >= 10:
            vals.append(lqcd.lqcd_plaquette(ctx, G))
    vals = np.array(vals)
    expect = beta / 18 + beta ** 2 / 216
    err = vals.std() / np.sqrt(len(vals))
    assert abs(vals.mean() - expect) < 4 * err + 2e-4


def test_f32_heatbath_equilibrium_and_unitarity(ctx):
    """At beta = 5.7 the FP32 and FP64 heatbaths reach the same plaquette; the
    FP32 result is written back reunitarised in FP64."""
    L = (8, 8, 8, 8)
    means = {}
    for prec in (lqcd.LQCD_F64, lqcd.LQCD_F32):
        G = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "cold")), L)
        vals = []
        for s in range(70):
            lqcd.lqcd_heatbath_sweep(ctx, G, 5.7, 79, s, n_or=1, prec=prec)
            if s >= 30:
                vals.append(lqcd.lqcd_plaquette(ctx, G))
        means[prec] = np.mean(vals)
        if prec == lqcd.LQCD_F32:
            got = _export(ctx, G, L)
            eye = np.eye(3)
            assert np.max(np.abs(got @ np.conj(np.transpose(got, (0, 1, 3, 2))) - eye)) < 1e-13
            assert np.max(np.abs(np.linalg.det(got) - 1)) < 1e-13
        G.free()
    assert 0.53 < means[lqcd.LQCD_F64] < 0.57
    assert abs(means[lqcd.LQCD_F32] - means[lqcd.LQCD_F64]) < 4e-3, means


@pytest.mark.parametrize("recon", [18, 12])
def test_f32_sweep_write_back_keeps_the_fp32_copy_current(ctx, recon):
    """After an FP32 sweep the library rewrites its FP32 link copy from the
    reunitarised FP64 field instead of converting it again: an FP32 hop on the
    swept field equals, bit for bit, the FP32 hop on a fresh import of the
    exported FP64 links (whose FP32 copy is made by the conversion), and the
    FP64 links are unitary to 1e-13 (the float-float Gram-Schmidt of the
    write-back)."""
    L = (8, 4, 6, 8)
    G = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "haar", seed=93)), L, recon=recon)
    for s in range(3):
        lqcd.lqcd_heatbath_sweep(ctx, G, 5.7, 94, s, n_or=1, prec=lqcd.LQCD_F32)
    U = _export(ctx, G, L)
    eye = np.eye(3)
    assert np.max(np.abs(U @ np.conj(np.transpose(U, (0, 1, 3, 2))) - eye)) < 1e-13
    G2 = lqcd.lqcd_gauge_import(ctx, dev(U), L, recon=recon)
    psi = inputs.gaussian_spinor(L, 95)
    outs = []
    for g in (G, G2):
        d, sc, _ = eo_full_from_lexi(ctx, L, psi, lqcd.LQCD_F32)
        fe, fo = half_views(L, d, sc, lqcd.LQCD_F32)
        od, osc = lqcd.alloc_field(L, lqcd.LQCD_FULL, lqcd.LQCD_F32)
        oe, _ = half_views(L, od, osc, lqcd.LQCD_F32)
        lqcd.lqcd_dslash(ctx, g, fo, oe, lqcd.LQCD_EVEN, 0)
        torch.cuda.synchronize()
        outs.append(od.clone())
    assert torch.equal(outs[0].view(torch.uint8), outs[1].view(torch.uint8))
    G.free()
    G2.free()


def test_f32_overrelaxation_preserves_action(ctx):
    L = (4, 4, 4, 4)
    G = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "near", seed=37, eps=0.8)), L)
    F = torch.zeros((4, inputs.volume(L), 8), dtype=torch.float64, device="cuda")
    G2 = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "cold")), L)
    lqcd.lqcd_heatbath_sweep(ctx, G, 5.7, 2, 0, prec=lqcd.LQCD_F32)
    lqcd.lqcd_gauge_copy(ctx, G, G2)
    lqcd.lqcd_heatbath_sweep(ctx, G, 5.7, 2, 1, n_or=0, prec=lqcd.LQCD_F32)
    lqcd.lqcd_heatbath_sweep(ctx, G2, 5.7, 2, 1, n_or=2, prec=lqcd.LQCD_F32)
    S1 = lqcd.lqcd_gauge_force(ctx, G, 5.7, F)
    S2 = lqcd.lqcd_gauge_force(ctx, G2, 5.7, F)
    assert abs(S2 - S1) < 1e-5 * abs(S1)
    assert np.abs(_export(ctx, G, L) - _export(ctx, G2, L)).max() > 0.3  # the links moved


def test_heatbath_rejects_other_precisions(ctx):
    L = (4, 4, 4, 4)
    G = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "cold")), L)
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.lqcd_heatbath_sweep(ctx, G, 5.7, 1, 0, prec=lqcd.LQCD_BF16S)
    assert e.value.status == lqcd.LQCD_ERR_INVALID


def test_ratio_force_matches_oracle(ctx, oracle):
    """Mass-preconditioning ratio S2 = phi2^+ W (Mhat^+ Mhat)^-1 W^+ phi2,
    W = Mhat(mu2): action and force against the oracle's."""
    L = (4, 4, 2, 4)
    V = inputs.volume(L)
    kappa, mu, mu2 = 0.14, 0.05, 0.3
    U = inputs.random_gauge(L, "near", seed=46, eps=0.4)
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    ev = ~oracle.parity_mask(L)
    phi2 = inputs.gaussian_spinor(L, 47) * ev[:, None, None]
    keep, fphi = _even_half_field(ctx, L, phi2)
    F = torch.zeros((4, V, 8), dtype=torch.float64, device="cuda")
    prm = lqcd.cg_params(tol=1e-13, max_iter=50000)
    S2, st = lqcd.lqcd_fermion_force_ratio(ctx, G, fphi, F, kappa, mu, mu2, prm)
    Sref, X = oracle.hasenbusch_action(U, phi2, L, kappa, mu, mu2, tol=1e-14)
    ref = oracle.hasenbusch_dSdw(U, phi2, X, L, kappa, mu, mu2)
    assert abs(S2 - Sref) < 1e-10 * abs(Sref)
    assert relerr(host(F), ref) < 1e-9


def test_hmc_mass_preconditioning(ctx, oracle):
    """HMC with mass preconditioning on three 2MN time scales (ratio, W, gauge):
    the start Hamiltonian is K + S_g + eta1^+ eta1 + eta2^+ eta2 (both
    pseudofermions drawn so), and dH is second order in the step size."""
    L = (4, 4, 2, 4)
    beta, kappa, mu, mu2, c1 = 3.9, 0.14, 0.05, 0.25, lqcd.TLSYM_C1
    U = inputs.random_gauge(L, "near", seed=48, eps=0.3)
    seed, traj = 91, 2
    dHs = {}
    for n in (2, 4):
        G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
        prm = lqcd.hmc_params(beta, kappa, mu, tau=0.5, nsteps=n, nf=1, seed=seed, traj=traj,
                              cg=lqcd.cg_params(tol=1e-13, max_iter=50000), integrator=lqcd.LQCD_2MN,
                              c1=c1, nsteps_gauge=2, mu2=mu2, nsteps_mid=2)
        st = lqcd.lqcd_hmc_trajectory(ctx, G, prm)
        dHs[n] = st["dH"]
        G.free()
    ev = ~oracle.parity_mask(L)
    eta1 = oracle.gaussian_spinor(L, seed, traj) * ev[:, None, None]
    eta2 = oracle.gaussian_spinor(L, seed ^ 0x9E3779B97F4A7C15, traj) * ev[:, None, None]
    P0 = oracle.momenta(L, seed, traj)
    H0 = (0.5 * np.sum(P0 ** 2) + oracle.gauge_action_sym(U, L, beta, c1) + np.vdot(eta1, eta1).real
          + np.vdot(eta2, eta2).real)
    assert abs(st["H0"] - H0) < 1e-9 * abs(H0)
    assert abs(dHs[2]) < 1.0
    assert 3.0 < dHs[2] / dHs[4] < 5.3, dHs


def test_hmc_mass_preconditioned_trajectory_matches_oracle(ctx, oracle):
    """One mass-preconditioned trajectory (Sec. 2.2) on three nested 2MN time
    scales -- ratio force outside, W = Mhat(mu2) force in the middle, tlSym
    gauge force inside -- from the same links and Philox streams as the
    oracle's three-scale integrator: H0, dH and the final links agree."""
    L = (4, 4, 2, 4)
    beta, kappa, mu, mu2, c1 = 3.9, 0.14, 0.05, 0.25, lqcd.TLSYM_C1
    U = inputs.random_gauge(L, "near", seed=49, eps=0.3)
    seed, traj = 93, 4
    G = lqcd.lqcd_gauge_import(ctx, dev(U), L)
    prm = lqcd.hmc_params(beta, kappa, mu, tau=0.5, nsteps=2, nf=1, seed=seed, traj=traj,
                          cg=lqcd.cg_params(tol=1e-13, max_iter=50000), integrator=lqcd.LQCD_2MN,
                          c1=c1, nsteps_gauge=2, mu2=mu2, nsteps_mid=2)
    st = lqcd.lqcd_hmc_trajectory(ctx, G, prm)
    ev = ~oracle.parity_mask(L)
    eta1 = oracle.gaussian_spinor(L, seed, traj) * ev[:, None, None]
    eta2 = oracle.gaussian_spinor(L, seed ^ 0x9E3779B97F4A7C15, traj) * ev[:, None, None]
    P0 = oracle.momenta(L, seed, traj)
    U1, P1, dH, (H0, H1), _ = oracle.hmc_md_2mn_hasenbusch(U, P0, eta1, eta2, L, beta, kappa, mu, mu2, c1=c1,
                                                           nsteps=2, nsteps_mid=2, nsteps_g=2, tau=0.5,
                                                           tol=1e-13)
    assert abs(st["H0"] - H0) < 1e-9 * abs(H0)
    assert abs(st["dH"] - dH) < 1e-7 * max(1.0, abs(dH))
    if st["accepted"]:
        assert relerr(_export(ctx, G, L), U1) < 1e-10
    else:
        assert np.array_equal(_export(ctx, G, L), U)
