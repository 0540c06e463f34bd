"""Statistical pins of the Monte Carlo (Sec. 2.2): what the samplers must get
right in distribution, not link by link.

- Creutz's equality <exp(-dH)> = 1 for the HMC's molecular dynamics
  (reversible and area-preserving: in equilibrium it holds for every
  proposal, accepted or not), with <dH> >= 0, pure gauge and with the
  twisted-mass doublet.
- The GPU heatbath and the oracle's heatbath, run as independent chains
  (different seeds), give the same mean plaquette at beta = 5.7.
- The heatbath and a pure-gauge HMC sample the same Wilson-action
  distribution: the same mean plaquette.

The chains are seeded, so the tests are deterministic; the bounds are four
standard errors, with the errors of the plaquette series taken from blocks
longer than their autocorrelation.
"""
import numpy as np
import pytest
import torch

from paper_1209_5942_gb300 import inputs, lqcd
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1209_5942_gb300 import build
    build.build()
    return lqcd.Context(0)


def _blocked(x, nblocks=10):
    """Mean and standard error of a correlated series from block means."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // nblocks * nblocks
    b = x[:n].reshape(nblocks, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / np.sqrt(nblocks)


def _thermalised(ctx, L, beta, sweeps, seed):
    G = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "cold")), L)
    for s in range(sweeps):
        lqcd.lqcd_heatbath_sweep(ctx, G, beta, seed, s, n_or=1)
    return G


def _chain(ctx, G, make_params, therm, meas):
    out = []
    for t in range(therm + meas):
        st = lqcd.lqcd_hmc_trajectory(ctx, G, make_params(t))
        if t >= therm:
            out.append(st)
    return out


@pytest.fixture(scope="module")
def gauge_chain(ctx):
    """Pure-gauge HMC at beta = 5.7 on 4^4 from a heatbath-thermalised field:
    leapfrog, tau = 1, 20 steps."""
    L = (4, 4, 4, 4)
    G = _thermalised(ctx, L, 5.7, 60, 61)
    return _chain(ctx, G, lambda t: lqcd.hmc_params(5.7, 0.0, 0.0, tau=1.0, nsteps=20, nf=0, seed=62, traj=t),
                  100, 900)


def _creutz(dH):
    """<exp(-dH)> with a blocked error, and <dH>."""
    w = np.exp(-np.asarray(dH))
    m, e = _blocked(w, 20)
    return m, e


def test_creutz_equality_pure_gauge(gauge_chain):
    dH = np.array([s["dH"] for s in gauge_chain])
    m, e = _creutz(dH)
    assert 0.02 < np.mean(np.abs(dH)) < 2.0, np.mean(np.abs(dH))  # dH is not ~0: the test has teeth
    assert abs(m - 1.0) < 4 * e, (m, e, dH.mean())
    assert dH.mean() > -4 * _blocked(dH, 20)[1]  # <dH> >= 0 (Jensen)


def test_creutz_equality_with_fermions(ctx):
    """The same for the twisted-mass doublet (every force through the CG and
    the adjoint kernel), kappa = 0.13, 2 kappa mu = 0.026, beta = 5.6."""
    L = (4, 4, 4, 4)
    G = _thermalised(ctx, L, 5.6, 60, 63)
    cg = lqcd.cg_params(tol=1e-11, outer_prec=lqcd.LQCD_DF64, inner_prec=lqcd.LQCD_F32, max_iter=50000)
    chain = _chain(ctx, G, lambda t: lqcd.hmc_params(5.6, 0.13, 0.1, tau=0.5, nsteps=10, nf=1, seed=64, traj=t,
                                                     cg=cg), 40, 360)
    dH = np.array([s["dH"] for s in chain])
    m, e = _creutz(dH)
    assert 0.01 < np.mean(np.abs(dH)) < 2.0, np.mean(np.abs(dH))
    assert abs(m - 1.0) < 4 * e, (m, e, dH.mean())
    assert np.mean([s["accepted"] for s in chain]) > 0.5


def test_heatbath_chain_matches_oracle_chain(ctx, oracle):
    L = (4, 4, 4, 4)
    beta, nsw, therm = 5.7, 240, 40
    G = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "cold")), L)
    gp = []
    for s in range(nsw):
        lqcd.lqcd_heatbath_sweep(ctx, G, beta, 4711, s)
        if s >= therm:
            gp.append(lqcd.lqcd_plaquette(ctx, G))
    U = inputs.random_gauge(L, "cold")
    op = []
    for s in range(nsw):
        U, _ = oracle.heatbath_sweep(U, L, beta, 815, s)
        if s >= therm:
            op.append(oracle.plaquette(U, L))
    mg, eg = _blocked(gp)
    mo, eo = _blocked(op)
    assert abs(mg - mo) < 4 * np.hypot(eg, eo), (mg, eg, mo, eo)
    assert 0.5 < mg < 0.62


def test_heatbath_and_pure_gauge_hmc_agree(ctx, gauge_chain):
    L = (4, 4, 4, 4)
    beta = 5.7
    G = lqcd.lqcd_gauge_import(ctx, dev(inputs.random_gauge(L, "cold")), L)
    hb = []
    for s in range(440):
        lqcd.lqcd_heatbath_sweep(ctx, G, beta, 77, s, n_or=1)
        if s >= 40:
            hb.append(lqcd.lqcd_plaquette(ctx, G))
    hmc = [s["plaquette"] for s in gauge_chain]
    mh, eh = _blocked(hb, 20)
    mm, em = _blocked(hmc, 20)
    assert np.mean([s["accepted"] for s in gauge_chain]) > 0.5
    assert abs(mh - mm) < 4 * np.hypot(eh, em), (mh, eh, mm, em)
