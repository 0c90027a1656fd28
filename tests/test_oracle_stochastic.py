"""Pins of the oracle's stochastic LapH estimator for general correlators (Sec. II-III:
noisy quark lines joined by the graphical rules; oracle/wick.py stochastic_expect) on a
4^3 x 4 lattice, against the brute-force Wick contraction with the exact G.

* the gamma_5 swap of a line estimate, Gamma' Q^dag Gamma', reproduces G itself
  (G = Gamma' G^dag Gamma' with Gamma' = gamma_4 gamma_5);
* full dilution: forward lines sourced at t0 and same-time lines with every projector
  solved make every estimate exact: isoscalar mesons (forward + same-time diagrams) and the
  I = 0, 1, 2 two-pion correlators (direct, crossed, box and vacuum diagrams), at zero and
  nonzero pion momentum;
* partial dilution: the I = 0 two-pion estimate is noisy for one noise set and its average
  over noise sets converges to the exact correlator (within 5.5 sigma).
"""
import numpy as np
import pytest

from oracle import dilution as dl
from oracle import laph, wick

GP = laph.GAMMA[3] @ laph.GAMMA5


def estimate(path, noise_id, dil, bs):
    saved = path.dil
    path.dil = dil
    try:
        _, x = path.line(noise_id, bs, method="lu")
    finally:
        path.dil = saved
    rho = path.rho(noise_id)
    coef = laph.sinks(path.evecs, x)
    rho_b = np.stack([laph.diluted_noise(rho, dil, b) for b in bs])
    return wick.line_estimate(coef, rho_b)


def fwd_projectors(dil, nt, nv, t0):
    nT, nS, nL = dl.counts(dil, nt, nv)
    kT, JT = dil[0]
    return [(bT * nS + bS) * nL + bL for bT in range(nT) if dl.projector_diag(kT, JT, nt, bT)[t0]
            for bS in range(nS) for bL in range(nL)]


def all_projectors(dil, nt, nv):
    nT, nS, nL = dl.counts(dil, nt, nv)
    return list(range(nT * nS * nL))


def line_sets(path, t0, dil_fwd, dil_smt, seed):
    nt, nv = path.wl.nt, path.wl.nv
    fwd = [estimate(path, seed + i, dil_fwd, fwd_projectors(dil_fwd, nt, nv, t0)) for i in range(4)]
    bwd = [wick.gamma_swap(q, nt, nv, GP) for q in fwd]
    smt = [estimate(path, seed + 10 + i, dil_smt, all_projectors(dil_smt, nt, nv)) for i in range(4)]
    return fwd, bwd, smt


@pytest.fixture(scope="module")
def setup(exact_4x4):
    path, G = exact_4x4
    N = path.wl.nt * 4 * path.wl.nv
    return path, G, G.reshape(N, N)


def _phi(path, mom):
    return laph.mom_overlaps(path.evecs, mom)


def test_gamma_swap_is_exact_on_G(setup):
    path, G, Q = setup
    assert np.abs(wick.gamma_swap(Q, path.wl.nt, path.wl.nv, GP) - Q).max() < 1e-12 * np.abs(Q).max()


@pytest.fixture(scope="module")
def full_lines(setup):
    path, _, _ = setup
    full = ((1, 0), (1, 0), (1, 0))
    return {t0: line_sets(path, t0, full, full, 100) for t0 in (1,)}


def test_full_dilution_isoscalar_exact(setup, full_lines):
    path, G, Q = setup
    nt, nv, t0 = path.wl.nt, path.wl.nv, 1
    fwd, bwd, smt = full_lines[t0]
    for ch in ("pion", "scalar"):
        c = laph.channel_c(ch)[0]
        one = np.eye(nv)
        r = 1.0 / np.sqrt(2.0)
        for dt in range(nt):
            tf = (t0 + dt) % nt
            snk = [(r, [wick.sink_bilinear(nt, nv, tf, c, one, f, f)]) for f in "ud"]
            src = [(r, [wick.source_bilinear(nt, nv, t0, c, one, f, f)]) for f in "ud"]
            ex = wick.correlator(snk, src, Q)
            st = wick.stochastic_correlator(snk, src, tf, t0, fwd, bwd, smt)
            assert abs(st - ex) < 1e-10 * max(1.0, abs(ex))


@pytest.mark.parametrize("mom", [(0, 0, 0), (1, 0, 0)])
@pytest.mark.parametrize("iso", [(2, 2), (1, 0), (0, 0)])
def test_full_dilution_two_pion_exact(setup, full_lines, mom, iso):
    path, G, Q = setup
    nt, nv, t0 = path.wl.nt, path.wl.nv, 1
    fwd, bwd, smt = full_lines[t0]
    c = laph.channel_c("pion")[0]
    ph, phm = _phi(path, mom), _phi(path, tuple(-m for m in mom))
    scale = 0.0
    for dt in range(nt):
        tf = (t0 + dt) % nt
        snk = wick.two_pion_sink(nt, nv, tf, c, ph[tf], phm[tf], iso)
        src = wick.two_pion_source(nt, nv, t0, c, ph[t0], phm[t0], iso)
        ex = wick.correlator(snk, src, Q)
        st = wick.stochastic_correlator(snk, src, tf, t0, fwd, bwd, smt)
        scale = max(scale, abs(ex))
        assert abs(st - ex) < 1e-9 * max(scale, 1e-30) + 1e-14


def test_partial_dilution_two_pion_i0_unbiased(setup):
    path, G, Q = setup
    nt, nv, t0, dt = path.wl.nt, path.wl.nv, 0, 1
    tf = (t0 + dt) % nt
    c = laph.channel_c("pion")[0]
    one = np.eye(nv)
    snk = wick.two_pion_sink(nt, nv, tf, c, one, one, (0, 0))
    src = wick.two_pion_source(nt, nv, t0, c, one, one, (0, 0))
    ex = wick.correlator(snk, src, Q)
    dil_fwd = ((1, 0), (1, 0), (3, 2))       # (TF, SF, LI2) from t0
    dil_smt = ((3, 2), (1, 0), (3, 2))       # (TI2, SF, LI2), every projector
    ests = []
    for s in range(24):
        fwd, bwd, smt = line_sets(path, t0, dil_fwd, dil_smt, 1000 + 100 * s)
        ests.append(wick.stochastic_correlator(snk, src, tf, t0, fwd, bwd, smt))
    ests = np.array(ests)
    assert abs(ests[0] - ex) > 1e-4 * abs(ex)                    # one noise set is not exact
    mean = ests.mean()
    sig_re = ests.real.std() / np.sqrt(len(ests))
    sig_im = ests.imag.std() / np.sqrt(len(ests))
    assert abs(mean.real - ex.real) < 5.5 * sig_re + 1e-12
    assert abs(mean.imag - ex.imag) < 5.5 * sig_im + 1e-12
