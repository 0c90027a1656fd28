"""End-to-end pins of the oracle's LapH path on small lattices.

* full time/spin/LapH dilution with Z4 noise makes the stochastic estimate
  exact (Sec. II: Z_N noise gives zero-variance diagonals; complete
  projectors), so every correlator must equal the exact distillation
  correlator built from G = V_s^dag Omega^{-1} V_s (dense LU);
* the gamma_5-swapped estimator Eq. (laphpropg5) equals the direct one;
* partial dilution is unbiased: the noise average converges to G;
* correlators are gauge invariant;
* sinks of an eigenvector "solution" reproduce unit coefficient vectors.
"""
import numpy as np
import pytest

import synth
from oracle import laph, noise
from oracle import dilution as dl
from oracle.pipeline import OraclePath


@pytest.fixture(scope="module")
def full(exact_4x4):
    return exact_4x4


def test_full_dilution_single_line_is_exact(full):
    path, G = full
    t0 = 1
    bs = path.projectors_for_time(t0)
    line, x = path.line(5, bs, method="lu")
    coef = laph.sinks(path.evecs, x)                               # [b, t, alpha, n]
    rho = path.rho(5)
    est = sum(np.einsum("tan,sm->tansm", coef[i], np.conj(laph.diluted_noise(rho, path.dil, b)[t0]))
              for i, b in enumerate(bs))
    assert np.abs(est - G[:, :, :, t0, :, :]).max() < 1e-12 * np.abs(G).max()


@pytest.mark.parametrize("channel", ["pion", "rho", "scalar"])
def test_full_dilution_meson_equals_exact(full, channel):
    path, G = full
    for t0 in (0, 2):
        bs = path.projectors_for_time(t0)
        l1, _ = path.line(0, bs, method="lu")
        l2, _ = path.line(1, bs, method="lu")
        c_st = laph.meson_connected(l1, l2, t0, channel)
        c_ex = laph.exact_meson_connected(G, t0, channel)
        assert np.abs(c_st - c_ex).max() < 1e-10 * np.abs(c_ex).max()
        if channel == "pion":
            assert np.all(c_ex.real > 0) and np.abs(c_ex.imag).max() < 1e-10 * c_ex.real.max()


def test_full_dilution_pipi_equals_exact(full):
    path, G = full
    t0 = 0
    bs = path.projectors_for_time(t0)
    lines = [path.line(s, bs, method="lu")[0] for s in range(4)]
    c_st = laph.pipi_i2(*lines, t0)
    c_ex = laph.exact_pipi_i2(G, t0)
    assert np.abs(c_st - c_ex).max() < 1e-10 * np.abs(c_ex).max()
    # the crossed term is not negligible, so the test constrains it
    d = laph.exact_meson_connected(G, t0, "pion") ** 2
    assert np.abs(d - c_ex).max() > 1e-3 * np.abs(c_ex).max()


def test_gamma5_swapped_estimator(full):
    """Eq. (laphprop) and Eq. (laphpropg5) estimate the two time orderings of
    the same exact G; with full dilution both are exact."""
    path, G = full
    t0 = 3
    bs = path.projectors_for_time(t0)
    rho = path.rho(7)
    rhs = np.stack([laph.dirac_rhs(path.evecs, rho, path.dil, b) for b in bs])
    x, _ = path.solve(rhs, "lu")
    coefs = laph.sinks(path.evecs, x)                                          # [b, t, alpha, n]
    pr = [laph.diluted_noise(rho, path.dil, b)[t0] for b in bs]               # [alpha, n] at t0
    est_direct = sum(np.einsum("tan,sm->tansm", coefs[i], np.conj(pr[i])) for i in range(len(bs)))
    rb = [-np.einsum("ab,bn->an", laph.G5G4, pr[i]) for i in range(len(bs))]
    fb = [np.einsum("ab,tbn->tan", laph.G5G4, coefs[i]) for i in range(len(bs))]
    est_swapped = sum(np.einsum("an,tbm->antbm", rb[i], np.conj(fb[i])) for i in range(len(bs)))
    scale = np.abs(G).max()
    assert np.abs(est_direct - G[:, :, :, t0, :, :]).max() < 1e-12 * scale
    assert np.abs(est_swapped - G[t0, :, :, :, :, :]).max() < 1e-12 * scale


def test_noise_average_converges_to_exact(full):
    path, G = full
    dil = ((1, 0), (0, 0), (3, 2))          # (TF, S none, LI2): off-diagonal noise survives
    path_p = path
    t0 = 0
    nT, nS, nL = dl.counts(dil, path.wl.nt, path.wl.nv)
    bs = [(t0 * nS + bS) * nL + bL for bS in range(nS) for bL in range(nL)]
    ests = []
    for s in range(48):
        rho = path_p.rho(100 + s)
        rhs = np.stack([laph.dirac_rhs(path.evecs, rho, dil, b) for b in bs])
        x, _ = path.solve(rhs, "lu")
        coef = laph.sinks(path.evecs, x)
        ests.append(sum(np.einsum("tan,sm->tansm", coef[i], np.conj(laph.diluted_noise(rho, dil, b)[t0]))
                        for i, b in enumerate(bs)))
    ests = np.array(ests)
    target = G[:, :, :, t0, :, :]
    mean = ests.mean(0)
    sigma = ests.std(0) / np.sqrt(len(ests))
    err = np.abs(mean - target)
    assert np.abs(ests[0] - target).max() > 1e-3 * np.abs(target).max()     # one noise is not exact
    mask = sigma > 1e-14
    assert np.all(err[mask] < 5.5 * sigma[mask] + 1e-12)
    assert np.all(err[~mask] < 1e-12)


def test_gauge_invariance(full):
    path, G = full
    wl = path.wl
    from oracle import gauge
    g = synth.random_gauge_transform(wl.ns, wl.nt, seed=77)
    path_g = OraclePath(wl, u0=gauge.gauge_transform_links(wl.gauge(), g))
    # fresh eigenvectors (own phases): full-dilution correlators are invariant
    t0 = 1
    bs = path.projectors_for_time(t0)
    for ch in ("pion", "rho"):
        a = laph.meson_connected(path.line(0, bs, "lu")[0], path.line(1, bs, "lu")[0], t0, ch)
        b = laph.meson_connected(path_g.line(0, bs, "lu")[0], path_g.line(1, bs, "lu")[0], t0, ch)
        assert np.abs(a - b).max() < 1e-10 * np.abs(a).max()
    # partial dilution with the transformed eigenvectors G v carried over: identical coefficients
    path_g.evecs = np.einsum("tzyxab,tnzyxb->tnzyxa", g, path.evecs.reshape(wl.nt, wl.nv, wl.ns, wl.ns, wl.ns, 3)).reshape(path.evecs.shape)
    dil = ((1, 0), (1, 0), (3, 2))
    path.dil = path_g.dil = dil
    try:
        bs = path.projectors_for_time(t0)
        a = laph.meson_connected(path.line(2, bs, "lu")[0], path.line(3, bs, "lu")[0], t0, "pion")
        b = laph.meson_connected(path_g.line(2, bs, "lu")[0], path_g.line(3, bs, "lu")[0], t0, "pion")
        assert np.abs(a - b).max() < 1e-10 * np.abs(a).max()
    finally:
        path.dil = ((1, 0), (1, 0), (1, 0))


def test_sinks_reproduce_unit_vectors(full):
    path, _ = full
    ev = path.evecs
    nt, nv = ev.shape[:2]
    for t, n, a in [(0, 0, 0), (2, 3, 1), (3, 1, 3)]:
        c = np.zeros((nt, 4, nv), dtype=complex)
        c[t, a, n] = 1.0
        x = laph.lapH_to_site(ev, c)
        assert np.abs(laph.sinks(ev, x) - c).max() < 1e-13
