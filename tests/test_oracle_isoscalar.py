"""Pins of the oracle's same-time quark lines (second term of Eq. (mesoncorr): the "smt"
diagram of the isoscalar mesons) on a 4^3 x 4 lattice.

* full time/spin/LapH dilution with every projector solved: the loops built from the
  site-space meson functions equal the exact ones from G = V_s^dag Omega^{-1} V_s, in both
  orientations, at zero and nonzero momentum, and so does the disconnected correlator;
* gamma_5-Hermiticity of K gives G^dag = (gamma_4 gamma_5) G (gamma_4 gamma_5), so the two
  exact orientations differ by the sign of (gamma_4 gamma_5) c (gamma_4 gamma_5) = s c:
  s = -1 for the pion, +1 for the rho and the scalar;
* time interlacing (TI2) leaves noise between the slices of one interlace class; the
  noise average of the loops converges to the exact loops (within 5.5 sigma) while one
  noise alone does not reproduce them;
* the exact loops are gauge invariant (fresh eigenvectors of the transformed field).
"""
import numpy as np
import pytest

import synth
from oracle import dilution as dl
from oracle import gauge, laph
from oracle.pipeline import OraclePath


def all_projectors(path):
    nT, nS, nL = dl.counts(path.dil, path.wl.nt, path.wl.nv)
    return list(range(nT * nS * nL))


@pytest.fixture(scope="module")
def full(exact_4x4):
    path, G = exact_4x4
    bs = all_projectors(path)
    lines = [path.line(s, bs, method="lu")[0] for s in (3, 4)]
    return path, G, lines


@pytest.mark.parametrize("channel", ["pion", "rho", "scalar"])
@pytest.mark.parametrize("mom", [None, (1, 0, 0), (0, 1, 1)])
def test_full_dilution_loops_are_exact(full, channel, mom):
    path, G, (l1, l2) = full
    phi = None if mom is None else laph.mom_overlaps(path.evecs, mom)
    for reverse in (False, True):
        st = laph.meson_loops(l1, channel, mom, reverse)
        ex = laph.exact_loops(G, channel, phi, reverse)
        assert np.abs(st - ex).max() < 1e-10 * np.abs(ex).max()
    c_st = laph.meson_disconnected(l1, l2, 2, channel, mom)
    c_ex = laph.exact_meson_disconnected(G, 2, channel, phi)
    assert np.abs(c_st - c_ex).max() < 1e-10 * np.abs(c_ex).max()


@pytest.mark.parametrize("channel,sign", [("pion", -1.0), ("rho", 1.0), ("scalar", 1.0)])
@pytest.mark.parametrize("mom", [None, (1, 0, 0)])
def test_orientations_related_by_gamma5_hermiticity(full, channel, sign, mom):
    path, G, _ = full
    phi = None if mom is None else laph.mom_overlaps(path.evecs, mom)
    fwd = laph.exact_loops(G, channel, phi)
    rev = laph.exact_loops(G, channel, phi, reverse=True)
    assert np.abs(fwd).max() > 1e-6
    assert np.abs(rev - sign * fwd).max() < 1e-10 * np.abs(fwd).max()


def test_time_interlaced_loops_are_unbiased(full):
    path, G, _ = full
    dil = ((3, 2), (1, 0), (1, 0))          # (TI2, SF, LF): slices t and t + 2 share a projector
    saved = path.dil
    path.dil = dil
    try:
        bs = all_projectors(path)
        exact = laph.exact_loops(G, "scalar")[0]
        ests = np.array([laph.meson_loops(path.line(200 + s, bs, method="lu")[0], "scalar")[0] for s in range(40)])
    finally:
        path.dil = saved
    mean = ests.mean(0)
    sigma = ests.std(0) / np.sqrt(len(ests))
    assert np.abs(ests[0] - exact).max() > 1e-4 * np.abs(exact).max()      # one noise is not exact
    assert np.all(np.abs(mean - exact) < 5.5 * sigma + 1e-12)


def test_exact_loops_gauge_invariant(full):
    path, G, _ = full
    wl = path.wl
    g = synth.random_gauge_transform(wl.ns, wl.nt, seed=91)
    path_g = OraclePath(wl, u0=gauge.gauge_transform_links(wl.gauge(), g))
    G_g = path_g.exact_G()
    for ch in ("pion", "scalar"):
        for mom in (None, (0, 0, 1)):
            phi = None if mom is None else laph.mom_overlaps(path.evecs, mom)
            phi_g = None if mom is None else laph.mom_overlaps(path_g.evecs, mom)
            a = laph.exact_loops(G, ch, phi)
            b = laph.exact_loops(G_g, ch, phi_g)
            assert np.abs(a - b).max() < 1e-10 * np.abs(a).max()


def test_isoscalar_combination():
    fwd, smt = np.array([3.0, 1.0]), np.array([0.5, 0.25])
    assert np.allclose(laph.isoscalar_meson(fwd, smt), [4.0, 1.5])
    assert np.allclose(laph.isoscalar_meson(fwd, smt, vev=0.25), [3.5, 1.0])
