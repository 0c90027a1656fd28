"""Pins of the brute-force Wick reference (oracle/wick.py) and, through it, of the signs
and flavour weights of the oracle's correlator formulas.

* the permutation formula for < B_1 ... B_m > equals a literal Gaussian Grassmann
  integral, < X > = int X e^{-qbar A q} / int e^{-qbar A q}, computed in the exterior
  algebra of 2 N generators on a tiny two-flavour space (m = 1..4, mixed flavours);
  the two-point function of that integral is <q_j qbar_i> = (A^{-1})_{ji};
* on a 4^3 x 4 lattice with Q = G = V_s^dag Omega^{-1} V_s:
  - the connected meson correlator (first term of Eq. (mesoncorr), sign included) of a
    flavour non-singlet, at zero and nonzero momentum, is <M(t_F) Mbar(t_0)>;
  - the I = 2 two-pion formula D - X is half of <pi+ pi+ (t_F) (pi+ pi+)bar (t_0)> (the
    two identical pions at each end double both diagrams), which fixes the sign of X;
  - the isoscalar (u-bar c u + d-bar c d)/sqrt(2) gives fwd + 2 smt (the flavour weights
    of the second term of Eq. (mesoncorr));
  - the two-pion isospin operators (pion triplet coupled by the Clebsch-Gordan
    coefficients of 1 x 1, momenta p and -p): all members of each multiplet have equal
    correlators, different isospins do not correlate, I = 1 vanishes at p = 0 and the
    I = 2 top state is twice D - X.
"""
import zlib

import numpy as np
import pytest

from oracle import laph, wick


from tests.grassmann import Grassmann, _mul


@pytest.fixture(scope="module")
def two_flavour():
    rng = np.random.default_rng(4)
    n = 2
    A0 = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * np.eye(n)
    A = np.zeros((2 * n, 2 * n), dtype=complex)
    A[:n, :n] = A0
    A[n:, n:] = A0
    return n, A0, Grassmann(A)


def test_grassmann_two_point(two_flavour):
    n, A0, g = two_flavour
    inv = np.linalg.inv(A0)
    for j in range(n):
        for i in range(n):
            assert abs(g.expect(_mul(g.q(j), g.qbar(i))) - inv[j, i]) < 1e-12
            assert abs(g.expect(_mul(g.q(n + j), g.qbar(n + i))) - inv[j, i]) < 1e-12
            assert abs(g.expect(_mul(g.q(j), g.qbar(n + i)))) < 1e-14     # flavours do not mix


FLAV = {"u": 0, "d": 1}


@pytest.mark.parametrize("pattern", [("uu",), ("ud",), ("uu", "uu"), ("ud", "du"), ("ud", "ud"), ("uu", "dd"),
                                     ("ud", "du", "uu"), ("ud", "du", "ud", "du"), ("du", "du", "ud", "ud"),
                                     ("uu", "dd", "uu", "ud")])
def test_expect_matches_grassmann(two_flavour, pattern):
    n, A0, g = two_flavour
    rng = np.random.default_rng(zlib.crc32("".join(pattern).encode()))
    Q = np.linalg.inv(A0)
    bils, x = [], {(): 1.0}
    for fb, f in pattern:                     # qbar flavour, q flavour
        M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        bils.append((M, fb, f))
        x = _mul(x, g.bilinear(M, FLAV[fb] * n, FLAV[f] * n))
    ref = g.expect(x)
    got = wick.expect(bils, Q)
    assert abs(got - ref) < 1e-10 * max(1.0, abs(ref))


# ---------------------------------------------------------------- correlators on a lattice
@pytest.fixture(scope="module")
def lattice(exact_4x4):
    path, G = exact_4x4
    N = path.wl.nt * 4 * path.wl.nv
    return path, G, G.reshape(N, N)


def _phi(path, mom):
    if mom is None:
        return np.broadcast_to(np.eye(path.wl.nv), (path.wl.nt, path.wl.nv, path.wl.nv))
    return laph.mom_overlaps(path.evecs, mom)


def _neg(mom):
    return None if mom is None else tuple(-m for m in mom)


@pytest.mark.parametrize("channel", ["pion", "rho", "scalar"])
@pytest.mark.parametrize("mom", [None, (1, 0, 0)])
def test_meson_connected_is_wick(lattice, channel, mom):
    path, G, Q = lattice
    nt, nv, t0 = path.wl.nt, path.wl.nv, 1
    ph, phm = _phi(path, mom), _phi(path, _neg(mom))
    exact = laph.exact_meson_connected(G, t0, channel, None if mom is None else ph)
    cs = laph.channel_c(channel)
    for dt in range(nt):
        tf = (t0 + dt) % nt
        w = sum(wick.correlator([(1.0, [wick.sink_bilinear(nt, nv, tf, c, ph[tf], "d", "u")])],
                                [(1.0, [wick.source_bilinear(nt, nv, t0, c, phm[t0], "d", "u")])], Q)
                for c in cs) / len(cs)
        assert abs(w - exact[dt]) < 1e-10 * np.abs(exact).max()


def test_pipi_i2_is_wick(lattice):
    path, G, Q = lattice
    nt, nv, t0 = path.wl.nt, path.wl.nv, 0
    c = laph.channel_c("pion")[0]
    one = np.eye(nv)
    exact = laph.exact_pipi_i2(G, t0)
    for dt in range(nt):
        tf = (t0 + dt) % nt
        snk = [(1.0, [wick.sink_bilinear(nt, nv, tf, c, one, "d", "u")] * 2)]
        src = [(1.0, [wick.source_bilinear(nt, nv, t0, c, one, "d", "u")] * 2)]
        w = wick.correlator(snk, src, Q)
        assert abs(0.5 * w - exact[dt]) < 1e-10 * np.abs(exact).max()
    # the crossed term matters: D alone is not the answer
    d = laph.exact_meson_connected(G, t0, "pion") ** 2
    assert np.abs(d - exact).max() > 1e-3 * np.abs(exact).max()


@pytest.mark.parametrize("channel", ["pion", "scalar"])
@pytest.mark.parametrize("mom", [None, (0, 1, 0)])
def test_isoscalar_is_wick(lattice, channel, mom):
    path, G, Q = lattice
    nt, nv, t0 = path.wl.nt, path.wl.nv, 2
    ph, phm = _phi(path, mom), _phi(path, _neg(mom))
    c = laph.channel_c(channel)[0]
    phi = None if mom is None else ph
    iso = laph.isoscalar_meson(laph.exact_meson_connected(G, t0, channel, phi),
                               laph.exact_meson_disconnected(G, t0, channel, phi))
    r = 1.0 / np.sqrt(2.0)
    for dt in range(nt):
        tf = (t0 + dt) % nt
        snk = [(r, [wick.sink_bilinear(nt, nv, tf, c, ph[tf], f, f)]) for f in "ud"]
        src = [(r, [wick.source_bilinear(nt, nv, t0, c, phm[t0], f, f)]) for f in "ud"]
        w = wick.correlator(snk, src, Q)
        assert abs(w - iso[dt]) < 1e-10 * np.abs(iso).max()


def _pipi(path, Q, tf, t0, snk_iso, src_iso, mom):
    nt, nv = path.wl.nt, path.wl.nv
    c = laph.channel_c("pion")[0]
    ph, phm = _phi(path, mom), _phi(path, _neg(mom))
    return wick.correlator(wick.two_pion_sink(nt, nv, tf, c, ph[tf], phm[tf], snk_iso),
                           wick.two_pion_source(nt, nv, t0, c, ph[t0], phm[t0], src_iso), Q)


@pytest.mark.parametrize("mom", [None, (1, 0, 0)])
def test_two_pion_isospin_multiplets(lattice, mom):
    """Degenerate u, d: every member of an isospin multiplet has the same correlator on each
    configuration, and operators of different isospin do not correlate."""
    path, G, Q = lattice
    t0 = 1
    for dt in (0, 1, 2):
        tf = (t0 + dt) % path.wl.nt
        c = {k: _pipi(path, Q, tf, t0, k, k, mom) for k in [(2, 2), (2, 1), (2, 0), (1, 1), (1, 0), (0, 0)]}
        scale = max(abs(v) for v in c.values())
        assert abs(c[(2, 1)] - c[(2, 2)]) < 1e-10 * scale and abs(c[(2, 0)] - c[(2, 2)]) < 1e-10 * scale
        assert abs(c[(1, 0)] - c[(1, 1)]) < 1e-10 * scale
        assert abs(c[(0, 0)] - c[(2, 2)]) > 1e-3 * scale          # I = 0 and I = 2 differ
        for a, b in [((2, 0), (0, 0)), ((0, 0), (2, 0)), ((1, 0), (0, 0)), ((2, 0), (1, 0))]:
            assert abs(_pipi(path, Q, tf, t0, a, b, mom)) < 1e-10 * scale
        if mom is None:
            # equal momenta: the isospin-antisymmetric operator vanishes identically
            assert abs(c[(1, 0)]) < 1e-12 * scale
            # the I = 2 top state doubles the D - X of exact_pipi_i2
            assert abs(c[(2, 2)] - 2.0 * laph.exact_pipi_i2(G, t0)[dt]) < 1e-10 * scale
        else:
            assert abs(c[(1, 0)]) > 1e-3 * scale
