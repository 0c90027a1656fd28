"""Pins of the oracle's momentum-projected meson functions (Sec. III, the phase of
Eq. (mesonfunc) without displacement) and of the LapH overlap matrices
Phi_p(t) = V_s^dag e^{-i p.x} V_s that carry the phase in coefficient space.

* Phi_0 is the identity (orthonormal eigenvectors);
* free field: the lowest N_v = 21 eigenvectors of -Delta span the plane waves of the
  momenta S = {0, +-e_x, +-e_y, +-e_z} (three colours each), so in any basis of that
  space sum |Phi_p|^2 = 3 #{k in S : k - p in S} -- 21, 6, 6, 3 and 0 for the momenta
  below on a 6^3 slice;
* translation: shifting the gauge field by a lattice vector a shifts each
  (non-degenerate) eigenvector, so diag Phi_p picks up e^{-i p.a} and |Phi_p| is
  unchanged; a shift along x and one along z tell the axes apart and fix the sign of
  the phase;
* full time/spin/LapH dilution: the site-space stochastic correlator with the phase on
  every site equals the exact distillation correlator with Phi_p between the lines
  (two routes that share no momentum code);
* gamma_5-Hermiticity: the exact correlator at -p is the complex conjugate of the one
  at p in every channel.
"""
import numpy as np
import pytest

import synth
from oracle import gauge, laph, laplacian


def unit_links(ns, nt):
    return np.broadcast_to(np.eye(3, dtype=complex), (nt, ns, ns, ns, 4, 3, 3)).copy()


def test_zero_momentum_overlap_is_identity():
    u = gauge.stout(synth.random_su3_field(4, 2, seed=5), 0.1, 2, spatial_only=True)
    _, v = laplacian.lowest_eigpairs(u, 6)
    phi = laph.mom_overlaps(v, (0, 0, 0))
    assert np.abs(phi - np.eye(6)[None]).max() < 1e-12


@pytest.fixture(scope="module")
def free_shell(free_shell_6):
    return free_shell_6


@pytest.mark.parametrize("mom,pairs", [((0, 0, 0), 7), ((1, 0, 0), 2), ((0, 1, 1), 2), ((0, 0, 2), 1),
                                       ((1, 1, 1), 0)])
def test_free_field_overlap_closed_form(free_shell, mom, pairs):
    phi = laph.mom_overlaps(free_shell, mom)
    assert abs(np.sum(np.abs(phi) ** 2) - 3 * pairs) < 1e-9


@pytest.fixture(scope="module")
def shifted_pair():
    ns, nt, nv = 4, 2, 6
    u = gauge.stout(synth.random_su3_field(ns, nt, seed=17), 0.1, 2, spatial_only=True)
    ev, v = laplacian.lowest_eigpairs(u, nv)
    assert np.diff(ev, axis=1).min() > 1e-6          # non-degenerate: eigenvectors fixed up to phases
    shifted = {}
    for axis, name in ((3, "x"), (1, "z")):          # link layout [t, z, y, x, mu, 3, 3]
        ev2, v2 = laplacian.lowest_eigpairs(np.roll(u, 1, axis=axis), nv)   # U'(x) = U(x - a)
        assert np.abs(ev2 - ev).max() < 1e-10
        shifted[name] = v2
    return ns, v, shifted


@pytest.mark.parametrize("shift,mom", [("x", (1, 0, 0)), ("x", (0, 0, 1)), ("z", (0, 0, 1)), ("z", (1, 0, 0)),
                                       ("x", (2, 1, 0))])
def test_translation_phase(shifted_pair, shift, mom):
    ns, v, shifted = shifted_pair
    a = {"x": (1, 0, 0), "z": (0, 0, 1)}[shift]
    phi = laph.mom_overlaps(v, mom)
    phi2 = laph.mom_overlaps(shifted[shift], mom)
    factor = np.exp(-2j * np.pi * np.dot(mom, a) / ns)
    d, d2 = np.einsum("tnn->tn", phi), np.einsum("tnn->tn", phi2)
    assert np.abs(d2 - factor * d).max() < 1e-10
    assert np.abs(np.abs(phi2) - np.abs(phi)).max() < 1e-10
    assert np.abs(d).max() > 1e-2                     # the diagonal is not trivially zero


@pytest.fixture(scope="module")
def full(exact_4x4):
    return exact_4x4


@pytest.mark.parametrize("channel", ["pion", "rho", "scalar"])
@pytest.mark.parametrize("mom", [(1, 0, 0), (0, 1, 1), (1, 1, 1)])
def test_full_dilution_momentum_meson_equals_exact(full, channel, mom):
    path, G = full
    t0 = 1
    bs = path.projectors_for_time(t0)
    l1, _ = path.line(0, bs, method="lu")
    l2, _ = path.line(1, bs, method="lu")
    c_st = laph.meson_connected(l1, l2, t0, channel, mom)
    c_ex = laph.exact_meson_connected(G, t0, channel, laph.mom_overlaps(path.evecs, mom))
    assert np.abs(c_st - c_ex).max() < 1e-10 * np.abs(c_ex).max()
    # the phase changes the correlator: it is not the zero-momentum one
    c0 = laph.exact_meson_connected(G, t0, channel)
    assert np.abs(c_ex - c0).max() > 1e-3 * np.abs(c0).max()


@pytest.mark.parametrize("channel", ["pion", "rho", "scalar"])
def test_opposite_momentum_is_conjugate(full, channel):
    path, G = full
    for mom in ((1, 0, 0), (0, 1, 1)):
        neg = tuple(-m for m in mom)
        cp = laph.exact_meson_connected(G, 2, channel, laph.mom_overlaps(path.evecs, mom))
        cm = laph.exact_meson_connected(G, 2, channel, laph.mom_overlaps(path.evecs, neg))
        assert np.abs(cm - np.conj(cp)).max() < 1e-10 * np.abs(cp).max()
        assert np.abs(cp.imag).max() > 1e-6 * np.abs(cp).max()    # complex at p != 0: the relation bites
