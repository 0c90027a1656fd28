"""The oracle's windowed smearing against its full-lattice smearing.

Large lattices (24^3 x 128) are too big for the oracle to smear whole inside a test; its
checks there use prepare_links_window, which smears only the slices around the one checked.
These pins show on a small lattice that the window's central slices equal the full
smearing's, and that one time slice of K x built on a three-slice piece of the window equals
that slice of K x on the full lattice (the stencil and the clover leaves reach one slice
forward and back)."""
import numpy as np

import synth
from oracle import gauge
from oracle.dirac import WilsonClover
from oracle.fast import FastK


def test_window_smearing_equals_full_on_central_slices():
    ns, nt, t0, halo = 4, 24, 13, 11
    u0 = synth.random_su3_field(ns, nt, seed=77)
    u, ut = gauge.prepare_links(u0, 0.1, 10, 2)
    uw, utw = gauge.prepare_links_window(u0, t0, halo, 0.1, 10, 2)
    for k in (-1, 0, 1):
        assert np.abs(uw[halo + k] - u[t0 + k]).max() < 1e-13
        assert np.abs(utw[halo + k] - ut[t0 + k]).max() < 1e-13
    # the slice next to the exact range is not exact: the window really is closed on itself (the
    # error is small there because each step passes on only a fraction rho of it)
    assert np.abs(uw[halo - 2] - u[t0 - 2]).max() > 1e-11


def test_window_smearing_wraps_the_lattice():
    ns, nt, halo = 4, 24, 11
    u0 = synth.random_su3_field(ns, nt, seed=78)
    u, _ = gauge.prepare_links(u0, 0.1, 10, 2)
    uw, _ = gauge.prepare_links_window(u0, 1, halo, 0.1, 10, 2)     # slices 14 .. 23, 0 .. 12
    for k in (-1, 0, 1):
        assert np.abs(uw[halo + k] - u[(1 + k) % nt]).max() < 1e-13


def test_three_slice_row_of_K():
    ns, nt, t0, halo, m0, csw, xi = 4, 24, 9, 11, -0.05, 1.0, 3.5
    u0 = synth.random_su3_field(ns, nt, seed=79)
    u, _ = gauge.prepare_links(u0, 0.1, 10, 2)
    uw, _ = gauge.prepare_links_window(u0, t0, halo, 0.1, 10, 2)
    x = synth.random_spinor(ns, nt, seed=80)
    full = FastK(WilsonClover(u, m0, csw, xi)).apply(x)[t0]
    piece = FastK(WilsonClover(np.ascontiguousarray(uw[halo - 1:halo + 2]), m0, csw, xi))
    row = piece.apply(np.ascontiguousarray(x[t0 - 1:t0 + 2]))[1]
    assert np.abs(row - full).max() < 1e-12 * np.abs(full).max()
