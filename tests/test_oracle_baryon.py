"""Pins of the oracle's baryon functions and correlators (Sec. III: three-quark elemental
operators, Eq. (baryonfunc), Eq. (baryoncorr)).

* the signed six-term contraction of three quarks with three antiquarks (the Wick orderings
  of Eq. (baryoncorr)) equals a literal Gaussian Grassmann integral in the exterior algebra,
  for distinct, two equal and three equal flavours and for permuted source flavours;
* the LapH tensor T_p(t)[n1, n2, n3] = sum_x e^{-ip.x} eps_abc V_n1 V_n2 V_n3 is totally
  antisymmetric, gauge invariant when the eigenvectors are carried along (det g = 1), and in
  the free field on a 6^3 slice sum |T_p|^2 = 6 #{(k1, k2, k3) in S^3 : k1 + k2 + k3 = p} / V_3
  with S = {0, +-e_x, +-e_y, +-e_z};
* full dilution: the stochastic correlator of Eq. (baryoncorr) equals the exact three-quark
  contraction with G, at zero and nonzero momentum and for the flavour patterns uds, uud and
  uuu; the exact correlator is gauge invariant (fresh eigenvectors).
"""
import itertools

import numpy as np
import pytest

import synth
from oracle import baryon, gauge
from oracle.pipeline import OraclePath
from tests.grassmann import Grassmann, _add, _mul

@pytest.mark.parametrize("snk,src", [("uds", "uds"), ("uud", "uud"), ("uuu", "uuu"), ("udu", "uud"),
                                     ("uds", "sud"), ("uud", "dud")])
def test_three_quark_contraction_is_grassmann(snk, src):
    """Each flavour present gets its own block of n generators (n = 3 when a flavour occurs
    three times, so that the three-quark monomial does not vanish by the exclusion rule)."""
    flavours = sorted(set(snk + src))
    blk = {f: i for i, f in enumerate(flavours)}
    n = 3 if max(snk.count(f) for f in flavours) == 3 else 2
    rng = np.random.default_rng(len(snk) + 7 * sum(map(ord, snk + src)))
    A0 = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * np.eye(n)
    g = Grassmann(np.kron(np.eye(len(flavours)), A0))
    T = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    Tb = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    B, Bbar = {}, {}
    for i0, i1, i2 in itertools.product(range(n), repeat=3):
        # q^A_i0 q^B_i1 q^C_i2  and  qbar^Cbar_j2 qbar^Bbar_j1 qbar^Abar_j0 (the paper's order)
        mono = _mul(_mul(g.q(blk[snk[0]] * n + i0), g.q(blk[snk[1]] * n + i1)), g.q(blk[snk[2]] * n + i2))
        B = _add(B, mono, T[i0, i1, i2])
        monob = _mul(_mul(g.qbar(blk[src[2]] * n + i2), g.qbar(blk[src[1]] * n + i1)), g.qbar(blk[src[0]] * n + i0))
        Bbar = _add(Bbar, monob, Tb[i0, i1, i2])
    ref = g.expect(_mul(B, Bbar))
    got = baryon.three_quark_contraction(T, Tb, np.linalg.inv(A0), tuple(snk), tuple(src))
    assert abs(got - ref) < 1e-10 * max(1.0, abs(ref))
    if sorted(snk) == sorted(src):
        assert abs(ref) > 1e-6
    else:
        assert abs(ref) < 1e-12


def test_lapH_tensor_antisymmetric_and_gauge_invariant():
    u = gauge.stout(synth.random_su3_field(4, 2, seed=41), 0.1, 2, spatial_only=True)
    from oracle import laplacian
    _, v = laplacian.lowest_eigpairs(u, 5)
    for mom in (None, (1, 0, -1)):
        T = baryon.lapH_tensor(v, mom)
        assert np.abs(T + np.transpose(T, (0, 2, 1, 3))).max() < 1e-13
        assert np.abs(T + np.transpose(T, (0, 1, 3, 2))).max() < 1e-13
        assert np.abs(T).max() > 1e-3
    g = synth.random_gauge_transform(4, 2, seed=3)
    vf = np.transpose(v.reshape(2, 5, 4, 4, 4, 3), (1, 0, 2, 3, 4, 5))
    vg = np.einsum("tzyxab,ntzyxb->ntzyxa", g, vf)
    vg = np.transpose(vg, (1, 0, 2, 3, 4, 5)).reshape(v.shape)
    assert np.abs(baryon.lapH_tensor(vg, (0, 1, 0)) - baryon.lapH_tensor(v, (0, 1, 0))).max() < 1e-12


@pytest.mark.parametrize("mom", [(0, 0, 0), (1, 0, 0), (1, 1, 0), (2, 0, 0), (1, 1, 1)])
def test_lapH_tensor_free_field_count(free_shell_6, mom):
    S = [np.zeros(3, dtype=int)] + [s * e for e in np.eye(3, dtype=int) for s in (1, -1)]
    count = sum(1 for k1, k2, k3 in itertools.product(S, repeat=3)
                if np.all((k1 + k2 + k3 - np.array(mom)) % 6 == 0))
    T = baryon.lapH_tensor(free_shell_6, mom)
    assert abs(np.sum(np.abs(T) ** 2) - 6.0 * count / 216) < 1e-10


def _c_tensor(seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((4, 4, 4)) + 1j * rng.standard_normal((4, 4, 4))


@pytest.fixture(scope="module")
def lines3(exact_4x4):
    path, G = exact_4x4
    t0 = 2
    bs = path.projectors_for_time(t0)
    return t0, [path.line(20 + k, bs, method="lu")[0] for k in range(3)]


@pytest.mark.parametrize("flav", ["uds", "uud", "uuu"])
@pytest.mark.parametrize("mom", [None, (1, 0, 0)])
def test_full_dilution_baryon_equals_exact(exact_4x4, lines3, flav, mom):
    path, G = exact_4x4
    t0, (l1, l2, l3) = lines3
    c_snk, c_src = _c_tensor(1), _c_tensor(2)
    f = tuple(flav)
    st = baryon.baryon_correlator(l1, l2, l3, t0, c_snk, c_src, f, f, mom)
    ex = baryon.exact_baryon_correlator(G, path.evecs, t0, c_snk, c_src, f, f, mom)
    assert np.abs(ex).max() > 1e-8
    assert np.abs(st - ex).max() < 1e-10 * np.abs(ex).max()


def test_exact_baryon_gauge_invariant(exact_4x4):
    path, G = exact_4x4
    wl = path.wl
    g = synth.random_gauge_transform(wl.ns, wl.nt, seed=19)
    path_g = OraclePath(wl, u0=gauge.gauge_transform_links(wl.gauge(), g))
    c = _c_tensor(5)
    a = baryon.exact_baryon_correlator(G, path.evecs, 1, c, c, tuple("uud"), tuple("uud"))
    b = baryon.exact_baryon_correlator(path_g.exact_G(), path_g.evecs, 1, c, c, tuple("uud"), tuple("uud"))
    assert np.abs(a - b).max() < 1e-9 * np.abs(a).max()
