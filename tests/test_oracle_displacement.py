"""Pins of the oracle's gauge-covariant displacements and displaced LapH overlaps
(Sec. II, the quark line D^(j) S Omega^{-1} S D^(k)dag; Eq. (quarkdef); the displaced
phase of Eq. (mesonfunc)).

* free field: a path is a plain shift of the field by its net displacement (np.roll on
  the numpy axis of each direction);
* gauge covariance D[U^g](g psi) = g D[U] psi; unitarity D^dag D = 1 with D^dag the
  reversed, negated path; adjointness <a, D b> = <D^dag a, b>;
* empty paths give the undisplaced overlaps Phi_p; displaced overlaps are gauge
  invariant when the eigenvectors are carried along (V -> g V);
* free field closed form: on a 6^3 slice the lowest 21 eigenvectors span the plane waves
  of S = {0, +-e_x, +-e_y, +-e_z}, and a plane wave e^{ik.x} picks up e^{ik.d} under a
  shift by d, so tr Phi_{0,jk} = 3 sum_{k in S} e^{i k.(d_k - d_j)} (basis independent);
* free field, p != 0: with the half-displacement phase the overlaps depend only on the
  relative displacement d_k - d_j (which fixes that phase's sign);
* the step order of a path, written out site by site with explicit indices;
* fields inside the LapH subspace: the site-space displaced meson function equals the
  coefficient form with Phi_{p,jk};
* full dilution: the site-space stochastic displaced correlator equals the exact one from
  G and the displaced overlaps, which equals the brute-force Wick contraction of the
  displaced sink bilinear with its source partner (Phi_{-p,kj}).
"""
import numpy as np
import pytest

import synth
from oracle import displacement as dsp
from oracle import gauge, laph, laplacian, wick

PATHS = [(1, 1, 1), (-2,), (3, -1), (2, 2, -3)]


def unit_links(ns, nt):
    return np.broadcast_to(np.eye(3, dtype=complex), (nt, ns, ns, ns, 4, 3, 3)).copy()


def rand_field(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.fixture(scope="module")
def links():
    return gauge.stout(synth.random_su3_field(4, 2, seed=23), 0.1, 1, spatial_only=True)


@pytest.mark.parametrize("path", PATHS)
def test_free_field_is_a_shift(path):
    ns, nt = 4, 2
    psi = rand_field((2, nt, ns, ns, ns, 3), 1)
    d = dsp.net_displacement(path)
    ref = psi
    for mu in range(3):                                  # psi(x + d): roll by -d on axis of mu
        ref = np.roll(ref, -d[mu], axis=1 + 3 - mu)
    assert np.abs(dsp.displace(unit_links(ns, nt), psi, path) - ref).max() < 1e-14


@pytest.mark.parametrize("path", PATHS)
def test_gauge_covariance_unitarity_adjoint(links, path):
    ns, nt = 4, 2
    psi = rand_field((nt, ns, ns, ns, 3), 2)
    chi = rand_field((nt, ns, ns, ns, 3), 3)
    g = synth.random_gauge_transform(ns, nt, seed=5)
    ug = gauge.gauge_transform_links(links, g)
    gpsi = np.einsum("tzyxab,tzyxb->tzyxa", g, psi)
    lhs = dsp.displace(ug, gpsi, path)
    rhs = np.einsum("tzyxab,tzyxb->tzyxa", g, dsp.displace(links, psi, path))
    assert np.abs(lhs - rhs).max() < 1e-12
    back = dsp.displace(links, dsp.displace(links, psi, path), dsp.adjoint_path(path))
    assert np.abs(back - psi).max() < 1e-12
    a = np.vdot(chi, dsp.displace(links, psi, path))
    b = np.vdot(dsp.displace(links, chi, dsp.adjoint_path(path)), psi)
    assert abs(a - b) < 1e-10 * abs(a)


def test_empty_paths_and_gauge_invariance(links):
    _, v = laplacian.lowest_eigpairs(links, 5)
    for mom in [(0, 0, 0), (1, 0, 0), (0, 1, -1)]:
        assert np.abs(dsp.displaced_overlaps(links, v, mom, (), ()) - laph.mom_overlaps(v, mom)).max() < 1e-13
    g = synth.random_gauge_transform(4, 2, seed=8)
    ug = gauge.gauge_transform_links(links, g)
    vf = dsp.evecs_as_fields(v)
    vg = np.einsum("tzyxab,ntzyxb->ntzyxa", g, vf)
    vg = np.transpose(vg, (1, 0, 2, 3, 4, 5)).reshape(v.shape)
    for mom, pb, p in [((1, 0, 0), (1, 1, 1), ()), ((0, 0, 1), (-2,), (3, -1))]:
        a = dsp.displaced_overlaps(links, v, mom, pb, p)
        b = dsp.displaced_overlaps(ug, vg, mom, pb, p)
        assert np.abs(a - b).max() < 1e-12


@pytest.fixture(scope="module")
def free_shell(free_shell_6):
    return free_shell_6


@pytest.mark.parametrize("pb,p", [((), (1, 1, 1)), ((), (1,)), ((2,), (-2,)), ((3, 3), ()), ((1, 2), (1, 2))])
def test_free_field_displaced_trace(free_shell, pb, p):
    S = [np.zeros(3)] + [s * e for e in np.eye(3) for s in (1, -1)]
    dd = dsp.net_displacement(p) - dsp.net_displacement(pb)
    ref = 3 * sum(np.exp(2j * np.pi * np.dot(k, dd) / 6) for k in S)
    phi = dsp.displaced_overlaps(unit_links(6, 1), free_shell, (0, 0, 0), pb, p)
    assert abs(np.trace(phi[0]) - ref) < 1e-9


@pytest.fixture(scope="module")
def full(exact_4x4):
    return exact_4x4


@pytest.mark.parametrize("c_name", ["pion", "rho"])
@pytest.mark.parametrize("mom,pb,p", [((0, 0, 0), (1, 1, 1), ()), ((1, 0, 0), (), (-2, -2, -2)),
                                      ((0, 1, 0), (3,), (-1, 2))])
def test_displaced_correlator_stochastic_exact_wick(full, c_name, mom, pb, p):
    path, G = full
    ut, ev = path.ut, path.evecs
    nt, nv, t0 = path.wl.nt, path.wl.nv, 1
    c = laph.channel_c(c_name)[0]
    neg = tuple(-m for m in mom)
    phi_snk = dsp.displaced_overlaps(ut, ev, mom, pb, p)
    phi_src = dsp.displaced_overlaps(ut, ev, neg, p, pb)
    exact = dsp.exact_meson_connected_displaced(G, t0, c, phi_snk, phi_src)
    bs = path.projectors_for_time(t0)
    l1, _ = path.line(0, bs, method="lu")
    l2, _ = path.line(1, bs, method="lu")
    st = dsp.meson_connected_displaced(ut, l1, l2, t0, c, mom, pb, p)
    assert np.abs(st - exact).max() < 1e-10 * np.abs(exact).max()
    Q = G.reshape(nt * 4 * nv, nt * 4 * nv)
    for dt in range(nt):
        tf = (t0 + dt) % nt
        w = wick.correlator([(1.0, [wick.sink_bilinear(nt, nv, tf, c, phi_snk[tf], "d", "u")])],
                            [(1.0, [wick.source_bilinear(nt, nv, t0, c, phi_src[t0], "d", "u")])], Q)
        assert abs(w - exact[dt]) < 1e-10 * np.abs(exact).max()
    # the displacement matters
    und = laph.exact_meson_connected(G, t0, c_name, None if mom == (0, 0, 0) else laph.mom_overlaps(ev, mom))
    if c_name == "pion":
        assert np.abs(exact - und).max() > 1e-3 * np.abs(und).max()


def test_path_order_pointwise(links):
    """(D psi)(x) = U_z(x) U_x(x + z - x)^dag psi(x + z - x) for the path (+z, -x), written
    out site by site with explicit indices (layout [t, z, y, x])."""
    ns = 4
    psi = rand_field((2, ns, ns, ns, 3), 6)
    got = dsp.displace(links, psi, (3, -1))
    for (t, z, y, x) in [(0, 0, 0, 0), (1, 3, 2, 1), (0, 2, 3, 3), (1, 1, 0, 2)]:
        z1, x1 = (z + 1) % ns, (x - 1) % ns                 # x + z_hat - x_hat
        u_z = links[t, z, y, x, 2]
        u_x_dag = np.conj(links[t, z1, y, x1, 0]).T         # U_{-x}(x + z_hat) = U_x(x + z_hat - x_hat)^dag
        ref = u_z @ u_x_dag @ psi[t, z1, y, x1]
        assert np.abs(got[t, z, y, x] - ref).max() < 1e-13


@pytest.mark.parametrize("mom", [(1, 0, 0), (1, 1, 0), (0, 1, 1)])
def test_free_field_depends_on_relative_displacement(free_shell, mom):
    """Free field: D is a shift, and with the half-displacement phase of Eq. (mesonfunc) the
    overlap depends only on d_k - d_j: substituting y = x + d_j leaves
    e^{-i p.(d_k - d_j)/2} sum_y V_n(y)^* e^{-i p.y} V_n'(y + d_k - d_j)."""
    u = unit_links(6, 1)
    a = dsp.displaced_overlaps(u, free_shell, mom, (), (1,))
    b = dsp.displaced_overlaps(u, free_shell, mom, (-1,), ())
    c = dsp.displaced_overlaps(u, free_shell, mom, (2, 3), (2, 3, 1))
    assert np.abs(a).max() > 1e-3
    assert np.abs(a - b).max() < 1e-12 and np.abs(a - c).max() < 1e-12


def test_site_space_function_matches_overlaps(full):
    """Fields in the LapH subspace, a = V alpha and b = V beta: the site-space displaced meson
    function equals sum conj(alpha) c Phi_{p,jk} beta (half-displacement phase included)."""
    path, _ = full
    ut, ev = path.ut, path.evecs
    nt, nv = path.wl.nt, path.wl.nv
    rng = np.random.default_rng(12)
    alpha = rng.standard_normal((2, nt, 4, nv)) + 1j * rng.standard_normal((2, nt, 4, nv))
    beta = rng.standard_normal((3, nt, 4, nv)) + 1j * rng.standard_normal((3, nt, 4, nv))
    a = np.stack([laph.lapH_to_site(ev, x) for x in alpha])
    b = np.stack([laph.lapH_to_site(ev, x) for x in beta])
    c = laph.channel_c("pion")[0]
    for mom, pb, p in [((1, 0, 0), (1,), ()), ((0, 1, 1), (2, 3), (-1,))]:
        site = dsp.meson_functions_displaced(ut, a, b, c, mom, pb, p)
        phi = dsp.displaced_overlaps(ut, ev, mom, pb, p)
        coef = np.einsum("ptan,ab,tnm,qtbm->pqt", np.conj(alpha), c, phi, beta)
        assert np.abs(site - coef).max() < 1e-12 * np.abs(coef).max()
