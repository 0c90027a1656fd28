"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed
forms (free-field spectra and propagators), algebraic identities (Clifford
algebra, projector algebra, gamma_5-Hermiticity, gauge covariance), an
independent construction (sparse matrices built block by block against the
np.roll stencils), library routines (numpy eigh, scipy eigsh, LU), and the
published Philox4x32-10 known-answer vectors.
"""
import itertools
import json
import os

import numpy as np
import pytest

import synth
from oracle import dilution as dl
from oracle import gauge, laplacian, noise
from oracle.dirac import WilsonClover, bicgstab, hop_weights
from oracle.gamma import GAMMA, GAMMA5, sigma
from oracle.lattice import dag, mm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- gamma matrices
def test_clifford_and_hermiticity():
    for mu, nu in itertools.product(range(4), range(4)):
        anti = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
        assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4), atol=0)
    for g in GAMMA:
        assert np.allclose(g, g.conj().T, atol=0)
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]), atol=0)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            s = sigma(mu, nu)
            assert np.allclose(s, s.conj().T)
            assert np.allclose(s @ GAMMA5, GAMMA5 @ s)          # block diagonal in chirality


# ---------------------------------------------------------------- stout smearing
@pytest.fixture(scope="module")
def small_field():
    return synth.random_su3_field(4, 4, seed=7)


def test_stout_unitary_and_identity(small_field):
    u = small_field
    assert gauge.unitarity_defect(u) < 1e-13
    s = gauge.stout(u, 0.1, 3, spatial_only=False)
    assert gauge.unitarity_defect(s) < 1e-13
    assert np.abs(gauge.stout_step(u, 0.0, False) - u).max() < 1e-14          # rho = 0
    one = np.broadcast_to(np.eye(3), u.shape).astype(complex)
    assert np.abs(gauge.stout_step(one, 0.1, False) - one).max() < 1e-14      # U = 1 fixed point
    s3 = gauge.stout(u, 0.1, 2, spatial_only=True)
    assert np.array_equal(s3[..., 3, :, :], u[..., 3, :, :])                  # time links untouched
    assert gauge.mean_plaquette(s) > gauge.mean_plaquette(u)                   # smoothing raises <P>


def test_stout_gauge_covariance(small_field):
    u = small_field
    g = synth.random_gauge_transform(4, 4, seed=11)
    ug = gauge.gauge_transform_links(u, g)
    for spatial in (False, True):
        lhs = gauge.stout(ug, 0.1, 2, spatial)
        rhs = gauge.gauge_transform_links(gauge.stout(u, 0.1, 2, spatial), g)
        assert np.abs(lhs - rhs).max() < 1e-12


def test_stout_small_rho_expansion(small_field):
    """exp(iQ) U = U + i Q U + O(rho^2): first-order check of the Q formula."""
    u = small_field
    rho = 1e-6
    s = gauge.stout_step(u, rho, False)
    for mu in range(4):
        c = gauge.staple_sum(u, mu, range(4))
        om = mm(c, dag(u[..., mu, :, :]))
        # the traceless anti-Hermitian part of Omega is what Q keeps
        a = 0.5 * (om - dag(om))
        a = a - np.trace(a, axis1=-2, axis2=-1)[..., None, None] / 3.0 * np.eye(3)
        pred = u[..., mu, :, :] + rho * mm(a, u[..., mu, :, :])
        assert np.abs(s[..., mu, :, :] - pred).max() < 1e-10


def test_clover_field_strength(small_field):
    u = small_field
    one = np.broadcast_to(np.eye(3), u.shape).astype(complex)
    g = synth.random_gauge_transform(4, 4, seed=5)
    ug = gauge.gauge_transform_links(u, g)
    for mu, nu in [(0, 1), (0, 3), (1, 2), (2, 3)]:
        f = gauge.field_strength(u, mu, nu)
        assert np.abs(f - dag(f)).max() < 1e-14
        assert np.abs(np.trace(f, axis1=-2, axis2=-1)).max() < 1e-14
        assert np.abs(gauge.field_strength(one, mu, nu)).max() < 1e-15
        assert np.abs(gauge.field_strength(u, nu, mu) + f).max() < 1e-14     # antisymmetric
        assert np.abs(gauge.field_strength(ug, mu, nu) - mm(mm(g, f), dag(g))).max() < 1e-13


def test_clover_abelian_closed_form():
    """U_x = exp(i a y) (abelian, colour-diagonal): F_xy = sin(a) per leaf, traceless part."""
    ns, nt, a = 4, 4, 2 * np.pi / 4
    u = np.broadcast_to(np.eye(3), (nt, ns, ns, ns, 4, 3, 3)).astype(complex).copy()
    y = np.arange(ns)[None, None, :, None]
    h = np.diag([1.0, -1.0, 0.0])
    for yy in range(ns):
        u[:, :, yy, :, 0] = np.diag(np.exp(1j * a * yy * np.diag(h)))
    f = gauge.field_strength(u, 0, 1)
    # each plaquette = exp(-i a h) (the x link at y+1 is traversed backwards)
    expect = -np.sin(a) * h
    assert np.abs(f - expect).max() < 1e-14


@pytest.mark.parametrize("mu,nu", list(itertools.combinations(range(4), 2)))
def test_clover_plane_weight_spectrum(mu, nu):
    """The clover term's weight per plane, from the spectrum of the site matrix A(x).

    An abelian, colour-diagonal field confined to the (mu, nu) plane, U_mu(x) = exp(i a x_nu h)
    with h = diag(1, -1, 0), has F_{mu nu} = -sin(a) h on every site (the closed form of the test
    above, any plane) and F = 0 in the five other planes.  sigma_{mu nu} squares to 1 with
    eigenvalues +1, +1, -1, -1, so A = (m0 + sum_mu w_mu) - (c_sw/2) w_{mu nu} sigma_{mu nu} F_{mu nu}
    has eigenvalues c0 and c0 +- (c_sw/2) w_{mu nu} sin(a), four times each.  The weight is
    (1 + 1/xi)/2 for the planes with the time direction and 1/xi for the spatial ones: a swap
    of the two, or one weight for every plane, moves the spread and fails here."""
    from oracle.dirac import diag_matrix
    ns = nt = 4
    a, xi, m0, csw = 2 * np.pi / 4, 3.5, -0.07, 1.3
    u = np.broadcast_to(np.eye(3), (nt, ns, ns, ns, 4, 3, 3)).astype(complex).copy()
    h = np.array([1.0, -1.0, 0.0])
    axis = {0: 3, 1: 2, 2: 1, 3: 0}[nu]          # array axis of coordinate x_nu ([t, z, y, x])
    for c in range(ns):
        sl = [slice(None)] * 4
        sl[axis] = c
        u[tuple(sl) + (mu,)] = np.diag(np.exp(1j * a * c * h))
    A = diag_matrix(u, m0, csw, xi)
    c0 = m0 + 3.0 / xi + 1.0
    w = 0.5 * (1.0 + 1.0 / xi) if nu == 3 else 1.0 / xi
    d = 0.5 * csw * w * np.sin(a)
    expect = np.sort(np.repeat([c0 - d, c0, c0 + d], 4))
    for site in [(0, 0, 0, 0), (1, 2, 3, 0), (3, 1, 0, 2)]:
        ev = np.linalg.eigvalsh(A[site])
        assert np.abs(np.sort(ev) - expect).max() < 1e-13, (mu, nu, ev, expect)


# ---------------------------------------------------------------- Laplacian
def test_free_laplacian_spectrum():
    ns = 4
    one = np.broadcast_to(np.eye(3), (1, ns, ns, ns, 4, 3, 3)).astype(complex)
    w, _ = np.linalg.eigh(laplacian.slice_matrix(one, 0).toarray())
    n = np.arange(ns)
    lam = (4 * np.sin(np.pi * n / ns) ** 2)
    exact = np.sort((lam[:, None, None] + lam[None, :, None] + lam[None, None, :]).ravel().repeat(3))
    assert np.abs(np.sort(w) - exact).max() < 1e-13
    # plane waves are eigenvectors of the stencil apply
    z, yy, x = np.meshgrid(n, n, n, indexing="ij")
    p = 2 * np.pi * np.array([1, 2, 3]) / ns
    wave = np.exp(1j * (p[0] * x + p[1] * yy + p[2] * z))[None, :, :, :, None] * np.array([1.0, 0.5j, -2.0])
    got = laplacian.apply_mlap(one, wave)
    assert np.abs(got - np.sum(4 * np.sin(p / 2) ** 2) * wave).max() < 1e-13


def test_laplacian_stencil_vs_sparse_and_bounds():
    ns, nt = 4, 3
    ut = synth.random_su3_field(ns, nt, seed=3)
    psi = synth.random_complex((nt, ns, ns, ns, 3), seed=4)
    got = laplacian.apply_mlap(ut, psi)
    for t in range(nt):
        m = laplacian.slice_matrix(ut, t)
        assert np.abs(m @ psi[t].ravel() - got[t].ravel()).max() < 1e-13
        d = m.toarray()
        assert np.abs(d - d.conj().T).max() < 1e-15
        w = np.linalg.eigvalsh(d)
        assert w.min() > -1e-12 and w.max() < 12 + 1e-12


def test_eigpairs_dense_vs_eigsh_and_covariance():
    ns, nt, nv = 4, 2, 8
    ut = gauge.stout(synth.random_su3_field(ns, nt, seed=21), 0.1, 4, spatial_only=True)
    ed, vd = laplacian.lowest_eigpairs(ut, nv, "dense")
    es, vs = laplacian.lowest_eigpairs(ut, nv, "sparse")
    assert np.abs(ed - es).max() < 1e-12 * 12
    assert laplacian.eigenprojector_distance(vd, vs) < 1e-9
    # eigen-equation, orthonormality and the phase rule
    for t in range(nt):
        v = vd[t].reshape(nv, -1)
        assert np.abs(v.conj() @ v.T - np.eye(nv)).max() < 1e-12
        lv = laplacian.apply_mlap(ut[t:t + 1], vd[t][:, None].reshape(nv, 1, ns, ns, ns, 3)).reshape(nv, -1)
        assert np.abs(lv - ed[t][:, None] * v).max() < 1e-11
        j = np.argmax(np.abs(v), axis=1)
        big = v[np.arange(nv), j]
        assert np.abs(big.imag).max() < 1e-15 and big.real.min() > 0
    # gauge covariance: eigenvalues invariant, eigenvectors rotate by G
    g = synth.random_gauge_transform(ns, nt, seed=9)
    ug = gauge.gauge_transform_links(ut, g)
    eg, vg = laplacian.lowest_eigpairs(ug, nv, "dense")
    assert np.abs(eg - ed).max() < 1e-12
    vrot = np.einsum("tzyxab,tnzyxb->tnzyxa", g, vd.reshape(nt, nv, ns, ns, ns, 3)).reshape(vd.shape)
    assert laplacian.eigenprojector_distance(vg, vrot) < 1e-10


def test_chebyshev():
    th = np.linspace(0, np.pi, 17)
    for n in range(0, 9):
        assert np.abs(laplacian.chebyshev_T(n, np.cos(th)) - np.cos(n * th)).max() < 1e-13
    lam_c, lam_l = 0.5, 15.0
    assert abs(laplacian.chebyshev_map(lam_c, lam_c, lam_l) - 1.0) < 1e-15
    assert abs(laplacian.chebyshev_map(lam_l, lam_c, lam_l) + 1.0) < 1e-15
    # the lowest eigenvalue of -Delta becomes the largest of T_n(B)
    lam = np.array([0.01, 0.1, 0.3, 0.6, 5.0, 12.0])
    v = laplacian.chebyshev_T(8, laplacian.chebyshev_map(lam, lam_c, lam_l))
    assert np.all(np.diff(v[:3]) < 0) and np.all(np.abs(v[3:]) <= 1.0 + 1e-12)


# ---------------------------------------------------------------- noise
def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.json")) as f:
        kat = json.load(f)
    for case in kat["cases"]:
        c = [int(v, 16) for v in case["counter"]]
        k = [int(v, 16) for v in case["key"]]
        out = noise.philox4x32_10(*c, *k)
        assert [int(v) for v in out] == [int(v, 16) for v in case["output"]]


def test_z4_noise_golden_and_statistics():
    with open(os.path.join(GOLDEN, "z4_noise.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        codes = noise.z4_codes(case["nt"], case["nv"], case["noise_id"], case["config_id"])
        assert codes.ravel()[:64].tolist() == case["first64"]
    codes = noise.z4_codes(64, 64, 3, 1001)
    vals = noise.z4_values(codes).ravel()
    n = vals.size
    assert np.allclose(np.abs(vals), 1.0)
    assert abs(vals.mean()) < 5.0 / np.sqrt(n)
    assert abs(np.mean(vals * vals)) < 5.0 / np.sqrt(n)             # E(rho^2) = 0 for Z4
    assert abs(np.mean(vals[1:] * np.conj(vals[:-1]))) < 5.0 / np.sqrt(n)
    counts = np.bincount(codes.ravel(), minlength=4) / n
    assert np.abs(counts - 0.25).max() < 5.0 * np.sqrt(0.25 * 0.75 / n)


# ---------------------------------------------------------------- dilution
@pytest.mark.parametrize("kind,J,N", [(0, 0, 8), (1, 0, 8), (2, 2, 8), (2, 4, 8), (3, 2, 8), (3, 4, 8),
                                      (1, 0, 4), (3, 8, 32), (2, 16, 32), (3, 16, 128)])
def test_projector_algebra(kind, J, N):
    nb = dl.n_projectors(kind, J, N)
    ps = [np.diag(dl.projector_diag(kind, J, N, b)) for b in range(nb)]
    assert np.array_equal(sum(ps), np.eye(N))                                  # completeness
    for a, b in itertools.product(range(nb), range(nb)):
        assert np.array_equal(ps[a] @ ps[b], ps[a] if a == b else np.zeros((N, N)))   # orthogonality


def test_projector_definitions_and_errors():
    assert dl.projector_diag(2, 2, 8, 1).tolist() == [0, 0, 0, 0, 1, 1, 1, 1]
    assert dl.projector_diag(3, 2, 8, 1).tolist() == [0, 1, 0, 1, 0, 1, 0, 1]
    with pytest.raises(ValueError):
        dl.n_projectors(3, 3, 8)
    dil = ((1, 0), (1, 0), (3, 8))
    tot = sum(dl.full_projector_diag(dil, 4, 16, b) for b in range(4 * 4 * 8))
    assert np.array_equal(tot, np.ones((4, 4, 16)))


# ---------------------------------------------------------------- Dirac matrix
@pytest.fixture(scope="module")
def tiny_dirac():
    u = gauge.stout(synth.random_su3_field(4, 4, seed=17), 0.1, 2, spatial_only=False)
    return WilsonClover(u, m0=-0.05, csw=1.0, xi=3.5)


def test_dirac_stencil_vs_sparse(tiny_dirac):
    psi = synth.random_spinor(4, 4, seed=1)
    ks = tiny_dirac.sparse()
    assert np.abs(ks @ psi.ravel() - tiny_dirac.apply(psi).ravel()).max() < 1e-13


def test_dirac_gamma5_hermiticity(tiny_dirac):
    v = synth.random_spinor(4, 4, seed=2)
    w = synth.random_spinor(4, 4, seed=3)
    g5 = np.diag(GAMMA5)[:, None]
    lhs = np.vdot(v, g5 * tiny_dirac.apply(g5 * w))
    rhs = np.vdot(tiny_dirac.apply(v), w)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    a = tiny_dirac.a
    assert np.abs(a - np.conj(np.swapaxes(a, -1, -2))).max() < 1e-14        # clover Hermitian
    assert np.abs(a[..., :6, 6:]).max() < 1e-15                            # chiral blocks


def test_dirac_gauge_covariance(tiny_dirac):
    g = synth.random_gauge_transform(4, 4, seed=8)
    ug = gauge.gauge_transform_links(tiny_dirac.u, g)
    kg = WilsonClover(ug, tiny_dirac.m0, tiny_dirac.csw, tiny_dirac.xi)
    psi = synth.random_spinor(4, 4, seed=4)
    gpsi = np.einsum("tzyxab,tzyxsb->tzyxsa", g, psi)
    lhs = kg.apply(gpsi)
    rhs = np.einsum("tzyxab,tzyxsb->tzyxsa", g, tiny_dirac.apply(psi))
    assert np.abs(lhs - rhs).max() < 1e-12


def _plane_wave(ns, nt, n):
    p = np.array([2 * np.pi * n[0] / ns, 2 * np.pi * n[1] / ns, 2 * np.pi * n[2] / ns,
                  (2 * n[3] + 1) * np.pi / nt])                   # antiperiodic in time
    t, z, y, x = np.meshgrid(np.arange(nt), np.arange(ns), np.arange(ns), np.arange(ns), indexing="ij")
    return p, np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))


def test_free_wilson_momentum_space():
    ns, nt, xi, m0 = 4, 6, 3.5, 0.2
    one = np.broadcast_to(np.eye(3), (nt, ns, ns, ns, 4, 3, 3)).astype(complex)
    k = WilsonClover(one, m0=m0, csw=1.0, xi=xi)
    w = hop_weights(xi)
    rng = np.random.default_rng(0)
    for n in [(0, 0, 0, 0), (1, 2, 3, 1), (3, 1, 0, 4)]:
        p, ph = _plane_wave(ns, nt, n)
        spin_col = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = ph[..., None, None] * spin_col
        kp = (m0 + np.sum(w * (1 - np.cos(p)))) * np.eye(4) + 1j * sum(w[m] * GAMMA[m] * np.sin(p[m]) for m in range(4))
        assert np.abs(k.apply(psi) - ph[..., None, None] * (kp @ spin_col)).max() < 1e-13
        # free propagator closed form: K^{-1}(p) = [M(p) - i sum w g sin p] / [M^2 + sum w^2 sin^2 p]
        mp = m0 + np.sum(w * (1 - np.cos(p)))
        kinv = (mp * np.eye(4) - 1j * sum(w[m] * GAMMA[m] * np.sin(p[m]) for m in range(4))) / (mp ** 2 + np.sum((w * np.sin(p)) ** 2))
        x, it, rr = bicgstab(k.apply, psi, tol=1e-13)
        assert np.abs(x - ph[..., None, None] * (kinv @ spin_col)).max() < 1e-11


def test_bicgstab_vs_lu(tiny_dirac):
    import scipy.linalg
    b = synth.random_spinor(4, 4, seed=12)
    x, it, rr = bicgstab(tiny_dirac.apply, b, tol=1e-12)
    assert rr < 1e-12
    kd = tiny_dirac.sparse().toarray()
    xl = scipy.linalg.lu_solve(scipy.linalg.lu_factor(kd), b.ravel())
    assert np.linalg.norm(x.ravel() - xl) / np.linalg.norm(xl) < 1e-10


def test_threaded_oracle_solve_is_bit_identical():
    """The opt-in site-split threads of the plain-C operator change no arithmetic: one
    BiCGStab solve gives the same iterate bit for bit on 1 and 4 threads, and the same as
    the per-right-hand-side batch solver."""
    from oracle.fast import FastK
    from oracle.pipeline import OraclePath
    wl = synth.WORKLOADS["tiny_4x8"]
    fk = FastK(OraclePath(wl).K)
    b = synth.random_spinor(wl.ns, wl.nt, seed=99)
    x1, i1, r1 = fk.solve_split(b, tol=1e-10, maxiter=1000, nthreads=1)
    x4, i4, r4 = fk.solve_split(b, tol=1e-10, maxiter=1000, nthreads=4)
    xb, ib, rb = fk.solve(b, tol=1e-10, maxiter=1000, nthreads=1)
    assert i1 == i4 == ib and r1 == r4 == rb
    assert np.array_equal(x1, x4) and np.array_equal(x1, xb)


def test_inversion_counts_match_the_paper():
    """The oracle's projector counts reproduce the inversion counts the paper prints (Sec. II;
    fixture tests/golden/inversion_counts.json): projectors solved per noise are the
    time projectors containing a source time (or all of them) x spin x eigenvector ones."""
    here = os.path.dirname(os.path.abspath(__file__))
    data = json.load(open(os.path.join(here, "golden", "inversion_counts.json")))
    per = []
    for c in data["cases"]:
        if "total" in c:
            assert 5 * per[0] + 2 * per[1] == c["total"]
            continue
        nT, nS, nL = dl.counts(tuple(tuple(d) for d in c["dil"]), c["nt"], c["nv"])
        n_time = c["source_times"] if c["source_times"] else nT   # full time dilution at chosen t0 only
        n = n_time * nS * nL
        assert n == c["inversions"], c["what"]
        per.append(n)


def test_mt19937_known_value_and_z4_extraction():
    """The paper's generator (Sec. IV: Mersenne twister, two bits per Z4 element), oracle only:
    MT19937 against the value fixed by the C++ standard (tests/golden/mt19937.json) and against
    numpy's MT19937 bit generator with the same legacy seeding; Z4 codes take the two-bit
    fields of each word least significant first."""
    here = os.path.dirname(os.path.abspath(__file__))
    gold = json.load(open(os.path.join(here, "golden", "mt19937.json")))
    w = noise.mt19937_words(gold["seed"], gold["index"])
    assert int(w[-1]) == gold["value"]
    bg = np.random.MT19937()
    if hasattr(bg, "_legacy_seeding"):                 # numpy's init_genrand path
        bg._legacy_seeding(123456789)
        assert np.array_equal(noise.mt19937_words(123456789, 1300), bg.random_raw(1300).astype(np.uint64))
    codes = noise.z4_codes_mt(4, 8, 3, 7)
    words = noise.mt19937_words(noise.noise_seed(3, 7), 8)
    flat = codes.ravel()
    for idx in (0, 1, 15, 16, 77, 127):
        assert flat[idx] == (int(words[idx // 16]) >> (2 * (idx % 16))) & 3
    big = noise.z4_codes_mt(64, 64, 1, 1).ravel()
    counts = np.bincount(big, minlength=4)
    expected = big.size / 4
    assert np.sum((counts - expected) ** 2 / expected) < 20.0          # chi^2 with 3 dof, far tail
