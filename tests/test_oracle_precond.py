"""Pins of the oracle's learned-preconditioner arithmetic: the analytic
gradients against central finite differences of the loss, the layer adjoint
against <y, F x> = <F^dag y, x>, and gauge covariance N(G psi; U^G) = G N(psi; U)."""
import numpy as np

import synth
from oracle import gauge, precond


def _setup(ns=2, nt=4, seed=3):
    u = gauge.stout(synth.random_su3_field(ns, nt, seed=seed), 0.1, 1, spatial_only=False)
    ws = precond.init_weights(seed=5, diag=2.0, nchan=2, nlayers=3, scale=0.3)
    return u, ws


def test_layer_adjoint():
    u, ws = _setup()
    w = ws[1]
    x = synth.random_complex((w.shape[2], 4, 2, 2, 2, 4, 3), 1)
    y = synth.random_complex((w.shape[1], 4, 2, 2, 2, 4, 3), 2)
    lhs = np.vdot(y, precond.layer(u, w, x))
    rhs = np.vdot(precond.layer_adjoint(u, w, y), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_gradients_match_finite_differences():
    u, ws = _setup()
    rhos = [synth.random_complex((4, 2, 2, 2, 4, 3), 10 + i) for i in range(2)]
    phis = [synth.random_complex((4, 2, 2, 2, 4, 3), 20 + i) for i in range(2)]
    loss, grads = precond.loss_and_grads(u, ws, rhos, phis)
    rng = np.random.default_rng(0)
    h = 1e-6
    for l in range(len(ws)):
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in ws[l].shape)
            for part, unit in (("re", 1.0), ("im", 1j)):
                wp = [w.copy() for w in ws]
                wm = [w.copy() for w in ws]
                wp[l][idx] += h * unit
                wm[l][idx] -= h * unit
                fd = (precond.loss_and_grads(u, wp, rhos, phis)[0] - precond.loss_and_grads(u, wm, rhos, phis)[0]) / (2 * h)
                g = grads[l][idx]
                an = 2 * g.real if part == "re" else 2 * g.imag
                assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (l, idx, part, fd, an)


def test_network_gauge_covariance():
    u, ws = _setup()
    g = synth.random_gauge_transform(2, 4, seed=9)
    ug = gauge.gauge_transform_links(u, g)
    psi = synth.random_spinor(2, 4, seed=4)
    gpsi = np.einsum("tzyxab,tzyxsb->tzyxsa", g, psi)
    lhs = precond.apply(ug, ws, gpsi)
    rhs = np.einsum("tzyxab,tzyxsb->tzyxsa", g, precond.apply(u, ws, psi))
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


def test_pack_roundtrip_and_shapes():
    ws = precond.init_weights(seed=1, diag=2.0)
    flat = precond.pack(ws)
    assert flat.size == 9 * 16 * (4 + 16 + 16 + 4)
    inter = np.empty(2 * flat.size)
    inter[0::2], inter[1::2] = flat.real, flat.imag
    for a, b in zip(ws, precond.unpack(inter)):
        assert np.array_equal(a, b)


def _unit_links(ns, nt):
    u = np.zeros((nt, ns, ns, ns, 4, 3, 3), dtype=complex)
    u[...] = np.eye(3)
    return u


def test_free_field_transport_is_a_shift():
    """Closed form at U = 1: a one-layer network whose only weight is W[1+mu] = 1 moves
    the field by one site, psi(x+mu), with the antiperiodic sign on the time wrap;
    W[5+mu] = 1 moves it the other way.  Checked against np.roll."""
    ns, nt = 2, 4
    u = _unit_links(ns, nt)
    psi = synth.random_spinor(ns, nt, seed=8)
    axis = {0: 3, 1: 2, 2: 1, 3: 0}            # field axes t, z, y, x
    for mu in range(4):
        for d, step in ((1 + mu, -1), (5 + mu, 1)):
            w = np.zeros((9, 1, 1, 4, 4), dtype=complex)
            w[d, 0, 0] = np.eye(4)
            got = precond.apply(u, [w], psi)
            ref = np.roll(psi, step, axis=axis[mu])
            if mu == 3:                       # hops across the time boundary flip sign
                if step == -1:
                    ref[-1] *= -1.0
                else:
                    ref[0] *= -1.0
            assert np.abs(got - ref).max() < 1e-14, (mu, d)


def test_scaled_identity_network():
    """Only W[0] nonzero, alpha_l times the identity in each layer: the network is the
    product of the alphas times the identity, channels and layers notwithstanding."""
    u, _ = _setup()
    alphas = [0.5 + 0.25j, -1.5, 2.0j]
    ws = []
    for l, shp in enumerate(precond.layer_shapes(1, 3)):
        w = np.zeros(shp, dtype=complex)
        w[0, 0, 0] = alphas[l] * np.eye(4)
        ws.append(w)
    psi = synth.random_spinor(2, 4, seed=12)
    got = precond.apply(u, ws, psi)
    assert np.abs(got - np.prod(alphas) * psi).max() < 1e-14
