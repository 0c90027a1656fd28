"""Learned gauge-covariant preconditioner: forward pass, loss and gradients (FP64).

The paper has no learned component; the workload asks for a small
gauge-covariant network of parallel-transported nearest-neighbour layers with
learned spin-colour channel mixing, trained on (rho, phi) pairs of the plain
solver and used as a right preconditioner in flexible GCR.  Reading taken:

  layer:  out_c(x) = sum_{c'} sum_{d=0..8} W[d][c][c'] (T_d in_{c'})(x)
    T_0 psi(x)     = psi(x)
    T_{1+mu} psi(x) = s U_mu(x) psi(x+mu)            (forward transport)
    T_{5+mu} psi(x) = s U_mu(x-mu)^dag psi(x-mu)     (backward transport)
    s = -1 for a hop across the time boundary (the fermion's antiperiodic
    condition, as in K), else +1;
    W[d][c][c'] a 4x4 complex matrix on spin, the identity on colour.  A
    general 12x12 spin-colour matrix would not commute with gauge
    transformations; colour enters only through the links, so
    N(G psi; U^G) = G N(psi; U).
  network: channels 1 -> C -> ... -> C -> 1 over L layers (C = 4, L = 4),
    linear (no nonlinearity), so N is a fixed linear operator.
  loss over a batch:  (1/B) sum_i ||N(rho_i) - phi_i||^2 / ||phi_i||^2.
Gradients are Wirtinger derivatives dL/d conj(W); the real gradient of Re W
is 2 Re(dL/d conj W) and of Im W is 2 Im(dL/d conj W).  The adjoint of a layer
swaps forward and backward transports and uses W^dag.

Weight layout (shared with the CUDA path through its specification only):
layers in order, each [9][c_out][c_in][4][4] complex.
"""
import numpy as np

from .lattice import fwd, bwd


def layer_shapes(nchan=4, nlayers=4):
    shapes = []
    for l in range(nlayers):
        cin = 1 if l == 0 else nchan
        cout = 1 if l == nlayers - 1 else nchan
        shapes.append((9, cout, cin, 4, 4))
    return shapes


def unpack(flat, nchan=4, nlayers=4):
    """Complex weight arrays from the flat layout (complex128 or interleaved reals)."""
    flat = np.asarray(flat)
    if not np.iscomplexobj(flat):
        flat = flat[0::2] + 1j * flat[1::2]
    out, o = [], 0
    for shp in layer_shapes(nchan, nlayers):
        n = int(np.prod(shp))
        out.append(flat[o:o + n].reshape(shp))
        o += n
    assert o == flat.size
    return out


def pack(ws):
    return np.concatenate([w.ravel() for w in ws])


def _sign_links(u):
    uf = u.copy()
    uf[-1, :, :, :, 3] *= -1.0
    return uf


def transport(u, psi, d):
    """T_d psi for a field psi[..., t, z, y, x, 4, 3] (u: gauge field)."""
    if d == 0:
        return psi
    lead = psi.ndim - 6
    uf = _sign_links(u)
    if d <= 4:
        mu = d - 1
        return np.einsum("tzyxab,...tzyxsb->...tzyxsa", uf[..., mu, :, :], fwd(psi, mu, lead))
    mu = d - 5
    return bwd(np.einsum("tzyxba,...tzyxsb->...tzyxsa", np.conj(uf[..., mu, :, :]), psi), mu, lead)


def layer(u, w, a):
    """out[c] = sum_{c', d} W[d][c][c'] T_d a[c'];  a: [c_in, ..., 4, 3]."""
    nd, cout, cin = w.shape[:3]
    out = np.zeros((cout,) + a.shape[1:], dtype=complex)
    for d in range(nd):
        for cp in range(cin):
            t = transport(u, a[cp], d)
            for c in range(cout):
                out[c] += np.einsum("ij,...jk->...ik", w[d, c, cp], t)
    return out


def layer_adjoint(u, w, g):
    """Adjoint of layer(): out[c'] = sum_{c, d} T_d^dag (W[d][c][c']^dag g[c])."""
    nd, cout, cin = w.shape[:3]
    adj = {0: 0, 1: 5, 2: 6, 3: 7, 4: 8, 5: 1, 6: 2, 7: 3, 8: 4}
    out = np.zeros((cin,) + g.shape[1:], dtype=complex)
    for d in range(nd):
        for c in range(cout):
            t = transport(u, g[c], adj[d])
            for cp in range(cin):
                out[cp] += np.einsum("ji,...jk->...ik", np.conj(w[d, c, cp]), t)
    return out


def forward(u, ws, r):
    """Activations [a_0 = r, a_1, ..., a_L] of the network on r[..., 4, 3]."""
    acts = [r[None]]
    for w in ws:
        acts.append(layer(u, w, acts[-1]))
    return acts


def apply(u, ws, r):
    return forward(u, ws, r)[-1][0]


def loss_and_grads(u, ws, rhos, phis):
    """Loss over pairs and dL/d conj(W) for every layer."""
    B = len(rhos)
    loss = 0.0
    grads = [np.zeros_like(w) for w in ws]
    for rho, phi in zip(rhos, phis):
        acts = forward(u, ws, rho)
        e = acts[-1][0] - phi
        nphi = np.vdot(phi, phi).real
        loss += np.vdot(e, e).real / nphi / B
        g = (e / (nphi * B))[None]         # dL/d conj(a_L)
        for l in range(len(ws) - 1, -1, -1):
            w, a = ws[l], acts[l]
            nd, cout, cin = w.shape[:3]
            for d in range(nd):
                for cp in range(cin):
                    t = transport(u, a[cp], d)
                    for c in range(cout):
                        grads[l][d, c, cp] += np.einsum("nsa,nta->st", g[c].reshape(-1, 4, 3),
                                                        np.conj(t).reshape(-1, 4, 3))
            g = layer_adjoint(u, w, g)
    return loss, grads


def init_weights(seed, diag, nchan=4, nlayers=4, scale=0.02):
    """Seeded start: the path through channel 0 is the identity scaled by 1/diag
    (a Jacobi-like first guess of K^{-1}); every other weight is small Gaussian."""
    rng = np.random.default_rng(seed)
    ws = []
    for l, shp in enumerate(layer_shapes(nchan, nlayers)):
        w = scale * (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) / np.sqrt(shp[0] * shp[2] * 4)
        w[0, 0, 0] += np.eye(4) * (1.0 / diag if l == nlayers - 1 else 1.0)
        ws.append(w)
    return ws
