"""Gauge-covariant displacements of LapH-smeared quark fields (test infrastructure).

Sec. II writes every quark line as Q = D^(j) S Omega^{-1} S D^(k)dag, and Eq. (quarkdef)
builds hadrons from q = D^(j) psi-tilde and qbar = psi-tilde-bar gamma_4 D^(j)dag: a
displacement of type j carries a field along a path of spatial links (the paper's are
typically three links in one direction, or several directions combined):
    (D psi)(x) = U_{s_1}(x) U_{s_2}(x + s_1) ... U_{s_L}(x + s_1 + ... + s_{L-1}) psi(x + s_1 + ... + s_L),
where a backward step uses U_{-mu}(y) = U_mu(y - mu)^dag.  A path is a tuple of signed
directions: +-1, +-2, +-3 for +-x, +-y, +-z.  The empty path is no displacement.

Sec. III, Eq. (mesonfunc): with displacements d_j (of qbar) and d_k (of q) the phase of
the meson function is e^{-i p.(x + (d_j + d_k)/2)}.  In LapH coordinates this becomes the
displaced overlap matrix
    Phi_{p,jk}(t)[n, n'] = sum_{x,c} conj((D^(j) V_n)(x, c)) e^{-i p.(x + (d_j + d_k)/2)} (D^(k) V_n')(x, c),
which is Phi_p of the undisplaced meson function when both paths are empty.  The source
partner of a displaced bilinear (c, p, j, k) is c*, -p with the roles of the paths
exchanged, i.e. Phi_{-p,kj} (qbar displaced by d_k, q by d_j).
"""
import numpy as np

from .lattice import bwd, fwd
from .laph import mom_phase


def step(ut: np.ndarray, psi: np.ndarray, s: int) -> np.ndarray:
    """One covariant link step.  ut [t,z,y,x,4,3,3]; psi [..., t,z,y,x,3].
    s = +mu: U_mu(x) psi(x + mu);  s = -mu: U_mu(x - mu)^dag psi(x - mu)  (mu = 1, 2, 3 for x, y, z)."""
    mu = abs(s) - 1
    lead = psi.ndim - 5
    u = ut[..., mu, :, :]
    if s > 0:
        return np.einsum("tzyxab,...tzyxb->...tzyxa", u, fwd(psi, mu, lead))
    return bwd(np.einsum("tzyxba,...tzyxb->...tzyxa", np.conj(u), psi), mu, lead)


def displace(ut: np.ndarray, psi: np.ndarray, path) -> np.ndarray:
    """(D psi)(x) for the path (s_1, ..., s_L): the step nearest the field acts first."""
    for s in reversed(tuple(path)):
        psi = step(ut, psi, s)
    return psi


def net_displacement(path) -> np.ndarray:
    """Net displacement vector (d_x, d_y, d_z) of a path, in lattice units."""
    d = np.zeros(3, dtype=int)
    for s in path:
        d[abs(s) - 1] += 1 if s > 0 else -1
    return d


def adjoint_path(path):
    """D^dag of a path is the reversed path with every step negated."""
    return tuple(-s for s in reversed(tuple(path)))


def evecs_as_fields(evecs: np.ndarray) -> np.ndarray:
    """[nt][nv][V3][3] -> [nv, t, z, y, x, 3]."""
    nt, nv, v3, _ = evecs.shape
    ns = round(v3 ** (1.0 / 3.0))
    return np.transpose(evecs.reshape(nt, nv, ns, ns, ns, 3), (1, 0, 2, 3, 4, 5))


def displaced_overlaps(ut: np.ndarray, evecs: np.ndarray, mom, path_bar, path) -> np.ndarray:
    """Phi_{p,jk}(t)[n, n'] for qbar displaced along path_bar (j) and q along path (k), [nt][nv][nv]."""
    nt, nv, v3, _ = evecs.shape
    ns = round(v3 ** (1.0 / 3.0))
    v = evecs_as_fields(evecs)
    dj = displace(ut, v, path_bar).reshape(nv, nt, v3, 3)
    dk = displace(ut, v, path).reshape(nv, nt, v3, 3)
    ph = mom_phase(ns, mom)
    half = np.exp(-1j * np.pi * np.dot(np.asarray(mom), net_displacement(path_bar) + net_displacement(path)) / ns)
    return half * np.einsum("ntxc,x,mtxc->tnm", np.conj(dj), ph, dk)


def exact_meson_connected_displaced(G: np.ndarray, t0: int, c: np.ndarray, phi_snk: np.ndarray,
                                    phi_src: np.ndarray) -> np.ndarray:
    """Connected meson correlator of one displaced elemental (spin matrix c) from the exact
    G, dt-indexed: phi_snk = Phi_{p,jk}, phi_src = Phi_{-p,kj} (the source partner);
        C(t_F) = - sum c_{ab} c*_{a'b'} phi_snk(t_F)[n, n'] phi_src(t_0)[m, m']
                   G[t_F b n'; t_0 b' m] G[t_0 a' m'; t_F a n]."""
    nt = G.shape[0]
    out = np.zeros(nt, dtype=complex)
    for tf in range(nt):
        out[(tf - t0) % nt] = -np.einsum("ab,pq,nN,mM,bNqm,pMan->", c, np.conj(c), phi_snk[tf], phi_src[t0],
                                         G[tf, :, :, t0, :, :], G[t0, :, :, tf, :, :])
    return out


def displace_spinor(ut: np.ndarray, f: np.ndarray, path) -> np.ndarray:
    """D acting on colour of a spinor field [..., t,z,y,x,4,3] (spin untouched)."""
    g = np.moveaxis(f, -2, 0)
    return np.moveaxis(displace(ut, g, path), 0, -2)


def meson_functions_displaced(ut, a_list, b_list, c, mom, path_bar, path) -> np.ndarray:
    """Eq. (mesonfunc) with displacements, site space:
    M[b1, b2, t] = sum_x e^{-i p.(x + (d_j + d_k)/2)} sum_{alpha beta} conj((D^(j) a^[b1])_alpha(x,t)) c_{alpha beta} (D^(k) b^[b2])_beta(x,t)."""
    nb1, nt, ns = a_list.shape[0], a_list.shape[1], a_list.shape[2]
    a = displace_spinor(ut, a_list, path_bar).reshape(nb1, nt, -1, 4, 3)
    b = displace_spinor(ut, b_list, path).reshape(b_list.shape[0], nt, -1, 4, 3)
    half = np.exp(-1j * np.pi * np.dot(np.asarray(mom), net_displacement(path_bar) + net_displacement(path)) / ns)
    cb = np.einsum("ab,ntxbc->ntxac", c, b) * mom_phase(ns, mom)[None, None, :, None, None]
    return half * np.einsum("ptxac,qtxac->pqt", np.conj(a), cb)


def meson_connected_displaced(ut, line1, line2, t0: int, c: np.ndarray, mom, path_bar, path) -> np.ndarray:
    """First term of Eq. (mesoncorr) for one displaced elemental (c, p, j, k), dt-indexed: the
    sink function M_l(phibar_1, phi_2; t_F) and the source function M_l(rhobar_1, rho_2; t_0),
    conjugated, with the same (c, p, j, k)."""
    nt = line1.varrho.shape[1]
    msink = meson_functions_displaced(ut, line1.varphi_bar, line2.varphi, c, mom, path_bar, path)
    msrc = meson_functions_displaced(ut, line1.varrho_bar, line2.varrho, c, mom, path_bar, path)[:, :, t0]
    ct = -np.einsum("pqt,pq->t", msink, np.conj(msrc))
    return np.roll(ct, -t0)
