"""Baryon functions and correlators (test infrastructure).

Sec. III, three-quark elemental operators at momentum p (no displacement):
    Phi^{ABC}_{alpha beta gamma}(p, t) = sum_x e^{-i p.x} eps_{abc} q^A_{a alpha}(x,t) q^B_{b beta}(x,t) q^C_{c gamma}(x,t),
the source operator Phibar = sum_x e^{+i p.x} eps_{abc} qbar^C_{c gamma} qbar^B_{b beta} qbar^A_{a alpha},
a baryon B_l = c^(l)_{alpha beta gamma} Phi_{alpha beta gamma} and its source partner with c*.
Eq. (baryonfunc), the baryon function of three quark lines:
    B^[b1 b2 b3](f1, f2, f3; t) = c_{alpha beta gamma} sum_x e^{-i p.x} eps_{abc} f1^[b1]_{a alpha}(x,t) f2^[b2]_{b beta}(x,t) f3^[b3]_{c gamma}(x,t),
Eq. (baryoncorr), the correlator: the sink function of the sinks phi_1, phi_2, phi_3 times the
conjugate of a signed sum over the six orderings of the sources at t0,
    C(t_F - t_0) = sum_{b} B^[b1 b2 b3](phi_1, phi_2, phi_3; t_F)
                   conj( sum_pi sgn(pi) delta(flavours) B^[b_pi0 b_pi1 b_pi2](rho_pi0, rho_pi1, rho_pi2; t_0) ),
where source slot s takes line pi(s) and the delta requires the flavour of sink quark pi(s)
to equal the flavour of source slot s.  In LapH coordinates the spatial sum becomes the tensor
    T_p(t)[n1, n2, n3] = sum_x e^{-i p.x} eps_{abc} V_{n1}(x)_a V_{n2}(x)_b V_{n3}(x)_c,
antisymmetric in its three indices.
"""
import itertools

import numpy as np

from .laph import mom_phase

EPS = np.zeros((3, 3, 3))
for _a, _b, _c in itertools.permutations(range(3)):
    EPS[_a, _b, _c] = np.linalg.det(np.eye(3)[[_a, _b, _c]])

SLOT_PERMS = [p for p in itertools.permutations(range(3))]


def perm_sign(p):
    return int(round(np.linalg.det(np.eye(3)[list(p)])))


def baryon_functions(f1, f2, f3, c, mom=None) -> np.ndarray:
    """B[b1, b2, b3, t] of Eq. (baryonfunc) from site fields f_k [nb_k, t, z, y, x, 4, 3]; c [4][4][4].
    Contracted in three plain steps per site: the colour epsilon with the first two fields,
    the spin tensor with the third, then the remaining spin-colour sum and the phase-weighted
    sum over sites."""
    nt, ns = f1.shape[1], f1.shape[2]
    a = f1.reshape(f1.shape[0], nt, -1, 4, 3)
    b = f2.reshape(f2.shape[0], nt, -1, 4, 3)
    d = f3.reshape(f3.shape[0], nt, -1, 4, 3)
    ph = np.ones(ns ** 3) if mom is None else mom_phase(ns, mom)
    pair = np.einsum("abc,itxpa,jtxqb->txijpqc", EPS, a, b)             # eps_abc f1_a f2_b
    third = np.einsum("pqr,ktxrc->txkpqc", c, d)                        # c_pqr f3_rc
    nx = a.shape[2]
    ni, nj, nk = a.shape[0], b.shape[0], d.shape[0]
    per_site = np.matmul(pair.reshape(nt, nx, ni * nj, 48), third.reshape(nt, nx, nk, 48).transpose(0, 1, 3, 2))
    out = np.einsum("txm,x->mt", per_site.reshape(nt, nx, ni * nj * nk), ph)
    return out.reshape(ni, nj, nk, nt)


def baryon_correlator(line1, line2, line3, t0: int, c_snk, c_src, flav_snk, flav_src, mom=None) -> np.ndarray:
    """Eq. (baryoncorr) for one source time, dt-indexed; lines carry varphi (sinks) and varrho
    (sources) as site fields; flav_snk = (A, B, C), flav_src = (Abar, Bbar, Cbar)."""
    lines = (line1, line2, line3)
    nt = line1.varrho.shape[1]
    snk = baryon_functions(line1.varphi, line2.varphi, line3.varphi, c_snk, mom)      # [b1, b2, b3, t]
    src = np.zeros(snk.shape[:3], dtype=complex)
    for pi in SLOT_PERMS:
        if any(flav_snk[pi[s]] != flav_src[s] for s in range(3)):
            continue
        f = baryon_functions(lines[pi[0]].varrho, lines[pi[1]].varrho, lines[pi[2]].varrho, c_src, mom)[..., t0]
        # slot s carries the dilution index of line pi(s): relabel to [b1, b2, b3]
        src += perm_sign(pi) * np.einsum(f, list(pi), [0, 1, 2])
    ct = np.einsum("ijkt,ijk->t", snk, np.conj(src))
    return np.roll(ct, -t0)


def lapH_tensor(evecs: np.ndarray, mom=None) -> np.ndarray:
    """T_p(t)[n1, n2, n3] = sum_x e^{-i p.x} eps_{abc} V_{n1}(x)_a V_{n2}(x)_b V_{n3}(x)_c, [nt][nv][nv][nv]."""
    nt, nv, v3, _ = evecs.shape
    ph = np.ones(v3) if mom is None else mom_phase(round(v3 ** (1.0 / 3.0)), mom)
    return np.stack([np.einsum("abc,x,ixa,jxb,kxc->ijk", EPS, ph, evecs[t], evecs[t], evecs[t], optimize=True)
                     for t in range(nt)])


def three_quark_contraction(T, Tbar, Q, flav_snk, flav_src) -> complex:
    """< (sum T[i0 i1 i2] q^A_i0 q^B_i1 q^C_i2) (sum Tbar[j0 j1 j2] qbar^Cbar_j2 qbar^Bbar_j1 qbar^Abar_j0) >
    with <q_i qbar_j> = Q[i, j] per flavour: sum over the slot permutations pi of
    sgn(pi) [flavour of q_pi(s) = flavour of slot s] sum T Tbar prod_s Q[i_pi(s), j_s]."""
    out = 0.0 + 0.0j
    for pi in SLOT_PERMS:
        if any(flav_snk[pi[s]] != flav_src[s] for s in range(3)):
            continue
        # prod_s Q[i_{pi(s)}, j_s]: einsum labels i0 i1 i2 = 0 1 2, j0 j1 j2 = 3 4 5
        ops = [T, [0, 1, 2], Tbar, [3, 4, 5]]
        for s in range(3):
            ops += [Q, [pi[s], 3 + s]]
        out += perm_sign(pi) * np.einsum(*ops, [], optimize=True)
    return out


def exact_baryon_correlator(G, evecs, t0: int, c_snk, c_src, flav_snk, flav_src, mom=None) -> np.ndarray:
    """Full-dilution limit of baryon_correlator from the exact G, dt-indexed: compound indices
    (spin, n), T = c (x) T_p(t_F), Tbar = conj(c_src) (x) conj(T_p(t0)), Q = G[t_F; t0]."""
    nt, nv = G.shape[0], G.shape[2]
    tp = lapH_tensor(evecs, mom)
    tbar = np.einsum("abc,ijk->aibjck", np.conj(c_src), np.conj(tp[t0])).reshape(4 * nv, 4 * nv, 4 * nv)
    out = np.zeros(nt, dtype=complex)
    for tf in range(nt):
        T = np.einsum("abc,ijk->aibjck", c_snk, tp[tf]).reshape(4 * nv, 4 * nv, 4 * nv)
        Q = G[tf, :, :, t0, :, :].reshape(4 * nv, 4 * nv)
        out[(tf - t0) % nt] = three_quark_contraction(T, tbar, Q, flav_snk, flav_src)
    return out
