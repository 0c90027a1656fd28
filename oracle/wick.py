"""Wick's theorem written out for products of quark bilinears in LapH coordinates.

Test infrastructure: the brute-force reference for the diagram bookkeeping of Sec. III
(meson functions joined by quark lines, Eq. (mesoncorr) and the two-meson figures).

A bilinear is B = sum_{i,j} M[i, j] qbar_f(i) q_g(j), with i, j compound (t, alpha, n)
indices of the whole LapH space (index (t * 4 + alpha) * N_v + n) and f, g flavour
labels.  With <q_g(j) qbar_f(i)> = delta_{fg} Q(j, i) and every bilinear Grassmann-even,
Gaussian Grassmann integration gives
    < B_1 ... B_m > = (-1)^m sum_{i, j} prod_k M_k[i_k, j_k] det[ Q(j_k, i_l) delta_{g_k f_l} ]_{k,l},
the (-1)^m from writing qbar q = -q qbar.  Expanding the determinant over permutations
sigma, each term factorises over the cycles of sigma:
    (-1)^m sgn(sigma) prod_{cycles (k, sigma k, sigma^2 k, ...)} tr(M_k Q M_{sigma k} Q ...),
and vanishes unless the flavour of q in B_k equals that of qbar in B_{sigma k} for every k.
Q is the LapH propagator V_s^dag Omega^{-1} V_s (degenerate flavours share it).

Operators follow the paper's conventions: the sink meson function of a bilinear
c_{alpha beta} qbar^A_alpha q^B_beta at momentum p carries e^{-i p.x} (Sec. III), which in
LapH coordinates is Phi_p(t) = V^dag e^{-i p.x} V between the colour-space indices; the
matching source operator is c*_{alpha beta} qbar^B_beta q^A_alpha with e^{+i p.x}, that is
Phi_{-p}.
"""
import itertools

import numpy as np


def lapH_index(nt, nv, t, alpha):
    """Slice of the compound indices (t, alpha, 0..nv-1)."""
    base = (t * 4 + alpha) * nv
    return slice(base, base + nv)


def sink_bilinear(nt, nv, t, c, phi_t, qbar_flavour, q_flavour):
    """sum_{alpha beta} c_{alpha beta} sum_{n n'} phi_t[n, n'] qbar(t, alpha, n) q(t, beta, n')."""
    m = np.zeros((nt * 4 * nv, nt * 4 * nv), dtype=complex)
    for a in range(4):
        for b in range(4):
            m[lapH_index(nt, nv, t, a), lapH_index(nt, nv, t, b)] = c[a, b] * phi_t
    return (m, qbar_flavour, q_flavour)


def source_bilinear(nt, nv, t, c, phi_minus_t, qbar_flavour_of_sink, q_flavour_of_sink):
    """Source partner of sink_bilinear(c, p, A, B): sum c*_{alpha beta} Phi_{-p}[n, n'] qbar^B(t, beta, n) q^A(t, alpha, n')."""
    m = np.zeros((nt * 4 * nv, nt * 4 * nv), dtype=complex)
    for a in range(4):
        for b in range(4):
            m[lapH_index(nt, nv, t, b), lapH_index(nt, nv, t, a)] = np.conj(c[a, b]) * phi_minus_t
    return (m, q_flavour_of_sink, qbar_flavour_of_sink)


def _cycles(perm):
    seen, out = set(), []
    for k in range(len(perm)):
        if k in seen:
            continue
        cyc, j = [], k
        while j not in seen:
            seen.add(j)
            cyc.append(j)
            j = perm[j]
        out.append(cyc)
    return out


def _sign(perm):
    return (-1) ** sum(len(c) - 1 for c in _cycles(perm))


def expect(bilinears, Q):
    """< B_1 ... B_m > by the permutation expansion above; bilinears = [(M, qbar_flavour, q_flavour)]."""
    m = len(bilinears)
    mq = [b[0] @ Q for b in bilinears]
    total = 0.0 + 0.0j
    for perm in itertools.permutations(range(m)):
        # q of B_k contracts with qbar of B_{perm[k]}
        if any(bilinears[k][2] != bilinears[perm[k]][1] for k in range(m)):
            continue
        term = 1.0 + 0.0j
        for cyc in _cycles(perm):
            prod = mq[cyc[0]]
            for k in cyc[1:]:
                prod = prod @ mq[k]
            term *= np.trace(prod)
        total += _sign(perm) * term
    return (-1) ** m * total


def correlator(sink_terms, source_terms, Q):
    """< O_sink O_source > for O = sum_r w_r prod(bilinears_r): sink_terms, source_terms are
    lists of (weight, [bilinears])."""
    out = 0.0 + 0.0j
    for ws, bs in sink_terms:
        for wr, br in source_terms:
            out += ws * wr * expect(list(bs) + list(br), Q)
    return out


# ---------------------------------------------------------------- pions and two-pion isospin states
# The bilinear qbar Gamma tau q transforms under isospin like tau in the adjoint; with
# tau_+ = E_ud as the top state, lowering gives the triplet
#     |1,+1> = u-bar d,   |1,0> = (d-bar d - u-bar u)/sqrt(2),   |1,-1> = -d-bar u,
# as (weight, (qbar flavour, q flavour)) lists.  Two-pion states couple these with the
# Clebsch-Gordan coefficients of 1 x 1; the first pion carries momentum p, the second -p
# (zero total momentum, the paper's two-pion operators of Sec. V).
_R2 = 1.0 / np.sqrt(2.0)
PION = {+1: [(1.0, ("u", "d"))], 0: [(-_R2, ("u", "u")), (_R2, ("d", "d"))], -1: [(-1.0, ("d", "u"))]}

CG_1x1 = {
    (2, 2): [(1.0, 1, 1)],
    (2, 1): [(_R2, 1, 0), (_R2, 0, 1)],
    (2, 0): [(1.0 / np.sqrt(6.0), 1, -1), (2.0 / np.sqrt(6.0), 0, 0), (1.0 / np.sqrt(6.0), -1, 1)],
    (1, 1): [(_R2, 1, 0), (-_R2, 0, 1)],
    (1, 0): [(_R2, 1, -1), (-_R2, -1, 1)],
    (0, 0): [(1.0 / np.sqrt(3.0), 1, -1), (-1.0 / np.sqrt(3.0), 0, 0), (1.0 / np.sqrt(3.0), -1, 1)],
}


def two_pion_sink(nt, nv, t, c, phi_p_t, phi_mp_t, iso):
    """Sink operator sum_CG w pi_{m1}(p, t) pi_{m2}(-p, t) as (weight, [B1, B2]) terms."""
    out = []
    for w, m1, m2 in CG_1x1[iso]:
        for w1, (fb1, f1) in PION[m1]:
            for w2, (fb2, f2) in PION[m2]:
                out.append((w * w1 * w2, [sink_bilinear(nt, nv, t, c, phi_p_t, fb1, f1),
                                          sink_bilinear(nt, nv, t, c, phi_mp_t, fb2, f2)]))
    return out


def two_pion_source(nt, nv, t, c, phi_p_t, phi_mp_t, iso):
    """Source partner of two_pion_sink: every bilinear replaced by its source partner
    (Phi_{-p} for the pion of momentum p) and every weight conjugated."""
    out = []
    for w, m1, m2 in CG_1x1[iso]:
        for w1, (fb1, f1) in PION[m1]:
            for w2, (fb2, f2) in PION[m2]:
                out.append((np.conj(w * w1 * w2), [source_bilinear(nt, nv, t, c, phi_mp_t, fb1, f1),
                                                   source_bilinear(nt, nv, t, c, phi_p_t, fb2, f2)]))
    return out


# ---------------------------------------------------------------- stochastic estimation (Sec. II-III)
# The stochastic LapH method replaces every quark line of a diagram by a noisy estimate
# built from one noise: with phi^[b] = G P^(b) rho (the sink coefficients of the solves)
# and rho^[b] = P^(b) rho, Q_hat = sum_b phi^[b] rho^[b]dag, whose noise average is G on the
# columns the projectors cover (Z_N noise, Sec. II).  The graphical rules of Sec. III then
# read, term by term of the Wick expansion above:
#   * a line leaving the source time t0 (qbar at t0) uses a forward line sourced at t0;
#   * a line from the sink time tF back to t0 uses a forward line through gamma_5
#     Hermiticity, Q(t0 <- tF) = Gamma' Q(tF <- t0)^dag Gamma', Gamma' = gamma_4 gamma_5
#     (which follows from K^dag = gamma_5 K gamma_5 and Omega = gamma_4 K);
#   * a line from tF to tF uses a same-time line (time interlacing, every projector solved);
#   * the lines of one term all carry different noises: propagators take the next unused
#     line of their kind in the order the term's cycles visit them.

def line_estimate(coef: np.ndarray, rho_b: np.ndarray) -> np.ndarray:
    """Q_hat = sum_b phi^[b] rho^[b]dag over the full LapH space; coef, rho_b [nb][nt][4][nv]."""
    nb = coef.shape[0]
    return coef.reshape(nb, -1).T @ np.conj(rho_b.reshape(nb, -1))


def gamma_swap(q_hat: np.ndarray, nt: int, nv: int, gamma_prime: np.ndarray) -> np.ndarray:
    """Gamma' Q_hat^dag Gamma' with Gamma' acting on the spin index of (t, alpha, n)."""
    g = np.kron(np.eye(nt), np.kron(gamma_prime, np.eye(nv)))
    return g @ q_hat.conj().T @ g


def stochastic_expect(bilinears, times, t0, fwd, bwd, smt):
    """< B_1 ... B_m > with every propagator of every Wick term replaced by a line estimate:
    fwd[i] (lines from t0), bwd[i] (the gamma_5-swapped forward lines, tF -> t0), smt[i]
    (same-time lines at tF); times[k] is the time slice of bilinear k."""
    m = len(bilinears)
    total = 0.0 + 0.0j
    for perm in itertools.permutations(range(m)):
        if any(bilinears[k][2] != bilinears[perm[k]][1] for k in range(m)):
            continue
        used = {"f": 0, "s": 0}
        term = 1.0 + 0.0j
        for cyc in _cycles(perm):
            prod = None
            for k in cyc:
                # Q(j_k, i_perm[k]): from qbar of B_perm[k] (its time) to q of B_k
                t_src, t_snk = times[perm[k]], times[k]
                if t_src == t0:
                    q = fwd[used["f"]]
                    used["f"] += 1
                elif t_snk == t0:
                    q = bwd[used["f"]]
                    used["f"] += 1
                else:
                    q = smt[used["s"]]
                    used["s"] += 1
                f = bilinears[k][0] @ q
                prod = f if prod is None else prod @ f
            term *= np.trace(prod)
        total += _sign(perm) * term
    return (-1) ** m * total


def stochastic_correlator(sink_terms, source_terms, tF, t0, fwd, bwd, smt):
    """Stochastic estimate of < O_sink(tF) O_source(t0) > (see stochastic_expect)."""
    out = 0.0 + 0.0j
    for ws, bs in sink_terms:
        for wr, br in source_terms:
            times = [tF] * len(bs) + [t0] * len(br)
            out += ws * wr * stochastic_expect(list(bs) + list(br), times, t0, fwd, bwd, smt)
    return out
