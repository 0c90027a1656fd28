"""Sources, sinks, meson functions and correlators (site-space route).

Sec. II, Eqs. (varrhodef), (varphidef): with no displacement (D = 1)
    varrho^[b] = V_s P^(b) rho                        (diluted source)
    varphi^[b] = S Omega^{-1} V_s P^(b) rho,  S = V_s V_s^dag,  Omega = gamma_4 K.
Solving Omega X = y is the same as solving K X = gamma_4 y.
Eq. (laphpropg5): varrho-bar = -gamma_5 gamma_4 varrho, varphi-bar = gamma_5 gamma_4 varphi.
Sec. IV: the stored quark-propagation coefficients are V_s^dag Omega^{-1} V_s P^(b) rho,
N_t N_v numbers per spin (reading: stored as coef[t][alpha][n]).

Sec. III meson function Eq. (mesonfunc) at zero momentum without displacement:
    M^[b1 b2](a, b; t) = c_{alpha beta} sum_x sum_colour a^[b1]_{alpha}(x,t)^* b^[b2]_{beta}(x,t)
and the connected meson correlator Eq. (mesoncorr), first term:
    C(t_F - t_0) = - sum_{b1,b2} M^[b1b2](varphi-bar_1, varphi_2; t_F) M^[b1b2](varrho-bar_1, varrho_2; t_0)^*.
Reading taken for the channels: the quark-bilinear psi-bar Gamma psi is
written with q-bar = psi-bar gamma_4 (Eq. (quarkdef)), so c = gamma_4 Gamma:
pion Gamma = gamma_5, rho Gamma = gamma_k (the three k averaged), scalar
Gamma = 1.  With these the pion correlator is positive.  Correlators are
summed over space (no 1/V) and averaged over the source times used (the
1/N_t sum over t_0 of Sec. III), indexed by dt = (t_F - t_0) mod N_t.

I = 2 two-pion (zero momenta, single-site pions): the paper gives only
diagrams (Figs. twomesontwomeson).  Reading (Wick's theorem, four independent
noises; lines 1 and 3 are the gamma_5-swapped lines):
    C = D - X,
    D = Cpi(1,2) * Cpi(3,4),
    X = sum_{b1..b4} M^[b1 b4](phibar_1, phi_4; t_F) M^[b3 b2](phibar_3, phi_2; t_F)
                     M^[b1 b2](rhobar_1, rho_2; t_0)^* M^[b3 b4](rhobar_3, rho_4; t_0)^*.

Momentum (Sec. III, the phase of Eq. (mesonfunc) without displacement): an operator
destroying momentum p carries sum_x e^{-i p.x}, p = 2 pi (p_x, p_y, p_z) / N_s with
integer components; the sink function M_l(tF) and the source function M_lbar(t0),
conjugated in Eq. (mesoncorr), both take that phase for the same p (reading: lbar is
the creation operator of the same momentum, so conj(M_lbar) carries e^{+i p.x}).
In LapH coordinates the phase enters through the overlap matrices
    Phi_p(t)[n, n'] = sum_{x,c} V(t,n,x,c)^* e^{-i p.x} V(t,n',x,c),
which are the identity at p = 0.

Same-time lines (second term of Eq. (mesoncorr), isoscalar mesons): each line closes on
one time slice, and the b sums of the two meson functions run separately:
    D(t_F - t_0) = sum_{b1} M^[b1 b1](varrho_1, varphi_1; t_F) (sum_{b2} M^[b2 b2](varphi_2, varrho_2; t_0))^*.
The paper names the two diagrams "fwd" (first term) and "smt" (second term) and, for its
isoscalars made of the two light flavours, plots their sum.  Reading taken for the
flavour weights: the operator (u-bar Gamma u + d-bar Gamma d)/sqrt(2) with degenerate u, d
gives the delta factors of Eq. (mesoncorr) the sums 1 (first term) and 2 (second term),
so C_isoscalar = fwd + 2 smt.  For the scalar the "smt" part has its vacuum expectation
value removed: smt - <L_1> <L_2>^*, with <L> the loop averaged over configurations, time
slices and noises.

This module works with full site-space fields (it builds varrho and varphi on
the lattice and sums over sites), an independent route from the coefficient-
space contractions of the CUDA path.
"""
import numpy as np

from .gamma import GAMMA, GAMMA5, ONE4
from . import dilution as dl

G4 = GAMMA[3]
G5G4 = GAMMA5 @ G4

CHANNELS = ("pion", "rho", "scalar")


def channel_c(channel: str):
    """List of the c matrices (c = gamma_4 Gamma) whose correlators are averaged."""
    if channel == "pion":
        return [G4 @ GAMMA5]
    if channel == "rho":
        return [G4 @ GAMMA[k] for k in range(3)]
    if channel == "scalar":
        return [G4 @ ONE4]
    raise ValueError(channel)


def lapH_to_site(evecs: np.ndarray, coef: np.ndarray) -> np.ndarray:
    """sum_n V(t,n,x,c) coef(t,alpha,n) -> field [t,z,y,x,4,3]."""
    nt, nv, v3, _ = evecs.shape
    ns = round(v3 ** (1.0 / 3.0))
    f = np.einsum("tnxc,tan->txac", evecs, coef)
    return f.reshape(nt, ns, ns, ns, 4, 3)


def diluted_noise(rho: np.ndarray, dil, b: int) -> np.ndarray:
    """P^(b) rho over (t, alpha, n)."""
    nt, _, nv = rho.shape
    return dl.full_projector_diag(dil, nt, nv, b) * rho


def source(evecs: np.ndarray, rho: np.ndarray, dil, b: int) -> np.ndarray:
    """varrho^[b] = V_s P^(b) rho as a site field."""
    return lapH_to_site(evecs, diluted_noise(rho, dil, b))


def dirac_rhs(evecs: np.ndarray, rho: np.ndarray, dil, b: int) -> np.ndarray:
    """Right-hand side for K: gamma_4 V_s P^(b) rho (Omega x = y <=> K x = gamma_4 y)."""
    y = source(evecs, rho, dil, b)
    return np.einsum("ab,...bc->...ac", G4, y)


def sinks(evecs: np.ndarray, x: np.ndarray) -> np.ndarray:
    """coef(t, alpha, n) = sum_{x,c} V(t,n,x,c)^* X(t,x,alpha,c)."""
    nt, nv, v3, _ = evecs.shape
    xf = x.reshape(x.shape[:-6] + (nt, v3, 4, 3))
    return np.einsum("tnxc,...txac->...tan", np.conj(evecs), xf)


def smear(evecs: np.ndarray, x: np.ndarray) -> np.ndarray:
    """varphi = V_s V_s^dag X (site field)."""
    return lapH_to_site(evecs, sinks(evecs, x))


def spin_mul(m: np.ndarray, f: np.ndarray) -> np.ndarray:
    return np.einsum("ab,...bc->...ac", m, f)


def mom_phase(ns: int, mom) -> np.ndarray:
    """e^{-i p.x} on one time slice, p = 2 pi mom / N_s, indexed like the slice's sites
    ((z N_s + y) N_s + x, x fastest)."""
    z, y, x = np.meshgrid(np.arange(ns), np.arange(ns), np.arange(ns), indexing="ij")
    px, py, pz = mom
    return np.exp(-2j * np.pi * (px * x + py * y + pz * z) / ns).ravel()


def mom_overlaps(evecs: np.ndarray, mom) -> np.ndarray:
    """Phi_p(t)[n, n'] = sum_{x,c} V(t,n,x,c)^* e^{-i p.x} V(t,n',x,c), [nt][nv][nv]."""
    nt, nv, v3, _ = evecs.shape
    ph = mom_phase(round(v3 ** (1.0 / 3.0)), mom)
    return np.einsum("tnxc,x,tmxc->tnm", np.conj(evecs), ph, evecs)


def meson_functions(a_list, b_list, c: np.ndarray, mom=None) -> np.ndarray:
    """M[b1, b2, t] = sum_{x,colour} e^{-i p.x} sum_{alpha beta} a^[b1]_alpha(x,t)^* c_{alpha beta} b^[b2]_beta(x,t).

    a_list, b_list: arrays [nb, t, z, y, x, 4, 3]; mom: integer 3-vector (None: p = 0)."""
    nb1, nt = a_list.shape[0], a_list.shape[1]
    a = a_list.reshape(nb1, nt, -1, 4, 3)
    b = b_list.reshape(b_list.shape[0], nt, -1, 4, 3)
    cb = np.einsum("ab,ntxbc->ntxac", c, b)
    if mom is not None:
        cb = cb * mom_phase(a_list.shape[2], mom)[None, None, :, None, None]
    return np.einsum("ptxac,qtxac->pqt", np.conj(a), cb)


class Line:
    """One quark line: its noise, dilution and, per solved projector, the
    diluted source varrho^[b] and sink varphi^[b] as site fields."""

    def __init__(self, evecs, rho, dil, bs, solutions):
        self.bs = list(bs)
        self.varrho = np.stack([source(evecs, rho, dil, b) for b in bs])
        self.varphi = np.stack([smear(evecs, x) for x in solutions])

    @property
    def varrho_bar(self):
        return -spin_mul(G5G4, self.varrho)

    @property
    def varphi_bar(self):
        return spin_mul(G5G4, self.varphi)


def meson_connected(line1: Line, line2: Line, t0: int, channel: str, mom=None) -> np.ndarray:
    """C(dt), dt = (t_F - t_0) mod N_t, of Eq. (mesoncorr) first term for one source time,
    at momentum mom (None: zero momentum)."""
    nt = line1.varrho.shape[1]
    out = np.zeros(nt, dtype=complex)
    for c in channel_c(channel):
        msink = meson_functions(line1.varphi_bar, line2.varphi, c, mom)       # [b1, b2, tF]
        msrc = meson_functions(line1.varrho_bar, line2.varrho, c, mom)[:, :, t0]
        ct = -np.einsum("pqt,pq->t", msink, np.conj(msrc))
        out += np.roll(ct, -t0)
    return out / len(channel_c(channel))


def meson_loops(line: Line, channel: str, mom=None, reverse=False) -> np.ndarray:
    """Same-time line closed on each slice: L_c(t) = sum_b M^[bb](varrho, varphi; t), or with
    reverse M^[bb](varphi, varrho; t), one row per c of the channel, [nc][nt].  Every t must
    be covered by the line's projectors (time interlacing with all of them solved)."""
    a, b = (line.varphi, line.varrho) if reverse else (line.varrho, line.varphi)
    return np.array([np.einsum("bbt->t", meson_functions(a, b, c, mom)) for c in channel_c(channel)])


def meson_disconnected(line1: Line, line2: Line, t0: int, channel: str, mom=None) -> np.ndarray:
    """Second term of Eq. (mesoncorr) for one source time, dt-indexed, averaged over the c of
    the channel: L_1(t0 + dt) conj(L_2(t0)) with L_1 from (varrho_1, varphi_1) and L_2 from
    (varphi_2, varrho_2)."""
    l1 = meson_loops(line1, channel, mom)
    l2 = meson_loops(line2, channel, mom, reverse=True)
    return np.mean(np.roll(l1, -t0, axis=1) * np.conj(l2[:, t0])[:, None], axis=0)


def isoscalar_meson(fwd: np.ndarray, smt: np.ndarray, vev=None) -> np.ndarray:
    """fwd + 2 (smt - vev): two degenerate light flavours; vev = <L_1> <L_2>^* (scalar only)."""
    return fwd + 2.0 * (smt - (0.0 if vev is None else vev))


def pipi_i2(l1: Line, l2: Line, l3: Line, l4: Line, t0: int) -> np.ndarray:
    """I = 2 two-pion correlator D - X for one source time (see module docstring)."""
    nt = l1.varrho.shape[1]
    c = channel_c("pion")[0]
    d = meson_connected(l1, l2, t0, "pion") * meson_connected(l3, l4, t0, "pion")
    m14 = meson_functions(l1.varphi_bar, l4.varphi, c)       # [b1, b4, tF]
    m32 = meson_functions(l3.varphi_bar, l2.varphi, c)       # [b3, b2, tF]
    s12 = meson_functions(l1.varrho_bar, l2.varrho, c)[:, :, t0]
    s34 = meson_functions(l3.varrho_bar, l4.varrho, c)[:, :, t0]
    x = np.einsum("adt,cbt,ab,cd->t", m14, m32, np.conj(s12), np.conj(s34))
    return d - np.roll(x, -t0)


# ----------------------------------------------------------------------------
# Exact (distillation) reference, Sec. II: G = V_s^dag Omega^{-1} V_s from the
# full inverse of K (tiny lattices only).
# ----------------------------------------------------------------------------

def exact_G(evecs: np.ndarray, kinv: np.ndarray) -> np.ndarray:
    """G[(t,alpha,n),(t',alpha',n')] = V^dag K^{-1} gamma_4 V in LapH x spin space.

    kinv: dense K^{-1} (12V x 12V) with component order (site, spin, colour)."""
    nt, nv, v3, _ = evecs.shape
    # W[(site,spin,colour), (t, alpha, n)] = V(t,n,x,c) delta_{spin alpha}
    w = np.zeros((nt, v3, 4, 3, nt, 4, nv), dtype=complex)
    for t in range(nt):
        for a in range(4):
            w[t, :, a, :, t, a, :] = np.transpose(evecs[t], (1, 2, 0))
    w = w.reshape(nt * v3 * 12, nt * 4 * nv)
    g4 = np.kron(np.eye(nt * v3), np.kron(G4, np.eye(3)))
    return (w.conj().T @ (kinv @ (g4 @ w))).reshape(nt, 4, nv, nt, 4, nv)


def exact_meson_connected(G: np.ndarray, t0: int, channel: str, phi=None) -> np.ndarray:
    """C(t_F, t_0) = - sum c_{ab} c^*_{a'b'} G[t0 a' m; tF a n] G[tF b n; t0 b' m], dt-indexed.

    With momentum overlaps phi = Phi_p [nt][nv][nv] the LapH indices of the two lines meet
    through them instead of directly:
        - sum c_{ab} c^*_{a'b'} Phi_p(t0)[m, m']^* Phi_p(tF)[n, n'] G[t0 a' m; tF a n] G[tF b n'; t0 b' m']."""
    nt = G.shape[0]
    out = np.zeros(nt, dtype=complex)
    for c in channel_c(channel):
        for tf in range(nt):
            g_src_snk = G[t0, :, :, tf, :, :]     # [a', m, a, n]
            g_snk_src = G[tf, :, :, t0, :, :]     # [b, n, b', m]
            if phi is None:
                out[(tf - t0) % nt] += -np.einsum("ab,pq,pman,bnqm->", c, np.conj(c), g_src_snk, g_snk_src)
            else:
                out[(tf - t0) % nt] += -np.einsum("ab,pq,mM,nN,pman,bNqM->", c, np.conj(c), np.conj(phi[t0]),
                                                  phi[tf], g_src_snk, g_snk_src)
    return out / len(channel_c(channel))


def exact_loops(G: np.ndarray, channel: str, phi=None, reverse=False) -> np.ndarray:
    """Full-dilution limit of meson_loops, [nc][nt]:
        L_c(t) = sum c_{ab} Phi(t)[n, n'] G[t b n'; t a n]            (varrho, varphi)
        L_c(t) = sum c_{ab} Phi(t)[n, n'] conj(G[t a n; t b n'])      (reverse: varphi, varrho)
    with Phi = 1 at zero momentum."""
    nt, nv = G.shape[0], G.shape[2]
    out = np.zeros((len(channel_c(channel)), nt), dtype=complex)
    for i, c in enumerate(channel_c(channel)):
        for t in range(nt):
            g = G[t, :, :, t, :, :]                         # [a, n, b, n']
            ph = np.eye(nv) if phi is None else phi[t]
            if reverse:
                out[i, t] = np.einsum("ab,nN,anbN->", c, ph, np.conj(g))
            else:
                out[i, t] = np.einsum("ab,nN,bNan->", c, ph, g)
    return out


def exact_meson_disconnected(G: np.ndarray, t0: int, channel: str, phi=None) -> np.ndarray:
    l1 = exact_loops(G, channel, phi)
    l2 = exact_loops(G, channel, phi, reverse=True)
    return np.mean(np.roll(l1, -t0, axis=1) * np.conj(l2[:, t0])[:, None], axis=0)


def exact_pipi_i2(G: np.ndarray, t0: int) -> np.ndarray:
    """D - X for the I = 2 two-pion correlator from the exact G."""
    nt = G.shape[0]
    c = channel_c("pion")[0]
    cpi = exact_meson_connected(G, t0, "pion")
    out = np.zeros(nt, dtype=complex)
    for tf in range(nt):
        a = G[t0, :, :, tf, :, :]   # d-type line, t0 <- tF : [a', m, a, n]
        b = G[tf, :, :, t0, :, :]   # u-type line, tF <- t0 : [b, n, b', m]
        # one loop: c^*(src1) Q_d(src1; snk1) c(snk1) Q_u(snk1; src2) c^*(src2) Q_d(src2; snk2) c(snk2) Q_u(snk2; src1)
        x = np.einsum("ab,pq,cd,rs,pman,bnsk,rkcl,dlqm->",
                      c, np.conj(c), c, np.conj(c), a, b, a, b)
        out[(tf - t0) % nt] = cpi[(tf - t0) % nt] ** 2 - x
    return out
