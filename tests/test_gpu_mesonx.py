"""GPU parity of the momentum, same-time and displaced pieces of the meson correlators (Sec. II
quark line with D^(j); Sec. III, the phase of Eq. (mesonfunc) and the second term of
Eq. (mesoncorr); Sec. V isoscalars) against
the oracle, on the 4^3 x 8 workload (N_v = 8) with the oracle's eigenvectors fed to both sides:

  laph_mom_overlaps       Phi_p = V^dag e^{-ip.x} V against oracle.laph.mom_overlaps: every
                          entry within 1e-12 of its Cauchy scale sum_{x,c} |V_n| |V_n'|
  correlate_mom           full dilution: the exact distillation correlator at momentum p
                          from dense LU (oracle.laph.exact_meson_connected with Phi_p)  1e-8 (floored)
  laph_meson_loops        full dilution, every projector solved (solves to 1e-12): the exact
                          loops from G in both orientations, at p = 0 and p != 0         1e-8 (floored)
                          + 1e-11 of the summed terms' size (the pion loop cancels ~1e4-fold)
  correlate_disconnected  the exact disconnected correlator; the isoscalar combination
                          fwd + 2 smt against the oracle's isoscalar_meson             1e-8 (floored)
  loops, partial dilution time interlacing (TI2) with every projector solved: the oracle's
                          site-space loops of the same noises and dense-LU solutions    1e-8 (floored)
  laph_displaced_overlaps Phi_{p,jk} for paths of 0 to 3 steps against
                          oracle.displacement.displaced_overlaps (Cauchy-scale bound as above)
  displaced correlator    correlate_mom with Phi_{p,jk}, full dilution, against the exact value
                          with the source partner Phi_{-p,kj}                           1e-8 (floored)

The floored relative bound is the correlator tolerance used everywhere:
|d| <= tol * max(|ref|, 1e-3 max|ref|)."""
import numpy as np
import pytest

import synth
from oracle import dilution as dl
from oracle import laph as olaph
from oracle.pipeline import OraclePath
from tests.gpu_util import context, dev, empty, host, lib, rel_err, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

MOMS = [(0, 0, 0), (1, 0, 0), (0, 1, 1), (1, -1, 2)]
CH = ["pion", "rho", "scalar"]


def close(gpu, ref, tol=1e-8):
    gpu, ref = np.asarray(gpu), np.asarray(ref)
    floor = 1e-3 * np.abs(ref).max()
    return bool(np.all(np.abs(gpu - ref) <= tol * np.maximum(np.abs(ref), floor)))


@pytest.fixture(scope="module")
def tiny():
    path = OraclePath(synth.WORKLOADS["tiny_4x8"])
    path._G = path.exact_G()
    return path


def _chan(L, name):
    return {"pion": L.CH_PION, "rho": L.CH_RHO, "scalar": L.CH_SCALAR}[name]


def _cauchy_scale(A, B):
    """sum_{x,c} |A_n| |B_n'| per slice and pair: the scale of the overlap sums."""
    return np.einsum("tnxc,tmxc->tnm", np.abs(A), np.abs(B))


def _loop_scale(G, channel, phi):
    """sum |c_ab| |Phi[n, n']| |G[t b n'; t a n]| per component and slice: the size of the terms that
    a loop sums, so its rounding and solve errors scale with this, not with the (cancelling) loop."""
    nt, nv = G.shape[0], G.shape[2]
    out = np.zeros((len(olaph.channel_c(channel)), nt))
    for i, c in enumerate(olaph.channel_c(channel)):
        for t in range(nt):
            ph = np.eye(nv) if phi is None else phi[t]
            out[i, t] = np.einsum("ab,nN,bNan->", np.abs(c), np.abs(ph), np.abs(G[t, :, :, t, :, :]))
    return out


def _gpu_line(L, tiny, noise_id, bs, dil, tol=1e-11):
    import torch
    wl = tiny.wl
    lat = L.lattice(wl.ns, wl.nt, wl.xi)
    rhs = empty((len(bs), wl.nt, wl.ns, wl.ns, wl.ns, 4, 3), torch.complex128)
    codes = torch.empty((wl.nt, 4, wl.nv), dtype=torch.uint8, device="cuda")
    L.laph_make_sources(context(), lat, dev(tiny.evecs), wl.nv, noise_id, wl.config_id, L.dilution(*dil), bs, rhs, codes)
    sol = torch.empty_like(rhs)
    L.dirac_solve_batch(context(), lat, dev(tiny.u), wl.m0, wl.csw, rhs, sol, len(bs),
                        L.solver_params(mode=L.MIXED_FP32, tol=tol))
    coef = empty((len(bs), wl.nt, 4, wl.nv), torch.complex128)
    L.laph_sinks(context(), lat, dev(tiny.evecs), wl.nv, sol, len(bs), coef)
    return coef, codes


def _gpu_phi(L, tiny, mom):
    import torch
    wl = tiny.wl
    phi = empty((1, wl.nt, wl.nv, wl.nv), torch.complex128)
    L.laph_mom_overlaps(context(), L.lattice(wl.ns, wl.nt, wl.xi), dev(tiny.evecs), wl.nv, [mom], phi)
    return phi[0]


def test_mom_overlaps(tiny):
    import torch
    L = lib()
    wl = tiny.wl
    phi = empty((len(MOMS), wl.nt, wl.nv, wl.nv), torch.complex128)
    L.laph_mom_overlaps(context(), L.lattice(wl.ns, wl.nt, wl.xi), dev(tiny.evecs), wl.nv, MOMS, phi)
    got = host(phi)
    scale = _cauchy_scale(tiny.evecs, tiny.evecs)
    for i, m in enumerate(MOMS):
        assert np.all(np.abs(got[i] - olaph.mom_overlaps(tiny.evecs, m)) <= 1e-12 * scale), m
    assert np.abs(got[0] - np.eye(wl.nv)[None]).max() <= 1e-12


def test_mom_overlaps_ragged_tiles():
    """6^3 x 2 slices, 21 random (not orthonormal) vectors: output tiles of 16 cut at 21, K = 648."""
    import torch
    L = lib()
    ns, nt, nv = 6, 2, 21
    V = synth.random_complex((nt, nv, ns ** 3, 3), seed=31)
    phi = empty((2, nt, nv, nv), torch.complex128)
    L.laph_mom_overlaps(context(), L.lattice(ns, nt, 3.5), dev(V), nv, [(2, 0, 1), (0, 3, -1)], phi)
    got = host(phi)
    scale = _cauchy_scale(V, V)
    for i, m in enumerate([(2, 0, 1), (0, 3, -1)]):
        assert np.all(np.abs(got[i] - olaph.mom_overlaps(V, m)) <= 1e-12 * scale)


@pytest.mark.parametrize("channel", CH)
def test_correlate_mom_full_dilution_vs_exact(tiny, channel):
    import torch
    L = lib()
    wl = tiny.wl
    t0, mom = 2, (1, 0, 0)
    bs = tiny.projectors_for_time(t0)
    lines = [_gpu_line(L, tiny, s, bs, tiny.dil) for s in (0, 1)]
    corr = empty((wl.nt,), torch.complex128)
    L.correlate_mom(context(), L.lattice(wl.ns, wl.nt, wl.xi), _chan(L, channel), t0, wl.nv, L.dilution(*tiny.dil),
                    bs, [c for c, _ in lines], [n for _, n in lines], _gpu_phi(L, tiny, mom), corr)
    ref = olaph.exact_meson_connected(tiny._G, t0, channel, olaph.mom_overlaps(tiny.evecs, mom))
    assert np.abs(ref).max() > 1e-8
    assert close(host(corr), ref)


@pytest.fixture(scope="module")
def all_lines(tiny):
    """Two lines (noises 20, 21) with every projector of full dilution solved, to 1e-12: the pion
    loop is a sum of 256 terms of order 1e-1 that cancels to order 1e-4, so it carries the
    solves' residual about a thousandfold."""
    L = lib()
    nT, nS, nL = dl.counts(tiny.dil, tiny.wl.nt, tiny.wl.nv)
    bs = list(range(nT * nS * nL))
    return bs, [_gpu_line(L, tiny, s, bs, tiny.dil, tol=1e-12) for s in (20, 21)]


@pytest.mark.parametrize("channel", CH)
@pytest.mark.parametrize("mom", [None, (0, 1, 1)])
def test_loops_and_disconnected_full_dilution_vs_exact(tiny, all_lines, channel, mom):
    import torch
    L = lib()
    wl = tiny.wl
    lat = L.lattice(wl.ns, wl.nt, wl.xi)
    bs, lines = all_lines
    nc = 3 if channel == "rho" else 1
    phi_g = None if mom is None else _gpu_phi(L, tiny, mom)
    phi_o = None if mom is None else olaph.mom_overlaps(tiny.evecs, mom)
    loops = []
    for k, reverse in ((0, 0), (1, 1)):
        lp = empty((nc, wl.nt), torch.complex128)
        coef, codes = lines[k]
        L.laph_meson_loops(context(), lat, _chan(L, channel), wl.nv, L.dilution(*tiny.dil), bs, coef, codes, phi_g,
                           reverse, lp)
        ref = olaph.exact_loops(tiny._G, channel, phi_o, reverse=bool(reverse))
        # solves to 1e-12: each loop carries about 1e-12 of the terms it sums, 1e-11 of them allowed
        got = host(lp)
        floor = 1e-3 * np.abs(ref).max()
        bound = 1e-8 * np.maximum(np.abs(ref), floor) + 1e-11 * _loop_scale(tiny._G, channel, phi_o)
        assert np.all(np.abs(got - ref) <= bound), (reverse, channel, mom)
        loops.append(lp)
    t0 = 3
    corr = empty((wl.nt,), torch.complex128)
    L.correlate_disconnected(context(), lat, t0, nc, loops[0], loops[1], 0.0, corr)
    smt_ref = olaph.exact_meson_disconnected(tiny._G, t0, channel, phi_o)
    assert close(host(corr), smt_ref)
    if mom is None:
        # isoscalar = fwd + 2 smt (two degenerate light flavours)
        fwd_ref = olaph.exact_meson_connected(tiny._G, t0, channel)
        fwd = empty((wl.nt,), torch.complex128)
        bs0 = tiny.projectors_for_time(t0)
        l2 = [_gpu_line(L, tiny, s, bs0, tiny.dil) for s in (30, 31)]
        L.correlate(context(), lat, _chan(L, channel), t0, wl.nv, L.dilution(*tiny.dil), bs0,
                    [c for c, _ in l2], [n for _, n in l2], fwd)
        iso = host(fwd) + 2.0 * host(corr)
        assert close(iso, olaph.isoscalar_meson(fwd_ref, smt_ref))


@pytest.mark.parametrize("channel", ["pion", "scalar"])
def test_loops_partial_dilution_same_noise(tiny, channel):
    """Time interlacing TI2 (with full spin and LapH dilution), every projector solved: the GPU
    loops of one noise equal the oracle's site-space loops of the same noise and dense-LU
    solutions, although both differ from the exact loops (the noise does not average out)."""
    import torch
    L = lib()
    wl = tiny.wl
    dil = ((3, 2), (1, 0), (1, 0))
    nT, nS, nL = dl.counts(dil, wl.nt, wl.nv)
    bs = list(range(nT * nS * nL))
    coef, codes = _gpu_line(L, tiny, 40, bs, dil)
    lp = empty((1, wl.nt), torch.complex128)
    L.laph_meson_loops(context(), L.lattice(wl.ns, wl.nt, wl.xi), _chan(L, channel), wl.nv, L.dilution(*dil), bs,
                       coef, codes, None, 0, lp)
    saved = tiny.dil
    tiny.dil = dil
    try:
        line = tiny.line(40, bs, "lu")[0]
    finally:
        tiny.dil = saved
    ref = olaph.meson_loops(line, channel)
    assert close(host(lp), ref)
    assert not close(ref, olaph.exact_loops(tiny._G, channel), 1e-4)


PATHS = [((), (1,)), ((2, 2), (-3,)), ((1, 2, 3), (-1, -1, -1)), ((-2,), ())]


@pytest.mark.parametrize("mom", [(0, 0, 0), (1, 0, 0), (0, -1, 2)])
@pytest.mark.parametrize("paths", PATHS)
def test_displaced_overlaps(tiny, mom, paths):
    """Phi_{p,jk} = e^{-ip.(d_j+d_k)/2} (D^(j) V)^dag e^{-ip.x} (D^(k) V) against
    oracle.displacement.displaced_overlaps (Sec. II quark line with D^(j), Eq. (quarkdef))."""
    import torch
    from oracle import displacement as od
    L = lib()
    wl = tiny.wl
    phi = empty((wl.nt, wl.nv, wl.nv), torch.complex128)
    L.laph_displaced_overlaps(context(), L.lattice(wl.ns, wl.nt, wl.xi), dev(tiny.ut), dev(tiny.evecs), wl.nv, mom,
                              paths[0], paths[1], phi)
    ref = od.displaced_overlaps(tiny.ut, tiny.evecs, mom, paths[0], paths[1])
    V = tiny.evecs
    scale = _cauchy_scale(od.displace(tiny.ut, od.evecs_as_fields(V), paths[0]).transpose(1, 0, 2, 3, 4, 5)
                          .reshape(V.shape), od.displace(tiny.ut, od.evecs_as_fields(V), paths[1])
                          .transpose(1, 0, 2, 3, 4, 5).reshape(V.shape))
    assert np.all(np.abs(host(phi) - ref) <= 1e-12 * scale)


@pytest.mark.parametrize("paths", PATHS[:3])
def test_displaced_correlator_full_dilution_vs_exact(tiny, paths):
    """The connected correlator of a displaced pion elemental (c = gamma_4 gamma_5, p, j, k) through
    correlate_mom with Phi_{p,jk}, against the exact value from G with Phi_{p,jk} at the sink and
    its source partner Phi_{-p,kj} (oracle.displacement.exact_meson_connected_displaced)."""
    import torch
    from oracle import displacement as od
    from oracle.gamma import GAMMA, GAMMA5
    L = lib()
    wl = tiny.wl
    t0, mom = 4, (1, 0, 0)
    lat = L.lattice(wl.ns, wl.nt, wl.xi)
    phi = empty((wl.nt, wl.nv, wl.nv), torch.complex128)
    L.laph_displaced_overlaps(context(), lat, dev(tiny.ut), dev(tiny.evecs), wl.nv, mom, paths[0], paths[1], phi)
    bs = tiny.projectors_for_time(t0)
    lines = [_gpu_line(L, tiny, s, bs, tiny.dil) for s in (50, 51)]
    corr = empty((wl.nt,), torch.complex128)
    L.correlate_mom(context(), lat, L.CH_PION, t0, wl.nv, L.dilution(*tiny.dil), bs, [c for c, _ in lines],
                    [n for _, n in lines], phi, corr)
    snk = od.displaced_overlaps(tiny.ut, tiny.evecs, mom, paths[0], paths[1])
    src = od.displaced_overlaps(tiny.ut, tiny.evecs, tuple(-m for m in mom), paths[1], paths[0])
    ref = od.exact_meson_connected_displaced(tiny._G, t0, GAMMA[3] @ GAMMA5, snk, src)
    assert np.abs(ref).max() > 1e-8
    assert close(host(corr), ref)
