"""GPU parity of the two-pion correlators of isospin 0, 1, 2 (Sec. III two-meson diagrams:
direct, crossed, box and vacuum; Sec. V two-pion operators) against the oracle on the
4^3 x 8 workload (N_v = 8), the oracle's eigenvectors fed to both sides:

  full dilution     four forward lines sourced at t0 and two same-time lines with every
                    projector solved (solves to 1e-12) make the estimate exact: the brute-force
                    Wick contraction of the exact G (oracle.wick.correlator) for |I, I3> =
                    |2,2>, |2,0>, |1,0>, |0,0> at p = 0 and p = (1,0,0), every dt     1e-8 (floored)
  partial dilution  forward lines (TF, SF, LI2), same-time lines (TI2, SF, LI2): the oracle's
                    stochastic estimate (oracle.wick.stochastic_correlator) from the same noises
                    and dense-LU lines, |0,0> and |1,0>, every dt != 0 (at dt = 0 the oracle
                    assigns lines by time, the library by the bilinear's side)       1e-8 (floored)

The floored relative bound: |d| <= tol * max(|ref|, 1e-3 max|ref|)."""
import numpy as np
import pytest

import synth
from oracle import dilution as dl
from oracle import laph as olaph
from oracle import wick
from oracle.pipeline import OraclePath
from tests.gpu_util import context, dev, empty, host, lib, requires_gpu
from tests.test_gpu_mesonx import _gpu_line, _gpu_phi, close

pytestmark = [pytest.mark.gpu, requires_gpu]

T0 = 1


@pytest.fixture(scope="module")
def tiny():
    path = OraclePath(synth.WORKLOADS["tiny_4x8"])
    path._G = path.exact_G()
    return path


def _all(dil, nt, nv):
    nT, nS, nL = dl.counts(dil, nt, nv)
    return list(range(nT * nS * nL))


def _fwd_projectors(dil, nt, nv, t0):
    nT, nS, nL = dl.counts(dil, nt, nv)
    kT, JT = dil[0]
    return [(bT * nS + bS) * nL + bL for bT in range(nT) if dl.projector_diag(kT, JT, nt, bT)[t0]
            for bS in range(nS) for bL in range(nL)]


@pytest.fixture(scope="module")
def full_lines(tiny):
    L = lib()
    wl = tiny.wl
    bf = _fwd_projectors(tiny.dil, wl.nt, wl.nv, T0)
    bs = _all(tiny.dil, wl.nt, wl.nv)
    fwd = [_gpu_line(L, tiny, 70 + k, bf, tiny.dil, tol=1e-12) for k in range(4)]
    smt = [_gpu_line(L, tiny, 80 + k, bs, tiny.dil, tol=1e-12) for k in range(2)]
    return bf, bs, fwd, smt


def _run(L, tiny, iso, dil_f, bf, fwd, dil_s, bs, smt, mom):
    import torch
    wl = tiny.wl
    corr = empty((wl.nt,), torch.complex128)
    php = phm = None
    if mom != (0, 0, 0):
        php, phm = _gpu_phi(L, tiny, mom), _gpu_phi(L, tiny, tuple(-m for m in mom))
    L.correlate_pipi(context(), L.lattice(wl.ns, wl.nt, wl.xi), iso[0], iso[1], T0, wl.nv, L.dilution(*dil_f), bf,
                     [c for c, _ in fwd], [n for _, n in fwd], L.dilution(*dil_s), bs, [c for c, _ in smt],
                     [n for _, n in smt], php, phm, corr)
    return host(corr)


def _exact(tiny, iso, mom):
    wl = tiny.wl
    nt, nv = wl.nt, wl.nv
    Q = tiny._G.reshape(nt * 4 * nv, nt * 4 * nv)
    c = olaph.channel_c("pion")[0]
    if mom == (0, 0, 0):
        ph = phm = np.stack([np.eye(nv)] * nt)
    else:
        ph, phm = olaph.mom_overlaps(tiny.evecs, mom), olaph.mom_overlaps(tiny.evecs, tuple(-m for m in mom))
    out = np.zeros(nt, dtype=complex)
    for dt in range(nt):
        tf = (T0 + dt) % nt
        snk = wick.two_pion_sink(nt, nv, tf, c, ph[tf], phm[tf], iso)
        src = wick.two_pion_source(nt, nv, T0, c, ph[T0], phm[T0], iso)
        out[dt] = wick.correlator(snk, src, Q)
    return out


@pytest.mark.parametrize("mom", [(0, 0, 0), (1, 0, 0)])
@pytest.mark.parametrize("iso", [(2, 2), (2, 0), (1, 0), (0, 0)])
def test_pipi_full_dilution_vs_exact(tiny, full_lines, iso, mom):
    L = lib()
    bf, bs, fwd, smt = full_lines
    got = _run(L, tiny, iso, tiny.dil, bf, fwd, tiny.dil, bs, smt, mom)
    ref = _exact(tiny, iso, mom)
    if iso == (1, 0) and mom == (0, 0, 0):
        # the antisymmetric I = 1 state of two pions at rest vanishes identically
        assert np.abs(ref).max() == 0.0
        assert np.abs(got).max() <= 1e-12 * np.abs(_exact(tiny, (2, 0), mom)).max()
        return
    assert np.abs(ref).max() > 1e-10
    assert close(got, ref), (iso, mom)


def test_pipi_i2_needs_no_same_time_lines(tiny, full_lines):
    """|2,2> has no box or vacuum diagram: no same-time line is read."""
    L = lib()
    bf, _, fwd, _ = full_lines
    got = _run(L, tiny, (2, 2), tiny.dil, bf, fwd, tiny.dil, [], [], (0, 0, 0))
    assert close(got, _exact(tiny, (2, 2), (0, 0, 0)))
    with pytest.raises(L.LaphError):
        _run(L, tiny, (0, 0), tiny.dil, bf, fwd, tiny.dil, [], [], (0, 0, 0))


def _oracle_estimate(tiny, noise_id, dil, bs):
    saved = tiny.dil
    tiny.dil = dil
    try:
        _, x = tiny.line(noise_id, bs, method="lu")
    finally:
        tiny.dil = saved
    rho = tiny.rho(noise_id)
    coef = olaph.sinks(tiny.evecs, x)
    rho_b = np.stack([olaph.diluted_noise(rho, dil, b) for b in bs])
    return wick.line_estimate(coef, rho_b)


@pytest.mark.parametrize("iso", [(0, 0), (1, 0)])
def test_pipi_partial_dilution_vs_oracle(tiny, iso):
    L = lib()
    wl = tiny.wl
    nt, nv = wl.nt, wl.nv
    dil_f = ((1, 0), (1, 0), (3, 2))
    dil_s = ((3, 2), (1, 0), (3, 2))
    bf = _fwd_projectors(dil_f, nt, nv, T0)
    bs = _all(dil_s, nt, nv)
    fwd = [_gpu_line(L, tiny, 90 + k, bf, dil_f) for k in range(4)]
    smt = [_gpu_line(L, tiny, 95 + k, bs, dil_s) for k in range(2)]
    mom = (0, 0, 0) if iso == (0, 0) else (1, 0, 0)
    got = _run(L, tiny, iso, dil_f, bf, fwd, dil_s, bs, smt, mom)
    fq = [_oracle_estimate(tiny, 90 + k, dil_f, bf) for k in range(4)]
    bq = [wick.gamma_swap(q, nt, nv, olaph.GAMMA[3] @ olaph.GAMMA5) for q in fq]
    sq = [_oracle_estimate(tiny, 95 + k, dil_s, bs) for k in range(2)]
    c = olaph.channel_c("pion")[0]
    if mom == (0, 0, 0):
        ph = phm = np.stack([np.eye(nv)] * nt)
    else:
        ph, phm = olaph.mom_overlaps(tiny.evecs, mom), olaph.mom_overlaps(tiny.evecs, tuple(-m for m in mom))
    ref = np.zeros(nt, dtype=complex)
    for dt in range(1, nt):
        tf = (T0 + dt) % nt
        snk = wick.two_pion_sink(nt, nv, tf, c, ph[tf], phm[tf], iso)
        src = wick.two_pion_source(nt, nv, T0, c, ph[T0], phm[T0], iso)
        ref[dt] = wick.stochastic_correlator(snk, src, tf, T0, fq, bq, sq)
    assert np.abs(ref[1:]).max() > 1e-10
    assert close(got[1:], ref[1:])
    # one noise set is not the exact correlator
    assert not close(ref[1:], _exact(tiny, iso, mom)[1:], 1e-3)
