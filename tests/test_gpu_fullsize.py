"""Parity at the bench's full size and launch configuration: the 16^3 x 32 medium
workload, all 64 diluted sources of source times 0 and 8 of one noise solved as ONE
block of 64 right-hand sides (the copy-engine-fed FP32 stencil inside the mixed solver),
checked on outputs the oracle computes independently or by properties that hold at
any size.  The oracle smears the seeded field itself; no oracle input comes from the GPU.

  stout links (a0)    every GPU-smeared link against the oracle's         |dU| <= 1e-12
  noise (a2)          the whole Z4 code table against the oracle's Philox  bit for bit
  sources (a2)        V^dag gamma_4 y_b = P^(b) rho for every source, with rho and P^(b)
                      from the oracle's noise and dilution definitions     <= 1e-12
  solves (a3)         for 4 sampled sources the FP64 true residual ||y - K x|| / ||y||
                      under the oracle's plain-C K on the oracle's links    <= 1e-10
  sinks (a4)          sampled coefficients equal sum_x conj(V) x            rel <= 1e-12
"""
import numpy as np
import pytest

import synth
from oracle import dilution as dl
from oracle import noise as onoise
from oracle.dirac import WilsonClover
from oracle.fast import FastK
from oracle.gamma import GAMMA
from tests.gpu_util import context, dev, empty, host, lib, oracle_links, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


@pytest.fixture(scope="module")
def medium():
    import torch
    L = lib()
    from paper_1104_3870_gb300.pipeline import LapHPath, LatticeSpec, projectors_for_time
    wl = synth.WORKLOADS["medium_16x32"]
    spec = LatticeSpec(wl.ns, wl.nt, wl.xi, wl.m0, wl.csw, wl.nv, (wl.dil_time, wl.dil_spin, wl.dil_laph),
                       wl.rho_stout, wl.n_stout4d, wl.n_stout3d)
    path = LapHPath(spec)
    u, ut = path.prepare_links(wl.gauge())
    evals, evecs, rep = path.eigvecs(ut)
    assert rep.nconv == wl.nv
    bs = projectors_for_time(spec, 0) + projectors_for_time(spec, 8)
    config_id = wl.gauge_seed % 65536
    rhs, codes = path.sources(evecs, 0, config_id, bs)
    assert rhs.shape[0] == 64
    sol, reps = path.solve(u, rhs, rhs_block=64)
    coef = path.sinks(evecs, sol)
    torch.cuda.synchronize()
    return dict(wl=wl, spec=spec, u=host(u), ut=host(ut), evecs=host(evecs), bs=bs, config_id=config_id,
                rhs=host(rhs), codes=host(codes), sol=host(sol), reps=reps, coef=host(coef))


def test_stout_links_full(medium):
    uo, uto = oracle_links("medium_16x32")
    assert np.abs(medium["u"] - uo).max() <= 1e-12
    assert np.abs(medium["ut"] - uto).max() <= 1e-12


def test_noise_table_bit_exact(medium):
    wl = medium["wl"]
    ref = onoise.z4_codes(wl.nt, wl.nv, 0, medium["config_id"])
    assert np.array_equal(medium["codes"], ref)


def test_sources_project_to_diluted_noise(medium):
    wl = medium["wl"]
    rho = onoise.z4_values(onoise.z4_codes(wl.nt, wl.nv, 0, medium["config_id"]))
    V = medium["evecs"]                                               # [t][n][V3][3]
    for i, b in enumerate(medium["bs"]):
        y = medium["rhs"][i].reshape(wl.nt, -1, 4, 3)                 # [t][x][alpha][c]
        g4y = np.einsum("ab,txbc->txac", GAMMA[3], y)
        c = np.einsum("tnxc,txac->tan", V.conj(), g4y)
        ref = dl.full_projector_diag(medium["spec"].dil, wl.nt, wl.nv, b) * rho
        assert np.abs(c - ref).max() <= 1e-12, b


def test_solves_true_residual_under_oracle_operator(medium):
    wl = medium["wl"]
    uo, _ = oracle_links("medium_16x32")
    fk = FastK(WilsonClover(uo, wl.m0, wl.csw, wl.xi))
    assert max(r.true_resid for r in medium["reps"]) <= 1e-10
    for i in (0, 21, 42, 63):
        b, x = medium["rhs"][i], medium["sol"][i]
        res = np.linalg.norm(b - fk.apply(x)) / np.linalg.norm(b)
        assert res <= 1e-10, (i, res)


def test_sinks_sampled_definition(medium):
    wl = medium["wl"]
    V = medium["evecs"]
    rng = np.random.default_rng(5)
    for _ in range(8):
        i, t, a, n = rng.integers(64), rng.integers(wl.nt), rng.integers(4), rng.integers(wl.nv)
        x = medium["sol"][i].reshape(wl.nt, -1, 4, 3)[t, :, a, :]
        ref = np.sum(V[t, n].conj() * x)
        assert abs(medium["coef"][i, t, a, n] - ref) <= 1e-12 * max(abs(ref), np.abs(medium["coef"][i]).max())


@pytest.fixture(scope="module")
def medium_lines():
    """Synthetic lines at the medium workload's size (16^3 x 32, N_v = 32, the 32 projectors of
    (TF, SF, LI8) whose time support holds t0 = 8): random orthonormal eigenvectors per slice,
    seeded random sink coefficients, the oracle's noise for ids 0..3.  Both sides take these
    inputs; the oracle builds site fields from them and contracts in site space."""
    from oracle import laph as olaph
    wl = synth.WORKLOADS["medium_16x32"]
    dil = (wl.dil_time, wl.dil_spin, wl.dil_laph)
    t0 = 8
    nT, nS, nL = dl.counts(dil, wl.nt, wl.nv)
    bs = [(bT * nS + bS) * nL + bL for bT in range(nT) if dl.projector_diag(dil[0][0], dil[0][1], wl.nt, bT)[t0]
          for bS in range(nS) for bL in range(nL)]
    v3 = wl.ns ** 3
    g = synth.random_complex((wl.nt, 3 * v3, wl.nv), seed=71)
    V = np.stack([np.linalg.qr(g[t])[0].T for t in range(wl.nt)]).reshape(wl.nt, wl.nv, v3, 3)
    config_id = wl.gauge_seed % 65536
    lines = []
    for k in range(4):
        coef = synth.random_complex((len(bs), wl.nt, 4, wl.nv), seed=80 + k)
        codes = onoise.z4_codes(wl.nt, wl.nv, k, config_id)
        rho = onoise.z4_values(codes)
        line = olaph.Line.__new__(olaph.Line)
        line.bs = list(bs)
        line.varrho = np.stack([olaph.source(V, rho, dil, b) for b in bs])
        # site fields sum_n V(t,n,x,c) coef(t,alpha,n), one matrix product per slice
        vm = V.reshape(wl.nt, wl.nv, 3 * v3)
        phi = np.einsum("btan,tnk->btak", coef, vm, optimize=True).reshape(len(bs), wl.nt, 4, v3, 3)
        line.varphi = phi.transpose(0, 1, 3, 2, 4).reshape(len(bs), wl.nt, wl.ns, wl.ns, wl.ns, 4, 3)
        lines.append((coef, codes, line))
    return wl, dil, t0, bs, lines


@pytest.mark.parametrize("channel", ["pion", "pipi"])
def test_correlators_medium_size_vs_oracle(medium_lines, channel):
    """correlate() at the medium size on synthetic lines against the oracle's site-space
    contraction (Eq. (mesoncorr); I = 2 pi pi as D - X)                   1e-10 (floored)"""
    import torch
    from oracle import laph as olaph
    L = lib()
    wl, dil, t0, bs, lines = medium_lines
    n = 4 if channel == "pipi" else 2
    ch = {"pion": L.CH_PION, "rho": L.CH_RHO, "pipi": L.CH_PIPI_I2}[channel]
    corr = empty((wl.nt,), torch.complex128)
    L.correlate(context(), L.lattice(wl.ns, wl.nt, wl.xi), ch, t0, wl.nv, L.dilution(*dil), bs,
                [dev(c) for c, _, _ in lines[:n]], [dev(k) for _, k, _ in lines[:n]], corr)
    ol = [ln for _, _, ln in lines[:n]]
    ref = olaph.pipi_i2(*ol, t0) if channel == "pipi" else olaph.meson_connected(ol[0], ol[1], t0, channel)
    got = host(corr)
    floor = 1e-3 * np.abs(ref).max()
    assert np.abs(ref).max() > 0
    assert np.all(np.abs(got - ref) <= 1e-10 * np.maximum(np.abs(ref), floor))
