"""GPU parity tests through the C ABI: gauge preparation, the Wilson-clover
matrix, solves, sources, sinks and correlators against the CPU oracle.

Tolerances (floating point, FP64 paths; derivations in the design notes):
  stout-smeared links          |dU| <= 1e-12      (different exp algorithms, O(1) entries)
  K applied to a field         rel <= 1e-12       (same arithmetic, different summation order)
  solves                       FP64 true residual <= 1e-10 (the method's target), and
                               ||x - x_LU|| / ||x_LU|| <= 1e-8 (residual times a condition number < 100)
  sources                      abs <= 1e-13       (sums of +-v, +-iv)
  sink coefficients            rel <= 1e-12
  correlators (same noise)     |dC(t)| <= 1e-8 max(|C(t)|, 1e-3 max|C|)
Z4 noise codes are compared bit for bit.
"""
import numpy as np
import pytest

import synth
from oracle import gauge, laph as olaph, laplacian, noise as onoise
from oracle import dilution as dl
from oracle.dirac import WilsonClover
from oracle.fast import FastK
from oracle.pipeline import OraclePath
from tests.gpu_util import context, dev, empty, host, lib, rel_err, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def corr_close(gpu, ref, tol=1e-8):
    gpu, ref = np.asarray(gpu), np.asarray(ref)
    floor = 1e-3 * np.abs(ref).max()
    return bool(np.all(np.abs(gpu - ref) <= tol * np.maximum(np.abs(ref), floor)))


@pytest.mark.parametrize("ns,nt,spatial", [(4, 4, False), (4, 6, True), (6, 4, False)])
def test_stout_parity(ns, nt, spatial):
    import torch
    L = lib()
    u0 = synth.random_su3_field(ns, nt, seed=100 + ns + nt)
    ref = gauge.stout(u0, 0.1, 3, spatial_only=spatial)
    d = dev(u0)
    L.laph_stout_smear(context(), L.lattice(ns, nt, 3.5), d, 0.1, 3, int(spatial))
    got = host(d)
    assert np.abs(got - ref).max() < 1e-12
    # host buffers through the same entry point
    h = np.ascontiguousarray(u0.copy())
    L.laph_stout_smear(context(), L.lattice(ns, nt, 3.5), h, 0.1, 3, int(spatial))
    assert np.abs(h - ref).max() < 1e-12


@pytest.mark.parametrize("ns,nt,nrhs", [(4, 8, 1), (4, 4, 3), (6, 4, 2), (8, 8, 1)])
def test_dirac_apply_parity(ns, nt, nrhs):
    L = lib()
    u = gauge.stout(synth.random_su3_field(ns, nt, seed=7 + ns), 0.1, 2, spatial_only=False)
    wc = WilsonClover(u, -0.05, 1.0, 3.5)
    psi = synth.random_spinor(ns, nt, seed=3, nrhs=nrhs)
    ref = wc.apply(psi)
    out = empty(psi.shape, dev(psi).dtype)
    L.laph_dirac_apply(context(), L.lattice(ns, nt, 3.5), dev(u), -0.05, 1.0, dev(psi), out, nrhs)
    assert rel_err(host(out), ref) < 1e-12


@pytest.fixture(scope="module")
def tiny():
    wl = synth.WORKLOADS["tiny_4x8"]
    return OraclePath(wl)


@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_solve_vs_dense_lu(tiny, mode):
    L = lib()
    wl = tiny.wl
    b = synth.random_spinor(wl.ns, wl.nt, seed=55, nrhs=5)
    x_lu, _ = tiny.solve(b, "lu")
    sol = empty(b.shape, dev(b).dtype)
    m = L.PLAIN_FP64 if mode == "plain" else L.MIXED_FP32
    prm = L.solver_params(tol=1e-10, mode=m, rhs_block=2 if mode == "plain" else 5)
    reps = L.dirac_solve_batch(context(), L.lattice(wl.ns, wl.nt, wl.xi), dev(tiny.u), wl.m0, wl.csw, dev(b), sol,
                               5, prm)
    x = host(sol)
    fk = FastK(tiny.K)
    for i in range(5):
        assert reps[i].status == 0 and reps[i].true_resid <= 1e-10
        res = np.linalg.norm(b[i] - fk.apply(x[i])) / np.linalg.norm(b[i])
        assert res <= 1.05e-10
        assert np.linalg.norm(x[i] - x_lu[i]) / np.linalg.norm(x_lu[i]) < 1e-8
        assert reps[i].iters > 0


@pytest.mark.parametrize("nrhs,block", [(32, 32), (40, 32)])
def test_solve_bf16_vs_dense_lu(tiny, nrhs, block):
    """LAPH_SOLVE_MIXED_BF16: FP64 defect correction around the BF16-stored inner BiCGStab.  The
    FP64 true residual decides convergence, so the solutions meet the same bounds as the other
    modes (residual <= 1e-10, LU distance <= 1e-8).  40 sources in blocks of 32: the tail block of
    8 runs the FP32 inner solver."""
    L = lib()
    wl = tiny.wl
    b = synth.random_spinor(wl.ns, wl.nt, seed=58, nrhs=nrhs)
    x_lu, _ = tiny.solve(b, "lu")
    sol = empty(b.shape, dev(b).dtype)
    prm = L.solver_params(tol=1e-10, mode=L.MIXED_BF16, rhs_block=block)
    reps = L.dirac_solve_batch(context(), L.lattice(wl.ns, wl.nt, wl.xi), dev(tiny.u), wl.m0, wl.csw, dev(b), sol,
                               nrhs, prm)
    x = host(sol)
    fk = FastK(tiny.K)
    for i in range(nrhs):
        assert reps[i].status == 0 and reps[i].true_resid <= 1e-10 and reps[i].fallback_used == 0
        res = np.linalg.norm(b[i] - fk.apply(x[i])) / np.linalg.norm(b[i])
        assert res <= 1.05e-10
        assert np.linalg.norm(x[i] - x_lu[i]) / np.linalg.norm(x_lu[i]) < 1e-8


@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_solve_cg_fallback(tiny, mode):
    """A Krylov budget far too small for BiCGStab (a host-side injected failure) hands every
    right-hand side to the FP64 CG solve of the normal equations (Sec. IV), which must still
    meet the tolerance; without the fallback the call reports non-convergence."""
    L = lib()
    wl = tiny.wl
    b = synth.random_spinor(wl.ns, wl.nt, seed=57, nrhs=3)
    x_lu, _ = tiny.solve(b, "lu")
    m = L.PLAIN_FP64 if mode == "plain" else L.MIXED_FP32
    lat = L.lattice(wl.ns, wl.nt, wl.xi)
    sol = empty(b.shape, dev(b).dtype)
    reps = L.dirac_solve_batch(context(), lat, dev(tiny.u), wl.m0, wl.csw, dev(b), sol, 3,
                               L.solver_params(tol=1e-10, mode=m, maxiter=10, fallback=1))
    x = host(sol)
    for i in range(3):
        assert reps[i].fallback_used == 1 and reps[i].status == 0
        assert reps[i].true_resid <= 1e-10
        assert np.linalg.norm(x[i] - x_lu[i]) / np.linalg.norm(x_lu[i]) < 1e-8
    reps = L.dirac_solve_batch(context(), lat, dev(tiny.u), wl.m0, wl.csw, dev(b), sol, 3,
                               L.solver_params(tol=1e-10, mode=m, maxiter=10, fallback=0), allow_not_converged=True)
    assert all(r.fallback_used == 0 and r.status == L.LAPH_ERR_NOT_CONVERGED for r in reps)


def test_solve_host_buffers_and_zero_rhs(tiny):
    L = lib()
    wl = tiny.wl
    b = synth.random_spinor(wl.ns, wl.nt, seed=56, nrhs=3)
    b[1] = 0.0
    sol = np.zeros_like(b)
    reps = L.dirac_solve_batch(context(), L.lattice(wl.ns, wl.nt, wl.xi), np.ascontiguousarray(tiny.u), wl.m0, wl.csw,
                               b, sol, 3, L.solver_params(mode=L.MIXED_FP32))
    assert np.all(sol[1] == 0.0)
    x_lu, _ = tiny.solve(b, "lu")
    for i in (0, 2):
        assert np.linalg.norm(sol[i] - x_lu[i]) / np.linalg.norm(x_lu[i]) < 1e-8
        assert reps[i].true_resid <= 1e-10


@pytest.mark.parametrize("dil", [((1, 0), (1, 0), (1, 0)), ((1, 0), (1, 0), (3, 2)), ((3, 2), (0, 0), (2, 4)),
                                 ((2, 4), (3, 2), (1, 0))])
def test_sources_and_noise(tiny, dil):
    L = lib()
    wl = tiny.wl
    nt, nv = wl.nt, wl.nv
    nT, nS, nL = dl.counts(dil, nt, nv)
    bs = list(range(0, nT * nS * nL, max(1, (nT * nS * nL) // 7)))
    rhs = empty((len(bs), nt, wl.ns, wl.ns, wl.ns, 4, 3), dev(tiny.evecs).dtype)
    import torch
    codes = torch.empty((nt, 4, nv), dtype=torch.uint8, device="cuda")
    L.laph_make_sources(context(), L.lattice(wl.ns, wl.nt, wl.xi), dev(tiny.evecs), nv, 3, wl.config_id,
                        L.dilution(*dil), bs, rhs, codes)
    assert np.array_equal(host(codes), onoise.z4_codes(nt, nv, 3, wl.config_id))
    rho = onoise.z4_values(onoise.z4_codes(nt, nv, 3, wl.config_id))
    ref = np.stack([olaph.dirac_rhs(tiny.evecs, rho, dil, b) for b in bs])
    assert np.abs(host(rhs) - ref).max() < 1e-13
    # the projector list may also live in device memory
    rhs2 = torch.empty_like(rhs)
    L.laph_make_sources(context(), L.lattice(wl.ns, wl.nt, wl.xi), dev(tiny.evecs), nv, 3, wl.config_id,
                        L.dilution(*dil), torch.tensor(bs, dtype=torch.int32, device="cuda"), rhs2, codes)
    assert torch.equal(rhs2, rhs)


def test_sinks_parity(tiny):
    L = lib()
    wl = tiny.wl
    x = synth.random_spinor(wl.ns, wl.nt, seed=9, nrhs=6)
    coef = empty((6, wl.nt, 4, wl.nv), dev(x).dtype)
    L.laph_sinks(context(), L.lattice(wl.ns, wl.nt, wl.xi), dev(tiny.evecs), wl.nv, dev(x), 6, coef)
    assert rel_err(host(coef), olaph.sinks(tiny.evecs, x)) < 1e-12


def test_dilution_rejects_bad_J(tiny):
    L = lib()
    wl = tiny.wl
    rhs = empty((1, wl.nt, wl.ns, wl.ns, wl.ns, 4, 3), dev(tiny.evecs).dtype)
    with pytest.raises(L.LaphError) as e:
        L.laph_make_sources(context(), L.lattice(wl.ns, wl.nt, wl.xi), dev(tiny.evecs), wl.nv, 0, 0,
                            L.dilution((3, 3), (1, 0), (1, 0)), [0], rhs)
    assert e.value.code == L.LAPH_ERR_ARG


def _gpu_line(L, tiny, noise_id, bs, dil):
    """Sources, solves and sinks of one quark line on the GPU; returns (coef, codes)."""
    import torch
    wl = tiny.wl
    lat = L.lattice(wl.ns, wl.nt, wl.xi)
    rhs = empty((len(bs), wl.nt, wl.ns, wl.ns, wl.ns, 4, 3), torch.complex128)
    codes = torch.empty((wl.nt, 4, wl.nv), dtype=torch.uint8, device="cuda")
    L.laph_make_sources(context(), lat, dev(tiny.evecs), wl.nv, noise_id, wl.config_id, L.dilution(*dil), bs, rhs, codes)
    sol = torch.empty_like(rhs)
    L.dirac_solve_batch(context(), lat, dev(tiny.u), wl.m0, wl.csw, rhs, sol, len(bs),
                        L.solver_params(mode=L.MIXED_FP32, tol=1e-11))
    coef = empty((len(bs), wl.nt, 4, wl.nv), torch.complex128)
    L.laph_sinks(context(), lat, dev(tiny.evecs), wl.nv, sol, len(bs), coef)
    return coef, codes


@pytest.mark.parametrize("channel", ["pion", "rho", "scalar", "pipi"])
def test_correlators_full_dilution_vs_exact(tiny, channel):
    """Full dilution makes the estimate exact: GPU correlators equal the exact
    distillation correlators of the oracle (dense LU)."""
    import torch
    L = lib()
    wl = tiny.wl
    G = tiny.exact_G() if not hasattr(tiny, "_G") else tiny._G
    tiny._G = G
    t0 = 3
    bs = tiny.projectors_for_time(t0)
    nl = 4 if channel == "pipi" else 2
    lines = [_gpu_line(L, tiny, s, bs, tiny.dil) for s in range(nl)]
    corr = empty((wl.nt,), torch.complex128)
    ch = {"pion": L.CH_PION, "rho": L.CH_RHO, "scalar": L.CH_SCALAR, "pipi": L.CH_PIPI_I2}[channel]
    L.correlate(context(), L.lattice(wl.ns, wl.nt, wl.xi), ch, t0, wl.nv, L.dilution(*tiny.dil), bs,
                [c for c, _ in lines], [n for _, n in lines], corr)
    ref = olaph.exact_pipi_i2(G, t0) if channel == "pipi" else olaph.exact_meson_connected(G, t0, channel)
    assert corr_close(host(corr), ref, 1e-8)


@pytest.mark.parametrize("channel", ["pion", "pipi"])
def test_correlators_partial_dilution_same_noise(tiny, channel):
    """Partial dilution: the GPU coefficient-space contraction equals the
    oracle's site-space contraction for the same noises and solutions."""
    import torch
    L = lib()
    wl = tiny.wl
    dil = ((1, 0), (1, 0), (3, 2))
    t0 = 5
    nT, nS, nL = dl.counts(dil, wl.nt, wl.nv)
    bs = [(t0 * nS + bS) * nL + bL for bS in range(nS) for bL in range(nL)]
    nl = 4 if channel == "pipi" else 2
    gl = [_gpu_line(L, tiny, 10 + s, bs, dil) for s in range(nl)]
    corr = empty((wl.nt,), torch.complex128)
    ch = L.CH_PIPI_I2 if channel == "pipi" else L.CH_PION
    L.correlate(context(), L.lattice(wl.ns, wl.nt, wl.xi), ch, t0, wl.nv, L.dilution(*dil), bs,
                [c for c, _ in gl], [n for _, n in gl], corr)
    saved = tiny.dil
    tiny.dil = dil
    try:
        ol = [tiny.line(10 + s, bs, "lu")[0] for s in range(nl)]
    finally:
        tiny.dil = saved
    ref = olaph.pipi_i2(*ol, t0) if channel == "pipi" else olaph.meson_connected(ol[0], ol[1], t0, "pion")
    assert corr_close(host(corr), ref, 1e-8)


def test_empty_inputs(tiny):
    """Zero right-hand sides or projectors are valid calls that write nothing; zero-sized
    correlator inputs and hops are rejected as argument errors."""
    import torch
    L = lib()
    wl = tiny.wl
    lat = L.lattice(wl.ns, wl.nt, wl.xi)
    u = dev(tiny.u)
    sentinel = torch.full((1, wl.nt, wl.ns, wl.ns, wl.ns, 4, 3), 7.0 + 7.0j, dtype=torch.complex128, device="cuda")
    reps = L.dirac_solve_batch(context(), lat, u, wl.m0, wl.csw, sentinel, sentinel, 0, L.solver_params())
    assert reps == [] and bool((sentinel == 7.0 + 7.0j).all())
    evecs = dev(tiny.evecs)
    coef = torch.full((1, wl.nt, 4, wl.nv), 7.0, dtype=torch.complex128, device="cuda")
    L.laph_sinks(context(), lat, evecs, wl.nv, sentinel, 0, coef)
    assert bool((coef == 7.0).all())
    codes = torch.zeros((wl.nt, 4, wl.nv), dtype=torch.uint8, device="cuda")
    L.laph_make_sources(context(), lat, evecs, wl.nv, 0, 1, L.dilution(*tiny.dil), [], sentinel, codes)
    assert bool((sentinel == 7.0 + 7.0j).all())
    vh = wl.ns ** 3 * wl.nt // 2
    x = torch.zeros((vh, 12, 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(L.LaphError) as e:
        L.laph_dslash_eo(context(), lat, u, wl.m0, wl.csw, 0, L.HOP_CLOVINV, L.PREC_FP64, x, None, x, 0)
    assert e.value.code == L.LAPH_ERR_ARG


@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_solve_nan_rhs_is_reported(tiny, mode):
    """A right-hand side carrying a NaN (a host-side injected fault) is reported as not
    converged with a NaN true residual; the other right-hand sides of its block still reach
    the tolerance."""
    L = lib()
    wl = tiny.wl
    b = synth.random_spinor(wl.ns, wl.nt, seed=58, nrhs=3)
    b[1, 0, 0, 0, 0, 0, 0] = np.nan
    sol = empty(b.shape, dev(b).dtype)
    m = L.PLAIN_FP64 if mode == "plain" else L.MIXED_FP32
    reps = L.dirac_solve_batch(context(), L.lattice(wl.ns, wl.nt, wl.xi), dev(tiny.u), wl.m0, wl.csw, dev(b), sol,
                               3, L.solver_params(tol=1e-10, mode=m, rhs_block=3), allow_not_converged=True)
    assert reps[1].status == L.LAPH_ERR_NOT_CONVERGED and np.isnan(reps[1].true_resid)
    x = host(sol)
    x_lu, _ = tiny.solve(b[[0, 2]], "lu")
    for i, k in enumerate((0, 2)):
        assert reps[k].status == 0 and reps[k].true_resid <= 1e-10
        assert np.linalg.norm(x[k] - x_lu[i]) / np.linalg.norm(x_lu[i]) < 1e-8
