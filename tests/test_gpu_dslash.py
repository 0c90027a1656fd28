"""GPU parity of the even-odd hopping call (laph_dslash_eo) in all three modes, both
precisions and both output parities, against the oracle's K = A + D.

The reference for output parity p, with q = 1 - p, is built from full-lattice fields:
  apply     (K x)_p with x_p = z, x_q = in
  clovinv   A_pp^{-1} (D x)_p with x_p = 0, x_q = in   (A_pp inverted site by site)
  xpay      z - clovinv
Right-hand-side counts cover the register-fed kernel (1, 5, and 96, which is not a power
of two) and the copy-engine-fed kernel (32: one RHS per lane; 64: two per lane; 128: two
per lane with two warps per site), on lattices whose sites do not fill the persistent grid
evenly.

Tolerances: FP64 rel <= 1e-12 (same arithmetic, another summation order).  FP32: the
inputs are rounded to FP32 before the reference sees them, so the error is the kernel's
own FP32 rounding of links, clover and about 100 products per output: rel <= 5e-6 in
norm and every element within 2e-5 of the largest reference element.
"""
import numpy as np
import pytest

import synth
from oracle import gauge
from oracle.dirac import WilsonClover
from tests.gpu_util import context, dev, empty, host, lib, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

M0, CSW, XI = -0.05, 1.0, 3.5


def parity_sites(ns, nt, p):
    """Lexicographic site indices (t, z, y, x order, x fastest) of parity p in cb order."""
    t, z, y, x = np.meshgrid(np.arange(nt), np.arange(ns), np.arange(ns), np.arange(ns), indexing="ij")
    lex = (((t * ns + z) * ns + y) * ns + x).ravel()
    par = ((t + z + y + x) % 2).ravel()
    sel = lex[par == p]
    assert np.all(sel >> 1 == np.arange(sel.size))
    return sel


def to_eo(full, p, ns, nt):
    """[nrhs][t][z][y][x][4][3] -> [cb][12][nrhs]."""
    nr = full.shape[0]
    f = full.reshape(nr, -1, 12)[:, parity_sites(ns, nt, p), :]
    return np.ascontiguousarray(f.transpose(1, 2, 0))


def from_eo(eo, p, ns, nt):
    nr = eo.shape[2]
    full = np.zeros((nr, ns ** 3 * nt, 12), dtype=eo.dtype)
    full[:, parity_sites(ns, nt, p), :] = eo.transpose(2, 0, 1)
    return full.reshape((nr, nt, ns, ns, ns, 4, 3))


@pytest.fixture(scope="module", params=[(4, 8), (6, 4)], ids=["4x8", "6x4"])
def lattice(request):
    ns, nt = request.param
    u = gauge.stout(synth.random_su3_field(ns, nt, seed=71), 0.1, 3, spatial_only=False)
    return ns, nt, u, WilsonClover(u, M0, CSW, XI)


def reference(K, ns, nt, p, mode, xin, zin):
    q = 1 - p
    nr = xin.shape[2]
    if mode == "apply":
        x = from_eo(xin, q, ns, nt) + from_eo(zin, p, ns, nt)
        return to_eo(K.apply(x), p, ns, nt)
    w = to_eo(K.apply_hop(from_eo(xin, q, ns, nt)), p, ns, nt)             # [cb][12][nr]
    a = K.a.reshape(-1, 12, 12)[parity_sites(ns, nt, p)]                    # [cb][12][12]
    y = np.linalg.solve(a, w)
    assert y.shape[2] == nr
    return y if mode == "clovinv" else zin - y


MODES = {"clovinv": 0, "xpay": 1, "apply": 2}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("nr", [1, 5, 32, 64, 96, 128])
def test_hop_parity(lattice, prec, mode, nr):
    import torch
    L = lib()
    ns, nt, u, K = lattice
    vh = ns ** 3 * nt // 2
    rng = np.random.default_rng(1000 + nr)
    cdt = np.complex128 if prec == "fp64" else np.complex64
    xin = (rng.standard_normal((vh, 12, nr)) + 1j * rng.standard_normal((vh, 12, nr))).astype(cdt)
    zin = (rng.standard_normal((vh, 12, nr)) + 1j * rng.standard_normal((vh, 12, nr))).astype(cdt)
    for p in (0, 1):
        out = empty(xin.shape, torch.complex128 if prec == "fp64" else torch.complex64)
        L.laph_dslash_eo(context(), L.lattice(ns, nt, XI), dev(u), M0, CSW, p, MODES[mode],
                         L.PREC_FP64 if prec == "fp64" else L.PREC_FP32, dev(xin),
                         None if mode == "clovinv" else dev(zin), out, nr)
        got = host(out).astype(np.complex128)
        ref = reference(K, ns, nt, p, mode, xin.astype(np.complex128), zin.astype(np.complex128))
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        if prec == "fp64":
            assert rel <= 1e-12, (p, rel)
        else:
            assert rel <= 5e-6, (p, rel)
            assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max(), p


def test_hop_rejects_bad_arguments(lattice):
    import torch
    L = lib()
    ns, nt, u, _ = lattice
    vh = ns ** 3 * nt // 2
    x = torch.zeros((vh, 12, 2), dtype=torch.complex128, device="cuda")
    out = torch.empty_like(x)
    lat = L.lattice(ns, nt, XI)
    for parity, mode, prec, z in ((2, 0, 0, None), (0, 3, 0, None), (0, 0, 3, None), (0, 1, 0, None),
                                  (0, 0, 2, None)):   # the last: BF16 with 2 right-hand sides
        with pytest.raises(L.LaphError) as e:
            L.laph_dslash_eo(context(), lat, dev(u), M0, CSW, parity, mode, prec, x, z, out, 2)
        assert e.value.code == L.LAPH_ERR_ARG


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("nr", [32, 64, 128])
def test_hop_parity_bf16(lattice, mode, nr):
    """BF16-stored spinors (the inner operator of LAPH_SOLVE_MIXED_BF16): the inputs are rounded
    to BF16 before the reference sees them, links, clover and arithmetic are FP32, and the output
    is rounded to BF16 (8 significant bits: unit roundoff 2^-8 per element).  Bound: every
    element within 2^-8 |ref| + 2e-5 max|ref|, and rel <= 3e-3 in norm."""
    import torch
    L = lib()
    ns, nt, u, K = lattice
    vh = ns ** 3 * nt // 2
    rng = np.random.default_rng(2000 + nr)

    def bf(a):
        return torch.from_numpy(a).to(torch.bfloat16).cuda()

    def cplx(t):
        f = t.float().cpu().numpy().astype(np.float64)
        return f[..., 0] + 1j * f[..., 1]

    xb, zb = bf(rng.standard_normal((vh, 12, nr, 2))), bf(rng.standard_normal((vh, 12, nr, 2)))
    xin, zin = cplx(xb), cplx(zb)
    for p in (0, 1):
        out = torch.empty((vh, 12, nr, 2), dtype=torch.bfloat16, device="cuda")
        L.laph_dslash_eo(context(), L.lattice(ns, nt, XI), dev(u), M0, CSW, p, MODES[mode], L.PREC_BF16, xb,
                         None if mode == "clovinv" else zb, out, nr)
        torch.cuda.synchronize()
        got = cplx(out)
        ref = reference(K, ns, nt, p, mode, xin, zin)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 3e-3, p
        assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 2e-5 * np.abs(ref).max()), p


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("mode", ["clovinv", "xpay"])
@pytest.mark.parametrize("nr", [32, 64])
def test_hop_parity_zblocked_order(prec, mode, nr):
    """16^3 x 4: the copy-engine-fed kernel visits the output sites in z-blocks of 8 planes
    (two blocks here; on the 4^3 and 6^3 lattices above the order is lexicographic).  Same
    tolerances as the FP32 and BF16 tests above."""
    import torch
    L = lib()
    ns, nt = 16, 4
    u = gauge.stout(synth.random_su3_field(ns, nt, seed=72), 0.1, 2, spatial_only=False)
    K = WilsonClover(u, M0, CSW, XI)
    vh = ns ** 3 * nt // 2
    rng = np.random.default_rng(3000 + nr)
    shape = (vh, 12, nr, 2)
    if prec == "fp32":
        xt = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
        zt = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
        out = torch.empty(shape, dtype=torch.float32, device="cuda")
    else:
        xt = torch.from_numpy(rng.standard_normal(shape)).to(torch.bfloat16).cuda()
        zt = torch.from_numpy(rng.standard_normal(shape)).to(torch.bfloat16).cuda()
        out = torch.empty(shape, dtype=torch.bfloat16, device="cuda")

    def cplx(t):
        f = t.float().cpu().numpy().astype(np.float64)
        return f[..., 0] + 1j * f[..., 1]

    xin, zin = cplx(xt), cplx(zt)
    for p in (0, 1):
        L.laph_dslash_eo(context(), L.lattice(ns, nt, XI), dev(u), M0, CSW, p, MODES[mode],
                         L.PREC_FP32 if prec == "fp32" else L.PREC_BF16, xt, None if mode == "clovinv" else zt,
                         out, nr)
        torch.cuda.synchronize()
        got = cplx(out)
        ref = reference(K, ns, nt, p, mode, xin, zin)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        if prec == "fp32":
            assert rel <= 5e-6 and np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max(), (p, rel)
        else:
            assert rel <= 3e-3, (p, rel)
            assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 2e-5 * np.abs(ref).max()), p
