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
    for parity, mode, prec, z in ((2, 0, 0, None), (0, 3, 0, None), (0, 0, 2, None), (0, 1, 0, None)):
        with pytest.raises(L.LaphError) as e:
            L.laph_dslash_eo(context(), lat, dev(u), M0, CSW, parity, mode, prec, x, z, out, 2)
        assert e.value.code == L.LAPH_ERR_ARG
