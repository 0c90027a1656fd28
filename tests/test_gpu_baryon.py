"""GPU parity of the baryon pieces (Sec. III three-quark operators, Eq. (baryonfunc),
Eq. (baryoncorr)) against the oracle, on the 4^3 x 8 workload (N_v = 8) with the oracle's
eigenvectors fed to both sides:

  laph_baryon_tensor   T_p(t)[n1 n2 n3] against oracle.baryon.lapH_tensor: every entry within
                       1e-12 of its Hadamard scale sum_x |V_n1(x)| |V_n2(x)| |V_n3(x)|; also
                       random (not orthonormal) vectors with N_v = 21 and 130 (thread strides)
  correlate_baryon     full dilution: the exact three-quark correlator from dense LU
                       (oracle.baryon.exact_baryon_correlator) for flavours uds, uud, uuu and
                       random spin tensors, at p = 0 and p != 0                     1e-8 (floored)
  correlate_baryon     partial dilution (spin block 2, LapH interlace 4): the oracle's
                       site-space baryon_correlator of the same noises and dense-LU lines,
                       with sink and source flavour labels in different orders     1e-8 (floored)

The floored relative bound: |d| <= tol * max(|ref|, 1e-3 max|ref|)."""
import numpy as np
import pytest

import synth
from oracle import baryon as ob
from oracle.pipeline import OraclePath
from tests.gpu_util import context, dev, empty, host, lib, requires_gpu
from tests.test_gpu_mesonx import _gpu_line, close

pytestmark = [pytest.mark.gpu, requires_gpu]


@pytest.fixture(scope="module")
def tiny():
    path = OraclePath(synth.WORKLOADS["tiny_4x8"])
    path._G = path.exact_G()
    return path


def _c_tensor(seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((4, 4, 4)) + 1j * rng.standard_normal((4, 4, 4))


def _hadamard_scale(V):
    """sum_x |V_n1(x)| |V_n2(x)| |V_n3(x)| (colour norms): |eps_abc a_a b_b c_c| <= |a| |b| |c|."""
    nrm = np.linalg.norm(V, axis=-1)
    return np.einsum("tix,tjx,tkx->tijk", nrm, nrm, nrm)


def _tensor(L, ns, nt, V, nv, mom):
    import torch
    T = empty((nt, nv, nv, nv), torch.complex128)
    L.laph_baryon_tensor(context(), L.lattice(ns, nt, 3.5), dev(V), nv, mom, T)
    return T


@pytest.mark.parametrize("mom", [(0, 0, 0), (1, 0, 0), (1, -1, 2)])
def test_baryon_tensor(tiny, mom):
    L = lib()
    wl = tiny.wl
    got = host(_tensor(L, wl.ns, wl.nt, tiny.evecs, wl.nv, mom))
    ref = ob.lapH_tensor(tiny.evecs, None if mom == (0, 0, 0) else mom)
    assert np.all(np.abs(got - ref) <= 1e-12 * _hadamard_scale(tiny.evecs)), mom
    assert np.abs(got + got.transpose(0, 2, 1, 3)).max() <= 1e-13 * np.abs(got).max()


@pytest.mark.parametrize("ns,nt,nv", [(6, 2, 21), (4, 2, 130)])
def test_baryon_tensor_ragged(ns, nt, nv):
    """Random vectors: 21 on 6^3 slices (216 sites = one full chunk of 128 and a ragged one of 88)
    and 130 on 4^3 slices (n3 beyond the 128 threads of a block, one ragged chunk of 64)."""
    L = lib()
    V = synth.random_complex((nt, nv, ns ** 3, 3), seed=37 + nv)
    got = host(_tensor(L, ns, nt, V, nv, (0, 2, 1)))
    ref = ob.lapH_tensor(V, (0, 2, 1))
    assert np.all(np.abs(got - ref) <= 1e-12 * _hadamard_scale(V))


@pytest.fixture(scope="module")
def lines3(tiny):
    L = lib()
    t0 = 2
    bs = tiny.projectors_for_time(t0)
    return t0, bs, [_gpu_line(L, tiny, 20 + k, bs, tiny.dil) for k in range(3)]


def _correlate(L, tiny, t0, dil, bs, lines, c_snk, c_src, fs, fr, mom):
    import torch
    wl = tiny.wl
    T = _tensor(L, wl.ns, wl.nt, tiny.evecs, wl.nv, (0, 0, 0) if mom is None else mom)
    corr = empty((wl.nt,), torch.complex128)
    L.correlate_baryon(context(), L.lattice(wl.ns, wl.nt, wl.xi), t0, wl.nv, L.dilution(*dil), bs, c_snk, c_src,
                       fs, fr, [c for c, _ in lines], [n for _, n in lines], T, corr)
    return host(corr)


@pytest.mark.parametrize("flav", ["uds", "uud", "uuu"])
@pytest.mark.parametrize("mom", [None, (1, 0, 0)])
def test_correlate_baryon_full_dilution_vs_exact(tiny, lines3, flav, mom):
    L = lib()
    t0, bs, lines = lines3
    c_snk, c_src = _c_tensor(1), _c_tensor(2)
    f = [ord(ch) for ch in flav]
    got = _correlate(L, tiny, t0, tiny.dil, bs, lines, c_snk, c_src, f, f, mom)
    ref = ob.exact_baryon_correlator(tiny._G, tiny.evecs, t0, c_snk, c_src, tuple(flav), tuple(flav), mom)
    assert np.abs(ref).max() > 1e-8
    assert close(got, ref), flav


@pytest.mark.parametrize("fs,fr", [("uud", "udu"), ("uuu", "uuu")])
def test_correlate_baryon_partial_dilution_vs_oracle(tiny, fs, fr):
    L = lib()
    wl = tiny.wl
    t0, mom = 5, (0, 1, 0)
    dil = ((1, 0), (2, 2), (3, 4))
    saved = tiny.dil
    tiny.dil = dil
    try:
        bs = tiny.projectors_for_time(t0)
        olines = [tiny.line(60 + k, bs, "lu")[0] for k in range(3)]
    finally:
        tiny.dil = saved
    glines = [_gpu_line(L, tiny, 60 + k, bs, dil) for k in range(3)]
    c_snk, c_src = _c_tensor(3), _c_tensor(4)
    got = _correlate(L, tiny, t0, dil, bs, glines, c_snk, c_src, [ord(c) for c in fs], [ord(c) for c in fr], mom)
    ref = ob.baryon_correlator(*olines, t0, c_snk, c_src, tuple(fs), tuple(fr), mom)
    assert len(bs) == 8 and np.abs(ref).max() > 1e-10
    assert close(got, ref)


def test_correlate_baryon_rejects_bad_sizes(tiny):
    import torch
    L = lib()
    wl = tiny.wl
    T = empty((wl.nt, wl.nv, wl.nv, wl.nv), torch.complex128)
    corr = empty((wl.nt,), torch.complex128)
    coef = empty((1, wl.nt, 4, wl.nv), torch.complex128)
    codes = torch.zeros((wl.nt, 4, wl.nv), dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LaphError):
        L.correlate_baryon(context(), L.lattice(wl.ns, wl.nt, wl.xi), wl.nt, wl.nv, L.dilution(*tiny.dil), [0],
                           _c_tensor(1), _c_tensor(2), [1, 2, 3], [1, 2, 3], [coef] * 3, [codes] * 3, T, corr)
