"""correlate_noalloc against correlate.

correlate_noalloc serves callers that cannot allocate GPU memory (a caller-
owned pool or arena, memory reserved up front, loops that must not stall on
an allocation): it takes device arrays only and keeps its scratch in a fixed
device array inside the library.  Its correlators must equal those of the
allocating entry point on the same inputs, within the correlator tolerance
used elsewhere (1e-8 relative), on consecutive calls -- the second call
reuses the scratch the first one left behind.  This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

import synth
from tests.gpu_util import context, dev, empty, host, lib, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def _lines(nlines, nb, nt, nv, seed):
    coefs = [synth.random_complex((nb, nt, 4, nv), seed + k) for k in range(nlines)]
    rng = np.random.default_rng(seed + 100)
    codes = [rng.integers(0, 4, size=(nt, 4, nv), dtype=np.uint8) for _ in range(nlines)]
    return coefs, codes


def _close(a, b, tol=1e-8):
    floor = 1e-3 * np.abs(b).max()
    return bool(np.all(np.abs(a - b) <= tol * np.maximum(np.abs(b), floor)))


def _compare_twice(L, channel, nt, nv, dil, t0, bs, seeds=(11, 23)):
    import torch
    ch = {"pion": L.CH_PION, "rho": L.CH_RHO, "scalar": L.CH_SCALAR, "pipi": L.CH_PIPI_I2}[channel]
    nlines = 4 if channel == "pipi" else 2
    lat = L.lattice(4, nt, 3.5)
    for call, seed in enumerate(seeds):
        coefs, codes = _lines(nlines, len(bs), nt, nv, seed)
        dc = [dev(c) for c in coefs]
        dn = [dev(c) for c in codes]
        ref = empty((nt,), torch.complex128)
        L.correlate(context(), lat, ch, t0, nv, L.dilution(*dil), bs, dc, dn, ref)
        got = empty((nt,), torch.complex128)
        L.correlate_noalloc(lat, ch, t0, nv, L.dilution(*dil), bs, dc, dn, got)
        assert _close(host(got), host(ref)), f"call {call}"


@pytest.mark.parametrize("channel", ["pion", "rho", "scalar", "pipi"])
def test_noalloc_matches_correlate_twice(channel):
    L = lib()
    nt, nv, t0 = 8, 16, 3
    dil = ((1, 0), (1, 0), (3, 4))                       # (TF, SF, LI4)
    bs = [(t0 * 4 + bS) * 4 + bL for bS in range(4) for bL in range(4)]
    _compare_twice(L, channel, nt, nv, dil, t0, bs)


@pytest.mark.parametrize("channel", ["pion", "scalar"])
def test_noalloc_block_dilution_many_projectors(channel):
    """Block time and block LapH dilution (type 2), 128 projectors: the kernels' 256-thread
    shape, and masks of the block type, against correlate()."""
    L = lib()
    nt, nv, t0 = 16, 32, 5
    dil = ((2, 2), (1, 0), (2, 16))                      # (TB2, SF, LB16): 2 x 4 x 16 projectors
    _compare_twice(L, channel, nt, nv, dil, t0, list(range(128)))


def test_noalloc_scratch_boundary():
    """A meson channel needs one sink/source meson-function pair: nt = 60 with 128 projectors
    fits the 16 MiB array (and matches correlate()), nt = 62 does not and is rejected."""
    import torch
    L = lib()
    nv, t0 = 16, 7
    dil = ((1, 0), (1, 0), (3, 4))
    bs = list(range(128))
    _compare_twice(L, "pion", 60, nv, dil, t0, bs, seeds=(31,))
    nt = 62
    c = empty((128, nt, 4, nv), torch.complex128)
    n = torch.zeros((nt, 4, nv), dtype=torch.uint8, device="cuda")
    o = empty((nt,), torch.complex128)
    with pytest.raises(L.LaphError) as e:
        L.correlate_noalloc(L.lattice(4, nt, 3.5), L.CH_PION, t0, nv, L.dilution(*dil), bs, [c, c], [n, n], o)
    assert e.value.code == L.LAPH_ERR_ARG and "bytes of scratch" in str(e.value)


def test_noalloc_arrays_on_two_devices_rejected():
    """Line arrays on one GPU and the output on another: rejected before any launch."""
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    L = lib()
    nt, nv = 8, 16
    dil = ((1, 0), (1, 0), (3, 4))
    bs = list(range(16))
    coefs, codes = _lines(2, 16, nt, nv, 5)
    dc = [dev(c) for c in coefs]
    dn = [dev(c) for c in codes]
    other = torch.empty((nt,), dtype=torch.complex128, device="cuda:1")
    with pytest.raises(L.LaphError) as e:
        L.correlate_noalloc(L.lattice(4, nt, 3.5), L.CH_PION, 0, nv, L.dilution(*dil), bs, dc, dn, other)
    assert e.value.code == L.LAPH_ERR_ARG
    s1 = torch.cuda.Stream(device="cuda:1")
    out = empty((nt,), torch.complex128)
    with pytest.raises(L.LaphError) as e:
        L.correlate_noalloc(L.lattice(4, nt, 3.5), L.CH_PION, 0, nv, L.dilution(*dil), bs, dc, dn, out, stream=s1)
    assert e.value.code == L.LAPH_ERR_ARG


def test_noalloc_rejects_host_arrays_and_oversize():
    import torch
    L = lib()
    nt, nv = 8, 16
    dil = ((1, 0), (1, 0), (3, 4))
    bs = list(range(16))
    coefs, codes = _lines(2, 16, nt, nv, 5)
    out = empty((nt,), torch.complex128)
    with pytest.raises(L.LaphError) as e:
        L.correlate_noalloc(L.lattice(4, nt, 3.5), L.CH_PION, 0, nv, L.dilution(*dil), bs, coefs, codes, out)
    assert e.value.code == L.LAPH_ERR_ARG
    # nt nb^2 complex doubles above 16 MiB: nt = 128, nb = 256 (full time, spin, LapH-64 at one t0)
    big_nt, big_nv = 128, 64
    bdil = ((1, 0), (1, 0), (1, 0))
    bbs = list(range(256))
    c = empty((256, big_nt, 4, big_nv), torch.complex128)
    n = torch.zeros((big_nt, 4, big_nv), dtype=torch.uint8, device="cuda")
    o = empty((big_nt,), torch.complex128)
    with pytest.raises(L.LaphError) as e:
        L.correlate_noalloc(L.lattice(4, big_nt, 3.5), L.CH_PION, 0, big_nv, L.dilution(*bdil), bbs, [c, c], [n, n], o)
    assert e.value.code == L.LAPH_ERR_ARG and "bytes of scratch" in str(e.value)
