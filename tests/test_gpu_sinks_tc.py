"""The sink coefficients of laph_sinks, computed on the tensor cores from exact integer slices,
against their definition coef[i][t][a][n] = sum_{x,c} conj(V[t][n][x][c]) X[i][t][x][a][c]
(oracle.laph.sinks, FP64).

Bound: every entry is scaled by a power of two taken from the largest entry of its row (V) or
column (X), at most twice that entry, and truncated to 48 bits; with the digit pairs the kernel
leaves out (a tenth of that), a coefficient's error is at most 2^-46 (max|V| sum|X| + max|X| sum|V|)
over its own product, plus FP64 sums; for entries of one order of magnitude that
is below 1e-12 of sum_{x,c} |V| |X|, the Cauchy scale of the sum.  Shapes exercise the tile
edges: N_v = 40 (80 of a tile's 128 rows), 5 right-hand sides (20 of 64 columns), K = 3 * 6^3 =
648 complex (1296 reals, not a multiple of the 32-real sub-chunk); also an all-zero column, an
all-zero eigenvector row, entries spread over 30 orders of magnitude (against the first bound),
and a right-hand side carrying a NaN, which gives NaN coefficients in its own columns only."""
import numpy as np
import pytest

import synth
from oracle import laph as olaph
from tests.gpu_util import context, dev, empty, host, lib, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def _check(ns, nt, nv, nrhs, V, X):
    L = lib()
    coef = empty((nrhs, nt, 4, nv), dev(X).dtype)
    L.laph_sinks(context(), L.lattice(ns, nt, 3.5), dev(V), nv, dev(X), nrhs, coef)
    got = host(coef)
    ref = olaph.sinks(V, X)
    # Cauchy scale of each coefficient: sum_{x,c} |V| |X|
    Xa = np.abs(X).reshape(nrhs, nt, ns ** 3, 4, 3)
    scale = np.einsum("tnxc,itxac->itan", np.abs(V), Xa)
    return got, ref, scale


@pytest.mark.parametrize("spread", [1.0, 30.0])
def test_sinks_tensor_core_ragged_shapes_and_magnitudes(spread):
    ns, nt, nv, nrhs = 6, 4, 40, 5
    rng = np.random.default_rng(17)
    V = synth.random_complex((nt, nv, ns ** 3, 3), seed=18)
    V *= 10.0 ** rng.uniform(-spread / 2, spread / 2, size=V.shape)
    V[1, 7] = 0.0                                            # an all-zero eigenvector row
    X = synth.random_spinor(ns, nt, seed=19, nrhs=nrhs)
    X *= 10.0 ** rng.uniform(-spread / 4, spread / 4, size=X.shape)
    X[3, :, :, :, :, 2, :] = 0.0                             # an all-zero column (i = 3, spin 2)
    got, ref, scale = _check(ns, nt, nv, nrhs, V, X)
    va = np.abs(V).reshape(nt, nv, -1)
    xa = np.abs(X).reshape(nrhs, nt, ns ** 3, 4, 3).transpose(0, 1, 3, 2, 4).reshape(nrhs, nt, 4, -1)
    bound = 2.0 ** -46 * (va.max(-1)[None, :, None, :] * xa.sum(-1)[..., None] +
                          xa.max(-1)[..., None] * va.sum(-1)[None, :, None, :]) + 1e-15 * scale
    assert np.all(np.abs(got - ref) <= bound + 1e-300)
    if spread == 1.0:
        assert np.all(np.abs(got - ref) <= 1e-12 * scale + 1e-300)
    assert np.all(got[3, :, 2, :] == 0.0) and np.all(got[:, 1, :, 7] == 0.0)


def test_sinks_tensor_core_unit_sources():
    """Sinks of eigenvector sources x = V_n (spin a) are unit vectors (the pin of the oracle's
    sinks), here through the tensor-core path on 8^3 x 4 with 64 eigenvectors (a full row tile)."""
    ns, nt, nv = 8, 4, 64
    rng = np.random.default_rng(20)
    q, _ = np.linalg.qr(rng.standard_normal((3 * ns ** 3, nv)) + 1j * rng.standard_normal((3 * ns ** 3, nv)))
    V = np.broadcast_to(q.T.reshape(1, nv, ns ** 3, 3), (nt, nv, ns ** 3, 3)).copy()
    nrhs = 16
    X = np.zeros((nrhs, nt, ns, ns, ns, 4, 3), dtype=complex)
    for i in range(nrhs):
        n, a = (5 * i) % nv, i % 4
        X[i, :, :, :, :, a, :] = V[:, n].reshape(nt, ns, ns, ns, 3)
    got, ref, scale = _check(ns, nt, nv, nrhs, V, X)
    for i in range(nrhs):
        n, a = (5 * i) % nv, i % 4
        e = np.zeros((nt, 4, nv), dtype=complex)
        e[:, a, n] = 1.0
        assert np.abs(got[i] - e).max() <= 2e-13   # 2^-46 (max|V| sum|X| + max|X| sum|V|) ~ 1.3e-13 here


def test_sinks_tensor_core_nan_stays_in_its_columns():
    ns, nt, nv, nrhs = 4, 4, 8, 3
    V = synth.random_complex((nt, nv, ns ** 3, 3), seed=21)
    X = synth.random_spinor(ns, nt, seed=22, nrhs=nrhs)
    X[1, 2, 0, 1, 3, 0, 2] = np.nan                          # right-hand side 1, slice 2, spin 0
    got, ref, scale = _check(ns, nt, nv, nrhs, V, X)
    assert np.all(np.isnan(got[1, 2, 0]))
    ok = np.ones(got.shape, dtype=bool)
    ok[1, 2, 0] = False
    assert np.all(np.isfinite(got[ok])) and np.all(np.abs(got - ref)[ok] <= 1e-12 * scale[ok])
