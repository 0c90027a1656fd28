"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds random numbers, lattice shapes and workload parameters only:
none of the stochastic-LapH arithmetic lives here (no smearing, no Laplacian,
no Dirac operator, no noise generator, no contraction).  Both the CPU oracle
and the GPU tests/benchmark draw their inputs from here, so the two sides see
bit-identical starting data while sharing no code of the method.

Array conventions (all numpy, complex128 unless stated):
  * a 4D site array has leading axes [t, z, y, x] (x fastest in memory);
  * a gauge field is [t, z, y, x, mu, a, b] with mu = 0,1,2,3 = x,y,z,t;
  * a spinor field is [..., t, z, y, x, spin, colour].

The gauge-field recipe is the workload definition of the benchmark: each link
is U = exp(i * 0.4 * H) with H a Gaussian traceless Hermitian 3x3 matrix drawn
from numpy's PCG64 stream seeded by the configuration's gauge seed.  (The
paper's RHMC ensembles are not available; these fields are a smooth stand-in,
so spectra and iteration counts differ from the paper's.)
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np

__all__ = [
    "Workload", "WORKLOADS", "random_hermitian_traceless", "random_su3_field",
    "random_gauge_transform", "random_spinor", "random_complex",
]


def random_hermitian_traceless(rng: np.random.Generator, shape) -> np.ndarray:
    """Gaussian traceless Hermitian 3x3 matrices of the given leading shape."""
    a = rng.standard_normal(tuple(shape) + (3, 3)) + 1j * rng.standard_normal(tuple(shape) + (3, 3))
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[..., None, None] * np.eye(3)
    return h


def _exp_i_hermitian(h: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*h) for Hermitian h via its eigendecomposition (input generation only)."""
    w, v = np.linalg.eigh(h)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ij,...j,...kj->...ik", v, ph, np.conj(v))


def random_su3_field(ns: int, nt: int, seed: int, eps: float = 0.4) -> np.ndarray:
    """Gauge field U[t,z,y,x,mu,a,b] = exp(i*eps*H), H Gaussian traceless Hermitian."""
    rng = np.random.default_rng(seed)
    h = random_hermitian_traceless(rng, (nt, ns, ns, ns, 4))
    return _exp_i_hermitian(h, eps)


def random_gauge_transform(ns: int, nt: int, seed: int, eps: float = 2.0) -> np.ndarray:
    """Random SU(3) matrix per site, G[t,z,y,x,a,b] (used by gauge-covariance tests)."""
    rng = np.random.default_rng(seed)
    h = random_hermitian_traceless(rng, (nt, ns, ns, ns))
    return _exp_i_hermitian(h, eps)


def random_complex(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(tuple(shape)) + 1j * rng.standard_normal(tuple(shape))


def random_spinor(ns: int, nt: int, seed: int, nrhs: Optional[int] = None) -> np.ndarray:
    """Gaussian complex spinor field [nrhs?, t, z, y, x, 4, 3]."""
    shape = (nt, ns, ns, ns, 4, 3)
    if nrhs is not None:
        shape = (nrhs,) + shape
    return random_complex(shape, seed)


# Dilution type codes: 0 none, 1 full, 2 block-J, 3 interlace-J.
DIL_NONE, DIL_FULL, DIL_BLOCK, DIL_INTERLACE = 0, 1, 2, 3


@dataclass(frozen=True)
class Workload:
    """One synthetic workload: lattice, action parameters and LapH parameters.

    m0 values were chosen by seeded bisection on the plain FP64 BiCGStab
    iteration count of the oracle (oracle/tune_m0.py writes them).
    """
    name: str
    ns: int
    nt: int
    xi: float
    csw: float
    m0: float
    nv: int
    gauge_seed: int
    n_stout4d: int = 10
    n_stout3d: int = 2
    rho_stout: float = 0.1
    dil_time: Tuple[int, int] = (DIL_FULL, 0)
    dil_spin: Tuple[int, int] = (DIL_FULL, 0)
    dil_laph: Tuple[int, int] = (DIL_FULL, 0)
    source_times: Tuple[int, ...] = (0,)
    n_noise: int = 2
    target_iters: int = 0

    @property
    def volume(self) -> int:
        return self.ns ** 3 * self.nt

    @property
    def config_id(self) -> int:
        return self.gauge_seed % 65536

    def gauge(self) -> np.ndarray:
        return random_su3_field(self.ns, self.nt, self.gauge_seed)


WORKLOADS = {
    # 4^3x8, N_v = 8, full time/spin/LapH dilution (the exact case).
    "tiny_4x8": Workload("tiny_4x8", ns=4, nt=8, xi=3.5, csw=1.0, m0=-0.04898, nv=8,
                         gauge_seed=1000, dil_time=(DIL_FULL, 0), dil_spin=(DIL_FULL, 0),
                         dil_laph=(DIL_FULL, 0), source_times=tuple(range(8)), n_noise=2,
                         target_iters=150),
    # 16^3x32, N_v = 32, (TF, SF, LI8) fixed-time quark lines at four widely separated
    # source times (as in the paper's production runs), 2 noises: 256 diluted sources.
    "medium_16x32": Workload("medium_16x32", ns=16, nt=32, xi=3.5, csw=1.0, m0=-0.0049, nv=32,
                             gauge_seed=1001, dil_time=(DIL_FULL, 0), dil_spin=(DIL_FULL, 0),
                             dil_laph=(DIL_INTERLACE, 8), source_times=(0, 8, 16, 24), n_noise=2,
                             target_iters=600),
    # 24^3x128, N_v = 64, (TI16, SF, LI8): 512 diluted sources per noise, four noises (two pion
    # lines and the four lines of the I = 2 pi pi correlator).  m0 from the seeded bisection of the
    # plain FP64 iteration count (1351 iterations to 1e-10, target 1500).
    "paper_24x128": Workload("paper_24x128", ns=24, nt=128, xi=3.5, csw=1.0, m0=-0.0003125, nv=64,
                             gauge_seed=1002, dil_time=(DIL_INTERLACE, 16), dil_spin=(DIL_FULL, 0),
                             dil_laph=(DIL_INTERLACE, 8), source_times=(0,), n_noise=4,
                             target_iters=1500),
    # The same lattice, field and mass with N_v = 112 (the eigenvector count of the paper's
    # 24^3 x 128 runs, Sec. V), (TI16, SF, LI8): 512 diluted sources per noise as before.
    "paper_24x128_nv112": Workload("paper_24x128_nv112", ns=24, nt=128, xi=3.5, csw=1.0, m0=-0.0003125, nv=112,
                                   gauge_seed=1002, dil_time=(DIL_INTERLACE, 16), dil_spin=(DIL_FULL, 0),
                                   dil_laph=(DIL_INTERLACE, 8), source_times=(0,), n_noise=4,
                                   target_iters=1500),
}
