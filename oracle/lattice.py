"""Lattice geometry for the oracle.

Site arrays carry leading axes [t, z, y, x]; direction mu = 0,1,2,3 means
x, y, z, t and lives on numpy axis 3 - mu of a site array.  Boundary
conditions are periodic for the gauge field; the fermion's antiperiodic time
boundary is applied inside the Dirac operator (oracle/dirac.py).
"""
import numpy as np


def axis_of(mu: int, lead: int = 0) -> int:
    """numpy axis of direction mu in a site array with `lead` leading batch axes."""
    return lead + 3 - mu


def fwd(f: np.ndarray, mu: int, lead: int = 0) -> np.ndarray:
    """f(x + mu_hat), periodic."""
    return np.roll(f, -1, axis=axis_of(mu, lead))


def bwd(f: np.ndarray, mu: int, lead: int = 0) -> np.ndarray:
    """f(x - mu_hat), periodic."""
    return np.roll(f, 1, axis=axis_of(mu, lead))


def dag(m: np.ndarray) -> np.ndarray:
    """Hermitian conjugate over the last two axes."""
    return np.conj(np.swapaxes(m, -1, -2))


def mm(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Batched matrix product over the last two axes."""
    return np.einsum("...ij,...jk->...ik", a, b)


def site_index(t, z, y, x, ns):
    """Lexicographic site index, x fastest."""
    return ((t * ns + z) * ns + y) * ns + x


def parity_of(shape_tzyx) -> np.ndarray:
    """(t + z + y + x) mod 2 for every site."""
    nt, nz, ny, nx = shape_tzyx
    t, z, y, x = np.meshgrid(np.arange(nt), np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (t + z + y + x) % 2
