"""Dilution projectors (Sec. II, noise-dilution projectors).

For a dilution type over a space of dimension N (time N = N_t, spin N = 4,
LapH N = N_v) the projectors are diagonal:
    none          P^(0)_ij = delta_ij                          b = 0
    full          P^(b)_ij = delta_ij delta_{b,i}              b = 0..N-1
    block-J       P^(b)_ij = delta_ij delta_{b, floor(J i / N)} b = 0..J-1
    interlace-J   P^(b)_ij = delta_ij delta_{b, i mod J}        b = 0..J-1
with N/J an integer.  The full projector is the product
P^(b) = P_T^(b_T) (x) P_S^(b_S) (x) P_L^(b_L); reading taken for the flat
index: b = (b_T * n_S + b_S) * n_L + b_L.
"""
import numpy as np

NONE, FULL, BLOCK, INTERLACE = 0, 1, 2, 3


def n_projectors(kind: int, J: int, N: int) -> int:
    if kind == NONE:
        return 1
    if kind == FULL:
        return N
    if kind in (BLOCK, INTERLACE):
        if J <= 0 or N % J != 0:
            raise ValueError(f"dilution J={J} must divide N={N}")
        return J
    raise ValueError(f"unknown dilution type {kind}")


def projector_diag(kind: int, J: int, N: int, b: int) -> np.ndarray:
    """Diagonal of P^(b) as a 0/1 float vector of length N."""
    n_projectors(kind, J, N)
    i = np.arange(N)
    if kind == NONE:
        return np.ones(N)
    if kind == FULL:
        return (i == b).astype(float)
    if kind == BLOCK:
        return ((J * i) // N == b).astype(float)
    return (i % J == b).astype(float)


def split_index(b: int, nT: int, nS: int, nL: int):
    bL = b % nL
    bS = (b // nL) % nS
    bT = b // (nL * nS)
    if bT >= nT:
        raise ValueError("projector index out of range")
    return bT, bS, bL


def full_projector_diag(dil, nt: int, nv: int, b: int) -> np.ndarray:
    """Diagonal of P^(b) over (t, alpha, n) as [nt, 4, nv]; dil = ((kT,JT),(kS,JS),(kL,JL))."""
    (kT, JT), (kS, JS), (kL, JL) = dil
    nT, nS, nL = n_projectors(kT, JT, nt), n_projectors(kS, JS, 4), n_projectors(kL, JL, nv)
    bT, bS, bL = split_index(b, nT, nS, nL)
    pt = projector_diag(kT, JT, nt, bT)
    ps = projector_diag(kS, JS, 4, bS)
    pl = projector_diag(kL, JL, nv, bL)
    return pt[:, None, None] * ps[None, :, None] * pl[None, None, :]


def counts(dil, nt: int, nv: int):
    (kT, JT), (kS, JS), (kL, JL) = dil
    return n_projectors(kT, JT, nt), n_projectors(kS, JS, 4), n_projectors(kL, JL, nv)
