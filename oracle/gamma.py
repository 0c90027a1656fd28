"""Dirac matrices for the oracle.

The paper fixes neither the basis nor the sign conventions (it uses
gamma_4 and gamma_5 in Eq. (laphpropg5) and the quark-field definition
q-bar = psi-bar gamma_4, Sec. III).  Reading taken: the chiral (DeGrand-Rossi)
basis,
    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],  gamma_4 = [[0, 1], [1, 0]],
    gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1),
all Hermitian, {gamma_mu, gamma_nu} = 2 delta_{mu nu}.  Spin index 0..3,
direction index mu = 0,1,2,3 for gamma_1..gamma_4.
sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu] is block-diagonal in this basis.
"""
import numpy as np

_s1 = np.array([[0, 1], [1, 0]], dtype=complex)
_s2 = np.array([[0, -1j], [1j, 0]], dtype=complex)
_s3 = np.array([[1, 0], [0, -1]], dtype=complex)
_z2 = np.zeros((2, 2), dtype=complex)
_i2 = np.eye(2, dtype=complex)


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = np.array([
    _block(_z2, -1j * _s1, 1j * _s1, _z2),
    _block(_z2, -1j * _s2, 1j * _s2, _z2),
    _block(_z2, -1j * _s3, 1j * _s3, _z2),
    _block(_z2, _i2, _i2, _z2),
])
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ONE4 = np.eye(4, dtype=complex)


def sigma(mu: int, nu: int) -> np.ndarray:
    """sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu]."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])
