"""Oracle driver for one workload: the steps of the path in the paper's order.

Sec. IV lists the tasks per configuration: smear the links, compute the
Laplacian eigenvectors slice by slice, solve Omega x = V_s P^(b) rho for the
diluted sources, form the sinks/coefficients, and assemble correlators.
This module strings the oracle's pieces together for tests and for the CPU
baseline of the benchmark; it adds no arithmetic of its own.
"""
import numpy as np
import scipy.linalg

from . import dilution as dl
from . import gauge, laplacian, laph, noise
from .dirac import WilsonClover, bicgstab


class OraclePath:
    def __init__(self, wl, u0=None, eig_method="auto"):
        self.wl = wl
        u0 = wl.gauge() if u0 is None else u0
        self.u, self.ut = gauge.prepare_links(u0, wl.rho_stout, wl.n_stout4d, wl.n_stout3d)
        self.K = WilsonClover(self.u, wl.m0, wl.csw, wl.xi)
        self.evals, self.evecs = laplacian.lowest_eigpairs(self.ut, wl.nv, eig_method)
        self.dil = (wl.dil_time, wl.dil_spin, wl.dil_laph)
        self._lu = None

    # ---- noise and projectors
    def rho(self, noise_id):
        return noise.z4_values(noise.z4_codes(self.wl.nt, self.wl.nv, noise_id, self.wl.config_id))

    def projectors_for_time(self, t0):
        """Flat projector indices b whose time part contains t0."""
        nT, nS, nL = dl.counts(self.dil, self.wl.nt, self.wl.nv)
        kT, JT = self.dil[0]
        out = []
        for bT in range(nT):
            if dl.projector_diag(kT, JT, self.wl.nt, bT)[t0] == 0:
                continue
            out.extend((bT * nS + bS) * nL + bL for bS in range(nS) for bL in range(nL))
        return out

    # ---- solves
    def dense_lu(self):
        if self._lu is None:
            self._lu = scipy.linalg.lu_factor(self.K.sparse().toarray())
        return self._lu

    def solve(self, rhs, method="bicgstab", tol=1e-12):
        if method == "lu":
            x = scipy.linalg.lu_solve(self.dense_lu(), rhs.reshape(rhs.shape[0], -1).T).T
            return x.reshape(rhs.shape), None
        xs, its = [], []
        for b in rhs:
            x, it, rr = bicgstab(self.K.apply, b, tol=tol)
            xs.append(x)
            its.append(it)
        return np.stack(xs), its

    def line(self, noise_id, bs, method="bicgstab"):
        r = self.rho(noise_id)
        rhs = np.stack([laph.dirac_rhs(self.evecs, r, self.dil, b) for b in bs])
        x, _ = self.solve(rhs, method)
        return laph.Line(self.evecs, r, self.dil, bs, x), x

    def exact_G(self):
        """G = V^dag K^{-1} gamma_4 V from the dense LU (tiny lattices)."""
        nt, nv = self.wl.nt, self.wl.nv
        v3 = self.evecs.shape[2]
        w = np.zeros((nt, v3, 4, 3, nt, 4, nv), dtype=complex)
        for t in range(nt):
            for a in range(4):
                w[t, :, a, :, t, a, :] = np.transpose(self.evecs[t], (1, 2, 0))
        w = w.reshape(nt * v3 * 12, nt * 4 * nv)
        g4w = np.einsum("ab,tsbcq->tsacq", laph.G4, w.reshape(nt, v3, 4, 3, -1)).reshape(w.shape)
        z = scipy.linalg.lu_solve(self.dense_lu(), g4w)
        return (w.conj().T @ z).reshape(nt, 4, nv, nt, 4, nv)
