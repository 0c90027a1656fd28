"""Sequencing of the C-ABI calls for one stochastic-LapH pass.

The steps follow the paper's task order (Sec. IV): stout-smeared links, the
Laplacian eigenvectors of every slice, diluted Z4 sources, the solves of
Omega x = V_s P^(b) rho, the sink coefficients and the meson correlators.  All
arithmetic runs in liblaph; this module only allocates device buffers with
torch and forwards pointers and sizes.
"""
from dataclasses import dataclass
from typing import List, Optional, Sequence

import torch

from . import laph as L


@dataclass
class LatticeSpec:
    ns: int
    nt: int
    xi: float
    m0: float
    csw: float
    nv: int
    dil: tuple            # ((kT, JT), (kS, JS), (kL, JL))
    rho_stout: float = 0.1
    n_stout4d: int = 10
    n_stout3d: int = 2


def n_projectors(kind, J, N):
    return {0: 1, 1: N}.get(kind, J)


def projectors_for_time(spec: LatticeSpec, t0: int) -> List[int]:
    """Flat projector indices b = (b_T n_S + b_S) n_L + b_L whose time part contains t0."""
    (kT, JT), (kS, JS), (kL, JL) = spec.dil
    nT, nS, nL = n_projectors(kT, JT, spec.nt), n_projectors(kS, JS, 4), n_projectors(kL, JL, spec.nv)
    if kT == 0:
        bts = [0]
    elif kT == 1:
        bts = [t0]
    elif kT == 2:
        bts = [(JT * t0) // spec.nt]
    else:
        bts = [t0 % JT]
    return [(bT * nS + bS) * nL + bL for bT in bts for bS in range(nS) for bL in range(nL)]


class LapHPath:
    def __init__(self, spec: LatticeSpec, device: int = 0):
        self.spec = spec
        self.device = device
        self.ctx = L.Context(device)
        self.lat = L.lattice(spec.ns, spec.nt, spec.xi)
        self.dil = L.dilution(*spec.dil)
        self.dev = torch.device("cuda", device)

    # a0: gauge preparation
    def prepare_links(self, u0):
        u = torch.as_tensor(u0).to(self.dev).contiguous()
        L.laph_stout_smear(self.ctx, self.lat, u, self.spec.rho_stout, self.spec.n_stout4d, 0)
        ut = u.clone()
        L.laph_stout_smear(self.ctx, self.lat, ut, self.spec.rho_stout, self.spec.n_stout3d, 1)
        return u, ut

    # a1
    def eigvecs(self, ut, evals=None, evecs=None, params=None):
        s = self.spec
        if evals is None:
            evals = torch.empty((s.nt, s.nv), dtype=torch.float64, device=self.dev)
        if evecs is None:
            evecs = torch.empty((s.nt, s.nv, s.ns ** 3, 3), dtype=torch.complex128, device=self.dev)
        rep = L.laph_eigvecs(self.ctx, self.lat, ut, s.nv, evals, evecs, params)
        return evals, evecs, rep

    def field(self, n):
        s = self.spec
        return torch.empty((n, s.nt, s.ns, s.ns, s.ns, 4, 3), dtype=torch.complex128, device=self.dev)

    # a2
    def sources(self, evecs, noise_id, config_id, bs, out=None, codes=None):
        s = self.spec
        out = self.field(len(bs)) if out is None else out
        codes = torch.empty((s.nt, 4, s.nv), dtype=torch.uint8, device=self.dev) if codes is None else codes
        L.laph_make_sources(self.ctx, self.lat, evecs, s.nv, noise_id, config_id, self.dil, bs, out, codes)
        return out, codes

    # a3
    def solve(self, u, rhs, mode=L.MIXED_FP32, tol=1e-10, rhs_block=0, sol=None, **kw):
        sol = torch.empty_like(rhs) if sol is None else sol
        prm = L.solver_params(tol=tol, mode=mode, rhs_block=rhs_block, **kw)
        reps = L.dirac_solve_batch(self.ctx, self.lat, u, self.spec.m0, self.spec.csw, rhs, sol, rhs.shape[0], prm)
        return sol, reps

    # a4
    def sinks(self, evecs, sol, out=None):
        s = self.spec
        n = sol.shape[0]
        out = torch.empty((n, s.nt, 4, s.nv), dtype=torch.complex128, device=self.dev) if out is None else out
        L.laph_sinks(self.ctx, self.lat, evecs, s.nv, sol, n, out)
        return out

    # a5
    def correlate(self, channel, t0, bs, coefs: Sequence, codes: Sequence, out=None):
        out = torch.empty((self.spec.nt,), dtype=torch.complex128, device=self.dev) if out is None else out
        L.correlate(self.ctx, self.lat, channel, t0, self.spec.nv, self.dil, bs, list(coefs), list(codes), out)
        return out

    def close(self):
        self.ctx.close()
