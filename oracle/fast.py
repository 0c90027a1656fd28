"""ctypes front end of the oracle's plain-C Dirac stencil and BiCGStab
(oracle/c/oracle_dirac.c).  Same definition of K as oracle/dirac.py (the mass +
clover matrix A(x) is built by the numpy oracle and passed in); the C code only
makes the loops fast enough for 16^3 x 32 and larger lattices.  Test
infrastructure: compiled by build() (oracle/build_c.py) with gcc."""
import ctypes
import os

import numpy as np

from .build_c import build_oracle_c

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_oracle_c())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        _lib.oracle_K_apply.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
        _lib.oracle_bicgstab_batch.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp,
                                               ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ip, dp]
        _lib.oracle_bicgstab_threaded.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp,
                                                  ctypes.c_double, ctypes.c_int, ctypes.c_int, dp]
        _lib.oracle_bicgstab_threaded.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class FastK:
    """Wraps an oracle.dirac.WilsonClover; apply() and solve() run the C loops."""

    def __init__(self, wc):
        self.wc = wc
        self.U = np.ascontiguousarray(wc.u, dtype=np.complex128)
        self.A = np.ascontiguousarray(wc.a, dtype=np.complex128)
        self.nt, self.ns = wc.shape[0], wc.shape[3]

    def apply(self, psi):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        out = np.empty_like(psi)
        lead = psi.shape[:-6]
        n = int(np.prod(lead)) if lead else 1
        fi = psi.reshape(n, -1)
        fo = out.reshape(n, -1)
        for k in range(n):
            lib().oracle_K_apply(_p(self.U), _p(self.A), self.ns, self.nt, self.wc.xi, _p(fi[k]), _p(fo[k]))
        return out

    def solve(self, b, tol=1e-12, maxiter=100000, nthreads=None):
        """Independent BiCGStab solves of K x = b[k]; returns (x, iters, relres)."""
        b = np.ascontiguousarray(b, dtype=np.complex128)
        single = b.ndim == 6
        if single:
            b = b[None]
        nrhs = b.shape[0]
        x = np.zeros_like(b)
        iters = np.zeros(nrhs, dtype=np.int32)
        rr = np.zeros(nrhs)
        nth = nthreads or os.cpu_count() or 1
        lib().oracle_bicgstab_batch(_p(self.U), _p(self.A), self.ns, self.nt, self.wc.xi, _p(b), _p(x), nrhs,
                                    tol, maxiter, nth, iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(rr))
        if single:
            return x[0], int(iters[0]), float(rr[0])
        return x, iters, rr

    def solve_split(self, b, tol=1e-12, maxiter=100000, nthreads=1):
        """One BiCGStab solve of K x = b with each application of K split over nthreads
        threads (the same arithmetic per site); returns (x, iters, relres)."""
        b = np.ascontiguousarray(b, dtype=np.complex128)
        x = np.zeros_like(b)
        rr = ctypes.c_double()
        it = lib().oracle_bicgstab_threaded(_p(self.U), _p(self.A), self.ns, self.nt, self.wc.xi, _p(b), _p(x),
                                            tol, maxiter, int(nthreads), ctypes.byref(rr))
        return x, int(it), float(rr.value)
