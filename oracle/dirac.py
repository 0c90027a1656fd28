"""Anisotropic Wilson-clover Dirac matrix K, and plain FP64 solves.

The paper uses "an improved anisotropic clover fermion action" (Sec. V,
ensembles) and solves Omega x = y with Omega = gamma_4 K (Sec. II, definition
of the quark line; Sec. IV solver).  It prints no formula for K.  Reading taken
(project definition, shared by the CUDA path through its specification only):

  K psi(x) = (m0 + sum_mu w_mu) psi(x)
             - 1/2 sum_mu w_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
                                + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
             - (c_sw/2) sum_{mu<nu} w_{mu nu} sigma_{mu nu} F_{mu nu}(x) psi(x)

  w_mu = 1/xi (spatial), 1 (temporal); w_{k4} = (1 + 1/xi)/2, w_{jk} = 1/xi;
  F_{mu nu} the traceless clover-leaf field strength (oracle/gauge.py);
  fermion boundary conditions periodic in space, antiperiodic in time.

Free field (U = 1): K(p) = m0 + sum w_mu (1 - cos p_mu) + i sum w_mu gamma_mu sin p_mu.
The diagonal part A(x) (mass + clover) is Hermitian and commutes with gamma_5,
so it is block diagonal in the two chiral halves (spins {0,1} and {2,3}).

Solves: plain BiCGStab (van der Vorst 1992) on the full K, and dense LU for
tiny lattices (scipy.linalg.lu_factor as the library step).
"""
import numpy as np
import scipy.linalg
import scipy.sparse

from .gamma import GAMMA, ONE4, sigma
from .gauge import field_strength
from .lattice import fwd, bwd, dag, site_index


def hop_weights(xi: float) -> np.ndarray:
    return np.array([1.0 / xi, 1.0 / xi, 1.0 / xi, 1.0])


def clover_weight(mu: int, nu: int, xi: float) -> float:
    if mu == 3 or nu == 3:
        return 0.5 * (1.0 + 1.0 / xi)
    return 1.0 / xi


def diag_matrix(u: np.ndarray, m0: float, csw: float, xi: float) -> np.ndarray:
    """A(x) = (m0 + sum w_mu) 1 - (c_sw/2) sum_{mu<nu} w_{mu nu} sigma_{mu nu} (x) F_{mu nu}(x).

    Returned as [t,z,y,x,12,12] with component index spin*3 + colour."""
    shp = u.shape[:4]
    a = np.zeros(shp + (12, 12), dtype=complex)
    a += (m0 + hop_weights(xi).sum()) * np.eye(12)
    if csw != 0.0:
        for mu in range(4):
            for nu in range(mu + 1, 4):
                f = field_strength(u, mu, nu)
                s = sigma(mu, nu)
                a -= 0.5 * csw * clover_weight(mu, nu, xi) * np.einsum("ab,...cd->...acbd", s, f).reshape(shp + (12, 12))
    return a


def fermion_links(u: np.ndarray) -> np.ndarray:
    """Links with the antiperiodic time boundary folded in: U_4(x) at t = N_t - 1
    carries a factor -1 (every hop across the time boundary flips sign)."""
    uf = u.copy()
    uf[-1, :, :, :, 3] *= -1.0
    return uf


class WilsonClover:
    """K for a given gauge field; apply() works on [..., t,z,y,x,4,3] fields."""

    def __init__(self, u: np.ndarray, m0: float, csw: float, xi: float):
        self.u = u
        self.uf = fermion_links(u)
        self.m0, self.csw, self.xi = m0, csw, xi
        self.w = hop_weights(xi)
        self.a = diag_matrix(u, m0, csw, xi)
        self.shape = u.shape[:4]

    def apply_diag(self, psi: np.ndarray) -> np.ndarray:
        lead = psi.ndim - 6
        p = psi.reshape(psi.shape[:lead] + self.shape + (12,))
        out = np.einsum("tzyxij,...tzyxj->...tzyxi", self.a, p)
        return out.reshape(psi.shape)

    def apply_hop(self, psi: np.ndarray) -> np.ndarray:
        """D psi = -1/2 sum_mu w_mu [(1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^dag psi(x-mu)]."""
        lead = psi.ndim - 6
        out = np.zeros_like(psi)
        for mu in range(4):
            umu = self.uf[..., mu, :, :]
            f = np.einsum("tzyxab,...tzyxsb->...tzyxsa", umu, fwd(psi, mu, lead))
            b = bwd(np.einsum("tzyxba,...tzyxsb->...tzyxsa", np.conj(umu), psi), mu, lead)
            out -= 0.5 * self.w[mu] * (np.einsum("sr,...rc->...sc", ONE4 - GAMMA[mu], f)
                                       + np.einsum("sr,...rc->...sc", ONE4 + GAMMA[mu], b))
        return out

    def apply(self, psi: np.ndarray) -> np.ndarray:
        return self.apply_diag(psi) + self.apply_hop(psi)

    def apply_dag(self, psi: np.ndarray) -> np.ndarray:
        """K^dag = gamma_5 K gamma_5 (gamma_5-Hermiticity, Sec. II)."""
        g5 = np.diag(GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3])[:, None]
        return g5 * self.apply(g5 * psi)

    def sparse(self) -> scipy.sparse.csr_matrix:
        """K as a sparse (12V x 12V) matrix assembled block by block (an
        independent construction used to check apply())."""
        nt, nz, ny, nx = self.shape
        ns = nx
        t, z, y, x = np.meshgrid(np.arange(nt), np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        t, z, y, x = t.ravel(), z.ravel(), y.ravel(), x.ravel()
        site = site_index(t, z, y, x, ns)
        rows, cols, vals = [], [], []
        ii, jj = np.meshgrid(np.arange(12), np.arange(12), indexing="ij")

        def add(rs, cs, blocks):
            rows.append((rs[:, None, None] * 12 + ii[None]).ravel())
            cols.append((cs[:, None, None] * 12 + jj[None]).ravel())
            vals.append(blocks.reshape(-1))

        add(site, site, self.a.reshape(-1, 12, 12)[site])
        coords = [x, y, z, t]
        dims = [nx, ny, nz, nt]
        for mu in range(4):
            c_f = list(coords)
            c_f[mu] = (coords[mu] + 1) % dims[mu]
            nb_f = site_index(c_f[3], c_f[2], c_f[1], c_f[0], ns)
            c_b = list(coords)
            c_b[mu] = (coords[mu] - 1) % dims[mu]
            nb_b = site_index(c_b[3], c_b[2], c_b[1], c_b[0], ns)
            u_here = self.u[t, z, y, x, mu]
            u_back = self.u[c_b[3], c_b[2], c_b[1], c_b[0], mu]
            sgn_f = np.ones(len(site))
            sgn_b = np.ones(len(site))
            if mu == 3:
                sgn_f[t == nt - 1] = -1.0
                sgn_b[t == 0] = -1.0
            bf = -0.5 * self.w[mu] * np.einsum("sr,nab->nsarb", ONE4 - GAMMA[mu], u_here).reshape(-1, 12, 12)
            bb = -0.5 * self.w[mu] * np.einsum("sr,nba->nsarb", ONE4 + GAMMA[mu], np.conj(u_back)).reshape(-1, 12, 12)
            add(site, nb_f, bf * sgn_f[:, None, None])
            add(site, nb_b, bb * sgn_b[:, None, None])
        n = 12 * len(site)
        return scipy.sparse.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def bicgstab(apply, b: np.ndarray, tol: float = 1e-12, maxiter: int = 100000, x0=None):
    """Plain BiCGStab (van der Vorst 1992).  Returns (x, iterations, relres).

    The relative residual is recomputed from scratch at the end."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply(x) if x0 is not None else b.copy()
    rhat = r.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    rho_old = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    it = 0
    while it < maxiter:
        it += 1
        rho = np.vdot(rhat, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = apply(p)
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        if np.linalg.norm(s) <= tol * bnorm:
            x = x + alpha * p
            r = s
            break
        t = apply(s)
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        if np.linalg.norm(r) <= tol * bnorm:
            break
    relres = np.linalg.norm(b - apply(x)) / bnorm
    return x, it, relres


def lu_solve_dense(kmat: np.ndarray, b: np.ndarray) -> np.ndarray:
    lu = scipy.linalg.lu_factor(kmat)
    return scipy.linalg.lu_solve(lu, b)
