"""3D gauge-covariant Laplacian, its lowest eigenpairs, and the phase convention.

Sec. II, Laplacian matrix:
    Delta^{ab}(x,y) = sum_{k=1..3} { U_k^{ab}(x) delta(y, x+k) + U_k^{ba}(y)^* delta(y, x-k)
                                   - 2 delta(x,y) delta^{ab} },
built from the stout-smeared spatial links; Hermitian and block diagonal in
time.  V_s holds, on each time slice, the eigenvectors of the N_v lowest
eigenvalues of -Delta (Sec. II, fixed-N_v approximation).  All eigenvalues of
-Delta lie in [0, 12] (a sum of six unitary hops bounded by 6 plus the 6 of the
diagonal), which is why lambda_L = 15 bounds the spectrum (Sec. IV).

Eigenpairs are the plain definition: the N_v smallest eigenpairs of the
Hermitian slice matrix, by numpy.linalg.eigh (dense, small slices) or
scipy.sparse.linalg.eigsh (larger slices) as the library step.

Phase convention (Sec. IV asks for one and does not give it).  Reading taken:
each eigenvector is multiplied by a phase so that its component of largest
modulus is real and positive; among components whose modulus is within a
relative 1e-8 of the largest, the first in storage order (site index with x
fastest, colour fastest within a site) is used.
"""
import numpy as np
import scipy.sparse
import scipy.sparse.linalg

from .lattice import fwd, bwd, site_index


def apply_mlap(ut: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(-Delta psi)(x) = 6 psi(x) - sum_k [U_k(x) psi(x+k) + U_k(x-k)^dag psi(x-k)].

    ut: [t,z,y,x,4,3,3] (spatial slots 0..2 used); psi: [..., t,z,y,x,3]."""
    lead = psi.ndim - 5
    out = 6.0 * psi
    for k in range(3):
        uk = ut[..., k, :, :]
        out = out - np.einsum("tzyxab,...tzyxb->...tzyxa", uk, fwd(psi, k, lead))
        out = out - bwd(np.einsum("tzyxba,...tzyxb->...tzyxa", np.conj(uk), psi), k, lead)
    return out


def slice_matrix(ut: np.ndarray, t: int) -> scipy.sparse.csr_matrix:
    """-Delta on time slice t as a sparse (3 V3) x (3 V3) matrix, built block by block."""
    ns = ut.shape[3]
    z, y, x = np.meshgrid(np.arange(ns), np.arange(ns), np.arange(ns), indexing="ij")
    z, y, x = z.ravel(), y.ravel(), x.ravel()
    site = site_index(0, z, y, x, ns)
    ii, jj = np.meshgrid(np.arange(3), np.arange(3), indexing="ij")
    rows = [(site[:, None, None] * 3 + ii[None]).ravel()]
    cols = [(site[:, None, None] * 3 + jj[None]).ravel()]
    vals = [np.broadcast_to(6.0 * np.eye(3), (len(site), 3, 3)).ravel().astype(complex)]
    c = [x, y, z]
    for k in range(3):
        cf = list(c)
        cf[k] = (c[k] + 1) % ns
        cb = list(c)
        cb[k] = (c[k] - 1) % ns
        nf = site_index(0, cf[2], cf[1], cf[0], ns)
        nb = site_index(0, cb[2], cb[1], cb[0], ns)
        u_here = ut[t, z, y, x, k]
        u_back = ut[t, cb[2], cb[1], cb[0], k]
        rows.append((site[:, None, None] * 3 + ii[None]).ravel())
        cols.append((nf[:, None, None] * 3 + jj[None]).ravel())
        vals.append((-u_here).ravel())
        rows.append((site[:, None, None] * 3 + ii[None]).ravel())
        cols.append((nb[:, None, None] * 3 + jj[None]).ravel())
        vals.append((-np.conj(np.swapaxes(u_back, -1, -2))).ravel())
    n = 3 * ns ** 3
    return scipy.sparse.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def phase_fix(v: np.ndarray) -> np.ndarray:
    """Apply the phase convention to each row of v ([..., n_components])."""
    v = np.array(v, dtype=complex, copy=True)
    flat = v.reshape(-1, v.shape[-1])
    for i in range(flat.shape[0]):
        mag = np.abs(flat[i])
        j = int(np.argmax(mag >= (1.0 - 1e-8) * mag.max()))
        flat[i] *= np.conj(flat[i, j]) / mag[j]
    return flat.reshape(v.shape)


def lowest_eigpairs(ut: np.ndarray, nv: int, method: str = "auto"):
    """Lowest nv eigenpairs of -Delta on every slice.

    Returns evals [nt, nv] (ascending) and evecs [nt, nv, V3, 3] with the
    phase convention applied."""
    nt, ns = ut.shape[0], ut.shape[3]
    n = 3 * ns ** 3
    if method == "auto":
        method = "dense" if n <= 3000 else "sparse"
    evals = np.zeros((nt, nv))
    evecs = np.zeros((nt, nv, ns ** 3, 3), dtype=complex)
    for t in range(nt):
        m = slice_matrix(ut, t)
        if method == "dense":
            w, v = np.linalg.eigh(m.toarray())
            w, v = w[:nv], v[:, :nv]
        else:
            w, v = scipy.sparse.linalg.eigsh(m, k=nv, which="SA", tol=1e-14, ncv=max(2 * nv + 16, 64))
            order = np.argsort(w)
            w, v = w[order], v[:, order]
        evals[t] = w
        evecs[t] = phase_fix(v.T).reshape(nv, ns ** 3, 3)
    return evals, evecs


def chebyshev_map(lam, lam_lo_cut: float, lam_hi: float):
    """Spectral map of Sec. IV written for an eigenvalue lam of -Delta:
    B = 1 + 2 (Delta + lambda_C)/(lambda_L - lambda_C)  ->  b = 1 - 2 (lam - lambda_C)/(lambda_L - lambda_C)."""
    return 1.0 - 2.0 * (np.asarray(lam) - lam_lo_cut) / (lam_hi - lam_lo_cut)


def chebyshev_T(n: int, x):
    """T_n(x) by the three-term recurrence T_0 = 1, T_1 = x, T_n = 2x T_{n-1} - T_{n-2} (Sec. IV)."""
    x = np.asarray(x, dtype=float)
    t0, t1 = np.ones_like(x), x
    if n == 0:
        return t0
    for _ in range(n - 1):
        t0, t1 = t1, 2.0 * x * t1 - t0
    return t1


def eigenprojector_distance(va: np.ndarray, vb: np.ndarray) -> float:
    """max over slices of || P_a - P_b ||_F, P = sum_n v_n v_n^dag over the N_v
    vectors of a slice (evecs [nt, nv, V3, 3]).  Insensitive to phases and to
    rotations inside the span.  Uses ||P_a - P_b||_F = sqrt(2) ||(1 - P_a) B||_F
    (equal ranks, orthonormal rows), which has no cancellation."""
    nt, nv = va.shape[:2]
    d = 0.0
    for t in range(nt):
        a = va[t].reshape(nv, -1)
        b = vb[t].reshape(nv, -1)
        r = b - (b @ a.conj().T) @ a
        d = max(d, float(np.sqrt(2.0) * np.linalg.norm(r)))
    return d
