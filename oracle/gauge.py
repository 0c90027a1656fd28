"""Gauge-field arithmetic of the oracle: stout smearing and the clover field.

Stout smearing (Sec. II: the spatial links are stout-smeared, only spatial
staples are used and temporal links are left alone; the recipe itself is the
cited Morningstar-Peardon stout step):
    C_mu(x) = rho * sum_{nu != mu} [ U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
                                    + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ]
    Omega   = C_mu U_mu^dag
    Q_mu    = (i/2)(Omega^dag - Omega) - (i/6) Tr(Omega^dag - Omega)
    U_mu   <- exp(i Q_mu) U_mu          (all links of a step updated at once)
The 4D variant (used as the synthetic "thermalisation" of the workload) sums
over all nu != mu and updates all four directions; the 3D variant used for the
Laplacian sums over spatial nu only and updates spatial mu only.

exp(i Q) is taken from the eigendecomposition of the Hermitian Q.
"""
import numpy as np

from .lattice import fwd, bwd, dag, mm


def _exp_iq(q: np.ndarray) -> np.ndarray:
    w, v = np.linalg.eigh(q)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), np.conj(v))


def staple_sum(u: np.ndarray, mu: int, nus) -> np.ndarray:
    """Sum of the upper and lower staples of U_mu(x) over the given nu."""
    c = np.zeros(u.shape[:4] + (3, 3), dtype=complex)
    umu = u[..., mu, :, :]
    for nu in nus:
        if nu == mu:
            continue
        unu = u[..., nu, :, :]
        # U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
        c += mm(mm(unu, fwd(umu, nu)), dag(fwd(unu, mu)))
        # U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
        unu_m = bwd(unu, nu)
        c += mm(mm(dag(unu_m), bwd(umu, nu)), fwd(unu_m, mu))
    return c


def stout_step(u: np.ndarray, rho: float, spatial_only: bool) -> np.ndarray:
    """One stout step on a gauge field u[t,z,y,x,mu,3,3]; returns a new field."""
    mus = (0, 1, 2) if spatial_only else (0, 1, 2, 3)
    nus = (0, 1, 2) if spatial_only else (0, 1, 2, 3)
    out = u.copy()
    for mu in mus:
        c = rho * staple_sum(u, mu, nus)
        om = mm(c, dag(u[..., mu, :, :]))
        a = dag(om) - om
        tr = np.trace(a, axis1=-2, axis2=-1)
        q = 0.5j * a - (1j / 6.0) * tr[..., None, None] * np.eye(3)
        out[..., mu, :, :] = mm(_exp_iq(q), u[..., mu, :, :])
    return out


def stout(u: np.ndarray, rho: float, nsteps: int, spatial_only: bool) -> np.ndarray:
    for _ in range(nsteps):
        u = stout_step(u, rho, spatial_only)
    return u


def prepare_links(u0: np.ndarray, rho: float, n4d: int, n3d: int):
    """Workload gauge preparation: n4d 4D stout steps give the Dirac links U;
    n3d further 3D (spatial-only) steps give the Laplacian links U-tilde."""
    u = stout(u0, rho, n4d, spatial_only=False)
    ut = stout(u, rho, n3d, spatial_only=True)
    return u, ut


def prepare_links_window(u0: np.ndarray, t0: int, halo: int, rho: float, n4d: int, n3d: int):
    """prepare_links on the time slices t0-halo .. t0+halo of u0 (periodic indices of the full
    lattice), smeared as a periodic lattice of 2 halo + 1 slices.

    A stout step (Sec. II recipe) updates each link from its staples, which reach one slice
    forward and back, so the error from closing the window on itself spreads inwards by one
    slice per 4D step; 3D steps do not spread in time.  Slices t0 - (halo - n4d) .. t0 + (halo -
    n4d) of the window (positions n4d .. 2 halo - n4d) therefore equal those of the full
    lattice's smearing exactly.  Returns (u, ut) of the window, slice t0 at position halo."""
    nt = u0.shape[0]
    idx = [(t0 + k) % nt for k in range(-halo, halo + 1)]
    return prepare_links(np.ascontiguousarray(u0[idx]), rho, n4d, n3d)


def plaquette(u: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """P_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag."""
    umu, unu = u[..., mu, :, :], u[..., nu, :, :]
    return mm(mm(mm(umu, fwd(unu, mu)), dag(fwd(umu, nu))), dag(unu))


def mean_plaquette(u: np.ndarray) -> float:
    s = 0.0
    n = 0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            s += np.trace(plaquette(u, mu, nu), axis1=-2, axis2=-1).real.mean() / 3.0
            n += 1
    return s / n


def clover_leaves(u: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """Sum of the four plaquettes in the mu-nu plane that touch x, each
    starting and ending at x (the clover leaf Q_{mu nu}(x))."""
    umu, unu = u[..., mu, :, :], u[..., nu, :, :]
    # leaf 1: x -> x+mu -> x+mu+nu -> x+nu -> x
    l1 = mm(mm(mm(umu, fwd(unu, mu)), dag(fwd(umu, nu))), dag(unu))
    # leaf 2: x -> x+nu -> x+nu-mu -> x-mu -> x
    umu_m = bwd(umu, mu)                     # U_mu(x-mu)
    unu_m = bwd(unu, mu)                     # U_nu(x-mu)
    l2 = mm(mm(mm(unu, dag(fwd(umu_m, nu))), dag(unu_m)), umu_m)
    # leaf 3: x -> x-mu -> x-mu-nu -> x-nu -> x
    umu_mm = bwd(umu_m, nu)                  # U_mu(x-mu-nu)
    unu_mm = bwd(unu_m, nu)                  # U_nu(x-mu-nu)
    unu_n = bwd(unu, nu)                     # U_nu(x-nu)
    l3 = mm(mm(mm(dag(umu_m), dag(unu_mm)), umu_mm), unu_n)
    # leaf 4: x -> x-nu -> x-nu+mu -> x+mu -> x
    umu_n = bwd(umu, nu)                     # U_mu(x-nu)
    l4 = mm(mm(mm(dag(unu_n), umu_n), fwd(unu_n, mu)), dag(umu))
    return l1 + l2 + l3 + l4


def field_strength(u: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """Clover field strength F_{mu nu} = (Q - Q^dag)/(8i), made traceless (Hermitian)."""
    q = clover_leaves(u, mu, nu)
    f = (q - dag(q)) / 8j
    tr = np.trace(f, axis1=-2, axis2=-1) / 3.0
    return f - tr[..., None, None] * np.eye(3)


def gauge_transform_links(u: np.ndarray, g: np.ndarray) -> np.ndarray:
    """U_mu(x) -> G(x) U_mu(x) G(x+mu)^dag."""
    out = np.empty_like(u)
    for mu in range(4):
        out[..., mu, :, :] = mm(mm(g, u[..., mu, :, :]), dag(fwd(g, mu)))
    return out


def unitarity_defect(u: np.ndarray) -> float:
    """max over links of |U U^dag - 1| and |det U - 1|."""
    e = np.abs(mm(u, dag(u)) - np.eye(3)).max()
    d = np.abs(np.linalg.det(u) - 1.0).max()
    return float(max(e, d))
