"""Finite-element core of the oracle (Sec. III of the paper), float64.

The paper discretises the linear-elastic potential energy
    P(u, v) = 1/2 u^T K(v) u,   K(v) = sum_e K_e(v)
on a regular grid and loads it with P_f = P - f^T u (Sec. III).  Here the
elements are trilinear hexahedra (hex8) on an nx x ny x nz voxel grid of edge
h, and the power-law (SIMP) parameterisation of Sec. III reads
    E_e = Emin + rho~_e^p (E0 - Emin).
Fixtures (Sec. III: fixed DOFs) are applied by elimination: with m the
free-DOF indicator,  K^ = diag(m) K diag(m) + diag(1 - m).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

# Local node order of an element (offsets in i, j, k), local DOF = 3*l + c.
LOCAL_NODES = np.array([(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
                        (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)], dtype=np.int64)


def constitutive(nu: float, E: float = 1.0) -> np.ndarray:
    """Isotropic 6x6 elasticity matrix in Voigt order (xx, yy, zz, xy, yz, zx)."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def shape_gradients(xi: np.ndarray, h: float) -> np.ndarray:
    """d N_a / d x at reference point xi in [0,1]^3 for the 8 trilinear shape functions."""
    g = np.zeros((8, 3))
    for a, off in enumerate(LOCAL_NODES):
        f = [xi[d] if off[d] else 1.0 - xi[d] for d in range(3)]
        s = [1.0 if off[d] else -1.0 for d in range(3)]
        g[a, 0] = s[0] * f[1] * f[2] / h
        g[a, 1] = f[0] * s[1] * f[2] / h
        g[a, 2] = f[0] * f[1] * s[2] / h
    return g


def strain_displacement(dN: np.ndarray) -> np.ndarray:
    """6x24 B matrix (engineering shear strains) from shape-function gradients."""
    B = np.zeros((6, 24))
    for a in range(8):
        dx, dy, dz = dN[a]
        c = 3 * a
        B[0, c] = dx
        B[1, c + 1] = dy
        B[2, c + 2] = dz
        B[3, c] = dy
        B[3, c + 1] = dx
        B[4, c + 1] = dz
        B[4, c + 2] = dy
        B[5, c] = dz
        B[5, c + 2] = dx
    return B


def ke_hex8(nu: float, h: float = 1.0, order: int = 2) -> np.ndarray:
    """Unit-modulus hex8 element stiffness K_e = int B^T D B dV by Gauss quadrature.

    ``order`` points per direction; 2 is exact for the trilinear cube (the
    integrand is at most quadratic in each coordinate).
    """
    pts, wts = np.polynomial.legendre.leggauss(order)
    pts = 0.5 * (pts + 1.0)
    wts = 0.5 * wts
    D = constitutive(nu)
    K = np.zeros((24, 24))
    for (a, wa), (b, wb), (c, wc) in itertools.product(zip(pts, wts), repeat=3):
        B = strain_displacement(shape_gradients(np.array([a, b, c]), h))
        K += (wa * wb * wc * h ** 3) * (B.T @ D @ B)
    return K


def young(rho_t: np.ndarray, E0: float, Emin: float, p: float) -> np.ndarray:
    """Modified SIMP modulus E_e = Emin + rho~^p (E0 - Emin)."""
    return Emin + rho_t ** p * (E0 - Emin)


def young_deriv(rho_t: np.ndarray, E0: float, Emin: float, p: float) -> np.ndarray:
    """dE_e/d rho~_e = p rho~^(p-1) (E0 - Emin)."""
    return p * rho_t ** (p - 1) * (E0 - Emin)


def element_nodes(nx: int, ny: int, nz: int) -> np.ndarray:
    """(E, 8) global node ids of every element, element id e = i + nx (j + ny k)."""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    out = np.empty((i.size, 8), dtype=np.int64)
    for l, (a, b, c) in enumerate(LOCAL_NODES):
        out[:, l] = (i + a) + (nx + 1) * ((j + b) + (ny + 1) * (k + c))
    return out


def element_dofs(nx: int, ny: int, nz: int) -> np.ndarray:
    """(E, 24) global DOF ids, local DOF 3*l + c."""
    en = element_nodes(nx, ny, nz)
    return (3 * en[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 24)


def free_mask(n_dof: int, fixed_dof: np.ndarray) -> np.ndarray:
    m = np.ones(n_dof)
    m[np.asarray(fixed_dof, dtype=np.int64)] = 0.0
    return m


def load_vector(n_dof: int, load_dof, load_val, fixed_dof) -> np.ndarray:
    """Dense f with fixed DOFs zeroed (elimination of the fixtures)."""
    f = np.zeros(n_dof)
    np.add.at(f, np.asarray(load_dof, dtype=np.int64), np.asarray(load_val, dtype=np.float64))
    f[np.asarray(fixed_dof, dtype=np.int64)] = 0.0
    return f


def assemble(nx: int, ny: int, nz: int, Ee: np.ndarray, ke: np.ndarray, fixed_dof) -> sp.csr_matrix:
    """CSR K^ = m K m + (1 - m): sum_e E_e P_e^T k_e P_e with fixtures eliminated."""
    ed = element_dofs(nx, ny, nz)
    n_dof = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    rows = np.repeat(ed, 24, axis=1).ravel()
    cols = np.tile(ed, (1, 24)).ravel()
    vals = (Ee[:, None] * ke.ravel()[None, :]).ravel()
    K = sp.coo_matrix((vals, (rows, cols)), shape=(n_dof, n_dof)).tocsr()
    m = sp.diags(free_mask(n_dof, fixed_dof))
    return (m @ K @ m + sp.diags(1.0 - free_mask(n_dof, fixed_dof))).tocsr()


def apply_matfree(nx: int, ny: int, nz: int, Ee: np.ndarray, ke: np.ndarray, fixed_dof,
                  u: np.ndarray) -> np.ndarray:
    """K^ u by an explicit loop over elements (gather u_e, y_e = E_e k_e u_e, scatter-add)."""
    n_dof = u.size
    m = free_mask(n_dof, fixed_dof)
    um = m * u
    ed = element_dofs(nx, ny, nz)
    ye = (um[ed] @ ke.T) * Ee[:, None]
    y = np.zeros(n_dof)
    np.add.at(y, ed.ravel(), ye.ravel())
    return m * y + (1.0 - m) * u


def jacobi_diagonal(nx: int, ny: int, nz: int, Ee: np.ndarray, ke: np.ndarray, fixed_dof) -> np.ndarray:
    """diag(K^): sum over elements of E_e k_e[ll], 1 on fixed DOFs."""
    n_dof = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    ed = element_dofs(nx, ny, nz)
    d = np.zeros(n_dof)
    np.add.at(d, ed.ravel(), (Ee[:, None] * np.diag(ke)[None, :]).ravel())
    m = free_mask(n_dof, fixed_dof)
    return m * d + (1.0 - m)


def element_energy(nx: int, ny: int, nz: int, ke: np.ndarray, u: np.ndarray) -> np.ndarray:
    """u_e^T k_e u_e for every element (unit modulus)."""
    ue = u[element_dofs(nx, ny, nz)]
    return np.einsum("ei,ij,ej->e", ue, ke, ue)
