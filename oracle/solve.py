"""Lower-level solvers of the oracle, float64.

* ``inner_sd``         -- n preconditioned steepest-descent steps on
  P_f(u) = 1/2 u^T K u - f^T u with the exact line search.  This widens the
  single step of Algorithm 1 (line 1) / Algorithm 3 (line 1) to a few steps
  warm-started from the previous u; each step moves along z = M^-1 r with
  beta = r^T z / z^T K z, the minimiser of P_f on that line.
* ``inner_richardson`` -- the literal constant-beta step of Algorithms 1 / 3,
  u <- u - beta M^-1 (K u - f).
* ``krylov_apply``     -- the Krylov preconditioner of Eq. (LSP) (Sec. IV-C):
  M^-1 b = sum_{i=0}^{D} c_i K^i b, with c minimising ||b - sum_{i=1}^{D+1}
  c_{i-1} K^i b||, on an orthonormal Arnoldi basis of that Krylov space
  (``krylov_apply_power``: the paper's Householder QR of the power basis).
  With beta = 1 in ``inner_richardson`` this is Algorithm CPFBTO.
* ``inner_pfbto``      -- Algorithm 2 (PFBTO): u <- u - beta K M^-1 M^-1 (K u - f),
  the preconditioned gradient step on the squared lower-level problem.
* ``solve_exact``      -- K^-1 f for the nested exact method (PGD, Sec. V):
  dense Cholesky when small, sparse LU otherwise.
* ``Multigrid``        -- a geometric-multigrid V-cycle used as M^-1.  The paper
  only cites multigrid as prior art (Sec. II, IV-A, IV-D); the cycle here is
  this library's own definition, restated independently on the GPU side:
  rediscretised hex8 coarse operators with element moduli averaged over the
  8 children, element size doubled per level, trilinear prolongation P,
  restriction P^T, damped Jacobi smoothing (omega, nu1 pre, nu2 post), and a
  dense Cholesky solve on the coarsest grid.  A coarse DOF is fixed when any
  fine DOF of the same component among the fine nodes {2I-1, 2I, 2I+1}^3 is.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem


def inner_sd(A, f: np.ndarray, u: np.ndarray, Minv, n: int):
    """Return (u_n, r_n, betas, r_0).  ``A`` and ``Minv`` are callables."""
    u = u.copy()
    r = f - A(u)
    r0 = r.copy()
    betas = []
    for _ in range(n):
        z = Minv(r)
        q = A(z)
        rz = float(r @ z)
        zq = float(z @ q)
        beta = rz / zq if (zq > 0.0 and rz != 0.0) else 0.0
        u = u + beta * z
        r = r - beta * q
        betas.append(beta)
    return u, r, betas, r0


def inner_richardson(A, f: np.ndarray, u: np.ndarray, Minv, n: int, beta: float):
    """Return (u_n, r_0): n constant-beta preconditioned Richardson steps."""
    u = u.copy()
    r0 = None
    for _ in range(n):
        r = f - A(u)
        if r0 is None:
            r0 = r.copy()
        u = u + beta * Minv(r)
    return u, r0


def krylov_apply(A, b: np.ndarray, D: int) -> np.ndarray:
    """M^-1 b of Eq. (LSP) (Sec. IV-C) for the operator ``A`` (a callable).

    Eq. (LSP) defines M^-1 b = sum_{i=0}^{D} c_i K^i b with c the minimiser of
    ||b - sum_{i=1}^{D+1} c_{i-1} K^i b||: the vector x of the Krylov space
    span{b, K b, ..., K^D b} whose K x is closest to b.  That space is spanned
    here by an orthonormal basis q_0 .. q_D built by the Arnoldi process
    (modified Gram-Schmidt; K q_j = sum_{i<=j+1} H_ij q_i), so that
    ||b - K Q y|| = || ||b|| e_1 - H y || and the minimiser is the small
    least-squares solution y.  (The paper solves the same least-squares problem
    on the power basis b, K b, ... with a Householder QR; in double precision
    that basis loses rank beyond D of about 8 on these problems, see
    ``krylov_apply_power``.)
    """
    beta0 = float(np.linalg.norm(b))
    if beta0 == 0.0:
        return np.zeros_like(b)
    Q = [b / beta0]
    H = np.zeros((D + 2, D + 1))
    m = D + 1
    for j in range(D + 1):
        w = A(Q[j])
        for i in range(j + 1):
            H[i, j] = float(Q[i] @ w)
            w = w - H[i, j] * Q[i]
        H[j + 1, j] = float(np.linalg.norm(w))
        # the space is invariant (K^-1 b lies in it) when the new direction vanishes
        # relative to ||K q_j|| = ||H[0..j+1, j]||
        if H[j + 1, j] <= 1e-12 * float(np.linalg.norm(H[:j + 2, j])):
            m = j + 1
            break
        Q.append(w / H[j + 1, j])
    e1 = np.zeros(m + 1)
    e1[0] = beta0
    y = np.linalg.lstsq(H[:m + 1, :m], e1, rcond=None)[0]
    return np.stack(Q[:m], axis=1) @ y


def krylov_apply_power(A, b: np.ndarray, D: int) -> np.ndarray:
    """The same least-squares problem as ``krylov_apply`` posed on the power basis,
    as the paper does: s_0 = b, s_i = K s_{i-1} / ||K s_{i-1}|| (normalising changes
    neither the span nor the minimiser), min_c ||b - [K s_0 ... K s_D] c|| by a
    Householder QR (numpy.linalg.qr: LAPACK geqrf), M^-1 b = [s_0 ... s_D] c.
    Agrees with ``krylov_apply`` while the power basis keeps full numerical rank."""
    S = [b.copy()]
    KS = []
    for i in range(D + 1):
        w = A(S[i])
        KS.append(w)
        if i < D:
            nw = float(np.linalg.norm(w))
            S.append(w / nw if nw > 0.0 else np.zeros_like(w))
    Q, R = np.linalg.qr(np.stack(KS, axis=1))
    c = np.linalg.lstsq(R, Q.T @ b, rcond=None)[0]
    return np.stack(S, axis=1) @ c


def inner_pfbto(A, f: np.ndarray, u: np.ndarray, Minv, n: int, beta: float):
    """Return (u_n, r_0): n steps of Algorithm PFBTO (Algorithm 2, lines 1-2):
    delta = M^-1 (K u - f), u <- u - beta K M^-1 delta, i.e. preconditioned gradient
    steps on the squared lower-level problem (1/2) ||K u - f||^2 (Eq. optBilevelSqr)."""
    u = u.copy()
    r0 = None
    for _ in range(n):
        b = A(u) - f
        if r0 is None:
            r0 = -b
        delta = Minv(b)
        u = u - beta * A(Minv(delta))
    return u, r0


def solve_exact(K: sp.spmatrix, f: np.ndarray) -> np.ndarray:
    n = K.shape[0]
    if n <= 6000:
        c = sla.cho_factor(K.toarray(), lower=True)
        return sla.cho_solve(c, f)
    return spla.spsolve(K.tocsc(), f)


def pcg(A, f: np.ndarray, Minv, tol: float = 1e-12, maxit: int = 100000, x0=None):
    """Preconditioned CG to ||r|| / ||f|| <= tol (used where a factorisation does not fit)."""
    x = np.zeros_like(f) if x0 is None else x0.copy()
    r = f - A(x)
    z = Minv(r)
    p = z.copy()
    rz = r @ z
    nf = np.linalg.norm(f)
    for it in range(maxit):
        if np.linalg.norm(r) <= tol * nf:
            return x, it
        q = A(p)
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        z = Minv(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit


# ----------------------------------------------------------------------------- multigrid

def auto_levels(nx: int, ny: int, nz: int) -> int:
    """1 + the largest t with every dimension divisible by 2^t and >= 2 after coarsening."""
    t = 0
    while (nx % (2 ** (t + 1)) == 0 and ny % (2 ** (t + 1)) == 0 and nz % (2 ** (t + 1)) == 0
           and min(nx, ny, nz) // 2 ** (t + 1) >= 2):
        t += 1
    return t + 1


def coarse_fixed(nx: int, ny: int, nz: int, fixed_dof: np.ndarray) -> np.ndarray:
    """Fixed DOFs of the 2x coarser grid (see module docstring)."""
    fm = np.zeros((nz + 1, ny + 1, nx + 1, 3), dtype=bool)
    fd = np.asarray(fixed_dof, dtype=np.int64)
    node, comp = fd // 3, fd % 3
    i = node % (nx + 1)
    j = (node // (nx + 1)) % (ny + 1)
    k = node // ((nx + 1) * (ny + 1))
    fm[k, j, i, comp] = True
    cx, cy, cz = nx // 2, ny // 2, nz // 2
    out = []
    for K in range(cz + 1):
        for J in range(cy + 1):
            for I in range(cx + 1):
                blk = fm[max(2 * K - 1, 0):min(2 * K + 1, nz) + 1,
                         max(2 * J - 1, 0):min(2 * J + 1, ny) + 1,
                         max(2 * I - 1, 0):min(2 * I + 1, nx) + 1]
                anyc = blk.reshape(-1, 3).any(axis=0)
                n = I + (cx + 1) * (J + (cy + 1) * K)
                for c in range(3):
                    if anyc[c]:
                        out.append(3 * n + c)
    return np.array(out, dtype=np.int64)


def coarse_modulus(nx: int, ny: int, nz: int, Ee: np.ndarray) -> np.ndarray:
    """Mean of the 8 child element moduli."""
    a = Ee.reshape(nz, ny, nx)
    return 0.125 * (a[0::2, 0::2, 0::2] + a[0::2, 0::2, 1::2] + a[0::2, 1::2, 0::2] + a[0::2, 1::2, 1::2]
                    + a[1::2, 0::2, 0::2] + a[1::2, 0::2, 1::2] + a[1::2, 1::2, 0::2] + a[1::2, 1::2, 1::2]).ravel()


def prolongation(cx: int, cy: int, cz: int) -> sp.csr_matrix:
    """Trilinear interpolation from a (cx,cy,cz)-element grid to the 2x finer one (DOF level)."""
    fx, fy, fz = 2 * cx, 2 * cy, 2 * cz

    def one_d(nc):
        nf = 2 * nc
        rows, cols, vals = [], [], []
        for i in range(nf + 1):
            if i % 2 == 0:
                rows.append(i); cols.append(i // 2); vals.append(1.0)
            else:
                rows += [i, i]; cols += [(i - 1) // 2, (i + 1) // 2]; vals += [0.5, 0.5]
        return sp.csr_matrix((vals, (rows, cols)), shape=(nf + 1, nc + 1))

    # node index is i + (nx+1)(j + (ny+1)k): kron order z (slowest), y, x (fastest)
    Pn = sp.kron(sp.kron(one_d(cz), one_d(cy)), one_d(cx)).tocsr()
    return sp.kron(Pn, sp.identity(3)).tocsr()


class Multigrid:
    """V-cycle M^-1 for K^(E) on an (nx, ny, nz) grid with element edge h."""

    def __init__(self, nx, ny, nz, h, Ee, nu, fixed_dof, levels=None, omega=0.5, nu1=2, nu2=2):
        L = auto_levels(nx, ny, nz) if not levels else levels
        self.omega, self.nu1, self.nu2 = omega, nu1, nu2
        ke1 = fem.ke_hex8(nu, 1.0)
        self.A, self.D, self.P, self.m = [], [], [], []
        dims = (nx, ny, nz)
        E = np.asarray(Ee, dtype=np.float64)
        fixed = np.asarray(fixed_dof, dtype=np.int64)
        for l in range(L):
            gx, gy, gz = dims
            hl = h * 2 ** l
            ke = hl * ke1          # 3-D elasticity: K_e scales linearly with the edge length
            self.A.append(fem.assemble(gx, gy, gz, E, ke, fixed))
            self.D.append(fem.jacobi_diagonal(gx, gy, gz, E, ke, fixed))
            n_dof = 3 * (gx + 1) * (gy + 1) * (gz + 1)
            self.m.append(fem.free_mask(n_dof, fixed))
            if l < L - 1:
                cx, cy, cz = gx // 2, gy // 2, gz // 2
                P = prolongation(cx, cy, cz)
                E = coarse_modulus(gx, gy, gz, E)
                fixed = coarse_fixed(gx, gy, gz, fixed)
                mc = fem.free_mask(3 * (cx + 1) * (cy + 1) * (cz + 1), fixed)
                self.P.append(sp.diags(self.m[l]) @ P @ sp.diags(mc))
                dims = (cx, cy, cz)
        self.L = L
        self.coarse = sla.cho_factor(self.A[-1].toarray(), lower=True)

    def vcycle(self, b: np.ndarray, l: int = 0) -> np.ndarray:
        if l == self.L - 1:
            return sla.cho_solve(self.coarse, b)
        A, D = self.A[l], self.D[l]
        x = np.zeros_like(b)
        for _ in range(self.nu1):
            x = x + self.omega * (b - A @ x) / D
        r = b - A @ x
        x = x + self.P[l] @ self.vcycle(self.P[l].T @ r, l + 1)
        for _ in range(self.nu2):
            x = x + self.omega * (b - A @ x) / D
        return x

    __call__ = vcycle
