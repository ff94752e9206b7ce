"""Reverse mode of a truncated lower-level solve, float64.

The compliance J(rho) = f^T u_T(rho) is taken through T constant-beta Jacobi
steps from u_0 = 0 (the literal lower-level step of Algorithms 1 / 3 with
M = diag K):
    r_j     = f - K^(rho~) u_j
    u_{j+1} = u_j + beta D(rho~)^-1 r_j.
Its gradient is written out as a plain reverse loop over the stored iterates
(lambda_T = f;  lambda_j = lambda_{j+1} - K^ s_j with s_j = beta D^-1 lambda_{j+1}):
    dJ/drho~_e = sum_j -E'_e [ (m s_j)_e^T k_e (m u_j)_e
                               + sum_{d in e} m_d k_e[dd] s_j,d r_j,d / D_d ]
and dJ/drho = C^T dJ/drho~.  As T grows, u_T -> K^-1 f and this tends to the
exact sensitivity -E'_e u_e^T k_e u_e of Sec. III.
"""
from __future__ import annotations

import numpy as np

from . import fem, filt


def forward(S, rho, T, beta):
    pb = S.pb
    rt, Ee, Ed = S.moduli(rho)
    K = S.K(Ee)
    D = fem.jacobi_diagonal(pb.nx, pb.ny, pb.nz, Ee, S.ke, pb.fixed_dof)
    u = np.zeros(pb.n_dof)
    us, rs = [], []
    for _ in range(T):
        r = S.f - K @ u
        us.append(u)
        rs.append(r)
        u = u + beta * r / D
    return float(S.f @ u), u, (K, D, Ed, us, rs)


def gradient(S, rho, T, beta):
    """Return (J, dJ/drho) for the truncated solve."""
    pb = S.pb
    J, uT, (K, D, Ed, us, rs) = forward(S, rho, T, beta)
    ed = fem.element_dofs(pb.nx, pb.ny, pb.nz)
    kd = np.diag(S.ke)
    lam = S.f.copy()
    gt = np.zeros(pb.n_elem)
    for j in range(T - 1, -1, -1):
        s = beta * lam / D
        ms, mu = S.m * s, S.m * us[j]
        term_k = np.einsum("ei,ij,ej->e", ms[ed], S.ke, mu[ed])
        diag_part = S.m * s * rs[j] / D
        term_d = (diag_part[ed] * kd[None, :]).sum(axis=1)
        gt += -Ed * (term_k + term_d)
        lam = lam - K @ s
    return J, filt.filter_transpose(S.H, S.Hs, gt)
