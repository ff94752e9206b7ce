"""Outer loop of the oracle: FBTO / CPFBTO (Algorithms 1 and 3) and the nested
exact method PGD (Sec. V, convergence analysis), float64, mirror of the GPU.

One outer iteration k = 1, 2, ... (u_1 = 0) does, in this order:
  1. rho~ = C(rho_k), E = Emin + rho~^p (E0 - Emin), E' = dE/drho~
     (Sec. III power law; Remark 3.1 filter)
  2. g~_e = -E'_e u_e^T k_e u_e at u_k, the iterate *before* this iteration's
     lower-level steps (the high-level line of Algorithms 1 / 3 uses u_k)
  3. J_k = f^T u_k
  4. u_{k+1} = n_inner lower-level steps from u_k with K(rho~_k) and M
     (Jacobi diagonal or the multigrid V-cycle); PGD uses K^-1 f instead
  5. g = C^T g~ (chain rule through the filter); optional mean projection
     g <- g - 1 1^T g / E (Sec. IV-B)
  6. alpha_k = alpha_0 k^-m (Sec. V: alpha_k = alpha_0 k^-3/4); when alpha_0
     is not given it is fixed once as  scale / ||g||_inf  at the first k with
     g != 0 (a scale-free choice of this library; the paper tunes alpha_0)
  7. rho_{k+1} = Proj_X(rho_k - alpha_k g)  (Algorithm 4)
The paper's termination quantities (Sec. V) are logged: ||K(v_k) u_k - f||_inf
(the residual at u_k) and ||rho_{k+1} - rho_k||_inf.
"""
from __future__ import annotations

import numpy as np

from . import fem, filt, project, solve


class Setup:
    """Problem data derived once: k_e, filter, fixtures, load vector."""

    def __init__(self, pb):
        self.pb = pb
        self.ke = fem.ke_hex8(pb.nu, pb.h)
        self.H, self.Hs = filt.filter_matrix(pb.nx, pb.ny, pb.nz, pb.rmin)
        self.m = fem.free_mask(pb.n_dof, pb.fixed_dof)
        self.f = fem.load_vector(pb.n_dof, pb.load_dof, pb.load_val, pb.fixed_dof)
        self.vbar = pb.volfrac * pb.n_elem

    def moduli(self, rho):
        pb = self.pb
        rt = filt.filter_forward(self.H, self.Hs, rho)
        return rt, fem.young(rt, pb.E0, pb.Emin, pb.p), fem.young_deriv(rt, pb.E0, pb.Emin, pb.p)

    def K(self, Ee):
        pb = self.pb
        return fem.assemble(pb.nx, pb.ny, pb.nz, Ee, self.ke, pb.fixed_dof)

    def sens_rho_tilde(self, Ed, u):
        pb = self.pb
        return -Ed * fem.element_energy(pb.nx, pb.ny, pb.nz, self.ke, self.m * u)

    def exact_compliance(self, rho):
        _, Ee, _ = self.moduli(rho)
        u = solve.solve_exact(self.K(Ee), self.f)
        return float(self.f @ u), u


def run(pb, n_outer, precond="jacobi", n_inner=5, inner_mode="sd", beta=0.5,
        alpha0=None, alpha_scale=0.2, m=0.75, mean_proj=False,
        mg_levels=None, mg_omega=0.5, nu1=2, nu2=2, setup=None, rho=None, u=None, k0=1, krylov_dim=20):
    """Run ``n_outer`` outer iterations; returns (rho, u, history, alpha0)."""
    S = setup or Setup(pb)
    rho = pb.rho0.copy() if rho is None else rho.copy()
    u = np.zeros(pb.n_dof) if u is None else u.copy()
    hist = []
    for k in range(k0, k0 + n_outer):
        rt, Ee, Ed = S.moduli(rho)
        gt = S.sens_rho_tilde(Ed, u)
        J = float(S.f @ u)
        K = S.K(Ee)
        A = lambda x: K @ x
        betas = []
        if precond == "exact":
            r0 = S.f - A(u)
            u_new = solve.solve_exact(K, S.f)
        else:
            if precond == "jacobi":
                D = fem.jacobi_diagonal(pb.nx, pb.ny, pb.nz, Ee, S.ke, pb.fixed_dof)
                Minv = lambda r: r / D
            elif precond == "mg":
                mg = solve.Multigrid(pb.nx, pb.ny, pb.nz, pb.h, Ee, pb.nu, pb.fixed_dof,
                                     levels=mg_levels, omega=mg_omega, nu1=nu1, nu2=nu2)
                Minv = mg
            elif precond == "none":
                Minv = lambda r: r
            elif precond == "krylov":   # Eq. (LSP); with inner_mode "richardson", beta = 1: CPFBTO
                Minv = lambda r: solve.krylov_apply(A, r, krylov_dim)
            else:
                raise ValueError(precond)
            if inner_mode == "sd":
                u_new, _, betas, r0 = solve.inner_sd(A, S.f, u, Minv, n_inner)
            elif inner_mode == "pfbto":
                u_new, r0 = solve.inner_pfbto(A, S.f, u, Minv, n_inner, beta)
            elif inner_mode == "pcg":   # n_inner conjugate-gradient iterations (the nested method's solve)
                r0 = S.f - A(u)
                u_new, _ = solve.pcg(A, S.f, Minv, tol=0.0, maxit=n_inner, x0=u)
            else:
                u_new, r0 = solve.inner_richardson(A, S.f, u, Minv, n_inner, beta)
        g = filt.filter_transpose(S.H, S.Hs, gt)
        if mean_proj:
            g = g - g.mean()
        gmax = float(np.abs(g).max())
        if alpha0 is None and gmax > 0.0:
            alpha0 = alpha_scale / gmax
        alpha = alpha0 * k ** (-m) if alpha0 is not None else 0.0
        w = rho - alpha * g
        rho_new, lam = project.project_alg4(w, S.vbar, pb.rho_min, pb.rho_max)
        hist.append(dict(k=k, J=J, res_inf=float(np.abs(r0).max()), res2=float(np.linalg.norm(r0)),
                         drho_inf=float(np.abs(rho_new - rho).max()), volume=float(rho_new.sum()),
                         lam=lam, alpha=alpha, betas=betas, gmax=gmax))
        rho, u = rho_new, u_new
    return rho, u, hist, alpha0
