"""Pins for the lower-level solvers: steepest descent with exact line search
(Algorithms 1 / 3 widened to a few steps), the multigrid V-cycle used as M, and
the truncated-solve reverse mode."""
import numpy as np
import scipy.sparse as sp

import workloads as W
from oracle import adjoint, fem, outer, solve


def _setup(nx=8, ny=4, nz=4, rho=None):
    pb = W.cantilever(nx, ny, nz)
    if rho is not None:
        pb.rho0 = rho(pb.n_elem)
    S = outer.Setup(pb)
    _, Ee, _ = S.moduli(pb.rho0)
    return pb, S, Ee


def test_steepest_descent_decreases_energy_every_step():
    pb, S, Ee = _setup(rho=lambda n: W.random_rho(n))
    K = S.K(Ee)
    D = fem.jacobi_diagonal(pb.nx, pb.ny, pb.nz, Ee, S.ke, pb.fixed_dof)
    energy = lambda u: 0.5 * u @ (K @ u) - S.f @ u
    u = np.zeros(pb.n_dof)
    last = energy(u)
    r0 = S.f - K @ u
    u1, r1, _, _ = solve.inner_sd(lambda x: K @ x, S.f, u, lambda r: r / D, 1)
    assert abs(r1 @ (r0 / D)) < 1e-12 * abs(r0 @ (r0 / D))
    for _ in range(20):
        u, r, betas, _ = solve.inner_sd(lambda x: K @ x, S.f, u, lambda r: r / D, 1)
        e = energy(u)
        assert e < last
        last = e
    # the recursively updated residual equals the true one
    assert np.abs(r - (S.f - K @ u)).max() < 1e-12 * np.abs(S.f).max()


def test_multigrid_galerkin_identity_uniform_modulus():
    """Rediscretised coarse operator = P^T A P for constant E (nested trilinear spaces)."""
    nx, ny, nz = 8, 4, 4
    ke = fem.ke_hex8(0.3)
    A = fem.assemble(nx, ny, nz, np.full(nx * ny * nz, 0.4), ke, [])
    P = solve.prolongation(nx // 2, ny // 2, nz // 2)
    Ac = fem.assemble(nx // 2, ny // 2, nz // 2, np.full(nx * ny * nz // 8, 0.4), 2.0 * ke, [])
    assert abs(P.T @ A @ P - Ac).max() < 1e-14
    # interpolation reproduces linear fields exactly
    k, j, i = np.meshgrid(np.arange(nz // 2 + 1), np.arange(ny // 2 + 1), np.arange(nx // 2 + 1), indexing="ij")
    lin = np.stack([2 * i.ravel() + 1.0, -j.ravel() * 2.0, 2 * k.ravel() * 0.5], axis=1).ravel()
    kf, jf, if_ = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    linf = np.stack([if_.ravel() + 1.0, -jf.ravel() * 1.0, kf.ravel() * 0.5], axis=1).ravel()
    assert np.abs(P @ lin - linf).max() < 1e-14


def test_multigrid_coarse_fixtures_and_modulus():
    pb = W.cantilever(8, 4, 4)
    cf = solve.coarse_fixed(8, 4, 4, pb.fixed_dof)
    assert cf.size == 3 * 3 * 3          # the clamped face of the 4x2x2 grid
    pbm = W.mbb_half(8, 4, 4)
    cfm = set(solve.coarse_fixed(8, 4, 4, pbm.fixed_dof).tolist())
    node = lambda i, j, k: i + 5 * (j + 3 * k)
    assert 3 * node(4, 0, 1) + 1 in cfm and 3 * node(4, 0, 0) + 2 in cfm and 3 * node(0, 2, 2) + 0 in cfm
    E = np.arange(8 * 4 * 4, dtype=float)
    Ec = solve.coarse_modulus(8, 4, 4, E)
    a = E.reshape(4, 4, 8)
    assert Ec[0] == a[:2, :2, :2].mean() and Ec[-1] == a[2:, 2:, 6:].mean()


def test_vcycle_symmetric_positive_definite_and_contracts():
    pb, S, Ee = _setup(16, 8, 8)
    mg = solve.Multigrid(pb.nx, pb.ny, pb.nz, pb.h, Ee, pb.nu, pb.fixed_dof)
    assert mg.L == 3
    r = np.random.default_rng(4)
    a, b = r.normal(size=pb.n_dof), r.normal(size=pb.n_dof)
    Va, Vb = mg(a), mg(b)
    assert abs(Va @ b - a @ Vb) < 1e-10 * abs(Va @ b)
    assert a @ Va > 0 and b @ Vb > 0
    # as a stationary iteration on the full-density problem the V-cycle contracts the residual
    pb1, S1, E1 = _setup(16, 8, 8, rho=lambda n: np.ones(n))
    K = S1.K(E1)
    mg1 = solve.Multigrid(pb1.nx, pb1.ny, pb1.nz, pb1.h, E1, pb1.nu, pb1.fixed_dof)
    u = np.zeros(pb1.n_dof)
    res = [np.linalg.norm(S1.f)]
    for _ in range(6):
        u = u + mg1(S1.f - K @ u)
        res.append(np.linalg.norm(S1.f - K @ u))
    assert all(res[i + 1] < 0.6 * res[i] for i in range(len(res) - 1))


def test_vcycle_single_level_is_exact_solve():
    pb, S, Ee = _setup(4, 2, 2)
    mg = solve.Multigrid(pb.nx, pb.ny, pb.nz, pb.h, Ee, pb.nu, pb.fixed_dof, levels=1)
    K = S.K(Ee)
    b = np.random.default_rng(5).normal(size=pb.n_dof)
    assert np.abs(K @ mg(b) - b).max() < 1e-9 * np.abs(b).max()


def test_truncated_solve_reverse_mode_matches_finite_differences():
    pb, S, _ = _setup(6, 4, 4, rho=lambda n: W.random_rho(n))
    T, beta = 6, 0.5
    J, g = adjoint.gradient(S, pb.rho0, T, beta)
    h = 1e-6
    for e in W.random_elements(pb.n_elem, 10):
        rp, rm = pb.rho0.copy(), pb.rho0.copy()
        rp[e] += h
        rm[e] -= h
        fd = (adjoint.forward(S, rp, T, beta)[0] - adjoint.forward(S, rm, T, beta)[0]) / (2 * h)
        assert abs(g[e] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max())


def test_truncated_gradient_tends_to_exact_sensitivity():
    pb, S, _ = _setup(4, 2, 2, rho=lambda n: W.random_rho(n))
    J, u = S.exact_compliance(pb.rho0)
    _, _, Ed = S.moduli(pb.rho0)
    from oracle import filt
    g_exact = filt.filter_transpose(S.H, S.Hs, S.sens_rho_tilde(Ed, u))
    JT, gT = adjoint.gradient(S, pb.rho0, 10000, 0.5)
    assert abs(JT - J) < 1e-8 * J
    assert np.abs(gT - g_exact).max() < 1e-9 * np.abs(g_exact).max()


# ----------------------------------------------------------------------------- Krylov preconditioner, Eq. (LSP)
def test_krylov_preconditioner_is_the_gmres_minimal_residual_vector():
    """Eq. (LSP) minimises ||b - K x|| over x in span{b, ..., K^D b}: the vector one
    restart cycle of GMRES(D + 1) from x = 0 returns (scipy's implementation)."""
    import scipy.sparse.linalg as spla
    pb, S, Ee = _setup(rho=lambda n: W.random_rho(n))
    K = S.K(Ee).tocsr()
    b = W.random_u(pb.n_dof)
    for D in (0, 1, 4, 20):
        x = solve.krylov_apply(lambda v: K @ v, b, D)
        xg, _ = spla.gmres(K, b, x0=np.zeros_like(b), rtol=1e-300, atol=0.0, restart=D + 1, maxiter=1)
        assert np.linalg.norm(x - xg) <= 1e-6 * np.linalg.norm(xg)
        rx, rg = np.linalg.norm(b - K @ x), np.linalg.norm(b - K @ xg)
        assert abs(rx - rg) <= 1e-10 * np.linalg.norm(b)


def test_krylov_preconditioner_power_basis_agrees_for_small_D():
    """The paper's Householder QR of the power basis solves the same problem."""
    pb, S, Ee = _setup(rho=lambda n: W.random_rho(n))
    K = S.K(Ee)
    b = W.random_u(pb.n_dof)
    for D in (0, 1, 2, 4):
        x = solve.krylov_apply(lambda v: K @ v, b, D)
        xp = solve.krylov_apply_power(lambda v: K @ v, b, D)
        assert np.linalg.norm(x - xp) <= 1e-9 * np.linalg.norm(x)


def test_krylov_residual_never_grows_with_D():
    """Nested Krylov spaces: the minimal residual is non-increasing in D."""
    pb, S, Ee = _setup(rho=lambda n: W.random_rho(n))
    K = S.K(Ee)
    b = W.random_u(pb.n_dof)
    last = np.linalg.norm(b)
    for D in range(0, 21):
        res = np.linalg.norm(b - K @ solve.krylov_apply(lambda v: K @ v, b, D))
        assert res <= last * (1 + 1e-10)
        last = res


def test_krylov_preconditioner_is_the_exact_inverse_on_a_complete_space():
    """One element (24 DOFs, 12 fixed): the Krylov space of dimension 24 holds K^-1 b."""
    pb = W.cantilever(1, 1, 1)
    S = outer.Setup(pb)
    _, Ee, _ = S.moduli(np.full(1, 0.7))
    K = S.K(Ee).toarray()
    b = W.random_u(pb.n_dof)
    x = solve.krylov_apply(lambda v: K @ v, b, 23)
    assert np.linalg.norm(x - np.linalg.solve(K, b)) <= 1e-8 * np.linalg.norm(np.linalg.solve(K, b))


def test_cpfbto_step_contracts_the_tracking_error():
    """Eq. (contractXi): with the Krylov preconditioner and beta = 1,
    ||K(v_k) u_{k+1} - f|| < ||K(v_k) u_k - f|| at every outer iteration
    (Algorithm CPFBTO, line 1)."""
    pb = W.cantilever(16, 8, 8)
    S = outer.Setup(pb)
    rho, u = pb.rho0.copy(), np.zeros(pb.n_dof)
    a0 = None
    for k in range(1, 9):
        _, Ee, _ = S.moduli(rho)
        K = S.K(Ee)
        before = np.linalg.norm(K @ u - S.f)
        u_next, _ = solve.inner_richardson(lambda v: K @ v, S.f, u, lambda r: solve.krylov_apply(lambda v: K @ v, r, 20), 1, 1.0)
        after = np.linalg.norm(K @ u_next - S.f)
        assert after < before
        rho, _, _, a0 = outer.run(pb, 1, precond="krylov", n_inner=1, inner_mode="richardson", beta=1.0,
                                  krylov_dim=20, setup=S, rho=rho, u=u, k0=k, alpha0=a0)
        u = u_next


# ----------------------------------------------------------------------------- PFBTO (Algorithm 2)
def test_pfbto_step_with_the_exact_preconditioner_solves_the_system():
    """M = K, beta = 1: u - K K^-1 K^-1 (K u - f) = K^-1 f in one step."""
    pb, S, Ee = _setup(rho=lambda n: W.random_rho(n))
    K = S.K(Ee).tocsc()
    lu = sp.linalg.splu(K)
    u0 = W.random_u(pb.n_dof)
    u0[pb.fixed_dof] = 0.0
    u1, _ = solve.inner_pfbto(lambda v: K @ v, S.f, u0, lu.solve, 1, 1.0)
    assert np.linalg.norm(u1 - lu.solve(S.f)) <= 1e-10 * np.linalg.norm(lu.solve(S.f))


def test_pfbto_squared_residual_decreases_with_a_small_step():
    """With M = I the step is gradient descent on (1/2)||K u - f||^2 (Eq. optBilevelSqr):
    every step with beta < 2 / lambda_max(K^2) lowers ||K u - f||."""
    pb, S, Ee = _setup(rho=lambda n: W.random_rho(n))
    K = S.K(Ee)
    lmax = float(sp.linalg.eigsh(K, k=1, which="LA", return_eigenvectors=False)[0])
    beta = 1.0 / lmax ** 2
    u = np.zeros(pb.n_dof)
    last = np.linalg.norm(K @ u - S.f)
    for _ in range(10):
        u, _ = solve.inner_pfbto(lambda v: K @ v, S.f, u, lambda r: r, 1, beta)
        now = np.linalg.norm(K @ u - S.f)
        assert now < last
        last = now


def test_pcg_matches_scipy_cg():
    """The oracle's preconditioned CG = scipy's CG with the same Jacobi preconditioner and
    iteration count (an independent implementation of the same recurrence)."""
    import scipy.sparse.linalg as spla
    pb, S, Ee = _setup(rho=lambda n: W.random_rho(n))
    K = S.K(Ee).tocsr()
    D = fem.jacobi_diagonal(pb.nx, pb.ny, pb.nz, Ee, S.ke, pb.fixed_dof)
    for it in (1, 5, 30):
        x, _ = solve.pcg(lambda v: K @ v, S.f, lambda r: r / D, tol=0.0, maxit=it)
        xs, _ = spla.cg(K, S.f, x0=np.zeros_like(S.f), rtol=1e-300, atol=0.0, maxiter=it,
                        M=spla.LinearOperator(K.shape, matvec=lambda r: r / D))
        assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)


def test_richardson_with_the_exact_inverse_solves_in_one_step():
    """Constant-beta step of Algorithms 1 / 3: with M = K^-1 and beta = 1, u_1 = u_0 +
    K^-1 (f - K u_0) is the exact solution from any u_0; r_0 = f - K u_0."""
    pb, S, Ee = _setup(4, 2, 2, rho=lambda n: W.random_rho(n))
    K = S.K(Ee).toarray()
    uex = np.linalg.solve(K, S.f)
    u0 = W.random_u(pb.n_dof, seed=3)
    u1, r0 = solve.inner_richardson(lambda v: K @ v, S.f, u0, lambda r: np.linalg.solve(K, r), 1, 1.0)
    assert np.linalg.norm(u1 - uex) <= 1e-10 * np.linalg.norm(uex)
    assert np.allclose(r0, S.f - K @ u0, rtol=0, atol=1e-14 * np.abs(S.f).max())


def test_richardson_jacobi_matches_the_iteration_matrix_power():
    """n Jacobi-preconditioned steps with constant beta: the error obeys
    e_n = (I - beta D^-1 K)^n e_0 (the closed form of the linear iteration, formed here as
    an explicit dense matrix power), and for beta < 2 / lambda_max(D^-1 K) it contracts in
    the energy norm at every step."""
    pb, S, Ee = _setup(4, 2, 2, rho=lambda n: W.random_rho(n))
    K = S.K(Ee).toarray()
    D = fem.jacobi_diagonal(pb.nx, pb.ny, pb.nz, Ee, S.ke, pb.fixed_dof)
    uex = np.linalg.solve(K, S.f)
    u0 = W.random_u(pb.n_dof, seed=4)
    lam = np.max(np.real(np.linalg.eigvals(K / D[:, None])))
    beta = 1.0 / lam
    G = np.eye(pb.n_dof) - beta * (K / D[:, None])
    n = 7
    un, _ = solve.inner_richardson(lambda v: K @ v, S.f, u0, lambda r: r / D, n, beta)
    en_ref = np.linalg.matrix_power(G, n) @ (u0 - uex)
    assert np.linalg.norm((un - uex) - en_ref) <= 1e-9 * np.linalg.norm(u0 - uex)
    enorm = lambda e: float(np.sqrt(e @ (K @ e)))
    u, prev = u0.copy(), enorm(u0 - uex)
    for _ in range(n):
        u, _ = solve.inner_richardson(lambda v: K @ v, S.f, u, lambda r: r / D, 1, beta)
        cur = enorm(u - uex)
        assert cur < prev
        prev = cur
