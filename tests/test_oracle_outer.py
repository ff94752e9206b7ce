"""Pins for the oracle's outer loop (Algorithms 1 / 3 and PGD, Sec. V)."""
import numpy as np

import workloads as W
from oracle import outer


def test_bilevel_with_converged_inner_solve_reproduces_nested_exact():
    """With the lower level run to convergence, FBTO is PGD (Sec. V)."""
    pb = W.cantilever(8, 4, 4)
    S = outer.Setup(pb)
    # u_1 = 0, so iteration 1 has g = 0; run PGD and a bilevel loop with many inner steps
    rho_p, u_p, hp, a_p = outer.run(pb, 6, precond="exact", setup=S)
    rho_b, u_b, hb, a_b = outer.run(pb, 6, precond="mg", n_inner=60, setup=S)
    assert abs(a_p - a_b) < 1e-10 * a_p
    assert np.abs(rho_p - rho_b).max() < 1e-10
    for a, b in zip(hp, hb):
        assert abs(a["J"] - b["J"]) <= 1e-10 * max(abs(a["J"]), 1e-30)


def test_outer_loop_feasible_schedule_and_tracks_nested_exact():
    pb = W.cantilever(8, 4, 4)
    S = outer.Setup(pb)
    rho, u, hist, a0 = outer.run(pb, 40, precond="mg", n_inner=2, setup=S)
    assert rho.min() >= pb.rho_min and rho.max() <= 1.0
    assert abs(rho.sum() - S.vbar) < 1e-9 * S.vbar or rho.sum() < S.vbar
    assert hist[0]["J"] == 0.0 and hist[0]["alpha"] == 0.0      # u_1 = 0, so g_1 = 0
    assert a0 is not None and hist[1]["alpha"] > 0
    # the alpha schedule is alpha_0 k^-3/4
    for h in hist[1:]:
        assert abs(h["alpha"] - a0 * h["k"] ** -0.75) < 1e-15 * a0
    # two multigrid-preconditioned steps per iteration follow PGD closely, and both descend
    rho_p, _, _, _ = outer.run(pb, 40, precond="exact", setup=S)
    J0 = S.exact_compliance(pb.rho0)[0]
    Jb = S.exact_compliance(rho)[0]
    Jp = S.exact_compliance(rho_p)[0]
    assert Jb < 0.8 * J0 and Jp < 0.8 * J0
    assert abs(Jb - Jp) < 0.05 * Jp


def test_resume_is_bitwise_identical():
    pb = W.cantilever(8, 4, 4)
    S = outer.Setup(pb)
    rho_a, u_a, _, a0 = outer.run(pb, 8, setup=S)
    rho_1, u_1, _, a01 = outer.run(pb, 3, setup=S)
    rho_b, u_b, _, _ = outer.run(pb, 5, setup=S, rho=rho_1, u=u_1, k0=4, alpha0=a01)
    assert np.array_equal(rho_a, rho_b) and np.array_equal(u_a, u_b)


# ----------------------------------------------------------------------------- mean projection (Sec. IV-B)
def _grad_at(S, pb, rho, u):
    """dJ/drho at (rho, u): the element sensitivity chained through the filter transpose."""
    from oracle import filt
    _, _, Ed = S.moduli(rho)
    return filt.filter_transpose(S.H, S.Hs, S.sens_rho_tilde(Ed, u))


def test_mean_projected_step_is_the_paper_projector():
    """One outer step with the mean projection equals w = rho - alpha (I - 1 1^T / E) g written
    with the projector as an explicit E x E matrix (Sec. IV-B), then projected onto X."""
    from oracle import project
    pb = W.cantilever(4, 2, 2)
    S = outer.Setup(pb)
    a0 = 0.05
    rho2, u2, h1, _ = outer.run(pb, 1, setup=S, alpha0=a0, mean_proj=True)      # k = 1: g = 0
    rho3, u3, h2, _ = outer.run(pb, 1, setup=S, rho=rho2, u=u2, k0=2, alpha0=a0, mean_proj=True)
    E = pb.n_elem
    Pm = np.eye(E) - np.ones((E, E)) / E
    g = _grad_at(S, pb, rho2, u2)
    alpha = a0 * 2.0 ** -0.75
    w = rho2 - alpha * (Pm @ g)
    ref, lam = project.project_alg4(w, S.vbar, pb.rho_min, pb.rho_max)
    assert np.abs(rho3 - ref).max() <= 1e-14
    assert abs(h2[0]["gmax"] - np.abs(Pm @ g).max()) <= 1e-14 * np.abs(g).max()
    assert abs(float(np.ones(E) @ (Pm @ g))) <= 1e-12 * np.abs(g).sum()   # 1^T P g = 0


def test_mean_projection_keeps_volume_when_no_bound_is_active():
    """With the volume and box bounds inactive the mean-projected step moves along
    1^perp: the volume stays at its start value exactly (up to rounding), while the
    plain gradient step changes it."""
    pb = W.cantilever(8, 4, 4, volfrac=0.9, rho_init=0.3)
    S = outer.Setup(pb)
    a0 = 1e-3
    rho_m, _, hm, _ = outer.run(pb, 6, setup=S, alpha0=a0, mean_proj=True)
    rho_p, _, hp, _ = outer.run(pb, 6, setup=S, alpha0=a0, mean_proj=False)
    assert rho_m.min() > pb.rho_min and rho_m.max() < pb.rho_max         # box inactive
    assert all(h["lam"] == 0.0 for h in hm)                               # volume bound inactive
    assert abs(rho_m.sum() - 0.3 * pb.n_elem) <= 1e-12 * pb.n_elem
    assert rho_p.sum() > 0.3 * pb.n_elem + 1e-3                           # compliance gradient < 0 adds volume


def test_mean_projection_only_shifts_the_multiplier_when_the_volume_bound_binds():
    """Proj_X(rho - alpha g) = Proj_X(rho - alpha (g - c 1)) when the volume bound is active
    and no box bound binds (the KKT multiplier absorbs c): same rho, lambda + alpha c."""
    from oracle import project
    pb = W.cantilever(4, 2, 2)
    S = outer.Setup(pb)
    r = W.rng(5)
    rho = r.uniform(0.25, 0.35, pb.n_elem)
    rho *= S.vbar / rho.sum()
    u = W.random_u(pb.n_dof) * 0.1
    g = _grad_at(S, pb, rho, u)
    alpha = 1e-3 / np.abs(g).max()
    a, la = project.project_alg4(rho - alpha * g, S.vbar, pb.rho_min, pb.rho_max)
    b, lb = project.project_alg4(rho - alpha * (g - g.mean()), S.vbar, pb.rho_min, pb.rho_max)
    assert la > 0.0
    assert np.abs(a - b).max() <= 1e-14
    assert abs((lb - la) - alpha * g.mean()) <= 1e-12 * abs(alpha * g.mean())
