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
