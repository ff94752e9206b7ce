"""GPU parity of the preconditioned-CG lower-level mode (the near-exact solve of the
nested method, PGD, Sec. V) against the oracle's CG.  Workload: the 16x8x8 cantilever,
rho ~ U[0, 1] (seeded) for the single solves, rho = 0.3 for the outer loop."""
import numpy as np
import pytest

import workloads as W
from oracle import fem, outer, solve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fb():
    import __graft_entry__ as g
    g.build()
    import paper_2204_06204_gb300 as fb
    return fb


@pytest.mark.parametrize("precond,iters", [("jacobi", 30), ("mg", 10)])
def test_pcg_iterations_match_oracle_fp64(precond, iters):
    fb = _fb()
    pb = W.cantilever(16, 8, 8)
    rho = W.random_rho(pb.n_elem)
    S = outer.Setup(pb)
    _, Ee, _ = S.moduli(rho)
    K = S.K(Ee)
    if precond == "jacobi":
        D = fem.jacobi_diagonal(pb.nx, pb.ny, pb.nz, Ee, S.ke, pb.fixed_dof)
        Minv = lambda r: r / D
    else:
        Minv = solve.Multigrid(pb.nx, pb.ny, pb.nz, pb.h, Ee, pb.nu, pb.fixed_dof)
    ref, _ = solve.pcg(lambda v: K @ v, S.f, Minv, tol=0.0, maxit=iters)
    pc = fb.TO_PRECOND_JACOBI if precond == "jacobi" else fb.TO_PRECOND_MG
    prm = fb.to_default_params(precision=fb.TO_FP64, precond=pc, inner_mode=fb.TO_INNER_PCG, n_inner=iters)
    with fb.Problem.from_workload(pb, prm) as P:
        P.set_design(torch.tensor(rho, dtype=torch.float64, device=P.device))
        u = P.dof()
        u.zero_()
        res = P.inner_solve(u, iters, want_res=True)
        u = u.cpu().numpy()
    assert np.linalg.norm(u - ref) <= 1e-8 * np.linalg.norm(ref)
    assert abs(res - np.linalg.norm(S.f - K @ ref)) <= 1e-8 * np.linalg.norm(S.f)


def test_nested_method_outer_loop_matches_oracle_fp64():
    """PGD with the lower level solved by 20 multigrid-preconditioned CG iterations."""
    fb = _fb()
    pb = W.cantilever(16, 8, 8)
    n = 5
    rho_o, u_o, hist, _ = outer.run(pb, n, precond="mg", n_inner=20, inner_mode="pcg")
    prm = fb.to_default_params(precision=fb.TO_FP64, precond=fb.TO_PRECOND_MG, inner_mode=fb.TO_INNER_PCG, n_inner=20)
    with fb.Problem.from_workload(pb, prm) as P:
        st = P.step(n, want_stats=True)
        rho = P.get_state()[0].cpu().numpy()
    d = [s if isinstance(s, dict) else s.as_dict() for s in st]
    for a, h in zip(d, hist):
        assert abs(a["J"] - h["J"]) <= 1e-8 * max(abs(h["J"]), 1e-30)
    assert np.abs(rho - rho_o).max() <= 1e-8
