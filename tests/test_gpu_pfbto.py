"""GPU parity of Algorithm PFBTO (Algorithm 2: u <- u - beta K M^-1 M^-1 (K u - f)) against
the oracle, with the Jacobi and the multigrid preconditioner.  Workload: the 16x8x8
cantilever, rho = 0.3.  The steps are below 2 / lambda_max(K M^-2 K) (Jacobi: about 12 ^ 2 /
4; multigrid V-cycle: lambda_max about 11.5, measured by power iteration in the oracle)."""
import numpy as np
import pytest

import workloads as W
from oracle import outer

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fb():
    import __graft_entry__ as g
    g.build()
    import paper_2204_06204_gb300 as fb
    return fb


@pytest.mark.parametrize("precond,beta", [("jacobi", 0.05), ("mg", 0.08)])
def test_pfbto_outer_loop_matches_oracle_fp64(precond, beta):
    fb = _fb()
    pb = W.cantilever(16, 8, 8)
    n = 6
    rho_o, u_o, hist, _ = outer.run(pb, n, precond=precond, n_inner=2, inner_mode="pfbto", beta=beta)
    pc = fb.TO_PRECOND_JACOBI if precond == "jacobi" else fb.TO_PRECOND_MG
    prm = fb.to_default_params(precision=fb.TO_FP64, precond=pc, inner_mode=fb.TO_INNER_PFBTO, beta=beta, n_inner=2)
    with fb.Problem.from_workload(pb, prm) as P:
        st = P.step(n, want_stats=True)
        rho, u, _, _ = P.get_state()
        rho, u = rho.cpu().numpy(), u.cpu().numpy()
    d = [s if isinstance(s, dict) else s.as_dict() for s in st]
    for a, h in zip(d, hist):
        assert abs(a["J"] - h["J"]) <= 1e-8 * max(abs(h["J"]), 1e-30)
        assert abs(a["res2"] - h["res2"]) <= 1e-8 * h["res2"]
    assert np.abs(rho - rho_o).max() <= 1e-8
    assert np.abs(u - u_o).max() <= 1e-8 * np.abs(u_o).max()


def test_pfbto_lower_level_contracts_fp32():
    """On a fixed design, repeated PFBTO steps with the Jacobi M lower ||K u - f||."""
    fb = _fb()
    pb = W.cantilever(32, 16, 16)
    prm = fb.to_default_params(precision=fb.TO_FP32_MIXED, precond=fb.TO_PRECOND_JACOBI,
                               inner_mode=fb.TO_INNER_PFBTO, beta=0.05, n_inner=1)
    with fb.Problem.from_workload(pb, prm) as P:
        u = P.dof()
        u.zero_()
        last = P.inner_solve(u, 0, want_res=True)
        for _ in range(5):
            now = P.inner_solve(u, 4, want_res=True)
            assert now < last
            last = now
