"""GPU parity of the mean-projected gradient step (Sec. IV-B: the step uses
g - 1 1^T g / E) against the oracle's outer loop, with the volume bound active
(the projection's multiplier absorbs the shift) and inactive (the mean projection
changes the design and keeps the volume)."""
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


CASES = {
    "bound_active": lambda: W.cantilever(16, 8, 8),
    "bound_inactive": lambda: W.cantilever(16, 8, 8, volfrac=0.9, rho_init=0.3),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mean_projected_outer_loop_matches_oracle(case, precision):
    fb = _fb()
    pb = CASES[case]()
    n = 10 if precision == "fp64" else 5
    prec = fb.TO_FP64 if precision == "fp64" else fb.TO_FP32_MIXED
    prm = fb.to_default_params(precision=prec, n_inner=5, mean_proj=1)
    with fb.Problem.from_workload(pb, prm) as P:
        rho0 = torch.tensor(pb.rho0, dtype=P.dtype, device=P.device)
        P.set_state(rho0, None, 1, 0.0)
        st = P.step(n)
        rho, u, k, a0 = P.get_state()
    rho_o, u_o, hist, a0_o = outer.run(pb, n, precond="jacobi", n_inner=5, mean_proj=True)
    rho = rho.double().cpu().numpy()
    if prec == fb.TO_FP64:
        assert abs(a0 - a0_o) <= 1e-10 * a0_o
        assert np.abs(rho - rho_o).max() <= 1e-10
        for s, h in zip(st, hist):
            assert abs(s["gmax"] - h["gmax"]) <= 1e-10 * max(h["gmax"], 1e-30)
            # lambda shifts w (values of order one): compare it on that scale
            assert abs(s["lambda"] - h["lam"]) <= 1e-10 * max(abs(h["lam"]), 1.0)
            assert abs(s["volume"] - h["volume"]) <= 1e-10 * h["volume"]
    else:
        assert abs(a0 - a0_o) <= 1e-4 * a0_o
        assert np.abs(rho - rho_o).max() <= 1e-4
        for s, h in zip(st, hist):
            assert abs(s["gmax"] - h["gmax"]) <= 1e-4 * max(h["gmax"], 1e-30)
    if case == "bound_inactive":
        # the step lies in 1^perp: the volume stays at 0.3 E while the bound is inactive
        assert all(s["lambda"] == 0.0 for s in st)
        tol = 1e-9 if prec == fb.TO_FP64 else 1e-3
        assert abs(st[-1]["volume"] - 0.3 * pb.n_elem) <= tol * pb.n_elem
