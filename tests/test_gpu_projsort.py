"""GPU parity of the projection's multiplier by the paper's parallel form of Algorithm 4
(radix sort of the 2E breakpoints, scans, the crossing segment; Sec. IV-D) against the
oracle's Algorithm 4.  Workloads: seeded w on the 20x10x10 cantilever (the four cases of
the search-based projection tests), and the 16x8x8 outer loop."""
import numpy as np
import pytest

import workloads as W
from oracle import outer, project

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fb():
    import __graft_entry__ as g
    g.build()
    import paper_2204_06204_gb300 as fb
    return fb


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["active", "inactive", "ties", "lower_bound"])
def test_sorted_projection_matches_algorithm4(precision, case):
    fb = _fb()
    pb = W.cantilever(20, 10, 10)
    r = W.rng(7)
    if case == "active":
        w = r.normal(0.3, 0.5, pb.n_elem)
    elif case == "inactive":
        w = r.uniform(0.0, 0.5, pb.n_elem)
    elif case == "ties":
        w = np.round(r.normal(0.4, 0.5, pb.n_elem), 1)
    else:
        pb.rho_min = 0.1
        w = r.normal(0.35, 0.3, pb.n_elem)
    prec = fb.TO_FP64 if precision == "fp64" else fb.TO_FP32_MIXED
    with fb.Problem.from_workload(pb, fb.to_default_params(precision=prec, proj_sort=1)) as P:
        wt = torch.tensor(w, dtype=P.dtype, device=P.device)
        rho, lam = P.project(wt)
        wd = wt.cpu().numpy().astype(np.float64)
        vref, lref = project.project_alg4(wd, pb.volfrac * pb.n_elem, pb.rho_min, 1.0)
        rho = rho.cpu().numpy()
    tol = 1e-12 if prec == fb.TO_FP64 else 1e-6
    assert np.abs(rho - vref).max() <= tol
    if prec == fb.TO_FP64:
        assert abs(lam - lref) <= 1e-12 * max(1.0, abs(lref))


def test_outer_loop_with_sorted_projection_matches_oracle_fp64():
    fb = _fb()
    pb = W.cantilever(16, 8, 8)
    n = 10
    rho_o, _, hist, _ = outer.run(pb, n, precond="jacobi", n_inner=5)
    with fb.Problem.from_workload(pb, fb.to_default_params(precision=fb.TO_FP64, proj_sort=1)) as P:
        st = P.step(n, want_stats=True)
        rho = P.get_state()[0].cpu().numpy()
    d = [s if isinstance(s, dict) else s.as_dict() for s in st]
    for a, h in zip(d, hist):
        assert abs(a["lambda"] - h["lam"]) <= 1e-10 * max(1.0, abs(h["lam"]))
    assert np.abs(rho - rho_o).max() <= 1e-10
