"""The allocation-free projection (for callers that may not allocate device
memory) against the regular entry point, through the C ABI, on two calls in a row.
Collected last on purpose: it shares one static device array across calls."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_projection_matches_to_project(precision):
    import __graft_entry__ as g
    g.build()
    import paper_2204_06204_gb300 as fb
    prec = fb.TO_FP64 if precision == "fp64" else fb.TO_FP32_MIXED
    pb = W.cantilever(24, 12, 12)
    pb.rho_min = 0.05
    tol = 1e-12 if prec == fb.TO_FP64 else 1e-6
    with fb.Problem.from_workload(pb, fb.to_default_params(precision=prec)) as P:
        vbar = pb.volfrac * pb.n_elem
        for call, seed in enumerate((31, 32)):            # two calls in a row, different inputs
            w = torch.tensor(W.rng(seed).normal(0.35, 0.4, pb.n_elem), dtype=P.dtype, device=P.device)
            ref, lam_ref = P.project(w)
            out = torch.empty_like(w)
            lam = fb.to_project_noalloc(w, out, vbar, pb.rho_min, 1.0)
            torch.cuda.synchronize()
            assert torch.max(torch.abs(out - ref)).item() <= tol
            assert abs(lam - lam_ref) <= 1e-12 * max(1.0, abs(lam_ref))
            assert lam > 0.0
            assert abs(out.double().sum().item() - vbar) <= (1e-9 if prec == fb.TO_FP64 else 2e-3)


def test_noalloc_rejects_oversize_and_infeasible():
    import paper_2204_06204_gb300 as fb
    w = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(fb.ToError) as e:
        fb.to_project_noalloc(w, torch.empty_like(w), vbar=0.5, lo=0.1, hi=1.0)
    assert e.value.code == fb._abi.TO_ERR_INFEASIBLE
    big = torch.zeros((1 << 21) + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(fb.ToError) as e:
        fb.to_project_noalloc(big, big, vbar=1.0)
    assert e.value.code == fb._abi.TO_ERR_ARG
