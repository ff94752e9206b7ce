"""The allocation-free projection (for callers that may not allocate device
memory) through the C ABI: against the regular entry point on two calls in a row,
against the oracle's Algorithm 4 (Sec. IV-B) at small and at the largest
allowed size, and its sticky device-side error word.  Collected last on purpose:
it shares one static device array across calls."""
import numpy as np
import pytest

import workloads as W
from oracle import project

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_MAX = 1 << 21


def _fb():
    import __graft_entry__ as g
    g.build()
    import paper_2204_06204_gb300 as fb
    return fb


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_projection_matches_to_project(precision):
    fb = _fb()
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


@pytest.mark.parametrize("n", [3456, 100_003, N_MAX])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_projection_matches_algorithm_4(precision, n):
    """The oracle's sorted-breakpoint walk (Algorithm 4) on the very values the GPU
    receives (FP32 inputs rounded first); the volume bound is active and both box
    bounds bind for some elements."""
    fb = _fb()
    dt = torch.float64 if precision == "fp64" else torch.float32
    w_h = W.rng(40 + n % 7).normal(0.3, 0.5, n).astype(np.float64)
    w_h = np.asarray(torch.tensor(w_h, dtype=dt).double().numpy())
    lo, hi, vbar = 0.05, 1.0, 0.25 * n
    ref, lam_ref = project.project_alg4(w_h, vbar, lo, hi)
    assert lam_ref > 0.0 and (ref == lo).any() and (ref == hi).any()
    w = torch.tensor(w_h, dtype=dt, device="cuda")
    out = torch.empty_like(w)
    for _ in range(2):
        lam = fb.to_project_noalloc(w, out, vbar, lo, hi)
        rho = out.double().cpu().numpy()
        if precision == "fp64":
            assert np.abs(rho - ref).max() <= 1e-12
            assert abs(lam - lam_ref) <= 1e-12 * max(1.0, abs(lam_ref))
        else:
            assert np.abs(rho - ref).max() <= 1e-6
            assert abs(lam - lam_ref) <= 1e-6 * max(1.0, abs(lam_ref))


def test_noalloc_errors_are_sticky_until_reported():
    """A NaN in w raises TO_ERR_NONFINITE on the device.  A call without lambda_out does
    not synchronise and returns TO_OK; the next call that asks for lambda reports the
    error and clears it, and the call after that is clean again."""
    fb = _fb()
    n = 4096
    w_h = W.rng(50).normal(0.3, 0.5, n)
    good = torch.tensor(w_h, dtype=torch.float32, device="cuda")
    bad = good.clone()
    bad[17] = float("nan")
    out = torch.empty_like(good)
    fb.to_project_noalloc(bad, out, 0.25 * n, 0.0, 1.0, want_lambda=False)
    with pytest.raises(fb.ToError) as e:
        fb.to_project_noalloc(good, out, 0.25 * n, 0.0, 1.0)
    assert e.value.code == fb._abi.TO_ERR_NONFINITE
    lam = fb.to_project_noalloc(good, out, 0.25 * n, 0.0, 1.0)
    ref, lam_ref = project.project_alg4(good.double().cpu().numpy(), 0.25 * n, 0.0, 1.0)
    assert np.abs(out.double().cpu().numpy() - ref).max() <= 1e-6
    assert abs(lam - lam_ref) <= 1e-6 * max(1.0, lam_ref)


def test_noalloc_rejects_oversize_and_infeasible():
    fb = _fb()
    w = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(fb.ToError) as e:
        fb.to_project_noalloc(w, torch.empty_like(w), vbar=0.5, lo=0.1, hi=1.0)
    assert e.value.code == fb._abi.TO_ERR_INFEASIBLE
    big = torch.zeros(N_MAX + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(fb.ToError) as e:
        fb.to_project_noalloc(big, big, vbar=1.0)
    assert e.value.code == fb._abi.TO_ERR_ARG
