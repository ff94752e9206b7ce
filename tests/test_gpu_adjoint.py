"""GPU parity of the differentiable compliance (truncated lower-level solve) against
the oracle's reverse mode, central finite differences, and the autograd path.
Workload: the 64x32x32 cantilever with rho ~ U[0.2, 1] (seeded), T = 5, beta = 0.5."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint, outer

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T_STEPS, BETA = 5, 0.5


def _fb():
    import __graft_entry__ as g
    g.build()
    import paper_2204_06204_gb300 as fb
    return fb


@pytest.fixture(scope="module")
def oracle_64():
    pb = W.cantilever_random_64x32x32()
    S = outer.Setup(pb)
    J, g = adjoint.gradient(S, pb.rho0, T_STEPS, BETA)
    return pb, J, g


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_truncated_compliance_and_gradient_match_oracle(oracle_64, precision):
    fb = _fb()
    pb, Jo, go = oracle_64
    prec = fb.TO_FP64 if precision == "fp64" else fb.TO_FP32_MIXED
    with fb.Problem.from_workload(pb, fb.to_default_params(precision=prec)) as P:
        rho = torch.tensor(pb.rho0, dtype=P.dtype, device=P.device)
        J = fb.to_compliance_truncated(P, rho, T_STEPS, BETA)
        g = P.elem()
        fb.to_compliance_truncated_grad(P, 1.0, g)
        g = g.cpu().numpy().astype(np.float64)
    if prec == fb.TO_FP64:
        assert abs(J - Jo) <= 1e-12 * abs(Jo)
        assert np.abs(g - go).max() <= 1e-10 * np.abs(go).max()
    else:
        assert abs(J - Jo) <= 1e-5 * abs(Jo)
        assert np.abs(g - go).max() <= 1e-4 * np.abs(go).max()


def test_gradient_matches_central_differences_fp64(oracle_64):
    """h = 1e-6 in FP64 on 100 seeded elements."""
    fb = _fb()
    pb, _, _ = oracle_64
    with fb.Problem.from_workload(pb, fb.to_default_params(precision=fb.TO_FP64)) as P:
        rho = torch.tensor(pb.rho0, dtype=torch.float64, device=P.device)
        fb.to_compliance_truncated(P, rho, T_STEPS, BETA)
        g = P.elem()
        fb.to_compliance_truncated_grad(P, 1.0, g)
        g = g.cpu().numpy()
        h = 1e-6
        gmax = np.abs(g).max()
        for e in W.random_elements(pb.n_elem, 100):
            rp = rho.clone()
            rp[int(e)] += h
            rm = rho.clone()
            rm[int(e)] -= h
            fd = (fb.to_compliance_truncated(P, rp, T_STEPS, BETA) - fb.to_compliance_truncated(P, rm, T_STEPS, BETA)) / (2 * h)
            assert abs(g[e] - fd) <= 1e-6 * gmax + 1e-4 * abs(fd)


def test_autograd_function(oracle_64):
    fb = _fb()
    from paper_2204_06204_gb300.autograd import compliance
    pb, Jo, go = oracle_64
    with fb.Problem.from_workload(pb, fb.to_default_params(precision=fb.TO_FP64)) as P:
        rho = torch.tensor(pb.rho0, dtype=torch.float64, device=P.device, requires_grad=True)
        J = compliance(rho, P, T_STEPS, BETA)
        (3.0 * J).backward()
        assert abs(J.item() - Jo) <= 1e-12 * abs(Jo)
        assert np.abs(rho.grad.cpu().numpy() - 3.0 * go).max() <= 1e-10 * 3.0 * np.abs(go).max()


def test_requires_jacobi_preconditioner():
    fb = _fb()
    pb = W.cantilever(8, 4, 4)
    with fb.Problem.from_workload(pb, fb.to_default_params(precond=fb.TO_PRECOND_MG)) as P:
        with pytest.raises(fb.ToError) as e:
            fb.to_compliance_truncated(P, torch.full((pb.n_elem,), 0.5, device=P.device), T_STEPS, BETA)
        assert e.value.code == 7


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("stride", [-1, 2, 3, 9])
def test_recompute_mode_is_bitwise_the_stored_mode(precision, stride):
    """Keeping every s-th iterate and recomputing the rest in the reverse sweep gives the
    very same gradient bits as keeping all of them (same kernels, same order)."""
    fb = _fb()
    pb = W.cantilever(24, 12, 12)
    rho_h = W.random_rho(pb.n_elem, 0.2, 1.0, seed=W.SEED + 21)
    prec = fb.TO_FP64 if precision == "fp64" else fb.TO_FP32_MIXED
    T = 9
    out = {}
    for s in (0, stride):
        with fb.Problem.from_workload(pb, fb.to_default_params(precision=prec, adj_stride=s)) as P:
            rho = torch.tensor(rho_h, dtype=P.dtype, device=P.device)
            J = fb.to_compliance_truncated(P, rho, T, BETA)
            g = P.elem()
            fb.to_compliance_truncated_grad(P, 1.0, g)
            out[s] = (J, g.cpu())
    assert out[0][0] == out[stride][0]
    assert torch.equal(out[0][1], out[stride][1])


def test_gradient_refuses_a_changed_design_and_autograd_is_reentrant(oracle_64):
    """Two forwards on one problem before backward: each graph still gets the gradient of
    its own rho (the Function re-runs its forward when the kept iterates are another's);
    the C call itself refuses a reverse sweep after the design changed."""
    fb = _fb()
    from paper_2204_06204_gb300.autograd import compliance
    pb = W.cantilever(16, 8, 8)
    r1 = W.random_rho(pb.n_elem, 0.2, 1.0, seed=W.SEED + 31)
    r2 = W.random_rho(pb.n_elem, 0.2, 1.0, seed=W.SEED + 32)
    with fb.Problem.from_workload(pb, fb.to_default_params(precision=fb.TO_FP64)) as P:
        ref = []
        for r in (r1, r2):
            rho = torch.tensor(r, dtype=torch.float64, device=P.device)
            fb.to_compliance_truncated(P, rho, T_STEPS, BETA)
            g = P.elem()
            fb.to_compliance_truncated_grad(P, 1.0, g)
            ref.append(g.clone())
        a = torch.tensor(r1, dtype=torch.float64, device=P.device, requires_grad=True)
        b = torch.tensor(r2, dtype=torch.float64, device=P.device, requires_grad=True)
        (compliance(a, P, T_STEPS, BETA) + 2.0 * compliance(b, P, T_STEPS, BETA)).backward()
        assert torch.equal(a.grad, ref[0])
        assert torch.equal(b.grad, 2.0 * ref[1])
        # the C-level reverse sweep after a design change is an error, not a wrong gradient
        fb.to_compliance_truncated(P, a.detach(), T_STEPS, BETA)
        assert fb.to_compliance_truncated_id(P) > 0
        P.set_design(b.detach())
        assert fb.to_compliance_truncated_id(P) == 0
        with pytest.raises(fb.ToError) as e:
            fb.to_compliance_truncated_grad(P, 1.0, P.elem())
        assert e.value.code == fb._abi.TO_ERR_STATE
