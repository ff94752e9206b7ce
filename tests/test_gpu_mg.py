"""GPU parity of the multigrid-preconditioned path against the oracle's V-cycle
(same definition, independent code): lower-level steps, and the outer loop on the
cantilever and on the MBB half model (different fixtures reach the coarse masks)."""
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


def _t(x, P):
    return torch.tensor(np.asarray(x), dtype=P.dtype, device=P.device)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dims", [(16, 8, 8), (24, 8, 16)])
def test_mg_inner_steps(precision, dims):
    fb = _fb()
    pb = W.cantilever(*dims)
    pb.rho0 = W.random_rho(pb.n_elem, 0.01, 1.0)
    prec = fb.TO_FP64 if precision == "fp64" else fb.TO_FP32_MIXED
    prm = fb.to_default_params(precision=prec, precond=fb.TO_PRECOND_MG, n_inner=2)
    with fb.Problem.from_workload(pb, prm) as P:
        P.set_design(_t(pb.rho0, P))
        S = outer.Setup(pb)
        _, Ee, _ = S.moduli(pb.rho0)
        K = S.K(Ee)
        mg = solve.Multigrid(pb.nx, pb.ny, pb.nz, pb.h, Ee, pb.nu, pb.fixed_dof)
        u0 = np.zeros(pb.n_dof)
        ut = _t(u0, P)
        res = P.inner_solve(ut, 4, want_res=True)
        uref, _, _, _ = solve.inner_sd(lambda x: K @ x, S.f, u0, mg, 4)
        u = ut.cpu().numpy()
        tol = 1e-10 if prec == fb.TO_FP64 else 2e-4
        assert np.abs(u - uref).max() <= tol * np.abs(uref).max()
        # the V-cycle contracts: four preconditioned steps reduce the residual
        assert res < 0.5 * np.linalg.norm(S.f)


@pytest.mark.parametrize("which", ["cantilever", "mbb"])
def test_mg_outer_loop_fp64_matches_oracle(which):
    fb = _fb()
    pb = W.cantilever(16, 8, 8) if which == "cantilever" else W.mbb_half(16, 8, 8)
    n = 15
    prm = fb.to_default_params(precision=fb.TO_FP64, precond=fb.TO_PRECOND_MG, n_inner=2)
    with fb.Problem.from_workload(pb, prm) as P:
        st = P.step(n)
        rho, u, k, a0 = P.get_state()
    rho_o, u_o, hist, a0_o = outer.run(pb, n, precond="mg", n_inner=2)
    assert np.abs(rho.cpu().numpy() - rho_o).max() <= 1e-8
    J = np.array([s["J"] for s in st])
    Jo = np.array([h["J"] for h in hist])
    assert np.abs(J - Jo).max() <= 1e-8 * np.abs(Jo).max()
    b = np.array([s["beta_first"] for s in st[1:]])
    bo = np.array([h["betas"][0] for h in hist[1:]])
    assert np.abs(b - bo).max() <= 1e-8 * np.abs(bo).max()


def test_mg_outer_loop_fp32_compliance():
    fb = _fb()
    pb = W.cantilever(32, 16, 16)
    n = 30
    prm = fb.to_default_params(precision=fb.TO_FP32_MIXED, precond=fb.TO_PRECOND_MG, n_inner=2)
    with fb.Problem.from_workload(pb, prm) as P:
        P.step(n)
        rho, u, k, a0 = P.get_state()
    rho_o, u_o, hist, a0_o = outer.run(pb, n, precond="mg", n_inner=2)
    S = outer.Setup(pb)
    Jg = S.exact_compliance(rho.cpu().numpy().astype(np.float64))[0]
    Jo = S.exact_compliance(rho_o)[0]
    assert abs(Jg - Jo) <= 1e-3 * Jo
    assert np.abs(rho.cpu().numpy() - rho_o).mean() <= 1e-2


def test_mg_rejects_grid_without_coarse_levels():
    fb = _fb()
    pb = W.cantilever(17, 9, 5)
    prm = fb.to_default_params(precond=fb.TO_PRECOND_MG)
    with pytest.raises(fb.ToError) as e:
        fb.Problem.from_workload(pb, prm)
    assert e.value.code == 1


def test_mg_repeatable_with_large_coarsest_inverse():
    """Two problem instances stepped the same way give bitwise identical designs.  The
    coarsest inverse (here 300 DOFs: the in-place Gauss-Jordan in global memory) runs on a
    forked stream branch; every refresh outside the outer iteration joins it at once, so a
    later iteration cannot reassemble the coarse operator under a running inverse."""
    fb = _fb()
    pb = W.batch_cantilevers(6)[1]   # 32 x 24 x 32: coarsest 4 x 3 x 4
    prm = fb.to_default_params(precision=fb.TO_FP64, precond=fb.TO_PRECOND_MG, n_inner=2)
    out = []
    for _ in range(3):
        with fb.Problem.from_workload(pb, prm) as P:
            st = P.step(4)
            out.append((P.get_state()[0].cpu().numpy(), [s["J"] for s in st]))
    for rho, J in out[1:]:
        assert np.array_equal(rho, out[0][0])
        assert J == out[0][1]


def test_mg_problems_with_different_tail_sizes_coexist():
    """The tail kernel's shared-memory opt-in is per kernel: creating a problem with a
    small coarse tail after one with a large tail must not break the first one."""
    fb = _fb()
    prm = fb.to_default_params(precision=fb.TO_FP32_MIXED, precond=fb.TO_PRECOND_MG, n_inner=2)
    big = fb.Problem.from_workload(W.cantilever(32, 16, 16), prm)     # tail from 16 x 8 x 8 (1024 elements)
    small = fb.Problem.from_workload(W.cantilever(16, 8, 8), prm)     # tail from 8 x 4 x 4 (128 elements)
    try:
        st_small = small.step(2)
        st_big = big.step(3)
        assert all(np.isfinite(s["J"]) for s in st_big + st_small)
        assert st_big[-1]["J"] > 0.0
    finally:
        big.close()
        small.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("which,dims", [("cantilever", (128, 64, 64)), ("cantilever", (64, 32, 32)), ("mbb", (64, 32, 48))])
def test_persistent_legs_are_bitwise_the_launch_per_step_v_cycle(which, dims, precision):
    """The cooperative down / up legs over levels 1 .. tail - 1 run the same steps on the same
    buffers in the same order as one launch per step: the outer iterations agree bit for bit."""
    fb = _fb()
    pb = W.cantilever(*dims) if which == "cantilever" else W.mbb_half(*dims)
    prec = fb.TO_FP64 if precision == "fp64" else fb.TO_FP32_MIXED
    out = {}
    for legs in (0, 1):
        prm = fb.to_default_params(precision=prec, precond=fb.TO_PRECOND_MG, n_inner=2, mg_legs=legs)
        with fb.Problem.from_workload(pb, prm) as P:
            st = P.step(4)
            rho, u, k, a0 = P.get_state()
            out[legs] = (rho.cpu(), u.cpu(), [s["J"] for s in st], [s["beta_first"] for s in st])
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] and out[0][3] == out[1][3]
