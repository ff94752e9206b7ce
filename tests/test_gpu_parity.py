"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, on the same
seeded inputs.  Tolerances:
  FP64 path   -- rounding only: element-wise 1e-12 relative to the vector's max
  FP32-mixed  -- K(rho)u: ||y - y_ref||_2 / || |K| |u| ||_2 <= 1e-5 (|K| the entrywise
                 absolute value; the plain relative error is amplified by cancellation),
                 sensitivities 1e-4 relative to max |g|, final compliance 1e-3,
                 mean per-element |drho| 1e-2
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import fem, filt, outer, project, solve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fb():
    import __graft_entry__ as g
    g.build()
    import paper_2204_06204_gb300 as fb
    return fb


def _problem(pb, precision, **kw):
    fb = _fb()
    prm = fb.to_default_params(precision=precision, **kw)
    return fb.Problem.from_workload(pb, prm)


def _t(x, P):
    return torch.tensor(np.asarray(x), dtype=P.dtype, device=P.device)


GRIDS = [(1, 1, 1), (3, 2, 5), (17, 9, 5), (32, 16, 16), (40, 20, 9)]
# grids for the TMA-staged kernel (op_kernel 1): one and several 64-column tiles, ragged x
# and y, tiles whose column element lies outside the grid, tiles of 8 node rows and fewer
TMA_GRIDS = [(17, 9, 5), (32, 16, 16), (40, 20, 9), (64, 8, 8), (65, 9, 3), (100, 23, 6), (130, 10, 4)]


@pytest.mark.parametrize("dims,precision,op_kernel",
                         [(d, p, 0) for d in GRIDS for p in ("fp64", "fp32")] + [(d, "fp32", 1) for d in TMA_GRIDS]
                         + [(d, "fp32", 2) for d in GRIDS + TMA_GRIDS[2:]])
def test_apply_K_matches_assembled_operator(dims, precision, op_kernel):
    fb = _fb()
    pb = W.cantilever(*dims)
    pb.rho0 = W.random_rho(pb.n_elem, 0.0, 1.0)
    prec = fb.TO_FP64 if precision == "fp64" else fb.TO_FP32_MIXED
    with _problem(pb, prec, op_kernel=op_kernel) as P:
        P.set_design(_t(pb.rho0, P))
        S = outer.Setup(pb)
        _, Ee_ref, _ = S.moduli(pb.rho0)
        # moduli from the device design so the comparison isolates the operator
        K = S.K(Ee_ref)
        for seed in (0, 1):
            u = W.random_u(pb.n_dof, seed=100 + seed)
            y = P.apply_K(_t(u, P)).cpu().numpy().astype(np.float64)
            yref = K @ u
            if prec == fb.TO_FP64:
                assert np.abs(y - yref).max() <= 1e-12 * np.abs(yref).max()
            else:
                Kabs = abs(K)
                scale = np.linalg.norm(Kabs @ np.abs(u))
                assert np.linalg.norm(y - yref) / scale <= 1e-5


def test_tensor_core_operator_is_the_kernel_that_runs():
    """op_kernel 2 computes K^ x with split-BF16 products on the tensor cores: within the
    FP32 tolerance of the general kernel's result, but not bitwise equal to it (a silent
    fall-back to the general kernel would be)."""
    fb = _fb()
    pb = W.cantilever(40, 20, 9)
    pb.rho0 = W.random_rho(pb.n_elem, 0.0, 1.0)
    u = W.random_u(pb.n_dof, seed=7)
    ys = []
    for ok in (0, 2):
        with _problem(pb, fb.TO_FP32_MIXED, op_kernel=ok) as P:
            P.set_design(_t(pb.rho0, P))
            ys.append(P.apply_K(_t(u, P)).cpu().numpy().astype(np.float64))
    S = outer.Setup(pb)
    _, Ee_ref, _ = S.moduli(pb.rho0)
    scale = np.linalg.norm(abs(S.K(Ee_ref)) @ np.abs(u))
    assert np.linalg.norm(ys[1] - ys[0]) / scale <= 1e-5
    assert not np.array_equal(ys[0], ys[1])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_filter_forward_and_transpose(precision):
    fb = _fb()
    for dims, r in (((7, 5, 4), 1.5), ((9, 6, 6), 2.5), ((3, 3, 3), 0.5)):
        pb = W.cantilever(*dims, rmin=r)
        prec = fb.TO_FP64 if precision == "fp64" else fb.TO_FP32_MIXED
        with _problem(pb, prec) as P:
            H, Hs = filt.filter_matrix(*dims, r)
            x = W.random_rho(pb.n_elem, -1.0, 1.0)
            tol = 1e-13 if prec == fb.TO_FP64 else 2e-6
            for tr in (False, True):
                y = P.filter(_t(x, P), transpose=tr).cpu().numpy()
                yref = filt.filter_transpose(H, Hs, x) if tr else filt.filter_forward(H, Hs, x)
                assert np.abs(y - yref).max() <= tol * max(np.abs(yref).max(), 1.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_filter_multi_tile_ragged(precision):
    """Grids spanning several 32 x 8 tiles and z chunks with ragged edges (100 = 3 * 32 + 4,
    50 = 6 * 8 + 2, 37 planes in chunks of 2), for both radii of the workloads."""
    fb = _fb()
    for dims, r in (((100, 50, 37), 1.5), ((70, 30, 21), 2.5)):
        pb = W.cantilever(*dims, rmin=r)
        prec = fb.TO_FP64 if precision == "fp64" else fb.TO_FP32_MIXED
        with _problem(pb, prec) as P:
            H, Hs = filt.filter_matrix(*dims, r)
            x = W.random_rho(pb.n_elem, -1.0, 1.0)
            tol = 1e-13 if prec == fb.TO_FP64 else 2e-6
            for tr in (False, True):
                y = P.filter(_t(x, P), transpose=tr).cpu().numpy()
                yref = filt.filter_transpose(H, Hs, x) if tr else filt.filter_forward(H, Hs, x)
                assert np.abs(y - yref).max() <= tol * max(np.abs(yref).max(), 1.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sensitivity(precision):
    fb = _fb()
    pb = W.cantilever(12, 6, 5)
    pb.rho0 = W.random_rho(pb.n_elem)
    prec = fb.TO_FP64 if precision == "fp64" else fb.TO_FP32_MIXED
    with _problem(pb, prec) as P:
        P.set_design(_t(pb.rho0, P))
        S = outer.Setup(pb)
        _, _, Ed = S.moduli(pb.rho0)
        u = W.random_u(pb.n_dof)
        g = P.sensitivity(_t(u, P)).cpu().numpy()
        gref = filt.filter_transpose(S.H, S.Hs, S.sens_rho_tilde(Ed, u))
        tol = 1e-12 if prec == fb.TO_FP64 else 1e-4
        assert np.abs(g - gref).max() <= tol * np.abs(gref).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["active", "inactive", "ties", "lower_bound"])
def test_projection(precision, case):
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
    with _problem(pb, prec) as P:
        wt = _t(w, P)
        rho, lam = P.project(wt)
        wd = wt.cpu().numpy().astype(np.float64)   # the same rounded input on both sides
        vref, lref = project.project_alg4(wd, pb.volfrac * pb.n_elem, pb.rho_min, 1.0)
        rho = rho.cpu().numpy()
        tol = 1e-12 if prec == fb.TO_FP64 else 1e-6
        assert np.abs(rho - vref).max() <= tol
        vol = rho.astype(np.float64).sum()
        if lref > 0:       # active bound: the volume is met with equality
            assert abs(vol - pb.volfrac * pb.n_elem) <= (1e-9 if prec == fb.TO_FP64 else 2e-3)
        else:
            assert vol <= pb.volfrac * pb.n_elem * (1 + 1e-12) and lam == 0.0
        assert (case == "inactive") == (lref == 0.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_inner_steps_jacobi_sd(precision):
    fb = _fb()
    pb = W.cantilever(16, 8, 8)
    pb.rho0 = W.random_rho(pb.n_elem)
    prec = fb.TO_FP64 if precision == "fp64" else fb.TO_FP32_MIXED
    with _problem(pb, prec, n_inner=5) as P:
        P.set_design(_t(pb.rho0, P))
        S = outer.Setup(pb)
        _, Ee, _ = S.moduli(pb.rho0)
        K = S.K(Ee)
        D = fem.jacobi_diagonal(pb.nx, pb.ny, pb.nz, Ee, S.ke, pb.fixed_dof)
        u0 = W.random_u(pb.n_dof) * S.m * 1e-2
        ut = _t(u0, P)
        res = P.inner_solve(ut, 7, want_res=True)
        uref, rref, _, _ = solve.inner_sd(lambda x: K @ x, S.f, u0, lambda r: r / D, 7)
        u = ut.cpu().numpy()
        tol = 1e-10 if prec == fb.TO_FP64 else 1e-4
        assert np.abs(u - uref).max() <= tol * np.abs(uref).max()
        assert abs(res - np.linalg.norm(S.f - K @ uref)) <= (1e-9 if prec == fb.TO_FP64 else 1e-3) * np.linalg.norm(S.f)


def test_outer_loop_fp64_matches_oracle_cantilever_32x16x16():
    """Plain FP64, Jacobi steepest descent x5, the 32x16x16 cantilever, 50 outer iterations."""
    fb = _fb()
    pb = W.cantilever_32x16x16()
    n = 50
    with _problem(pb, fb.TO_FP64, n_inner=5) as P:
        st = P.step(n)
        rho, u, k, a0 = P.get_state()
    rho_o, u_o, hist, a0_o = outer.run(pb, n, precond="jacobi", n_inner=5)
    assert k == n + 1
    assert abs(a0 - a0_o) <= 1e-10 * a0_o
    J = np.array([s["J"] for s in st])
    Jo = np.array([h["J"] for h in hist])
    assert np.abs(J - Jo).max() <= 1e-8 * np.abs(Jo).max()
    assert np.abs(rho.cpu().numpy() - rho_o).max() <= 1e-8
    for s, h in zip(st, hist):
        assert abs(s["volume"] - h["volume"]) <= 1e-8 * h["volume"]
        assert abs(s["res_inf"] - h["res_inf"]) <= 1e-8 * max(h["res_inf"], 1e-30)


@pytest.mark.parametrize("op_kernel", [0, 1, 2])
def test_outer_loop_fp32_mixed_matches_oracle_compliance(op_kernel):
    fb = _fb()
    pb = W.cantilever_32x16x16()
    n = 50
    with _problem(pb, fb.TO_FP32_MIXED, n_inner=5, op_kernel=op_kernel) as P:
        P.step(n)
        rho, u, k, a0 = P.get_state()
    rho_o, u_o, hist, a0_o = outer.run(pb, n, precond="jacobi", n_inner=5)
    S = outer.Setup(pb)
    Jg = S.exact_compliance(rho.cpu().numpy().astype(np.float64))[0]
    Jo = S.exact_compliance(rho_o)[0]
    assert abs(Jg - Jo) <= 1e-3 * Jo
    assert np.abs(rho.cpu().numpy() - rho_o).mean() <= 1e-2


def test_resume_bitwise_identical():
    fb = _fb()
    pb = W.cantilever(16, 8, 8)
    with _problem(pb, fb.TO_FP32_MIXED) as P:
        P.step(6, want_stats=False)
        rho_a, u_a, k_a, a0_a = P.get_state()
    with _problem(pb, fb.TO_FP32_MIXED) as P:
        P.step(2, want_stats=False)
        rho_m, u_m, k_m, a0_m = P.get_state()
    with _problem(pb, fb.TO_FP32_MIXED) as P:
        P.set_state(rho_m, u_m, k_m, a0_m)
        P.step(4, want_stats=False)
        rho_b, u_b, k_b, a0_b = P.get_state()
    assert k_a == k_b == 7
    assert torch.equal(rho_a, rho_b) and torch.equal(u_a, u_b)


def test_apply_K_full_size_sampled_nodes():
    """128x64x64 in the launch configuration of the benchmark: y at 300 sampled nodes
    computed by the oracle one node at a time (the 8 surrounding elements)."""
    fb = _fb()
    pb = W.cantilever_128x64x64()
    pb.rho0 = W.random_rho(pb.n_elem, 0.0, 1.0)
    with _problem(pb, fb.TO_FP32_MIXED) as P:
        P.set_design(_t(pb.rho0, P))
        u = W.random_u(pb.n_dof)
        y = P.apply_K(_t(u, P)).cpu().numpy().astype(np.float64)
    S_ke = fem.ke_hex8(pb.nu)
    H, Hs = filt.filter_matrix(pb.nx, pb.ny, pb.nz, pb.rmin)
    Ee = fem.young(filt.filter_forward(H, Hs, pb.rho0), pb.E0, pb.Emin, pb.p)
    m = fem.free_mask(pb.n_dof, pb.fixed_dof)
    um = m * u
    nx, ny, nz = pb.nx, pb.ny, pb.nz
    r = W.rng(11)
    nodes = r.integers(0, pb.n_node, 300)
    for n in nodes:
        i, j, k = n % (nx + 1), (n // (nx + 1)) % (ny + 1), n // ((nx + 1) * (ny + 1))
        acc = np.zeros(3)
        absacc = np.zeros(3)
        for dk in (-1, 0):
            for dj in (-1, 0):
                for di in (-1, 0):
                    ei, ej, ek = i + di, j + dj, k + dk
                    if not (0 <= ei < nx and 0 <= ej < ny and 0 <= ek < nz):
                        continue
                    e = ei + nx * (ej + ny * ek)
                    l = [tuple(o) for o in fem.LOCAL_NODES].index((-di, -dj, -dk))
                    dofs = fem.element_dofs(1, 1, 1)[0]
                    gn = [(ei + a) + (nx + 1) * ((ej + b) + (ny + 1) * (ek + c)) for a, b, c in fem.LOCAL_NODES]
                    ue = np.array([um[3 * q + c] for q in gn for c in range(3)])
                    acc += Ee[e] * (S_ke[3 * l:3 * l + 3] @ ue)
                    absacc += Ee[e] * (np.abs(S_ke[3 * l:3 * l + 3]) @ np.abs(ue))
        for c in range(3):
            d = 3 * n + c
            ref = acc[c] * m[d] + (1 - m[d]) * u[d]
            assert abs(y[d] - ref) <= 1e-5 * max(absacc[c], 1e-30) + 1e-7 * abs(u[d]) * (1 - m[d])


def test_error_paths_do_not_trap():
    fb = _fb()
    pb = W.cantilever(4, 2, 2)
    mat = dict(E0=1.0, Emin=1e-9, nu=0.3, p=3.0, volfrac=0.3, rmin=1.5, rho_min=0.5, rho_max=1.0)
    with pytest.raises(fb.ToError) as e:
        fb.Problem(4, 2, 2, mat, pb.load_dof, pb.load_val, pb.fixed_dof)
    assert e.value.code == 4                              # infeasible: vbar < n lo
    mat["rho_min"] = 0.0
    with pytest.raises(fb.ToError) as e:
        fb.Problem(4, 2, 2, mat, pb.load_dof, pb.load_val, [])
    assert e.value.code == 6                              # no fixture: singular
    with _problem(pb, fb.TO_FP32_MIXED) as P:
        bad = torch.full((pb.n_elem,), float("nan"), dtype=P.dtype, device=P.device)
        P.set_design(bad)
        with pytest.raises(fb.ToError) as e:
            P.check()
        assert e.value.code == 3                          # non-finite design reported, context alive
        y = P.apply_K(torch.zeros(pb.n_dof, dtype=P.dtype, device=P.device))
        torch.cuda.synchronize()
