"""Batched problems (one launch per phase for all) against the same problems
advanced one at a time, and against the oracle."""
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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_matches_single_problem_path(precision):
    fb = _fb()
    pbs = W.batch_cantilevers(6)
    prec = fb.TO_FP64 if precision == "fp64" else fb.TO_FP32_MIXED
    prm = fb.to_default_params(precision=prec, n_inner=5)
    n = 8
    singles = []
    for pb in pbs:
        with fb.Problem.from_workload(pb, prm) as P:
            st = P.step(n)
            rho, u, k, a0 = P.get_state()
            singles.append((rho.cpu().numpy().astype(np.float64), st))
    probs = [fb.Problem.from_workload(pb, prm) for pb in pbs]
    with fb.Batch(probs) as B:
        stats = B.step(n)
    tol = 1e-10 if prec == fb.TO_FP64 else 1e-4
    for P, (rho_s, st_s), st_b in zip(probs, singles, stats):
        rho_b, _, k, _ = P.get_state()
        assert k == n + 1
        assert np.abs(rho_b.cpu().numpy() - rho_s).max() <= tol
        for a, b in zip(st_s, st_b):
            assert abs(a["J"] - b["J"]) <= tol * max(abs(a["J"]), 1e-30) * 10
            assert abs(a["volume"] - b["volume"]) <= tol * a["volume"] * 10
        P.close()


def test_batch_against_oracle_and_uneven_sizes():
    fb = _fb()
    pbs = [W.cantilever(16, 8, 8), W.cantilever(24, 16, 8, volfrac=0.25), W.cantilever(12, 6, 6, load_k=3)]
    prm = fb.to_default_params(precision=fb.TO_FP64, n_inner=5)
    probs = [fb.Problem.from_workload(pb, prm) for pb in pbs]
    with fb.Batch(probs) as B:
        stats = B.step(12)
    for pb, P, st in zip(pbs, probs, stats):
        rho, _, _, _ = P.get_state()
        rho_o, _, hist, _ = outer.run(pb, 12, precond="jacobi", n_inner=5)
        assert np.abs(rho.cpu().numpy() - rho_o).max() <= 1e-8
        for s, h in zip(st, hist):
            assert abs(s["J"] - h["J"]) <= 1e-8 * max(abs(h["J"]), 1e-30)
        P.close()


def test_batch_rejects_mixed_settings():
    fb = _fb()
    a = fb.Problem.from_workload(W.cantilever(8, 4, 4), fb.to_default_params(n_inner=5))
    b = fb.Problem.from_workload(W.cantilever(8, 4, 4), fb.to_default_params(n_inner=3))
    with pytest.raises(fb.ToError):
        fb.Batch([a, b])
    a.close()
    b.close()


def test_batch_tile_autotuner_picks_a_candidate():
    fb = _fb()
    pbs = W.batch_cantilevers(4)
    probs = [fb.Problem.from_workload(p, fb.to_default_params(precision=fb.TO_FP32_MIXED)) for p in pbs]
    try:
        with fb.Batch(probs) as B:
            kc, us = B.tile()
            assert kc in (2, 4, 8, 16, 32) and us > 0.0
            B.step(2, want_stats=False)
    finally:
        for P in probs:
            P.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_mg_matches_single_problem_path(precision):
    """Multigrid-preconditioned batches (the V-cycle's steps batched per level, every
    problem's coarse tail in one launch) against the same problems stepped alone."""
    fb = _fb()
    pbs = W.batch_cantilevers(6)
    prec = fb.TO_FP64 if precision == "fp64" else fb.TO_FP32_MIXED
    prm = fb.to_default_params(precision=prec, precond=fb.TO_PRECOND_MG, n_inner=2)
    n = 8
    singles = []
    for pb in pbs:
        with fb.Problem.from_workload(pb, prm) as P:
            st = P.step(n)
            rho, u, k, a0 = P.get_state()
            singles.append((rho.cpu().numpy().astype(np.float64), u.cpu().numpy().astype(np.float64), st))
    probs = [fb.Problem.from_workload(pb, prm) for pb in pbs]
    with fb.Batch(probs) as B:
        stats = B.step(n)
    tol = 1e-10 if prec == fb.TO_FP64 else 1e-4
    for P, (rho_s, u_s, st_s), st_b in zip(probs, singles, stats):
        rho_b, u_b, k, _ = P.get_state()
        assert k == n + 1
        assert np.abs(rho_b.cpu().numpy() - rho_s).max() <= tol
        assert np.abs(u_b.cpu().numpy() - u_s).max() <= tol * np.abs(u_s).max() * 10
        for a, b in zip(st_s, st_b):
            assert abs(a["J"] - b["J"]) <= tol * max(abs(a["J"]), 1e-30) * 10
            assert abs(a["beta_first"] - b["beta_first"]) <= tol * max(abs(a["beta_first"]), 1e-30) * 10
        P.close()


def test_batch_mg_against_oracle_uneven_depths():
    """Problems whose V-cycles differ in depth (one or two levels before the coarse
    tail, or a tail of the dense solve alone), fixtures (cantilever, MBB) and
    coarsest size (135 to 315 DOFs, so the batch inverts every coarsest operator in
    global memory), against the oracle."""
    fb = _fb()
    pbs = [W.cantilever(16, 8, 8), W.cantilever(48, 16, 16), W.mbb_half(16, 8, 8), W.cantilever(24, 16, 8, volfrac=0.25),
           W.cantilever(8, 4, 4, load_k=1)]   # two levels: the coarse "tail" is the dense solve alone
    prm = fb.to_default_params(precision=fb.TO_FP64, precond=fb.TO_PRECOND_MG, n_inner=2)
    probs = [fb.Problem.from_workload(pb, prm) for pb in pbs]
    n = 10
    with fb.Batch(probs) as B:
        stats = B.step(n)
    for pb, P, st in zip(pbs, probs, stats):
        rho, _, _, _ = P.get_state()
        rho_o, _, hist, _ = outer.run(pb, n, precond="mg", n_inner=2)
        assert np.abs(rho.cpu().numpy() - rho_o).max() <= 1e-8
        for s, h in zip(st, hist):
            assert abs(s["J"] - h["J"]) <= 1e-8 * max(abs(h["J"]), 1e-30)
        P.close()


def test_batch_mg_rejections():
    fb = _fb()
    mg = fb.to_default_params(precond=fb.TO_PRECOND_MG, n_inner=2)
    jac = fb.to_default_params(n_inner=2)
    a = fb.Problem.from_workload(W.cantilever(16, 8, 8), mg)
    b = fb.Problem.from_workload(W.cantilever(16, 8, 8), jac)
    c = fb.Problem.from_workload(W.cantilever(16, 8, 8), fb.to_default_params(precond=fb.TO_PRECOND_MG, n_inner=2,
                                                                            mg_nu_pre=3))
    try:
        for group in ([a, b], [a, c]):
            with pytest.raises(fb.ToError) as e:
                fb.Batch(group)
            assert e.value.code == 1
    finally:
        for P in (a, b, c):
            P.close()
