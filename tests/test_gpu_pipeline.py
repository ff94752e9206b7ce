"""The pipelined outer iteration (the next design's moduli, diagonals and coarsest
inverse built on a branch beside the lower-level steps, into a second buffer set) is
scheduling only: every call pattern of to_step gives the same iterates bit for bit,
and after a step the live moduli are those of the current design.  Workloads: 32x16x16
cantilever (multigrid: two launched levels and the coarse tail) and 16x8x8 (Jacobi)."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fb():
    import __graft_entry__ as g
    g.build()
    import paper_2204_06204_gb300 as fb
    return fb


CASES = {
    "mg": (lambda: W.cantilever(32, 16, 16), "TO_PRECOND_MG", 2),
    "jacobi": (lambda: W.cantilever(16, 8, 8), "TO_PRECOND_JACOBI", 5),
}


def _params(fb, case, precision):
    _, pre, n_inner = CASES[case]
    prec = fb.TO_FP64 if precision == "fp64" else fb.TO_FP32_MIXED
    return fb.to_default_params(precision=prec, precond=getattr(fb, pre), n_inner=n_inner)


def _run(fb, case, precision, pattern):
    """pattern: list of ("step", n) / ("reset",) / ("probe",) applied in order."""
    pb = CASES[case][0]()
    stats = []
    with fb.Problem.from_workload(pb, _params(fb, case, precision)) as P:
        for op in pattern:
            if op[0] == "step":
                stats += P.step(op[1])
            elif op[0] == "reset":   # the same state written back: the next step starts afresh
                rho, u, k, a0 = P.get_state()
                P.set_state(rho, u, k, a0)
            else:                    # read-only calls between steps
                rho, u, k, a0 = P.get_state()
                P.apply_K(u)
                P.inner_solve(u.clone(), 0, want_res=True)
        rho, u, k, a0 = P.get_state()
        return rho.cpu(), u.cpu(), k, a0, [(s["J"], s["beta_first"], s["lambda"], s["volume"]) for s in stats]


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_call_patterns_agree_bitwise(case, precision):
    fb = _fb()
    ref = _run(fb, case, precision, [("step", 6)])
    for pattern in ([("step", 1)] * 6,
                    [("step", 2), ("step", 1), ("step", 3)],
                    [("step", 2), ("reset",), ("step", 1), ("probe",), ("step", 3)]):
        got = _run(fb, case, precision, pattern)
        assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1]), pattern
        assert ref[2] == got[2] == 7 and ref[3] == got[3]
        assert ref[4] == got[4], pattern


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_live_moduli_belong_to_the_current_design(precision):
    """After to_step the operator is K(rho) of the design to_step left: the same K u as a
    problem given that design directly."""
    fb = _fb()
    pb = CASES["mg"][0]()
    prm = _params(fb, "mg", precision)
    with fb.Problem.from_workload(pb, prm) as P:
        P.step(3)
        rho, u, k, a0 = P.get_state()
        y1 = P.apply_K(u).cpu()
    with fb.Problem.from_workload(pb, prm) as Q:
        Q.set_design(rho)
        y2 = Q.apply_K(u).cpu()
    assert torch.equal(y1, y2)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("change", ["none", "last_entry_one_ulp", "every_entry"])
@pytest.mark.parametrize("no_graph", [0, 1])
def test_set_state_rebuilds_only_a_changed_design(case, precision, change, no_graph):
    """After a pipelined step, to_set_state compares the design it brings with the one the
    live set was built for, on the device; the next step's rebuild kernels do nothing
    unless they differ.  Unchanged, changed in one bit of the last entry, or changed
    everywhere: the iterates (and K u right after the call) must equal those of the plain
    rebuild bit for bit.  The plain rebuild is forced by to_set_design before to_set_state
    (a design set that way is not compared)."""
    fb = _fb()
    pb = CASES[case][0]()

    def run(plain):
        prm = _params(fb, case, precision)
        prm.no_graph = no_graph
        with fb.Problem.from_workload(pb, prm) as P:
            stats = P.step(2)
            rho, u, k, a0 = P.get_state()
            new = rho.clone()
            if change == "every_entry":
                new.mul_(0.97).add_(0.01)
            elif change == "last_entry_one_ulp":
                new[-1] = torch.nextafter(new[-1], torch.zeros_like(new[-1]))
                assert not torch.equal(new, rho)
            if plain:
                P.set_design(new)
            P.set_state(new, None, k, a0)
            y = P.apply_K(u).cpu()   # the moduli of the design just set are live
            stats += P.step(3)
            rho2, u2, k2, a02 = P.get_state()
            return rho2.cpu(), u2.cpu(), k2, a02, y, [(s["J"], s["beta_first"], s["lambda"]) for s in stats]

    ref = run(True)
    got = run(False)
    assert torch.equal(ref[4], got[4])
    assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])
    assert ref[2] == got[2] and ref[3] == got[3]
    assert ref[5] == got[5]


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_step_host_is_set_state_plus_step(case, precision):
    """to_step_host (design in from host memory, one outer iteration, design and record out,
    one synchronisation) against the device-side calls it stands for: fed back its own
    designs it continues the device loop bit for bit; given a changed design it equals
    to_set_state with that design (k and alpha0 kept) followed by to_step(1)."""
    fb = _fb()
    pb = CASES[case][0]()
    prm = _params(fb, case, precision)
    with fb.Problem.from_workload(pb, prm) as P, fb.Problem.from_workload(pb, prm) as Q:
        ref = P.step(6)
        Q.step(2)
        rho, u, k, a0 = Q.get_state()
        hb = [rho.cpu().pin_memory(), torch.empty_like(rho, device="cpu").pin_memory()]
        rec = torch.empty(C_sizeof(fb), dtype=torch.uint8).pin_memory()
        got = []
        for i in range(4):
            fb.to_step_host(Q, hb[i % 2], hb[(i + 1) % 2], rec)
            got.append(fb.to_stats.from_address(rec.data_ptr()).J)
        assert [s["J"] for s in ref[2:]] == got
        rho_p, u_p, k_p, a0_p = P.get_state()
        rho_q, u_q, k_q, a0_q = Q.get_state()
        assert torch.equal(rho_p, rho_q) and torch.equal(hb[0], rho_q.cpu()) and torch.equal(u_p, u_q)
        assert k_p == k_q == 7 and a0_p == a0_q
        # a changed design from pageable memory (copied, not read in place), without
        # rho_out and stats_out
        new = rho_q.clone().mul_(0.97).add_(0.01)
        fb.to_step_host(Q, new.cpu())
        P.set_state(new, None, k_p, a0_p)
        P.step(1)
        rho_p, u_p, k_p, a0_p = P.get_state()
        rho_q, u_q, k_q, a0_q = Q.get_state()
        assert torch.equal(rho_p, rho_q) and torch.equal(u_p, u_q) and k_p == k_q == 8 and a0_p == a0_q
        # pageable output
        out = torch.empty_like(rho_q, device="cpu")
        fb.to_step_host(Q, rho_q.cpu(), out)
        P.step(1)
        assert torch.equal(out, P.get_state()[0].cpu())


def C_sizeof(fb):
    import ctypes
    return ctypes.sizeof(fb.to_stats)


def test_batched_call_patterns_agree_bitwise():
    """The pipelined batched iteration: one call of 4 iterations, four calls of one, and
    a member's state rewritten between calls (the next call starts afresh) agree."""
    fb = _fb()
    pbs = [W.cantilever(16, 8, 8), W.cantilever(32, 16, 16), W.cantilever(16, 16, 16)]
    prm = fb.to_default_params(precision=fb.TO_FP32_MIXED, precond=fb.TO_PRECOND_MG, n_inner=2, tile_z=8)

    def run(pattern):
        probs = [fb.Problem.from_workload(pb, prm) for pb in pbs]
        try:
            B = fb.Batch(probs)
            try:
                for op in pattern:
                    if op[0] == "step":
                        B.step(op[1], want_stats=False)
                    else:
                        torch.cuda.synchronize()
                        rho, u, k, a0 = probs[1].get_state()
                        probs[1].set_state(rho, u, k, a0)
                torch.cuda.synchronize()
                return [tuple(x.cpu() if torch.is_tensor(x) else x for x in P.get_state()) for P in probs]
            finally:
                B.close()
        finally:
            for P in probs:
                P.close()

    ref = run([("step", 4)])
    for pattern in ([("step", 1)] * 4, [("step", 2), ("reset",), ("step", 2)]):
        got = run(pattern)
        for a, b in zip(ref, got):
            assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and a[2] == b[2] and a[3] == b[3]


def test_get_stats_reads_the_last_step_records_without_a_synchronising_step():
    """to_get_stats after to_step(stats_out = NULL) delivers the records to_step itself
    returns with stats_out, field for field; n outside [1, the last call's n_outer] is
    refused."""
    import ctypes
    fb = _fb()
    pb = W.cantilever(32, 16, 16)
    prm = fb.to_default_params(precision=fb.TO_FP32_MIXED, precond=fb.TO_PRECOND_MG, n_inner=2)
    with fb.Problem.from_workload(pb, prm) as P:
        ref = P.step(3, want_stats=True)
    with fb.Problem.from_workload(pb, prm) as P:
        P.step(3, want_stats=False)
        buf = torch.empty(3 * ctypes.sizeof(fb.to_stats), dtype=torch.uint8, pin_memory=True)
        fb.to_get_stats(P, 3, buf)
        torch.cuda.synchronize()
        got = [fb.to_stats.from_address(buf.data_ptr() + i * ctypes.sizeof(fb.to_stats)).as_dict() for i in range(3)]
        for a, b in zip(ref, got):
            assert a == b
        for bad in (0, 4):
            with pytest.raises(fb.ToError):
                fb.to_get_stats(P, bad, buf)
