"""Failure detection on the GPU without a GPU fault: a device-side wait that runs
out returns an error status that the host reads, and the context stays usable."""
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fb():
    import __graft_entry__ as g
    g.build()
    import paper_2204_06204_gb300 as fb
    return fb


def test_grid_barrier_times_out_and_the_context_survives():
    fb = _fb()
    pb = W.cantilever(8, 4, 4)
    with fb.Problem.from_workload(pb, fb.to_default_params(precision=fb.TO_FP32_MIXED)) as P:
        fb.to_barrier_selftest(P, -1, 1 << 14)            # every block arrives: no timeout
        for limit in (1 << 10, 1 << 12):
            with pytest.raises(fb.ToError) as e:           # block 0 never arrives: the others give up
                fb.to_barrier_selftest(P, 0, limit)
            assert e.value.code == fb._abi.TO_ERR_TIMEOUT
        fb.to_barrier_selftest(P, -1, 1 << 14)            # the barrier words were cleared
        st = P.step(3)                                      # normal work still runs, status clean
        assert all(s["status"] == 0 for s in st)
        P.check()
        y = P.apply_K(torch.ones(P.n_dof, dtype=P.dtype, device=P.device))
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
    with pytest.raises(fb.ToError) as e:
        with fb.Problem.from_workload(pb) as P:
            fb.to_barrier_selftest(P, 0, 0)
    assert e.value.code == fb._abi.TO_ERR_ARG
