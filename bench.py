#!/usr/bin/env python
"""Benchmark of the first-order bilevel topology optimiser on one GB300.

A step is one outer iteration (Algorithms 1 / 3) of the whole hot path: density
filter and moduli, preconditioner refresh, the lower-level steps (operator
applies, dot products, updates), the fused sensitivity, the filter transpose
and the projection onto X.  Workload: the 128x64x64 cantilever (524,288 hex8
elements, 1,635,075 DOFs), seeded synthetic inputs (``workloads``).

Reported: outer iterations/s of the FP32-mixed path (``value``), the same for
plain FP64, and GDOF/s of K(rho)u for both, with the roofline of the operator
kernel measured live with CUDA events on the launching stream.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 512 << 20       # > 129 MB L2: written between timed steps
# DRAM bytes (read + written) of one K(rho)u launch at 128x64x64, FP32, from one ncu capture of the current
# operator kernel (dram__bytes_read.sum + dram__bytes_write.sum); below the algorithmic bytes because the
# working set stays in L2.  Set to None whenever the operator kernel changes until it is measured again.
APPLY_TRAFFIC_128 = 9249536


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=None)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-diff", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-mbb", action="store_true", help="skip the 512x256x256 MBB line")
    ap.add_argument("--no-cpfbto", action="store_true", help="skip the CPFBTO (Krylov preconditioner) line")
    ap.add_argument("--no-pgd", action="store_true", help="skip the FBTO vs nested-exact (PGD) time-to-quality line")
    ap.add_argument("--quality-steps", type=int, default=200,
                    help="outer iterations of the FP32-mixed vs FP64 compliance comparison (0: skip)")
    ap.add_argument("--precond", default="auto", choices=["auto", "mg", "jacobi"])
    ap.add_argument("--apply-only", nargs=3, type=int, metavar=("NX", "NY", "NZ"),
                    help="time only K(rho)u on a cantilever of this size (random design), FP32-mixed")
    ap.add_argument("--fp64", action="store_true", help="with --apply-only: the plain FP64 operator")
    ap.add_argument("--op-kernel", type=int, default=0, choices=[0, 1, 2],
                    help="operator kernel: 0 the general kernel (default), 1 the TMA-staged FP32 kernel, "
                         "2 the tensor-core FP32 kernel")
    ap.add_argument("--mg-legs", type=int, default=0, choices=[0, 1],
                    help="multigrid levels below the fine grid: 0 one launch per step, 1 two cooperative launches per V-cycle")
    ap.add_argument("--mg-cluster", type=int, default=None, choices=[0, 1],
                    help="the multigrid level above the coarse tail in one 16-CTA cluster (default: the library's)")
    ap.add_argument("--oracle-worker", nargs=3, metavar=("WARM", "ITERS", "BUDGET_S"), help=argparse.SUPPRESS)
    return ap.parse_args()


def apply_only(args):
    """K(rho)u alone on an nx x ny x nz cantilever with rho ~ U[0, 1]: GDOF/s and GB/s."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2204_06204_gb300 as fb
    import workloads as W
    pb = W.cantilever(*args.apply_only)
    prec = fb.TO_FP64 if args.fp64 else fb.TO_FP32_MIXED
    P = fb.Problem.from_workload(pb, fb.to_default_params(precision=prec, op_kernel=args.op_kernel))
    P.set_design(torch.tensor(W.random_rho(pb.n_elem, 0.0, 1.0), dtype=P.dtype, device=P.device))
    u = torch.tensor(W.random_u(pb.n_dof), dtype=P.dtype, device=P.device)
    y = P.dof()
    for _ in range(max(args.warmup, 3)):
        P.apply_K(u, y)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=P.device)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for a, b in ev:          # L2 flushed before every timed apply
        flush.zero_()
        a.record(stream)
        P.apply_K(u, y)
        b.record(stream)
    torch.cuda.synchronize()
    ts = sorted(a.elapsed_time(b) / 1000.0 for a, b in ev)
    t = ts[len(ts) // 2]
    s = 8 if args.fp64 else 4
    byts = 2 * 3 * pb.n_node * s + pb.n_elem * s + pb.n_node
    print(json.dumps({"apply_only": list(args.apply_only), "precision": "fp64" if args.fp64 else "fp32",
                      "op_kernel": args.op_kernel,
                      "us_median": t * 1e6, "us_min": ts[0] * 1e6, "gdofs": pb.n_dof / t / 1e9,
                      "gbs": byts / t / 1e9, "bytes": byts}))
    return 0


# ----------------------------------------------------------------------------- ranks
def max_over_ranks(value, dist, device):
    """The largest of a per-rank scalar, on every rank (the job's time is its slowest
    rank's); the value itself without a process group."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, seconds, world):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:   # sampling runs before the timed region starts
                time.sleep(0.01)
            self.lines.clear()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ----------------------------------------------------------------------------- oracle baseline
ORACLE_WORKLOAD = "cantilever 128x64x64 hex8 (1,635,075 DOFs), MG-preconditioned steepest descent x2"
THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS")


def oracle_worker(warm, iters, budget_s):
    """Time the FP64 oracle's outer iteration on the benchmark workload itself (no
    scaling): the oracle's setup (element matrix, filter matrix, fixtures) untimed,
    ``warm`` untimed outer iterations, then up to ``iters`` timed ones, stopping early
    once ``budget_s`` seconds are spent (at least one is always timed).  Runs in its
    own process so that the BLAS / OpenMP thread count set in its environment holds.
    Prints one JSON object."""
    import numpy as np
    import workloads as W
    from oracle import outer
    pb = W.cantilever_128x64x64()
    t0 = time.perf_counter()
    S = outer.Setup(pb)
    t_setup = time.perf_counter() - t0
    rho, u, a0, k = pb.rho0.copy(), np.zeros(pb.n_dof), None, 1
    for _ in range(warm):
        rho, u, _, a0 = outer.run(pb, 1, precond="mg", n_inner=2, setup=S, rho=rho, u=u, k0=k, alpha0=a0)
        k += 1
    times = []
    while len(times) < max(1, iters):
        t0 = time.perf_counter()
        rho, u, _, a0 = outer.run(pb, 1, precond="mg", n_inner=2, setup=S, rho=rho, u=u, k0=k, alpha0=a0)
        times.append(time.perf_counter() - t0)
        k += 1
        if sum(times) > budget_s:
            break
    threads = os.environ.get("OMP_NUM_THREADS", "")
    print(json.dumps({"seconds": times, "setup_s": t_setup, "warm": warm, "first_k": k - len(times),
                      "threads": int(threads) if threads.isdigit() else None}), flush=True)


def oracle_timing(threads, warm=0, iters=1, budget_s=30.0):
    """Run ``oracle_worker`` in a fresh interpreter with every BLAS / OpenMP pool set to
    ``threads``; returns its JSON record."""
    env = dict(os.environ)
    for k in THREAD_ENV:
        env[k] = str(threads)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-worker", str(warm), str(iters), str(budget_s)]
    p = subprocess.run(cmd, env=env, capture_output=True, text=True, cwd=ROOT)
    if p.returncode != 0:
        raise RuntimeError(f"oracle timing failed: {p.stderr[-2000:]}")
    return json.loads(p.stdout.strip().splitlines()[-1])


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline_line():
    """The oracle on all host cores and on one thread, one outer iteration each."""
    cores = host_cores()
    out = {}
    for name, th in (("all_cores", cores), ("one_thread", 1)):
        r = oracle_timing(th, warm=0, iters=1, budget_s=1.0)
        out[name] = {"outer_iters_per_s": len(r["seconds"]) / sum(r["seconds"]), "cores": th,
                     "seconds": r["seconds"], "setup_s": r["setup_s"]}
    return {"value": out["all_cores"]["outer_iters_per_s"], "unit": "outer_iters/s", "cores": cores,
            "kind": "oracle",
            "sample": "one outer iteration (k = 1) of the benchmark workload itself, " + ORACLE_WORKLOAD
                      + ", FP64 numpy/scipy; the oracle's setup untimed; BLAS/OpenMP pools set to the core count "
                        "(the CSR assembly and sparse products are single-threaded in scipy)",
            "one_thread": out["one_thread"], "all_cores": out["all_cores"]}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = host_cores()
    # the reference arm is the oracle itself: each step is one full outer iteration of the
    # benchmark workload; the warm-up is capped at one iteration and the timed steps at what
    # fits in about two minutes (both reported as run)
    warm = min(args.warmup, 1)
    r = oracle_timing(cores, warm=warm, iters=args.steps, budget_s=120.0)
    n = len(r["seconds"])
    t = sum(r["seconds"])
    ips = n / t
    line = {"impl": "reference", "metric": "outer TO iters/s (FP32-mixed) with K(rho)u GDOF/s, 1 GB300",
            "value": ips, "unit": "outer_iters/s", "n_gpus": args.gpus, "steps": n, "warmup": warm,
            "steps_requested": args.steps, "warmup_requested": args.warmup,
            "ms_per_step": 1000.0 * t / n, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": ORACLE_WORKLOAD, "parallelism": "host CPU"},
            "cpu_baseline": {"value": ips, "unit": "outer_iters/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} full outer iterations (k = {r['first_k']} ..) of the benchmark workload "
                                       f"after {warm} untimed; the oracle's setup ({r['setup_s']:.1f} s) untimed"},
            "e2e": {"value": ips, "unit": "outer_iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- ours
def main():
    args = parse()
    if args.oracle_worker:
        oracle_worker(int(args.oracle_worker[0]), int(args.oracle_worker[1]), float(args.oracle_worker[2]))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    if args.apply_only:
        return apply_only(args)

    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if dist:
        dist.barrier()
    import paper_2204_06204_gb300 as fb
    import workloads as W

    pb = W.cantilever_128x64x64()
    use_mg = args.precond == "mg" or (args.precond == "auto" and _mg_available(fb))
    precond = fb.TO_PRECOND_MG if use_mg else fb.TO_PRECOND_JACOBI
    n_inner = 2 if use_mg else 5
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def make(precision):
        prm = fb.to_default_params(precision=precision, precond=precond, n_inner=n_inner, op_kernel=args.op_kernel,
                                   mg_legs=args.mg_legs,
                                   **({} if args.mg_cluster is None else {"mg_cluster": args.mg_cluster}))
        return fb.Problem.from_workload(pb, prm, device=local)

    def time_steps(P, K, W_):
        P.step(W_, want_stats=False)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            P.step(1, want_stats=False)
            b.record(stream)
        torch.cuda.synchronize()
        P.check()
        return sum(a.elapsed_time(b) for a, b in ev) / 1000.0

    def time_apply(P, reps=50):
        rho, u, k, a0 = P.get_state()
        x = torch.tensor(W.random_u(pb.n_dof), dtype=P.dtype, device=dev) if k <= 1 else u
        y = P.dof()
        for _ in range(5):
            P.apply_K(x, y)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        torch.cuda.synchronize()
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            P.apply_K(x, y)
            b.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / reps / 1000.0

    s_el = 4
    n_node = pb.n_node
    apply_bytes = lambda s: 2 * 3 * n_node * s + pb.n_elem * s + n_node   # u read, y write, E read, mask
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)

    # --- FP32-mixed: the headline
    P32 = make(fb.TO_FP32_MIXED)
    with ClockSampler(local) as clk:
        t32 = time_steps(P32, args.steps, args.warmup)
    t_apply32 = time_apply(P32)
    ips32 = args.steps / t32

    # --- end to end through the C ABI with host buffers: rho in, rho + stats out each step,
    # one to_step_host call per step (the design copied in from pinned host memory and
    # compared with the live one on the device, one outer iteration, the new design and
    # the step's record copied out, one synchronisation; a device-side error raises).
    # Two pinned host buffers take turns: step i reads its design from one and leaves the
    # new design in the other, which is the next step's input (no host-side copy).
    rho_hb = [torch.empty(pb.n_elem, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    stats_h = torch.empty(ctypes.sizeof(fb.to_stats), dtype=torch.uint8, pin_memory=True)
    rho_hb[0].copy_(P32.get_state()[0])
    ke = max(3, min(args.steps, 100))
    we = max(3, args.warmup)   # untimed: the first host-fed steps capture their graph variants

    def e2e_step(i):
        fb.to_step_host(P32, rho_hb[i % 2], rho_hb[(i + 1) % 2], stats_h)

    for i in range(we):
        e2e_step(i)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(we, we + ke):
        e2e_step(i)
    t_e2e = time.perf_counter() - t0

    # --- differentiable compliance: forward + backward through T = 5 Jacobi steps, 256x128x128, FP32
    diff = None
    if not args.no_diff:
        pbd = W.cantilever_random_256x128x128()
        Pd = fb.Problem.from_workload(pbd, fb.to_default_params(precision=fb.TO_FP32_MIXED), device=local)
        rho_d = torch.tensor(pbd.rho0, dtype=torch.float32, device=dev)
        gd = Pd.elem()
        for _ in range(2):
            fb.to_compliance_truncated(Pd, rho_d, 5, 0.5, want_J=False)
            fb.to_compliance_truncated_grad(Pd, 1.0, gd)
        torch.cuda.synchronize()
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nrep = 5
        a_.record(stream)
        for _ in range(nrep):
            fb.to_compliance_truncated(Pd, rho_d, 5, 0.5, want_J=False)
            fb.to_compliance_truncated_grad(Pd, 1.0, gd)
        b_.record(stream)
        torch.cuda.synchronize()
        td = a_.elapsed_time(b_) / 1000.0 / nrep
        Pd.close()
        # the same with the iterates recomputed (every ceil(sqrt(T))-th kept, adj_stride = -1)
        Pr = fb.Problem.from_workload(pbd, fb.to_default_params(precision=fb.TO_FP32_MIXED, adj_stride=-1),
                                      device=local)
        for _ in range(2):
            fb.to_compliance_truncated(Pr, rho_d, 5, 0.5, want_J=False)
            fb.to_compliance_truncated_grad(Pr, 1.0, gd)
        torch.cuda.synchronize()
        a_.record(stream)
        for _ in range(nrep):
            fb.to_compliance_truncated(Pr, rho_d, 5, 0.5, want_J=False)
            fb.to_compliance_truncated_grad(Pr, 1.0, gd)
        b_.record(stream)
        torch.cuda.synchronize()
        tr = a_.elapsed_time(b_) / 1000.0 / nrep
        Pr.close()
        diff = {"workload": "cantilever 256x128x128, rho ~ U[0.2,1], T = 5, beta = 0.5, FP32",
                "fwd_bwd_per_s": 1.0 / td, "ms": td * 1e3,
                "recompute_mode": {"adj_stride": "ceil(sqrt(T)) = 3",
                                   "vectors_kept": "u_0 and u_3 plus a segment of 4: 6, as many as the stored mode at "
                                                   "T = 5 (about 2 sqrt(T) against T + 1 in general); one more forward",
                                   "fwd_bwd_per_s": 1.0 / tr, "ms": tr * 1e3}}
        del rho_d, gd

    # --- batched: 64 independent cantilevers of seeded uneven sizes, one launch per phase + a graph;
    # the Jacobi x5 batch and the multigrid x2 batch (V-cycle steps batched per level, the coarse
    # tails of all problems in one launch), each with the mean ||K u_k - f|| after 24 iterations
    batch = None
    if not args.no_batch:
        pbs = W.batch_cantilevers(64)
        ndof_b = sum(pb_.n_dof for pb_ in pbs)
        kb = 20

        def run_batch(prm_b):
            probs = [fb.Problem.from_workload(pb_, prm_b, device=local) for pb_ in pbs]
            with fb.Batch(probs) as Bt:
                tile_kc, tile_us = Bt.tile()
                Bt.step(3, want_stats=False)
                torch.cuda.synchronize()
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a_.record(stream)
                Bt.step(kb, want_stats=False)
                b_.record(stream)
                torch.cuda.synchronize()
                tb = a_.elapsed_time(b_) / 1000.0
                st = Bt.step(1, want_stats=True)
            res = float(np.mean([s_[-1]["res2"] for s_ in st]))
            for P_ in probs:
                P_.close()
            return tb, tile_kc, tile_us, res

        tb, tile_kc, tile_us, res_j = run_batch(fb.to_default_params(precision=fb.TO_FP32_MIXED, n_inner=5))
        batch = {"workload": "64 seeded cantilevers 16x16x16 .. 64x32x32, FP32-mixed, Jacobi steepest descent x5",
                 "problems": 64, "total_dofs": ndof_b, "batched_iterations": kb,
                 "ms_per_batched_iteration": tb * 1e3 / kb,
                 "outer_iters_per_s_aggregate": 64 * kb / tb,
                 "apply_gdofs_effective": ndof_b * 6 * kb / tb / 1e9,
                 "autotuned_tile_planes": tile_kc, "autotuned_batched_apply_us": tile_us,
                 "mean_residual_norm_at_24": res_j}
        tbm, tile_kc, tile_us, res_m = run_batch(fb.to_default_params(precision=fb.TO_FP32_MIXED,
                                                                     precond=fb.TO_PRECOND_MG, n_inner=2))
        batch["multigrid"] = {"workload": "the same 64 cantilevers, FP32-mixed, multigrid-preconditioned steepest "
                                          "descent x2 (batched V-cycles)",
                              "ms_per_batched_iteration": tbm * 1e3 / kb,
                              "outer_iters_per_s_aggregate": 64 * kb / tbm,
                              "autotuned_tile_planes": tile_kc,
                              "mean_residual_norm_at_24": res_m}

    # --- plain FP64
    res64 = None
    if not args.no_fp64:
        P64 = make(fb.TO_FP64)
        k64 = args.fp64_steps or max(3, args.steps // 4)
        t64 = time_steps(P64, k64, 3)
        t_apply64 = time_apply(P64, reps=10)
        res64 = {"outer_iters_per_s": k64 / t64, "apply_ms": t_apply64 * 1e3,
                 "apply_gdofs": pb.n_dof / t_apply64 / 1e9, "steps": k64}
        P64.close()

    # --- FP32-mixed vs FP64 plain from the same start: compliance after the same iterations
    quality = None
    if not args.no_fp64 and args.quality_steps > 0:
        nq = args.quality_steps
        res = {}
        for name, prec in (("fp32", fb.TO_FP32_MIXED), ("fp64", fb.TO_FP64)):
            Pq = make(prec)
            st = Pq.step(nq, want_stats=True)
            rho_q = Pq.get_state()[0].double().cpu().numpy()
            res[name] = (st[-1] if isinstance(st[-1], dict) else st[-1].as_dict(), rho_q)
            Pq.close()
        J32, J64 = res["fp32"][0]["J"], res["fp64"][0]["J"]
        quality = {"workload": f"cantilever 128x64x64, {nq} outer iterations from rho = 0.3, u = 0",
                   "J_fp32": J32, "J_fp64": J64, "J_rel_diff": abs(J32 - J64) / abs(J64),
                   "mean_abs_drho": float(np.mean(np.abs(res["fp32"][1] - res["fp64"][1]))),
                   "volume_fp32": res["fp32"][0]["volume"], "volume_fp64": res["fp64"][0]["volume"]}
        # against the FP64 oracle's own run of the same iterations (stored by a script that calls only
        # the oracle): exact compliance f^T K^-1 f of each final design
        gold = os.path.join(ROOT, "tests", "golden", f"cantilever_128x64x64_mg2_{nq}.json")
        if os.path.exists(gold):
            rec = json.load(open(gold))
            prm_e = fb.to_default_params(precision=fb.TO_FP64, precond=fb.TO_PRECOND_MG,
                                         inner_mode=fb.TO_INNER_PCG, n_inner=1)
            Pe = fb.Problem.from_workload(pb, prm_e, device=local)
            Pe.set_design(torch.as_tensor(res["fp32"][1], dtype=torch.float64, device=dev))
            ue = Pe.dof()
            ue.zero_()
            Pe.inner_solve(ue, 200)
            fvec = np.zeros(pb.n_dof)
            np.add.at(fvec, pb.load_dof, pb.load_val)
            J_ex = float(np.dot(fvec, ue.cpu().numpy()))
            Pe.close()
            idx = np.asarray(rec["rho_sample_index"], dtype=np.int64)
            quality["vs_oracle"] = {
                "J_exact_fp32_design": J_ex, "J_exact_oracle_design": rec["J_exact_final"],
                "J_rel_vs_oracle": abs(J_ex - rec["J_exact_final"]) / abs(rec["J_exact_final"]),
                "J_tracked_rel_vs_oracle": abs(J32 - rec["J"][-1]) / abs(rec["J"][-1]),
                "mean_abs_drho_on_sample": float(np.mean(np.abs(res["fp32"][1][idx] - np.asarray(rec["rho_sample"])))),
                "oracle_record": os.path.relpath(gold, ROOT)}

    # --- Algorithm CPFBTO: Krylov preconditioner of Eq. (LSP), D = 20, beta = 1, one step per iteration
    cpfbto = None
    if not args.no_cpfbto:
        prm_k = fb.to_default_params(precision=fb.TO_FP32_MIXED, precond=fb.TO_PRECOND_KRYLOV,
                                     inner_mode=fb.TO_INNER_RICHARDSON, beta=1.0, n_inner=1, krylov_dim=20)
        Pk = fb.Problem.from_workload(pb, prm_k, device=local)
        stk = Pk.step(10, want_stats=True)
        kk = 10
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        Pk.step(kk, want_stats=False)
        b_.record(stream)
        torch.cuda.synchronize()
        Pk.check()
        tk = a_.elapsed_time(b_) / 1000.0
        dk = [x if isinstance(x, dict) else x.as_dict() for x in stk]
        cpfbto = {"workload": "cantilever 128x64x64, Algorithm CPFBTO: Krylov preconditioner D = 20 (22 applies of "
                              "K per iteration), beta = 1, FP32-mixed",
                  "outer_iters_per_s": kk / tk, "ms_per_iter": tk * 1e3 / kk,
                  "tracking_residual_first_10": [x["res2"] for x in dk]}
        Pk.close()

    # --- time to quality: FBTO (MG x2 steepest descent) against the nested method (PGD: the lower
    # level re-solved by 30 MG-preconditioned CG iterations each outer iteration), same start
    pgd = None
    if not args.no_pgd:
        f_dev = torch.zeros(pb.n_dof, dtype=torch.float32, device=dev)
        f_dev[torch.as_tensor(pb.load_dof, device=dev)] = torch.as_tensor(pb.load_val, dtype=torch.float32, device=dev)

        def exact_J(rho_t):
            prm_e = fb.to_default_params(precision=fb.TO_FP32_MIXED, precond=fb.TO_PRECOND_MG,
                                         inner_mode=fb.TO_INNER_PCG, n_inner=1)
            Pe = fb.Problem.from_workload(pb, prm_e, device=local)
            Pe.set_design(rho_t)
            ue = Pe.dof()
            ue.zero_()
            Pe.inner_solve(ue, 100)
            J = float(torch.dot(f_dev, ue).item())
            Pe.close()
            return J

        def run(prm, n):
            Pr = fb.Problem.from_workload(pb, prm, device=local)
            torch.cuda.synchronize()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            st = Pr.step(n, want_stats=True)
            b_.record(stream)
            torch.cuda.synchronize()
            rho_f = Pr.get_state()[0].clone()
            Pr.close()
            J = [x["J"] if isinstance(x, dict) else x.as_dict()["J"] for x in st]
            return a_.elapsed_time(b_) / 1000.0, J, rho_f

        n_f, n_p = 200, 30
        tf, Jf, rho_fb = run(fb.to_default_params(precision=fb.TO_FP32_MIXED, precond=fb.TO_PRECOND_MG, n_inner=2), n_f)
        tp, Jp, rho_pg = run(fb.to_default_params(precision=fb.TO_FP32_MIXED, precond=fb.TO_PRECOND_MG,
                                                  inner_mode=fb.TO_INNER_PCG, n_inner=30), n_p)
        k_same = max(1, min(n_f, int(round(n_f * tp / tf))))
        pgd = {"workload": "cantilever 128x64x64 from rho = 0.3, FP32-mixed; compliance of each final design from "
                           "100 MG-preconditioned CG iterations",
               "fbto": {"iterations": n_f, "seconds": tf, "J_exact_final": exact_J(rho_fb),
                        "J_tracked_every_20": Jf[::20]},
               "pgd": {"iterations": n_p, "seconds": tp, "cg_iterations_per_outer": 30,
                       "J_exact_final": exact_J(rho_pg), "J_every_5": Jp[::5]},
               "fbto_iterations_in_pgd_time": k_same}

    # --- large single problem: MBB half model 512x256x256 (101.6M DOFs), filter radius 2.5, MG, FP32-mixed
    mbb = None
    if not args.no_mbb:
        pbm = W.mbb_512x256x256()
        prm_m = fb.to_default_params(precision=fb.TO_FP32_MIXED, precond=fb.TO_PRECOND_MG, n_inner=2)
        Pm = fb.Problem.from_workload(pbm, prm_m, device=local)
        Pm.step(2, want_stats=False)
        torch.cuda.synchronize()
        km = 5
        evm = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(km)]
        for a, b in evm:
            a.record(stream)
            Pm.step(1, want_stats=False)
            b.record(stream)
        torch.cuda.synchronize()
        Pm.check()
        tm = sum(a.elapsed_time(b) for a, b in evm) / 1000.0
        Pm_rho, um = Pm.get_state()[:2]
        ym = Pm.dof()
        for _ in range(3):
            Pm.apply_K(um, ym)
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        for _ in range(10):
            Pm.apply_K(um, ym)
        b_.record(stream)
        torch.cuda.synchronize()
        tam = a_.elapsed_time(b_) / 1000.0 / 10
        bytes_m = 2 * 3 * pbm.n_node * 4 + pbm.n_elem * 4 + pbm.n_node
        Pm.close()
        # the same apply with the TMA-staged (op_kernel 1) and the tensor-core (op_kernel 2) FP32
        # kernels, same design and input
        tam_alt = {}
        for okern in (1, 2):
            prm_t = fb.to_default_params(precision=fb.TO_FP32_MIXED, precond=fb.TO_PRECOND_MG, n_inner=2,
                                         op_kernel=okern)
            Pt = fb.Problem.from_workload(pbm, prm_t, device=local)
            Pt.set_design(Pm_rho)
            yt = Pt.dof()
            for _ in range(3):
                Pt.apply_K(um, yt)
            a_.record(stream)
            for _ in range(10):
                Pt.apply_K(um, yt)
            b_.record(stream)
            torch.cuda.synchronize()
            tam_alt[okern] = a_.elapsed_time(b_) / 1000.0 / 10
            Pt.close()
            del yt
        tam_tma, tam_tc = tam_alt[1], tam_alt[2]
        mbb = {"workload": "MBB half model 512x256x256 (101,649,411 DOFs), volfrac 0.15, r = 2.5, FP32-mixed, "
                           "MG-preconditioned steepest descent x2 (inputs far larger than L2)",
               "outer_iters_per_s": km / tm, "ms_per_iter": tm * 1e3 / km,
               "apply_K_us": tam * 1e6, "apply_gdofs": pbm.n_dof / tam / 1e9,
               "apply_GBs": bytes_m / tam / 1e9, "apply_frac_of_hbm": bytes_m / tam / 1e9 / hbm,
               "apply_K_us_tma_kernel": tam_tma * 1e6, "apply_frac_of_hbm_tma_kernel": bytes_m / tam_tma / 1e9 / hbm,
               "apply_K_us_tensor_core_kernel": tam_tc * 1e6,
               "apply_frac_of_hbm_tensor_core_kernel": bytes_m / tam_tc / 1e9 / hbm}
        del um, ym, Pm_rho

    # max over ranks (the timed region and the end-to-end loop)
    t32 = max_over_ranks(t32, dist, dev)
    t_e2e = max_over_ranks(t_e2e, dist, dev)
    ips32 = args.steps / t32

    if rank != 0:
        dist.destroy_process_group()
        return 0

    cpu = None
    if not args.no_cpu:
        cpu = cpu_baseline_line()

    ach = apply_bytes(s_el) / t_apply32 / 1e9
    launches_per_step = _launches_per_step(use_mg, n_inner, cluster=bool(args.mg_cluster))
    line = {
        "metric": "outer TO iters/s (FP32-mixed) with K(rho)u GDOF/s, 1 GB300",
        "value": job_rate(args.steps, t32, world),
        "unit": "outer_iters/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1000.0 * t32 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (dots, norms, step sizes and lambda in f64)",
        "data": "synthetic",
        "config": {"workload": "cantilever 128x64x64 hex8 (1,635,075 DOFs), FP32-mixed, "
                               + ("MG-preconditioned steepest descent x2" if use_mg else "Jacobi steepest descent x5"),
                   "l2": "flushed (512 MB write) before every timed step and every timed apply",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "apply_K": {"fp32_gdofs": pb.n_dof / t_apply32 / 1e9, "fp32_us": t_apply32 * 1e6,
                    "fp64_gdofs": res64["apply_gdofs"] if res64 else None,
                    "fp64_us": res64["apply_ms"] * 1e3 if res64 else None},
        "fp64_plain": res64,
        "fp32_over_fp64_iters": (ips32 / res64["outer_iters_per_s"]) if res64 else None,
        "fp32_vs_fp64_quality": quality,
        "cpfbto": cpfbto,
        "fbto_vs_pgd": pgd,
        "differentiable_compliance": diff,
        "batched": batch,
        "mbb_large": mbb,
        "roofline": {"kernel": "k_operator (K(rho)u, FP32)", "bound": "hbm", "achieved": ach, "peak": hbm,
                     "unit": "GB/s", "frac": ach / hbm, "traffic": APPLY_TRAFFIC_128,
                     "algorithmic_bytes": apply_bytes(s_el),
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs" if pk else "fallback 6800"},
        "e2e": {"value": job_rate(ke, t_e2e, world), "unit": "outer_iters/s", "h2d_bytes_per_step": pb.n_elem * 4,
                "d2h_bytes_per_step": pb.n_elem * 4 + ctypes.sizeof(fb.to_stats)},
        "gpu_launches": launches_per_step * args.steps * world,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def _mg_available(fb):
    import workloads as W
    pb = W.cantilever(4, 2, 2)
    try:
        prm = fb.to_default_params(precond=fb.TO_PRECOND_MG)
        fb.Problem.from_workload(pb, prm).close()
        return True
    except fb.ToError:
        return False


def _mg_levels(nx, ny, nz):
    t = 0
    while all(d % (2 << t) == 0 for d in (nx, ny, nz)) and min(nx, ny, nz) // (2 << t) >= 2:
        t += 1
    return t + 1


def _launches_per_step(mg, n_inner, dims=(128, 64, 64), nu1=2, nu2=2, cluster=False):
    """Kernel launches of one outer iteration (one to_step(1) call), as issued by the library
    (cluster: the FP32 level just above the coarse tail runs as two 16-CTA cluster launches)."""
    # stats-slot reset (once per to_step call), filter + moduli, diag, residual with the fused
    # sensitivity, (Q + update) per step, filter^T with the step-size statistics, the projection
    # (first pass, multiplier search, final pass), the design's copy to a host buffer (returns
    # at once unless to_step_host set one), record
    base = 1 + 1 + 1 + 1 + 2 * n_inner + 1 + 3 + 1 + 1
    if not mg:
        return base
    L = _mg_levels(*dims)
    if L == 1:
        return base + 2 + n_inner                   # dense assemble + invert, one dense solve per step
    refresh = 2 * (L - 1) + 2                       # coarsen + diag per coarse level, dense assemble + invert
    # levels from the first one (>= 1, above the coarsest) with at most 1024 elements run as one kernel
    elems = [(dims[0] >> l) * (dims[1] >> l) * (dims[2] >> l) for l in range(L)]
    tail = next((l for l in range(1, L - 1) if elems[l] <= 1024), 0)
    host_levels = tail if tail else L - 1
    # first sweep on the finest level (coarser ones come out of the restriction), per host level:
    # nu1 - 1 sweeps, b - K x, restriction, prolongation, nu2 sweeps; the dense solve or the tail kernel
    vcycle = 1 + host_levels * ((nu1 - 1) + 1 + 1 + 1 + nu2) + 1
    if cluster and tail >= 2 and nu1 >= 1:
        l = tail - 1
        nx, ny, nz = (d >> l for d in dims)
        if nz <= 16 and nx * ny <= 512 and (nx + 1) * (ny + 1) <= 640 and (nx // 2 + 1) * (ny // 2 + 1) <= 192:
            vcycle -= ((nu1 - 1) + 1 + 1 + 1 + nu2) - 2   # that level's steps in two launches
    return base + refresh + vcycle * n_inner        # one V-cycle per step (r^T z fused into the last sweep)


if __name__ == "__main__":
    sys.exit(main())
