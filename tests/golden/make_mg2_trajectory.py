"""Write the oracle's multigrid x2 trajectory of a seeded workload to a JSON fixture.

Run from the repository root, e.g.

    python tests/golden/make_mg2_trajectory.py cantilever 128 64 64 200 \
        tests/golden/cantilever_128x64x64_mg2_200.json

It calls only ``oracle/`` (and ``workloads`` for the inputs): the FP64 outer
loop of Algorithms 1 / 3 with two multigrid-preconditioned steepest-descent
steps per outer iteration (``oracle.outer.run``), then the exact compliance
f^T K(rho)^-1 f of the final design (Sec. V, the nested method's objective),
computed by multigrid-preconditioned CG to ||r|| / ||f|| <= 1e-12.

Stored: every iteration's J_k = f^T u_k, residual norms, volume, multiplier,
step sizes; the final exact compliance; and the final design at a seeded sample
of elements (``workloads.random_elements``), so that a test can check the mean
per-element |rho_gpu - rho_oracle| on that sample without a multi-megabyte file.
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import outer, solve  # noqa: E402

SAMPLE = 4096
SAMPLE_SEED = W.SEED + 7


def main(argv):
    kind, nx, ny, nz, n_outer, out = argv[0], int(argv[1]), int(argv[2]), int(argv[3]), int(argv[4]), argv[5]
    pb = W.cantilever(nx, ny, nz) if kind == "cantilever" else W.mbb_half(nx, ny, nz)
    S = outer.Setup(pb)
    rho, u = pb.rho0.copy(), np.zeros(pb.n_dof)
    hist, a0 = [], None
    t0 = time.time()
    for k in range(1, n_outer + 1):
        rho, u, h, a0 = outer.run(pb, 1, precond="mg", n_inner=2, setup=S, rho=rho, u=u, k0=k, alpha0=a0)
        hist += h
        print(f"k={k} J={h[0]['J']:.12g} res2={h[0]['res2']:.3e} t={time.time() - t0:.0f}s", flush=True)
    _, Ee, _ = S.moduli(rho)
    K = S.K(Ee)
    mg = solve.Multigrid(pb.nx, pb.ny, pb.nz, pb.h, Ee, pb.nu, pb.fixed_dof)
    ue, its = solve.pcg(lambda x: K @ x, S.f, mg, tol=1e-12, maxit=2000)
    J_exact = float(S.f @ ue)
    idx = W.random_elements(pb.n_elem, SAMPLE, seed=SAMPLE_SEED)
    rec = {
        "what": f"oracle FP64 outer loop, {pb.name}, multigrid-preconditioned steepest descent x2, "
                f"{n_outer} outer iterations from rho = volfrac, u = 0",
        "command": "python tests/golden/make_mg2_trajectory.py " + " ".join(argv),
        "citation": "Algorithms 1 and 3 (outer loop), Algorithm 4 (projection), Sec. V (exact compliance)",
        "alpha0": a0,
        "J": [h["J"] for h in hist],
        "res2": [h["res2"] for h in hist],
        "volume": [h["volume"] for h in hist],
        "lam": [h["lam"] for h in hist],
        "beta_first": [h["betas"][0] if h["betas"] else 0.0 for h in hist],
        "J_exact_final": J_exact,
        "pcg_iterations": its,
        "rho_sample_seed": SAMPLE_SEED,
        "rho_sample_index": idx.tolist(),
        "rho_sample": rho[idx].tolist(),
        "rho_mean": float(rho.mean()),
        "oracle_seconds": time.time() - t0,
    }
    with open(out, "w") as fh:
        json.dump(rec, fh, indent=0)
    print(f"J_exact_final={J_exact:.12g} pcg_its={its} -> {out}")


if __name__ == "__main__":
    main(sys.argv[1:])
