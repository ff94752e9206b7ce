"""Seeded synthetic design problems for the first-order bilevel topology optimiser.

This module only *describes* inputs: grid sizes, which degrees of freedom are
loaded and with what value, which are clamped, the initial design, and seeded
random fields.  It holds none of the method's arithmetic, so both the FP64
oracle (``oracle/``) and the CUDA path (tests, ``bench.py``) draw the same
bytes from it without sharing any computation.

Conventions (fixed for both sides):

* node index  n = i + (nx+1) * (j + (ny+1) * k),  0 <= i <= nx, ...
* DOF index   d = 3*n + c,  c in {0: x, 1: y, 2: z}
* element     e = i + nx * (j + ny * k),  0 <= i < nx, ...
* axes: x is the beam length (nx), y is vertical (ny), z is depth (nz).

The paper's experiments are 2-D benchmark geometries from suites that are not
available here; the 3-D cantilever and MBB half-model below stand in for them
with the sizes and loads of the five workloads the library is measured on.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

SEED = 20220413


@dataclasses.dataclass
class Problem:
    nx: int
    ny: int
    nz: int
    h: float
    E0: float
    Emin: float
    nu: float
    p: float
    volfrac: float
    rmin: float
    rho_min: float
    rho_max: float
    load_dof: np.ndarray      # int64 global DOF indices
    load_val: np.ndarray      # float64 values
    fixed_dof: np.ndarray     # int64 global DOF indices (u = 0)
    rho0: np.ndarray          # float64 initial design, length n_elem
    name: str = ""

    @property
    def n_elem(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_node(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_dof(self) -> int:
        return 3 * self.n_node

    def node(self, i, j, k):
        return np.asarray(i) + (self.nx + 1) * (np.asarray(j) + (self.ny + 1) * np.asarray(k))


def _node(nx, ny, i, j, k):
    return np.asarray(i, dtype=np.int64) + (nx + 1) * (np.asarray(j, dtype=np.int64) + (ny + 1) * np.asarray(k, dtype=np.int64))


def cantilever(nx: int, ny: int, nz: int, volfrac: float = 0.3, rmin: float = 1.5,
               rho_init: Optional[float] = None, load_k: Optional[int] = None,
               E0: float = 1.0, Emin: float = 1e-9, nu: float = 0.3, p: float = 3.0,
               rho_min: float = 0.0, name: str = "") -> Problem:
    """3-D cantilever: the x=0 face fully clamped, a unit downward (-y) load.

    ``load_k=None`` spreads the unit load uniformly over the nodes of the
    bottom edge at x = L, i.e. nodes (nx, 0, k) for k = 0..nz each carry
    f_y = -1/(nz+1).  An integer ``load_k`` puts the whole unit load on node
    (nx, 0, load_k) instead (the batched workload's point load).
    """
    ks = np.arange(nz + 1)
    fixed_nodes = _node(nx, ny, 0, *np.meshgrid(np.arange(ny + 1), ks, indexing="ij")).ravel()
    fixed = np.sort((3 * fixed_nodes[:, None] + np.arange(3)[None, :]).ravel()).astype(np.int64)
    if load_k is None:
        ln = _node(nx, ny, nx, 0, ks)
        ldof = (3 * ln + 1).astype(np.int64)
        lval = np.full(nz + 1, -1.0 / (nz + 1))
    else:
        ldof = np.array([3 * int(_node(nx, ny, nx, 0, load_k)) + 1], dtype=np.int64)
        lval = np.array([-1.0])
    rho0 = np.full(nx * ny * nz, volfrac if rho_init is None else rho_init, dtype=np.float64)
    return Problem(nx, ny, nz, 1.0, E0, Emin, nu, p, volfrac, rmin, rho_min, 1.0,
                   ldof, lval, fixed, rho0, name or f"cantilever {nx}x{ny}x{nz}")


def mbb_half(nx: int, ny: int, nz: int, volfrac: float = 0.15, rmin: float = 2.5,
             E0: float = 1.0, Emin: float = 1e-9, nu: float = 0.3, p: float = 3.0,
             rho_min: float = 0.0, name: str = "") -> Problem:
    """MBB-bridge half model.

    Symmetry u_x = 0 on every node of the x=0 face; a roller u_y = 0 on the
    bottom edge at the far end, nodes (nx, 0, k) for all k (the roller extruded
    along z); u_z = 0 at the single node (nx, 0, 0) to remove the z rigid
    motion; a unit downward line load on the top edge at x = 0, nodes (0, ny, k)
    each carrying f_y = -1/(nz+1).
    """
    ks = np.arange(nz + 1)
    jj, kk = np.meshgrid(np.arange(ny + 1), ks, indexing="ij")
    sym = 3 * _node(nx, ny, 0, jj, kk).ravel() + 0
    roller = 3 * _node(nx, ny, nx, 0, ks) + 1
    zfix = np.array([3 * int(_node(nx, ny, nx, 0, 0)) + 2])
    fixed = np.unique(np.concatenate([sym, roller, zfix])).astype(np.int64)
    ldof = (3 * _node(nx, ny, 0, ny, ks) + 1).astype(np.int64)
    lval = np.full(nz + 1, -1.0 / (nz + 1))
    rho0 = np.full(nx * ny * nz, volfrac, dtype=np.float64)
    return Problem(nx, ny, nz, 1.0, E0, Emin, nu, p, volfrac, rmin, rho_min, 1.0,
                   ldof, lval, fixed, rho0, name or f"mbb_half {nx}x{ny}x{nz}")


def batch_cantilevers(n: int = 64, seed: int = SEED) -> List[Problem]:
    """Independent cantilevers of uneven sizes (the batched workload).

    nx in {16, 24, ..., 64}, ny and nz in {16, 24, 32} (multiples of 8), volume
    fraction ~ U[0.2, 0.4], a unit -y point load on node (nx, 0, k) with k drawn
    uniformly from {0..nz}; all drawn from one PCG64 stream.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(n):
        nx = int(rng.choice(np.arange(16, 65, 8)))
        ny = int(rng.choice([16, 24, 32]))
        nz = int(rng.choice([16, 24, 32]))
        vf = float(rng.uniform(0.2, 0.4))
        lk = int(rng.integers(0, nz + 1))
        out.append(cantilever(nx, ny, nz, volfrac=vf, load_k=lk, name=f"batch[{b}] {nx}x{ny}x{nz}"))
    return out


def rng(seed: int = SEED) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_rho(n_elem: int, lo: float = 0.2, hi: float = 1.0, seed: int = SEED) -> np.ndarray:
    """Design field drawn i.i.d. uniform[lo, hi] (the differentiation workload)."""
    return rng(seed).uniform(lo, hi, size=n_elem)


def random_u(n_dof: int, seed: int = SEED + 1) -> np.ndarray:
    """Displacement-like vector drawn i.i.d. uniform[-1, 1]."""
    return rng(seed).uniform(-1.0, 1.0, size=n_dof)


def random_elements(n_elem: int, count: int, seed: int = SEED + 2) -> np.ndarray:
    """``count`` distinct element indices (finite-difference sample)."""
    return np.sort(rng(seed).choice(n_elem, size=min(count, n_elem), replace=False)).astype(np.int64)


# The five measured workloads, by what they are.
def cantilever_32x16x16() -> Problem:          # plain FP64, Jacobi inner steps, 50 outer iterations
    return cantilever(32, 16, 16)


def cantilever_128x64x64() -> Problem:         # FP32-mixed vs FP64, MG inner steps, 200 outer iterations
    return cantilever(128, 64, 64)


def cantilever_random_64x32x32() -> Problem:   # differentiation check, rho ~ U[0.2, 1]
    pb = cantilever(64, 32, 32)
    pb.rho0 = random_rho(pb.n_elem)
    return pb


def cantilever_random_256x128x128() -> Problem:  # differentiation timing
    pb = cantilever(256, 128, 128)
    pb.rho0 = random_rho(pb.n_elem)
    return pb


def mbb_512x256x256() -> Problem:              # large single problem
    return mbb_half(512, 256, 256)
