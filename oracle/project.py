"""Projection onto X = {lo <= v <= hi, 1^T v <= vbar} -- Sec. IV-B, Algorithm 4.

If the box projection already satisfies the volume bound it is the answer.
Otherwise the KKT conditions give v = clamp(w - lambda, lo, hi) with lambda
solving the piecewise-linear equation (piecewiseLinearEQ)
    vbar = sum_e clamp(w_e - lambda, lo, hi),
whose 2E breakpoints are w_e - lo ("left" nodes: the element reaches its
lower bound) and w_e - hi ("right" nodes: the element leaves its upper bound).
Algorithm 4 sorts them and walks the running slope and right-hand side.
The paper has hi = 1; it is a parameter here.
"""
from __future__ import annotations

import numpy as np


def project_box(w: np.ndarray, lo: float, hi: float = 1.0) -> np.ndarray:
    return np.clip(w, lo, hi)


def project_alg4(w: np.ndarray, vbar: float, lo: float, hi: float = 1.0):
    """Return (v, lambda).  lambda = 0 when the volume bound is inactive.

    Ties: lambda is not unique on a flat segment; v is.  The smallest lambda
    of the crossing segment is reported.
    """
    w = np.asarray(w, dtype=np.float64)
    E = w.size
    if vbar < E * lo:
        raise ValueError("infeasible volume bound: vbar < E * lo")
    box = project_box(w, lo, hi)
    if box.sum() <= vbar:
        return box, 0.0
    # Breakpoints: kind +1 for w - lo (element hits lo, slope gains +1),
    #              kind -1 for w - hi (element leaves hi, slope gains -1).
    lam_nodes = np.concatenate([w - lo, w - hi])
    kind = np.concatenate([np.ones(E), -np.ones(E)])
    order = np.argsort(lam_nodes, kind="stable")
    slope = 0.0
    rhs = E * hi                  # every element at hi for lambda below all nodes
    last = 0.0
    nodes_lam = []
    nodes_rhs = []
    for idx in order:
        lam = lam_nodes[idx]
        rhs = rhs + slope * (lam - last)
        if kind[idx] < 0:
            slope -= 1.0
        else:
            slope += 1.0
        nodes_lam.append(lam)
        nodes_rhs.append(rhs)
        last = lam
    # Walk consecutive nodes for the segment through vbar (rhs is non-increasing).
    for a in range(len(nodes_lam) - 1):
        la, ra = nodes_lam[a], nodes_rhs[a]
        lb, rb = nodes_lam[a + 1], nodes_rhs[a + 1]
        if ra >= vbar >= rb:
            lam = la if ra == rb else la + (ra - vbar) * (lb - la) / (ra - rb)
            return project_box(w - lam, lo, hi), float(lam)
    # vbar at or below E*lo: every element at its lower bound.
    lam = nodes_lam[-1]
    return project_box(w - lam, lo, hi), float(lam)


def volume_residual(w: np.ndarray, lam: float, vbar: float, lo: float, hi: float = 1.0) -> float:
    return float(project_box(w - lam, lo, hi).sum() - vbar)
