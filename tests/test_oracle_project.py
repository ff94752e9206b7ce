"""Pins for the projection onto X (Sec. IV-B, Eq. piecewiseLinearEQ, Algorithm 4)."""
import itertools
import os

import numpy as np
import pytest

from oracle import project

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_force(w, vbar, lo, hi):
    """Enumerate every active-set assignment (lower / free / upper) and keep the
    feasible KKT point; on E <= 7 elements this is exhaustive."""
    E = w.size
    box = np.clip(w, lo, hi)
    if box.sum() <= vbar:
        return box
    best = None
    for assign in itertools.product((0, 1, 2), repeat=E):
        a = np.array(assign)
        free = a == 1
        fixed_sum = lo * (a == 0).sum() + hi * (a == 2).sum()
        if free.sum() == 0:
            if abs(fixed_sum - vbar) > 1e-12:
                continue
            lam_lo = max([w[e] - lo for e in range(E) if a[e] == 0] + [-np.inf])
            lam_hi = min([w[e] - hi for e in range(E) if a[e] == 2] + [np.inf])
            if lam_lo > lam_hi + 1e-12:
                continue
            v = np.where(a == 0, lo, hi).astype(float)
        else:
            lam = (w[free].sum() + fixed_sum - vbar) / free.sum()
            v = np.where(a == 0, lo, np.where(a == 2, hi, w - lam))
            if np.any(v[free] < lo - 1e-12) or np.any(v[free] > hi + 1e-12):
                continue
            if np.any(w[a == 0] - lam > lo + 1e-12) or np.any(w[a == 2] - lam < hi - 1e-12):
                continue
        d = np.sum((v - w) ** 2)
        if best is None or d < best[0] - 1e-14:
            best = (d, v)
    return best[1]


@pytest.mark.parametrize("seed", range(6))
def test_alg4_equals_brute_force(seed):
    r = np.random.default_rng(seed)
    E = 1 + seed % 7
    w = r.normal(0.4, 0.6, E)
    lo = [0.0, 0.1][seed % 2]
    vbar = r.uniform(E * lo, E * 0.8)
    v, lam = project.project_alg4(w, vbar, lo, 1.0)
    vb = brute_force(w, vbar, lo, 1.0)
    assert np.abs(v - vb).max() < 1e-12


def test_alg4_kkt_and_idempotent_and_bisection():
    r = np.random.default_rng(7)
    w = r.normal(0.3, 0.5, 5000)
    vbar = 0.3 * 5000
    v, lam = project.project_alg4(w, vbar, 0.0, 1.0)
    assert v.min() >= 0.0 and v.max() <= 1.0
    assert abs(v.sum() - vbar) <= 1e-12 * 5000
    assert np.abs(v - np.clip(w - lam, 0.0, 1.0)).max() < 1e-15
    v2, lam2 = project.project_alg4(v, vbar, 0.0, 1.0)
    assert np.abs(v2 - v).max() < 1e-12
    # plain bisection on the monotone volume function gives the same point
    a, b = w.min() - 1.0, w.max()
    for _ in range(200):
        c = 0.5 * (a + b)
        if np.clip(w - c, 0, 1).sum() > vbar:
            a = c
        else:
            b = c
    assert np.abs(v - np.clip(w - c, 0.0, 1.0)).max() < 1e-12


def test_alg4_inactive_bound_returns_box():
    w = np.array([1.4, -0.2, 0.5, 0.3])
    v, lam = project.project_alg4(w, 3.0, 0.0, 1.0)
    assert lam == 0.0 and np.array_equal(v, [1.0, 0.0, 0.5, 0.3])


def test_alg4_infeasible_raises():
    with pytest.raises(ValueError):
        project.project_alg4(np.zeros(4), 0.3, 0.1, 1.0)


def test_golden_hand_example():
    """tests/golden/projection_hand.txt: worked by hand from Eq. (piecewiseLinearEQ)."""
    rows = {}
    for line in open(os.path.join(GOLDEN, "projection_hand.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            rows[k.strip()] = np.array([float(t) for t in v.split()])
    v, lam = project.project_alg4(rows["w"], float(rows["vbar"][0]), float(rows["lo"][0]), 1.0)
    assert np.abs(v - rows["v"]).max() < 1e-15
    assert abs(lam - float(rows["lambda"][0])) < 1e-15
