"""Pins for the density filter (Remark 3.1) and the compliance sensitivity
(Sec. III exact gradient)."""
import numpy as np

import workloads as W
from oracle import filt, outer


def test_filter_preserves_constants_and_is_adjoint():
    H, Hs = filt.filter_matrix(6, 5, 4, 1.5)
    x = np.full(120, 0.37)
    assert np.abs(filt.filter_forward(H, Hs, x) - 0.37).max() < 1e-15
    r = np.random.default_rng(2)
    a, b = r.normal(size=120), r.normal(size=120)
    lhs = filt.filter_forward(H, Hs, a) @ b
    rhs = a @ filt.filter_transpose(H, Hs, b)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_filter_radius_below_one_is_identity():
    H, Hs = filt.filter_matrix(4, 3, 2, 0.9)
    x = np.random.default_rng(3).uniform(size=24)
    assert np.abs(filt.filter_forward(H, Hs, x) - x).max() < 1e-16


def test_filter_stencil_sizes_and_hand_example():
    # interior element: 19 neighbours within r = 1.5 (self, 6 faces, 12 edges), 81 within r = 2.5
    H, _ = filt.filter_matrix(7, 7, 7, 1.5)
    assert H[3 + 7 * (3 + 7 * 3)].nnz == 19
    H, _ = filt.filter_matrix(7, 7, 7, 2.5)
    assert H[3 + 7 * (3 + 7 * 3)].nnz == 81
    # 3 x 1 x 1 row, r = 1.5: weights 1.5 (self) and 0.5 (neighbour at distance 1)
    H, Hs = filt.filter_matrix(3, 1, 1, 1.5)
    rho = np.array([1.0, 0.0, 0.0])
    out = filt.filter_forward(H, Hs, rho)
    assert np.allclose(out, [1.5 / 2.0, 0.5 / 2.5, 0.0], atol=1e-15)


def test_sensitivity_matches_central_differences_of_exact_compliance():
    pb = W.cantilever(6, 4, 4)
    pb.rho0 = W.random_rho(pb.n_elem)
    S = outer.Setup(pb)
    J, u = S.exact_compliance(pb.rho0)
    _, _, Ed = S.moduli(pb.rho0)
    g = filt.filter_transpose(S.H, S.Hs, S.sens_rho_tilde(Ed, u))
    h = 1e-6
    for e in W.random_elements(pb.n_elem, 12):
        rp, rm = pb.rho0.copy(), pb.rho0.copy()
        rp[e] += h
        rm[e] -= h
        fd = (S.exact_compliance(rp)[0] - S.exact_compliance(rm)[0]) / (2 * h)
        assert abs(g[e] - fd) <= 1e-6 * abs(fd) + 1e-12
    # compliance is non-increasing in every design variable
    assert np.all(g <= 0)


def test_filter_at_sampled_elements_equals_the_full_filter():
    """The per-element loop (used where the full H does not fit) gives the full filter's
    values, for both workload radii, at interior, edge and corner elements."""
    for dims, r in (((9, 7, 6), 1.5), ((11, 8, 7), 2.5)):
        H, Hs = filt.filter_matrix(*dims, r)
        x = W.random_rho(dims[0] * dims[1] * dims[2], 0.0, 1.0, seed=W.SEED + 40)
        full = filt.filter_forward(H, Hs, x)
        els = [0, 1, dims[0] - 1, dims[0] * dims[1] * dims[2] - 1] + list(W.random_elements(x.size, 20, seed=W.SEED + 41))
        at = filt.filter_forward_at(*dims, r, x, els)
        assert np.abs(at - full[els]).max() <= 1e-15
