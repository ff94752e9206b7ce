"""Pins for the oracle's finite-element core (Sec. III): element matrix, assembly,
matrix-free loop, Jacobi diagonal.  Each check is fixed by mechanics or
mathematics, not by the oracle itself."""
import itertools

import numpy as np
import pytest

import workloads as W
from oracle import fem, outer, solve


def rigid_modes():
    """3 translations and 3 infinitesimal rotations of the unit cube's 8 nodes."""
    X = fem.LOCAL_NODES.astype(float)
    modes = []
    for c in range(3):
        m = np.zeros((8, 3)); m[:, c] = 1.0; modes.append(m.ravel())
    for axis in np.eye(3):
        modes.append(np.cross(axis, X).ravel())
    return np.array(modes).T  # 24 x 6


def test_ke_symmetric_rowsum_nullspace():
    ke = fem.ke_hex8(0.3)
    assert np.allclose(ke, ke.T, atol=1e-15)
    assert np.abs(ke.sum(axis=1)).max() < 1e-14
    ev = np.linalg.eigvalsh(ke)
    scale = np.abs(ev).max()
    assert (np.abs(ev) < 1e-12 * scale).sum() == 6
    assert ev.min() > -1e-12 * scale
    R = rigid_modes()
    assert np.abs(ke @ R).max() < 1e-13 * scale
    # every zero mode lies in span(R): projecting the null space onto R loses nothing
    w, V = np.linalg.eigh(ke)
    N = V[:, :6]
    Q, _ = np.linalg.qr(R)
    assert np.linalg.norm(N - Q @ (Q.T @ N)) < 1e-10


def test_ke_quadrature_orders_agree_and_h_scaling():
    k2 = fem.ke_hex8(0.3, 1.0, order=2)
    k3 = fem.ke_hex8(0.3, 1.0, order=3)
    assert np.abs(k2 - k3).max() < 1e-14
    assert np.abs(fem.ke_hex8(0.3, 2.5) - 2.5 * k2).max() < 1e-13


def test_ke_closed_form_exact_integration():
    """Exact rational integral of the Lame bilinear form over the unit cube.

    K[(a,i),(b,j)] = lam G_ij[a,b] + mu G_ji[a,b] + mu delta_ij sum_k G_kk[a,b],
    G_ij[a,b] = int d_i N_a d_j N_b, with N_a a product of the 1-D hats 1-t, t.
    Separable, so each entry is a product of three exact 1-D integrals; no
    quadrature points and no B matrix are involved.
    """
    from fractions import Fraction as Fr
    X = fem.LOCAL_NODES

    def one_d(p, q, dp, dq):
        sp_, sq = (1 if p else -1), (1 if q else -1)
        if dp and dq:
            return Fr(sp_ * sq)
        if dp:
            return Fr(sp_, 2)
        if dq:
            return Fr(sq, 2)
        return Fr(1, 3) if p == q else Fr(1, 6)

    def G(i, j, a, b):
        out = Fr(1)
        for d in range(3):
            out *= one_d(X[a][d], X[b][d], d == i, d == j)
        return out

    nu = Fr(3, 10)
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1 / (2 * (1 + nu))
    K = np.zeros((24, 24))
    for a in range(8):
        for b in range(8):
            for i in range(3):
                for j in range(3):
                    v = lam * G(i, j, a, b) + mu * G(j, i, a, b)
                    if i == j:
                        v += mu * sum(G(k, k, a, b) for k in range(3))
                    K[3 * a + i, 3 * b + j] = float(v)
    assert np.abs(K - fem.ke_hex8(0.3)).max() < 1e-15


def test_patch_test_constant_strain():
    """u = eps x: interior nodal forces vanish; energy = 1/2 eps^T D eps * volume."""
    nx, ny, nz = 4, 3, 3
    ke = fem.ke_hex8(0.3)
    Ee = np.ones(nx * ny * nz)
    eps = np.array([[1e-3, 2e-4, -3e-4], [2e-4, -5e-4, 1e-4], [-3e-4, 1e-4, 7e-4]])  # symmetric gradient
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    P = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(float)
    u = (P @ eps.T).ravel()
    y = fem.apply_matfree(nx, ny, nz, Ee, ke, [], u)
    interior = (P[:, 0] > 0) & (P[:, 0] < nx) & (P[:, 1] > 0) & (P[:, 1] < ny) & (P[:, 2] > 0) & (P[:, 2] < nz)
    assert np.abs(y.reshape(-1, 3)[interior]).max() < 1e-16
    D = fem.constitutive(0.3)
    v = np.array([eps[0, 0], eps[1, 1], eps[2, 2], 2 * eps[0, 1], 2 * eps[1, 2], 2 * eps[0, 2]])
    energy = 0.5 * u @ y
    assert abs(energy - 0.5 * v @ D @ v * nx * ny * nz) < 1e-14


def test_cantilever_full_density_matches_beam_theory():
    """Tip deflection of a slender (L/h = 10) full-density cantilever vs
    Euler-Bernoulli + Timoshenko shear, P L^3/(3EI) + P L/(kGA), k = 5/6;
    the gap closes under refinement."""
    errs = []
    for n in (4, 8):
        pb = W.cantilever(10 * n, n, n)
        pb.rho0[:] = 1.0
        S = outer.Setup(pb)
        J, u = S.exact_compliance(pb.rho0)
        tip = -u[pb.load_dof].mean()
        L, h, b = 10 * n, n, n
        I = b * h ** 3 / 12.0
        G = 1.0 / (2 * 1.3)
        theory = L ** 3 / (3 * I) + L / (5.0 / 6.0 * G * b * h)
        errs.append(abs(tip - theory) / theory)
        # J = f^T u equals the load-weighted tip deflection
        assert abs(J - tip) < 1e-9 * tip
    assert errs[1] < 0.03
    assert errs[1] < errs[0]


def test_matrix_free_equals_assembled_and_diagonal():
    nx, ny, nz = 5, 3, 4
    r = np.random.default_rng(1)
    Ee = r.uniform(1e-3, 1.0, nx * ny * nz)
    ke = fem.ke_hex8(0.3)
    pb = W.cantilever(nx, ny, nz)
    u = r.uniform(-1, 1, pb.n_dof)
    K = fem.assemble(nx, ny, nz, Ee, ke, pb.fixed_dof)
    y1 = K @ u
    y2 = fem.apply_matfree(nx, ny, nz, Ee, ke, pb.fixed_dof, u)
    assert np.abs(y1 - y2).max() <= 1e-13 * np.abs(y1).max()
    d = fem.jacobi_diagonal(nx, ny, nz, Ee, ke, pb.fixed_dof)
    assert np.abs(d - K.diagonal()).max() < 1e-14
    # fixed rows / columns are the identity
    fx = pb.fixed_dof
    assert np.all(K[fx][:, fx].toarray() == np.eye(fx.size))
    assert np.abs(y2[fx] - u[fx]).max() == 0.0


def test_node_and_element_numbering():
    en = fem.element_nodes(3, 2, 2)
    # element (1, 1, 1): id 1 + 3 (1 + 2*1) = 10; its node (0,0,0) is node 1 + 4 (1 + 3*1) = 17
    assert en[10, 0] == 17
    assert en[10, 6] == (2) + 4 * (2 + 3 * 2)
    pb = W.cantilever(3, 2, 2)
    assert pb.fixed_dof.size == 3 * 3 * 3
    assert abs(pb.load_val.sum() + 1.0) < 1e-15
