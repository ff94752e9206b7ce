"""Linear (cone) density filter and its transpose -- Remark 3.1, material filtering.

The paper plugs a smooth convolution C into K(v) = sum_e A_e(C(v)) K_e and
uses a Gaussian; the workloads here use the standard linear density filter
    rho~_e = sum_i H_ei rho_i / Hs_e,   H_ei = max(0, r - |c_e - c_i|),
    Hs_e   = sum_i H_ei,
over in-domain element centres c (distances in voxels).  Its transpose, the
chain rule of the sensitivity through C, is  (C^T g)_i = sum_e H_ei g_e / Hs_e.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def filter_matrix(nx: int, ny: int, nz: int, rmin: float):
    """Sparse H (E x E) and row sums Hs for a cone of radius ``rmin`` voxels."""
    E = nx * ny * nz
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    R = int(np.ceil(rmin)) + 1
    rows, cols, vals = [], [], []
    for dk in range(-R, R + 1):
        for dj in range(-R, R + 1):
            for di in range(-R, R + 1):
                w = rmin - np.sqrt(di * di + dj * dj + dk * dk)
                if w <= 0:
                    continue
                ii, jj, kk = i + di, j + dj, k + dk
                ok = (ii >= 0) & (ii < nx) & (jj >= 0) & (jj < ny) & (kk >= 0) & (kk < nz)
                e = (i + nx * (j + ny * k))[ok]
                n = (ii + nx * (jj + ny * kk))[ok]
                rows.append(e)
                cols.append(n)
                vals.append(np.full(e.size, w))
    H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(E, E)).tocsr()
    Hs = np.asarray(H.sum(axis=1)).ravel()
    return H, Hs


def filter_forward(H, Hs, x: np.ndarray) -> np.ndarray:
    return (H @ x) / Hs


def filter_transpose(H, Hs, g: np.ndarray) -> np.ndarray:
    return H.T @ (g / Hs)


def filter_forward_at(nx: int, ny: int, nz: int, rmin: float, x: np.ndarray, elements) -> np.ndarray:
    """rho~_e = sum_i H_ei x_i / Hs_e at the listed elements only, by the same cone
    and in-domain rule as ``filter_matrix`` written as a plain loop over each
    element's neighbours (for grids whose full H does not fit in memory)."""
    R = int(np.ceil(rmin)) + 1
    out = np.empty(len(elements))
    for q, e in enumerate(elements):
        e = int(e)
        i, j, k = e % nx, (e // nx) % ny, e // (nx * ny)
        num = den = 0.0
        for dk in range(-R, R + 1):
            for dj in range(-R, R + 1):
                for di in range(-R, R + 1):
                    w = rmin - np.sqrt(di * di + dj * dj + dk * dk)
                    ii, jj, kk = i + di, j + dj, k + dk
                    if w <= 0 or not (0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz):
                        continue
                    num += w * x[ii + nx * (jj + ny * kk)]
                    den += w
        out[q] = num / den
    return out
