// Per-node bodies of the multigrid level operations: the grid transfers
// (trilinear prolongation P and its transpose, fixed DOFs masked on both sides)
// and the inverse Jacobi diagonal, shared by the per-level kernels, the coarse
// tail and the batched kernels.
#pragma once

#include "internal.cuh"

namespace to {

// b_c = m_c P^T (m_f t) at coarse node (I, J, K); with xc, also the coarse
// level's first damped Jacobi sweep from x = 0: x = omega b / d (DINV: dc holds
// 1 / d, the layout of the multigrid levels).  IX is the index type (32-bit where
// the level is small).
template <typename T, typename IX = long long, bool DINV = false>
__device__ __forceinline__ void restrict_node(int cx, int cy, int cz, int I, int J, int K, const T* __restrict__ tf,
                                              const uint8_t* __restrict__ mf, const uint8_t* __restrict__ mc,
                                              T* __restrict__ bc, const T* __restrict__ dc, T* __restrict__ xc, T omega) {
    const int fx = 2 * cx, fy = 2 * cy, fz = 2 * cz;
    const IX n = I + (IX)(cx + 1) * (J + (IX)(cy + 1) * K);
    T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int dk = -1; dk <= 1; ++dk) {
        const int k = 2 * K + dk;
        const T wk = dk ? T(0.5) : T(1);
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj) {
            const int j = 2 * J + dj;
            const T wj = dj ? T(0.5) : T(1);
#pragma unroll
            for (int di = -1; di <= 1; ++di) {
                const int i = 2 * I + di;
                const bool in = k >= 0 && k <= fz && j >= 0 && j <= fy && i >= 0 && i <= fx;
                const IX fnode = in ? i + (IX)(fx + 1) * (j + (IX)(fy + 1) * k) : 0;
                const T w = (di ? T(0.5) : T(1)) * wj * wk;
                const uint8_t m = in ? mf[fnode] : 7;
                const T v0 = in ? tf[3 * fnode + 0] : T(0), v1 = in ? tf[3 * fnode + 1] : T(0),
                        v2 = in ? tf[3 * fnode + 2] : T(0);
                acc[0] += (m & 1) ? T(0) : w * v0;
                acc[1] += (m & 2) ? T(0) : w * v1;
                acc[2] += (m & 4) ? T(0) : w * v2;
            }
        }
    }
    const uint8_t m = mc[n];
    for (int c = 0; c < 3; ++c) {
        const T v = ((m >> c) & 1) ? T(0) : acc[c];
        bc[3 * n + c] = v;
        if (xc) xc[3 * n + c] = DINV ? omega * v * dc[3 * n + c] : omega * v / dc[3 * n + c];
    }
}

// x_f += m_f P (m_c x_c) at fine node (i, j, k)
template <typename T, typename IX = long long>
__device__ __forceinline__ void prolong_node(int cx, int cy, int cz, int i, int j, int k, const T* __restrict__ xc,
                                             const uint8_t* __restrict__ mc, const uint8_t* __restrict__ mf,
                                             T* __restrict__ xf) {
    const int fx = 2 * cx, fy = 2 * cy;
    (void)cz;
    const IX n = i + (IX)(fx + 1) * (j + (IX)(fy + 1) * k);
    const uint8_t m = mf[n];
    if (m == 7) return;
    const int i0 = i >> 1, i1 = (i + 1) >> 1, j0 = j >> 1, j1 = (j + 1) >> 1, k0 = k >> 1, k1 = (k + 1) >> 1;
    T acc[3] = {T(0), T(0), T(0)};
    const T w = ((i & 1) ? T(0.5) : T(1)) * ((j & 1) ? T(0.5) : T(1)) * ((k & 1) ? T(0.5) : T(1));
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int ic = (q & 1) ? i1 : i0, jc = (q & 2) ? j1 : j0, kc = (q & 4) ? k1 : k0;
        // a coordinate with an even fine index has one parent: count it once
        const bool use = (!(q & 1) || i1 != i0) && (!(q & 2) || j1 != j0) && (!(q & 4) || k1 != k0);
        const IX cn = ic + (IX)(cx + 1) * (jc + (IX)(cy + 1) * kc);
        const uint8_t mcn = use ? mc[cn] : 7;
        const T v0 = use ? xc[3 * cn + 0] : T(0), v1 = use ? xc[3 * cn + 1] : T(0), v2 = use ? xc[3 * cn + 2] : T(0);
        acc[0] += (mcn & 1) ? T(0) : w * v0;
        acc[1] += (mcn & 2) ? T(0) : w * v1;
        acc[2] += (mcn & 4) ? T(0) : w * v2;
    }
    for (int c = 0; c < 3; ++c)
        if (!((m >> c) & 1)) xf[3 * n + c] += acc[c];
}

// 1 / diag(K^) at node (i, j, k): diag(K^) is kdiag times the sum of the moduli of
// the (up to 8) elements around the node, 1 on fixed DOFs; one divide per DOF here,
// multiplications where it is used
template <typename T>
__device__ __forceinline__ void diag_node(int nx, int ny, int nz, int i, int j, int k, const T* __restrict__ E,
                                          const uint8_t* __restrict__ mask, T* __restrict__ dinv, double kdiag) {
    const long long n = i + (long long)(nx + 1) * (j + (long long)(ny + 1) * k);
    T s = T(0);
    for (int dk = -1; dk <= 0; ++dk)
        for (int dj = -1; dj <= 0; ++dj)
            for (int di = -1; di <= 0; ++di) {
                const int ei = i + di, ej = j + dj, ek = k + dk;
                if (ei < 0 || ei >= nx || ej < 0 || ej >= ny || ek < 0 || ek >= nz) continue;
                s += E[ei + (long long)nx * (ej + (long long)ny * ek)];
            }
    const uint8_t mk = mask[n];
    const T v = T(1) / ((T)kdiag * s);
    for (int c = 0; c < 3; ++c) dinv[3 * n + c] = ((mk >> c) & 1) ? T(1) : v;
}

}  // namespace to
