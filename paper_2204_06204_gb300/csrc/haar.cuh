// The hex8 element matrix applied in the sum/difference (Haar) basis of its
// 2x2x2 nodes: 45 non-zeros (kHaarRow / kHaarCol), shared by the operator kernel
// and the coarse multigrid levels' element-parallel operator.
#pragma once

#include "internal.cuh"

namespace to {

// v = K^ u in the sum/difference basis (45 non-zeros, order of kHaarRow/kHaarCol)
template <typename T>
__device__ __forceinline__ void haar_apply(const T* __restrict__ k, const T u[24], T v[24]) {
    v[0] = v[1] = v[2] = T(0);
    v[3] = k[0] * u[3] + k[1] * u[7] + k[2] * u[14];
    v[7] = k[3] * u[3] + k[4] * u[7] + k[5] * u[14];
    v[14] = k[6] * u[3] + k[7] * u[7] + k[8] * u[14];
    v[4] = k[9] * u[4] + k[10] * u[6];
    v[6] = k[11] * u[4] + k[12] * u[6];
    v[5] = k[13] * u[5] + k[14] * u[12];
    v[12] = k[15] * u[5] + k[16] * u[12];
    v[8] = k[17] * u[8] + k[18] * u[13];
    v[13] = k[19] * u[8] + k[20] * u[13];
    v[9] = k[21] * u[9] + k[22] * u[20];
    v[20] = k[23] * u[9] + k[24] * u[20];
    v[10] = k[25] * u[10] + k[26] * u[17];
    v[17] = k[27] * u[10] + k[28] * u[17];
    v[15] = k[29] * u[15] + k[30] * u[19];
    v[19] = k[31] * u[15] + k[32] * u[19];
    v[11] = k[33] * u[11] + k[34] * u[16] + k[35] * u[18];
    v[16] = k[36] * u[11] + k[37] * u[16] + k[38] * u[18];
    v[18] = k[39] * u[11] + k[40] * u[16] + k[41] * u[18];
    v[21] = k[42] * u[21];
    v[22] = k[43] * u[22];
    v[23] = k[44] * u[23];
}

// y = E k_e u for one element: u, y in the local node order (0,0,0), (1,0,0),
// (1,1,0), (0,1,0), (0,0,1), (1,0,1), (1,1,1), (0,1,1), three components each.
// Forward butterflies u -> T u along x, y, z; the 45 products; the transposed
// butterflies scaled by E (the same factorisation as the operator kernel's).
template <typename T>
__device__ __forceinline__ void elem_apply_haar(const T* __restrict__ kh, T E, const T (&u)[24], T (&y)[24]) {
    // local node of (x, y, z) offsets
    constexpr int kNode[2][2][2] = {{{0, 4}, {3, 7}}, {{1, 5}, {2, 6}}};   // [x][y][z]
    T uh[24];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T F[2][4];   // per z-face: (sum x, sum y), (diff x, sum y), (sum x, diff y), (diff x, diff y)
#pragma unroll
        for (int z = 0; z < 2; ++z) {
            const T a00 = u[3 * kNode[0][0][z] + c], a10 = u[3 * kNode[1][0][z] + c];
            const T a01 = u[3 * kNode[0][1][z] + c], a11 = u[3 * kNode[1][1][z] + c];
            const T sx0 = a10 + a00, dx0 = a10 - a00, sx1 = a11 + a01, dx1 = a11 - a01;
            F[z][0] = sx1 + sx0;
            F[z][1] = dx1 + dx0;
            F[z][2] = sx1 - sx0;
            F[z][3] = dx1 - dx0;
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            uh[3 * f + c] = F[1][f] + F[0][f];
            uh[12 + 3 * f + c] = F[1][f] - F[0][f];
        }
    }
    T v[24];
    haar_apply(kh, uh, v);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int z = 0; z < 2; ++z) {
            T G[4];
#pragma unroll
            for (int f = 0; f < 4; ++f) G[f] = z ? E * (v[3 * f + c] + v[12 + 3 * f + c]) : E * (v[3 * f + c] - v[12 + 3 * f + c]);
            const T sx0 = G[0] - G[2], sx1 = G[0] + G[2], dx0 = G[1] - G[3], dx1 = G[1] + G[3];
            y[3 * kNode[0][0][z] + c] = sx0 - dx0;
            y[3 * kNode[1][0][z] + c] = sx0 + dx0;
            y[3 * kNode[0][1][z] + c] = sx1 - dx1;
            y[3 * kNode[1][1][z] + c] = sx1 + dx1;
        }
    }
}

}  // namespace to
