// Matrix-free hex8 operator  y = K^(E) x  on a voxel grid (Sec. III:
// K = sum_e E_e K_e, fixtures eliminated), with fused epilogues for the
// lower-level steps (Algorithms 1 / 3, line 1) and the multigrid smoother.
//
// Work decomposition.  A CTA of TX x TY threads owns a (TX-1) x (TY-1) block of
// node columns and a range of node planes [kb, ke); thread (tx, ty) walks the
// element column (X0-1+tx, Y0-1+ty) upwards in z through element layers
// kb-1 .. ke-1 (one halo column / layer of recomputed elements per tile).
// Per element layer:
//   1. the CTA stages the (TX+1) x (TY+1) node plane k+1 in shared memory
//      (coalesced: consecutive threads read consecutive xyz words);
//   2. each thread forms the sum/difference coefficients of its element's top
//      face (2 x 12 butterfly adds); the bottom face is carried in registers
//      from the previous layer, so a z butterfly completes the 24 coefficients;
//   3. the element matrix is applied in that basis (45 products), scaled by E_e;
//   4. the inverse z butterfly splits the result into bottom-face and top-face
//      parts; the top part is carried to the next layer, the bottom part plus
//      the carry of the previous layer is the column's complete contribution
//      to node plane k, brought back to nodes by the inverse face butterflies;
//   5. the four columns around each owned node add their corner contributions
//      in a fixed order (no atomics: bitwise reproducible).
#include "device.cuh"

namespace to {

template <typename T>
struct OpArgs {
    int nx, ny, nz, kchunk;
    const T* x;
    T* y;
    const T* b;       // f (RESID) or right-hand side (SMOOTH / BMINUS)
    const T* d;       // diag(K^) (RESID with Jacobi z, SMOOTH)
    T* z;             // RESID: z = r / d (optional)
    const T* E;
    const T* Ed;      // RESID: dE/drho~ for the fused sensitivity (optional)
    T* gt;            // RESID: -E'_e u_e^T k_e u_e (optional)
    const uint8_t* mask;
    HaarK<T> kh;
    T omega;
    double* red;
    unsigned* counter;
    DevScalars* sc;
    int first_step;   // Q: record beta as the first step size of the iteration;
                      // RESID: this is the residual at u_k (record norms and J)
};

// top-face coefficients (ss, sd, ds, dd per component) from four nodes
template <typename T>
__device__ __forceinline__ void face_forward(const T* p00, const T* p10, const T* p01, const T* p11, T F[12]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T sx0 = p10[c] + p00[c], dx0 = p10[c] - p00[c];
        const T sx1 = p11[c] + p01[c], dx1 = p11[c] - p01[c];
        F[0 + c] = sx1 + sx0;
        F[3 + c] = dx1 + dx0;
        F[6 + c] = sx1 - sx0;
        F[9 + c] = dx1 - dx0;
    }
}

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

template <typename T, int TX, int TY, int MODE>
__global__ void __launch_bounds__(TX * TY) k_operator(const OpArgs<T> a) {
    __shared__ T plane[TY + 1][TX + 1][3];
    __shared__ T corner[4][TY][TX][3];
    __shared__ double sh_red[32 * kRedQ];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + TX * ty;
    const int X0 = blockIdx.x * (TX - 1), Y0 = blockIdx.y * (TY - 1);
    const int kb = blockIdx.z * a.kchunk;
    const int ke = min(kb + a.kchunk, a.nz + 1);
    const int nxn = a.nx + 1, nyn = a.ny + 1;
    const int ie = X0 - 1 + tx, je = Y0 - 1 + ty;
    const bool col_in = ie >= 0 && ie < a.nx && je >= 0 && je < a.ny;
    const int ni = X0 + tx, nj = Y0 + ty;
    const bool owner = tx < TX - 1 && ty < TY - 1 && ni < nxn && nj < nyn;

    // per-thread partial reductions (accumulated in T across the walk)
    T acc0 = T(0), acc1 = T(0), acc3 = T(0);
    T accmax = T(0);

    auto load_plane = [&](int kp) {
        const int row = 3 * (TX + 1);
        for (int e = tid; e < row * (TY + 1); e += TX * TY) {
            const int py = e / row, off = e - py * row, px = off / 3, c = off - 3 * px;
            const int gi = X0 - 1 + px, gj = Y0 - 1 + py;
            T v = T(0);
            if (kp >= 0 && kp <= a.nz && gi >= 0 && gi < nxn && gj >= 0 && gj < nyn) {
                const long long node = gi + (long long)nxn * (gj + (long long)nyn * kp);
                if (!((a.mask[node] >> c) & 1)) v = a.x[3 * node + c];
            }
            plane[py][px][c] = v;
        }
    };

    T Fb[12], Gc[12];
    load_plane(kb - 1);
    __syncthreads();
    face_forward(plane[ty][tx], plane[ty][tx + 1], plane[ty + 1][tx], plane[ty + 1][tx + 1], Fb);
#pragma unroll
    for (int i = 0; i < 12; ++i) Gc[i] = T(0);
    __syncthreads();

    for (int k = kb - 1; k < ke; ++k) {
        load_plane(k + 1);
        __syncthreads();
        T Ft[12];
        face_forward(plane[ty][tx], plane[ty][tx + 1], plane[ty + 1][tx], plane[ty + 1][tx + 1], Ft);
        T S[12];
        const bool elem_in = col_in && k >= 0 && k < a.nz;
        if (elem_in) {
            const long long e = ie + (long long)a.nx * (je + (long long)a.ny * k);
            const T Ee = a.E[e];
            T uh[24], v[24];
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                uh[i] = Ft[i] + Fb[i];
                uh[12 + i] = Ft[i] - Fb[i];
            }
            haar_apply(a.kh.v, uh, v);
            if (MODE == OP_RESID) {
                // fused sensitivity: element owned when its (1,1,1) corner node is owned
                if (a.gt && owner && k + 1 >= kb && k + 1 < ke) {
                    T en = T(0);
#pragma unroll
                    for (int i = 3; i < 24; ++i) en += uh[i] * v[i];
                    a.gt[e] = -a.Ed[e] * en;
                }
            }
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                const T s = Ee * v[i], dd = Ee * v[12 + i];
                S[i] = Gc[i] + (s - dd);
                Gc[i] = s + dd;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                S[i] = Gc[i];
                Gc[i] = T(0);
            }
        }
#pragma unroll
        for (int i = 0; i < 12; ++i) Fb[i] = Ft[i];

        const bool out_plane = k >= kb;   // plane k complete and owned by this CTA
        if (out_plane) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T ss = S[0 + c], sd = S[3 + c], ds = S[6 + c], dd = S[9 + c];
                const T sx0 = ss - ds, sx1 = ss + ds, dx0 = sd - dd, dx1 = sd + dd;
                corner[0][ty][tx][c] = sx0 - dx0;   // node (0,0) of the column face
                corner[1][ty][tx][c] = sx0 + dx0;   // (1,0)
                corner[2][ty][tx][c] = sx1 - dx1;   // (0,1)
                corner[3][ty][tx][c] = sx1 + dx1;   // (1,1)
            }
        }
        __syncthreads();
        if (out_plane && owner) {
            const long long node = ni + (long long)nxn * (nj + (long long)nyn * k);
            const uint8_t mk = a.mask[node];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const long long dof = 3 * node + c;
                T Kx = corner[3][ty][tx][c] + corner[2][ty][tx + 1][c] + corner[1][ty + 1][tx][c] +
                       corner[0][ty + 1][tx + 1][c];
                const bool fixed = (mk >> c) & 1;
                if (fixed) Kx = a.x[dof];          // K^ is the identity on fixed DOFs
                if (MODE == OP_APPLY) {
                    a.y[dof] = Kx;
                } else if (MODE == OP_Q) {
                    a.y[dof] = Kx;
                    acc0 += a.x[dof] * Kx;
                } else if (MODE == OP_BMINUS) {
                    a.y[dof] = a.b[dof] - Kx;
                } else if (MODE == OP_SMOOTH) {
                    const T xv = a.x[dof];
                    a.y[dof] = xv + a.omega * (a.b[dof] - Kx) / a.d[dof];
                } else if (MODE == OP_RESID) {
                    const T fv = a.b[dof];
                    const T rv = fv - Kx;
                    a.y[dof] = rv;
                    if (a.z) {
                        const T zv = rv / a.d[dof];
                        a.z[dof] = zv;
                        acc0 += rv * zv;
                    }
                    acc1 += rv * rv;
                    accmax = fmax(accmax, fabs(rv));
                    acc3 += fv * a.x[dof];
                }
            }
        }
    }

    if (MODE == OP_Q) {
        double v[1] = {(double)acc0};
        const int kind[1] = {0};
        double tot[1];
        block_reduce<1>(v, kind, sh_red);
        if (finish_reduction<1>(v, kind, a.red, a.counter, tot, sh_red) && tid == 0) {
            DevScalars* sc = a.sc;
            sc->zq = tot[0];
            const double rz = sc->rz;
            double beta = (tot[0] > 0.0 && rz != 0.0) ? rz / tot[0] : 0.0;
            if (!isfinite(beta)) {
                set_err(&sc->err, TO_ERR_NONFINITE);
                beta = 0.0;
            }
            sc->beta = beta;
            if (a.first_step) sc->beta_first = beta;
            sc->n_inner_done += 1;
        }
    } else if (MODE == OP_RESID) {
        double v[4] = {(double)acc0, (double)acc1, (double)accmax, (double)acc3};
        const int kind[4] = {0, 0, 1, 0};
        double tot[4];
        block_reduce<4>(v, kind, sh_red);
        if (finish_reduction<4>(v, kind, a.red, a.counter, tot, sh_red) && tid == 0) {
            DevScalars* sc = a.sc;
            sc->rz = tot[0];
            if (a.first_step) {   // the residual at u_k: tracking error and compliance estimate
                sc->res2 = sqrt(tot[1]);
                sc->res_inf = tot[2];
                sc->J = tot[3];
            }
            if (!isfinite(tot[1]) || !isfinite(tot[0])) set_err(&sc->err, TO_ERR_NONFINITE);
        }
    }
}

template <typename T>
static void fill_haar(const to_problem* P, double scale_h, HaarK<T>& kh) {
    for (int n = 0; n < kHaarNnz; ++n) kh.v[n] = (T)(P->haar[n] * scale_h);
}

template <typename T, int TX, int TY>
static int launch_t(to_problem* P, int level, int mode, const void* x, void* y, const void* b,
                    cudaStream_t s, double omega, int first) {
    const Level& L = P->lv[level];
    OpArgs<T> a{};
    a.nx = L.nx;
    a.ny = L.ny;
    a.nz = L.nz;
    a.x = (const T*)x;
    a.y = (T*)y;
    a.b = (const T*)b;
    a.d = (const T*)L.d;
    a.E = (const T*)L.E;
    a.mask = L.mask;
    fill_haar<T>(P, L.h / P->g.h, a.kh);
    a.omega = (T)omega;
    a.red = P->red;
    a.sc = P->sc;
    a.first_step = first;
    if (mode == OP_RESID) {
        a.counter = P->counters + 0;
        a.z = (P->prm.precond == TO_PRECOND_JACOBI && level == 0) ? (T*)P->z : nullptr;
        a.Ed = (const T*)P->Ed;
        a.gt = (T*)P->gt;
    } else if (mode == OP_Q) {
        a.counter = P->counters + 1;
    }
    const int gx = (L.nx + 1 + TX - 2) / (TX - 1);
    const int gy = (L.ny + 1 + TY - 2) / (TY - 1);
    int kchunk = P->tile_z;
    if (kchunk <= 0) {
        // enough CTAs for two per SM, at least 4 planes per walk
        const long long per_plane = (long long)gx * gy;
        const long long want = 2LL * P->num_sms;
        long long gz = (want + per_plane - 1) / per_plane;
        kchunk = (int)((L.nz + 1 + gz - 1) / gz);
        if (kchunk < 4) kchunk = 4;
    }
    if (kchunk > L.nz + 1) kchunk = L.nz + 1;
    a.kchunk = kchunk;
    const int gz = (L.nz + 1 + kchunk - 1) / kchunk;
    if ((long long)gx * gy * gz > kMaxRedBlocks && (mode == OP_RESID || mode == OP_Q))
        return fail(TO_ERR_ARG, "operator grid exceeds the reduction scratch; raise tile_z");
    dim3 grid(gx, gy, gz), block(TX, TY);
    switch (mode) {
        case OP_APPLY: k_operator<T, TX, TY, OP_APPLY><<<grid, block, 0, s>>>(a); break;
        case OP_RESID: k_operator<T, TX, TY, OP_RESID><<<grid, block, 0, s>>>(a); break;
        case OP_Q: k_operator<T, TX, TY, OP_Q><<<grid, block, 0, s>>>(a); break;
        case OP_SMOOTH: k_operator<T, TX, TY, OP_SMOOTH><<<grid, block, 0, s>>>(a); break;
        case OP_BMINUS: k_operator<T, TX, TY, OP_BMINUS><<<grid, block, 0, s>>>(a); break;
        default: return fail(TO_ERR_ARG, "bad operator mode");
    }
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

int launch_operator(to_problem* P, int level, int mode, const void* x, void* y, const void* b,
                    cudaStream_t s, double omega, int first) {
    if (P->prec == TO_FP64) return launch_t<double, 32, 8>(P, level, mode, x, y, b, s, omega, first);
    return launch_t<float, 32, 8>(P, level, mode, x, y, b, s, omega, first);
}

}  // namespace to
