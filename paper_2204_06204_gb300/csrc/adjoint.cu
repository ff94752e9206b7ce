// Compliance through a truncated lower-level solve, and its gradient.
//
// J(rho) = f^T u_T with u_0 = 0 and T constant-beta Jacobi steps (the literal
// lower-level step of Algorithms 1 / 3 with M = diag K):
//     r_j = f - K^ u_j,   z_j = r_j / D,   u_{j+1} = u_j + beta z_j.
// Reverse mode over the stored iterates (z_j = (u_{j+1} - u_j) / beta, so the
// residuals need not be kept):
//     lambda_T = f;  for j = T-1 .. 0:
//         s = beta lambda / D
//         dJ/drho~_e += -E'_e [ s_e^T k_e u_j,e + sum_{d in e} k_dd s_d z_j,d ]
//         lambda <- lambda - K^ s
//     dJ/drho = C^T dJ/drho~
// (u_j, s and z_j vanish on fixed DOFs; the element terms are evaluated in the
// sum/difference basis, where x^T y = (T x)^T (T y) / 8.)  As T grows, u_T tends
// to K^-1 f and the gradient to the exact sensitivity of Sec. III.
#include <algorithm>
#include <cstring>

#include "device.cuh"

namespace to {

int launch_filter_prescaled_T(to_problem* P, const void* x, void* y, cudaStream_t s);

// Haar coefficients (sum / difference basis) of one element's 24 nodal values
template <typename T>
__device__ __forceinline__ void element_haar(const T nv[2][2][2][3], T uh[24]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T F[2][4];
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2) {
            const T sx0 = nv[c2][0][1][c] + nv[c2][0][0][c], dx0 = nv[c2][0][1][c] - nv[c2][0][0][c];
            const T sx1 = nv[c2][1][1][c] + nv[c2][1][0][c], dx1 = nv[c2][1][1][c] - nv[c2][1][0][c];
            F[c2][0] = sx1 + sx0;
            F[c2][1] = dx1 + dx0;
            F[c2][2] = sx1 - sx0;
            F[c2][3] = dx1 - dx0;
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            uh[3 * f + c] = F[1][f] + F[0][f];
            uh[12 + 3 * f + c] = F[1][f] - F[0][f];
        }
    }
}

// a^T K^ b in the sum/difference basis (45 non-zeros, order of kHaarRow / kHaarCol)
template <typename T>
__device__ __forceinline__ T haar_bilinear(const T* k, const T a[24], const T b[24]) {
    T r = T(0);
    r += a[3] * (k[0] * b[3] + k[1] * b[7] + k[2] * b[14]);
    r += a[7] * (k[3] * b[3] + k[4] * b[7] + k[5] * b[14]);
    r += a[14] * (k[6] * b[3] + k[7] * b[7] + k[8] * b[14]);
    r += a[4] * (k[9] * b[4] + k[10] * b[6]) + a[6] * (k[11] * b[4] + k[12] * b[6]);
    r += a[5] * (k[13] * b[5] + k[14] * b[12]) + a[12] * (k[15] * b[5] + k[16] * b[12]);
    r += a[8] * (k[17] * b[8] + k[18] * b[13]) + a[13] * (k[19] * b[8] + k[20] * b[13]);
    r += a[9] * (k[21] * b[9] + k[22] * b[20]) + a[20] * (k[23] * b[9] + k[24] * b[20]);
    r += a[10] * (k[25] * b[10] + k[26] * b[17]) + a[17] * (k[27] * b[10] + k[28] * b[17]);
    r += a[15] * (k[29] * b[15] + k[30] * b[19]) + a[19] * (k[31] * b[15] + k[32] * b[19]);
    r += a[11] * (k[33] * b[11] + k[34] * b[16] + k[35] * b[18]);
    r += a[16] * (k[36] * b[11] + k[37] * b[16] + k[38] * b[18]);
    r += a[18] * (k[39] * b[11] + k[40] * b[16] + k[41] * b[18]);
    r += a[21] * k[42] * b[21] + a[22] * k[43] * b[22] + a[23] * k[44] * b[23];
    return r;
}

// gt_e (+)= -scale E'_e [ s_e^T k_e u_e + kdiag sum_d s_d z_d ],  z = (u1 - u0) / beta
template <typename T>
__global__ void __launch_bounds__(256) k_adjoint_elem(int nx, int ny, int nz, const T* __restrict__ svec,
                                                      const T* __restrict__ u0, const T* __restrict__ u1,
                                                      const uint8_t* __restrict__ mask, const T* __restrict__ Ed,
                                                      T* __restrict__ gt, HaarK<T> kh, T kdiag, T inv_beta,
                                                      T scale, int accumulate) {
    const Idx3 t = idx3(nx, ny, nz);
    if (!t.ok) return;
    const int i = t.i, j = t.j, k = t.k;
    const long long e = i + (long long)nx * (j + (long long)ny * k);
    const int nxn = nx + 1, nyn = ny + 1;
    T sv[2][2][2][3], uv[2][2][2][3], zv[2][2][2][3];
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
        for (int b2 = 0; b2 < 2; ++b2)
#pragma unroll
            for (int a2 = 0; a2 < 2; ++a2) {
                const long long node = (i + a2) + (long long)nxn * ((j + b2) + (long long)nyn * (k + c2));
                const uint8_t mk = mask[node];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const bool fx = (mk >> c) & 1;
                    const long long d = 3 * node + c;
                    const T a = u0[d];
                    sv[c2][b2][a2][c] = fx ? T(0) : svec[d];
                    uv[c2][b2][a2][c] = fx ? T(0) : a;
                    zv[c2][b2][a2][c] = fx ? T(0) : (u1[d] - a) * inv_beta;
                }
            }
    T sh[24], uh[24], zh[24];
    element_haar<T>(sv, sh);
    element_haar<T>(uv, uh);
    element_haar<T>(zv, zh);
    T dz = T(0);
#pragma unroll
    for (int q = 0; q < 24; ++q) dz = fma(sh[q], zh[q], dz);
    const T term = haar_bilinear<T>(kh.v, sh, uh) + kdiag * dz * T(0.125);
    const T v = -scale * Ed[e] * term;
    gt[e] = accumulate ? gt[e] + v : v;
}

// out = u + beta z
template <typename T>
__global__ void k_axpy_out(long long n, const T* __restrict__ u, const T* __restrict__ z, T beta, T* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = u[i] + beta * z[i];
}

// s = beta lambda / d (dinv = 1 / d)
template <typename T>
__global__ void k_adj_s(long long n, const T* __restrict__ lam, const T* __restrict__ dinv, T beta, T* __restrict__ s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s[i] = beta * lam[i] * dinv[i];
}

// lambda -= q
template <typename T>
__global__ void k_sub_inplace(long long n, T* __restrict__ lam, const T* __restrict__ q) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        lam[i] -= q[i];
}

// J = f^T u
template <typename T>
__global__ void __launch_bounds__(256) k_dot_J(long long n, const T* __restrict__ f, const T* __restrict__ u, double* red,
                                               unsigned* counter, DevScalars* sc) {
    __shared__ double sh[32 * kRedQ];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T fv = f[i];
        if (fv != T(0)) acc += (double)fv * (double)u[i];
    }
    double v[1] = {acc};
    const int kind[1] = {0};
    double tot[1];
    block_reduce<double, 1>(v, kind, sh);
    if (finish_reduction<double, 1>(v, kind, red, counter, tot, sh, linear_block(), grid_blocks()) && threadIdx.x == 0) sc->J = tot[0];
}

static int grid_n(long long n, int num_sms) {
    long long b = (n + 255) / 256;
    if (b > 8LL * num_sms) b = 8LL * num_sms;
    return (int)(b < 1 ? 1 : b);
}

// Iterate storage.  Stride s = 1: slot j holds u_j (j = 0 .. T).  Stride s > 1:
// slots 0 .. nck-1 hold the kept iterates u_0, u_s, u_2s, ... (nck = ceil(T / s)),
// slots nck .. nck+s hold one segment u_ms .. u_ms+s being walked.
// slots are n_dof entries rounded up to 256 bytes apart, so that every slot is aligned
// like the problem's other vectors (and takes the same operator kernel)
template <typename T>
static size_t slot_ld(const to_problem* P) {
    const size_t per = 256 / sizeof(T);
    return ((size_t)P->n_dof + per - 1) / per * per;
}
template <typename T>
static T* slot(to_problem* P, int j) {
    return (T*)P->iters + (size_t)j * slot_ld<T>(P);
}

static int stride_for(const to_problem* P, int Tn) {
    int s = P->prm.adj_stride;
    if (s == -1) {
        s = 1;
        while ((long long)s * s < Tn) ++s;   // ceil(sqrt(T))
    }
    if (s < 1) s = 1;
    if (s > Tn && Tn > 0) s = Tn;
    return s;
}

static int n_slots(int Tn, int s) {
    if (s <= 1) return Tn + 1;
    const int nck = (Tn + s - 1) / s;
    return nck + s + 1;
}

// u_out = u_in + beta D^-1 (f - K^ u_in): the residual with the fused Jacobi epilogue
// (z = r / d into P->z), then the update
template <typename T>
static int fwd_step(to_problem* P, const T* u_in, T* u_out, double beta, cudaStream_t s) {
    int rc = launch_operator(P, 0, OP_RESID, u_in, P->r, P->f, s, 0.0, 0);
    if (rc) return rc;
    const int nb = grid_n(P->n_dof, P->num_sms);
    k_axpy_out<T><<<nb, 256, 0, s>>>(P->n_dof, u_in, (const T*)P->z, (T)beta, u_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TO_ERR_CUDA, std::string("axpy: ") + cudaGetErrorString(e));
    return TO_OK;
}

// walk segment m (stride s > 1) from its kept iterate: segment slots 0 .. len hold
// u_ms .. u_ms+len afterwards
template <typename T>
static int walk_segment(to_problem* P, int m, int len, int nck, double beta, cudaStream_t s) {
    const size_t bytes = (size_t)P->n_dof * sizeof(T);
    TO_CUDA(cudaMemcpyAsync(slot<T>(P, nck), slot<T>(P, m), bytes, cudaMemcpyDeviceToDevice, s));
    for (int i = 0; i < len; ++i)
        if (int rc = fwd_step<T>(P, slot<T>(P, nck + i), slot<T>(P, nck + i + 1), beta, s)) return rc;
    return TO_OK;
}

template <typename T>
static int forward_t(to_problem* P, const void* rho, int Tn, double beta, cudaStream_t s) {
    const size_t bytes = (size_t)P->n_dof * sizeof(T);
    const int st = stride_for(P, Tn);
    const int need = n_slots(Tn, st);
    P->fwd_id = 0;
    if (need > P->iters_cap) {
        TO_CUDA(cudaStreamSynchronize(s));
        if (P->iters) cudaFree(P->iters);
        P->iters = nullptr;
        P->iters_cap = 0;
        TO_CUDA(cudaMalloc(&P->iters, slot_ld<T>(P) * sizeof(T) * (size_t)need));
        P->iters_cap = need;
    }
    TO_CUDA(cudaMemcpyAsync(P->rho, rho, P->n_elem * sizeof(T), cudaMemcpyDeviceToDevice, s));
    int rc = launch_moduli(P, s);
    if (rc) return rc;
    if ((rc = launch_diag(P, 0, s))) return rc;
    P->precond_stale = 1;   // a new design: the next to_inner_solve refreshes the preconditioner
    P->pipe_ready = 0;
    P->design_check = 0;
    TO_CUDA(cudaMemsetAsync(slot<T>(P, 0), 0, bytes, s));
    void* gt = P->gt;
    P->gt = nullptr;   // no fused sensitivity in these residuals
    const T* uT = nullptr;
    if (st == 1) {
        for (int j = 0; j < Tn && !rc; ++j) rc = fwd_step<T>(P, slot<T>(P, j), slot<T>(P, j + 1), beta, s);
        uT = slot<T>(P, Tn);
    } else {
        // keep u_ms at slot m; the segment's last iterate seeds the next kept one
        const int nck = (Tn + st - 1) / st;
        for (int m = 0; m < nck && !rc; ++m) {
            const int len = std::min(st, Tn - m * st);
            rc = walk_segment<T>(P, m, len, nck, beta, s);
            if (!rc && m + 1 < nck)
                if (cudaMemcpyAsync(slot<T>(P, m + 1), slot<T>(P, nck + len), bytes, cudaMemcpyDeviceToDevice, s) !=
                    cudaSuccess)
                    rc = fail(TO_ERR_CUDA, "kept iterate copy");
            if (!rc && m + 1 == nck) uT = slot<T>(P, nck + len);
        }
        if (Tn == 0) uT = slot<T>(P, 0);
    }
    P->gt = gt;
    if (rc) return rc;
    const int nb = grid_n(P->n_dof, P->num_sms);
    k_dot_J<T><<<nb, 256, 0, s>>>(P->n_dof, (const T*)P->f, uT, P->red, P->counters + 7, P->sc);
    TO_CUDA(cudaGetLastError());
    P->iters_T = Tn;
    P->iters_beta = beta;
    P->iters_stride = st;
    P->fwd_id = ++P->fwd_count;
    return TO_OK;
}

template <typename T>
static int backward_t(to_problem* P, double scale, void* g, cudaStream_t s) {
    const int Tn = P->iters_T;
    const int st = P->iters_stride;
    const double beta = P->iters_beta;
    const int nb = grid_n(P->n_dof, P->num_sms);
    T* lam = (T*)P->tmp_v;
    T* sv = (T*)P->z;
    T* q = (T*)P->q;
    TO_CUDA(cudaMemcpyAsync(lam, P->f, P->n_dof * sizeof(T), cudaMemcpyDeviceToDevice, s));
    HaarK<T> kh;
    for (int n = 0; n < kHaarNnz; ++n) kh.v[n] = (T)P->haar[n];
    const dim3 eg = grid3(P->g.nx, P->g.ny, P->g.nz);
    if (Tn == 0) TO_CUDA(cudaMemsetAsync(P->gt, 0, P->n_elem * sizeof(T), s));
    // one reverse step j with u_j, u_{j+1}; lambda holds lambda_{j+1} on entry, lambda_j on exit
    auto rstep = [&](int j, const T* uj, const T* uj1) -> int {
        k_adj_s<T><<<nb, 256, 0, s>>>(P->n_dof, lam, (const T*)P->lv[0].dinv, (T)beta, sv);
        TO_CUDA(cudaGetLastError());
        k_adjoint_elem<T><<<eg, block3(), 0, s>>>(P->g.nx, P->g.ny, P->g.nz, sv, uj, uj1, P->lv[0].mask,
                                                  (const T*)P->Ed, (T*)P->gt, kh, (T)P->kdiag, (T)(1.0 / beta),
                                                  (T)scale, j < Tn - 1);
        TO_CUDA(cudaGetLastError());
        if (j > 0) {
            int rc = launch_operator(P, 0, OP_APPLY, sv, q, nullptr, s);
            if (rc) return rc;
            k_sub_inplace<T><<<nb, 256, 0, s>>>(P->n_dof, lam, q);
            TO_CUDA(cudaGetLastError());
        }
        return TO_OK;
    };
    if (st == 1) {
        for (int j = Tn - 1; j >= 0; --j)
            if (int rc = rstep(j, slot<T>(P, j), slot<T>(P, j + 1))) return rc;
    } else {
        // segments last to first: recompute the segment's iterates (the residual scratch r and
        // z are free here: lambda lives in tmp_v, s is rewritten at each reverse step), then
        // run its reverse steps
        const int nck = (Tn + st - 1) / st;
        void* gt = P->gt;
        for (int m = nck - 1; m >= 0; --m) {
            const int len = std::min(st, Tn - m * st);
            P->gt = nullptr;
            int rc = walk_segment<T>(P, m, len, nck, beta, s);
            P->gt = gt;
            if (rc) return rc;
            for (int i = len - 1; i >= 0; --i)
                if ((rc = rstep(m * st + i, slot<T>(P, nck + i), slot<T>(P, nck + i + 1)))) return rc;
        }
    }
    return launch_filter_prescaled_T(P, P->gt, g, s);
}

}  // namespace to

using namespace to;

extern "C" int to_compliance_truncated(to_problem* P, const void* rho_dev, int32_t T_steps, double beta,
                                       double* J_out, void* stream) {
    if (!P) return fail(TO_ERR_ARG, "null problem");
    if (!rho_dev || T_steps < 0 || !(beta > 0.0)) return fail(TO_ERR_ARG, "need rho, T >= 0 and beta > 0");
    if (P->prm.precond != TO_PRECOND_JACOBI)
        return fail(TO_ERR_STATE, "the truncated compliance is defined with the Jacobi preconditioner");
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(P->device) != cudaSuccess) return fail(TO_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = P->prec == TO_FP64 ? forward_t<double>(P, rho_dev, T_steps, beta, s)
                                : forward_t<float>(P, rho_dev, T_steps, beta, s);
    if (!rc && J_out) {
        DevScalars h;
        if (cudaMemcpyAsync(&h, P->sc, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = fail(TO_ERR_CUDA, "reading J failed");
        else {
            *J_out = h.J;
            if (h.err) rc = fail(h.err, "device-side error in the truncated solve");
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}

extern "C" int to_compliance_truncated_grad(to_problem* P, double scale, void* g_dev, void* stream) {
    if (!P) return fail(TO_ERR_ARG, "null problem");
    if (!g_dev) return fail(TO_ERR_ARG, "null gradient");
    if (P->iters_T < 0 || P->fwd_id == 0)
        return fail(TO_ERR_STATE, P->iters_T < 0 ? "call to_compliance_truncated first"
                                                 : "the design changed since the last to_compliance_truncated");
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(P->device) != cudaSuccess) return fail(TO_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = P->prec == TO_FP64 ? backward_t<double>(P, scale, g_dev, s) : backward_t<float>(P, scale, g_dev, s);
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}

extern "C" int to_compliance_truncated_id(const to_problem* P, int64_t* id_out) {
    if (!P || !id_out) return fail(TO_ERR_ARG, "null argument");
    *id_out = P->fwd_id;
    return TO_OK;
}
