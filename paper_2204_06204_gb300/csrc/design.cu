// Design-side kernels: the density filter of Remark 3.1 (a linear cone of
// radius rmin), the power-law moduli of Sec. III, the Jacobi diagonal, and the
// chain rule of the sensitivity through the filter.
#include "device.cuh"

namespace to {

// ----------------------------------------------------------------------------- filter
// forward:   y_e = sum_s w_s x_{e+s} / Hs_e
// transpose: y_i = sum_s w_s x_{i+s} / Hs_{i+s}   (the stencil is symmetric)
// Also reports max |y| and sum y (used when the output is the gradient).
template <typename T, bool TRANSPOSE, bool STATS>
__global__ void __launch_bounds__(256) k_filter(int nx, int ny, int nz, const T* __restrict__ x, T* __restrict__ y,
                                                const T* __restrict__ Hs, const int4* __restrict__ st,
                                                const T* __restrict__ w, int ns, double* red, unsigned* counter,
                                                DevScalars* sc, double alpha0_param, double alpha_scale, double m_exp) {
    __shared__ double sh[32 * kRedQ];
    const long long n = (long long)nx * ny * nz;
    double amax = 0.0, sum = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % nx);
        const int j = (int)((e / nx) % ny);
        const int k = (int)(e / ((long long)nx * ny));
        T acc = T(0);
        for (int s = 0; s < ns; ++s) {
            const int4 o = st[s];
            const int ii = i + o.x, jj = j + o.y, kk = k + o.z;
            if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
            const long long m = ii + (long long)nx * (jj + (long long)ny * kk);
            if (TRANSPOSE)
                acc += w[s] * x[m] / Hs[m];
            else
                acc += w[s] * x[m];
        }
        const T out = TRANSPOSE ? acc : acc / Hs[e];
        y[e] = out;
        if (STATS) {
            amax = fmax(amax, fabs((double)out));
            sum += (double)out;
        }
    }
    if (STATS) {
        double v[2] = {amax, sum};
        const int kind[2] = {1, 0};
        double tot[2];
        block_reduce<2>(v, kind, sh);
        if (finish_reduction<2>(v, kind, red, counter, tot, sh) && threadIdx.x == 0) {
            sc->gmax = tot[0];
            sc->gsum = tot[1];
            if (!isfinite(tot[0]) || !isfinite(tot[1])) set_err(&sc->err, TO_ERR_NONFINITE);
            // high-level step alpha_k = alpha0 k^-m; alpha0 fixed at the first k with g != 0
            double a0 = alpha0_param > 0.0 ? alpha0_param : sc->alpha0;
            if (!(a0 > 0.0) && tot[0] > 0.0) a0 = alpha_scale / tot[0];
            sc->alpha0 = a0 > 0.0 ? a0 : 0.0;
            sc->alpha = a0 > 0.0 ? a0 * pow((double)sc->k, -m_exp) : 0.0;
        }
    }
}

template <typename T>
__global__ void k_filter_rowsum(int nx, int ny, int nz, T* Hs, const int4* st, const T* w, int ns) {
    const long long n = (long long)nx * ny * nz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((long long)nx * ny));
        T acc = T(0);
        for (int s = 0; s < ns; ++s) {
            const int4 o = st[s];
            const int ii = i + o.x, jj = j + o.y, kk = k + o.z;
            if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
            acc += w[s];
        }
        Hs[e] = acc;
    }
}

// E = Emin + rho~^p (E0 - Emin),  E' = p rho~^(p-1) (E0 - Emin)
template <typename T>
__device__ __forceinline__ void simp(T rt, double E0, double Emin, double p, T& E, T& Ed) {
    const T dE = (T)(E0 - Emin);
    T pw, pw1;
    if (p == 3.0) {
        pw1 = rt * rt;
        pw = pw1 * rt;
    } else if (p == 1.0) {
        pw1 = T(1);
        pw = rt;
    } else if (p == 2.0) {
        pw1 = rt;
        pw = rt * rt;
    } else {
        pw1 = (T)pow((double)rt, p - 1.0);
        pw = pw1 * rt;
    }
    E = (T)Emin + pw * dE;
    Ed = (T)p * pw1 * dE;
}

template <typename T>
__global__ void k_moduli(long long n, const T* rt, T* E, T* Ed, double E0, double Emin, double p, int* err) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const T r = rt[e];
        if (!isfinite((double)r)) set_err(err, TO_ERR_NONFINITE);
        T a, b;
        simp<T>(r, E0, Emin, p, a, b);
        E[e] = a;
        Ed[e] = b;
    }
}

// diag(K^): kdiag * sum of the moduli of the (up to 8) elements around a node; 1 on fixed DOFs
template <typename T>
__global__ void k_diag(int nx, int ny, int nz, const T* E, const uint8_t* mask, T* d, double kdiag) {
    const long long nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn; n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % (nx + 1)), j = (int)((n / (nx + 1)) % (ny + 1)), k = (int)(n / ((long long)(nx + 1) * (ny + 1)));
        T s = T(0);
        for (int dk = -1; dk <= 0; ++dk)
            for (int dj = -1; dj <= 0; ++dj)
                for (int di = -1; di <= 0; ++di) {
                    const int ei = i + di, ej = j + dj, ek = k + dk;
                    if (ei < 0 || ei >= nx || ej < 0 || ej >= ny || ek < 0 || ek >= nz) continue;
                    s += E[ei + (long long)nx * (ej + (long long)ny * ek)];
                }
        const uint8_t mk = mask[n];
        const T v = (T)kdiag * s;
        for (int c = 0; c < 3; ++c) d[3 * n + c] = ((mk >> c) & 1) ? T(1) : v;
    }
}

static int grid_for(long long n, int threads, int num_sms) {
    long long b = (n + threads - 1) / threads;
    const long long cap = 8LL * num_sms;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename T>
static int filter_t(to_problem* P, const void* x, void* y, int transpose, int stats, cudaStream_t s) {
    const int nb = grid_for(P->n_elem, 256, P->num_sms);
    const T* Hs = (const T*)P->Hs;
    const T* w = (const T*)P->stencil_w;
    if (transpose) {
        if (stats)
            k_filter<T, true, true><<<nb, 256, 0, s>>>(P->g.nx, P->g.ny, P->g.nz, (const T*)x, (T*)y, Hs, P->stencil, w,
                                                       P->n_stencil, P->red, P->counters + 2, P->sc, P->prm.alpha0,
                                                       P->prm.alpha_scale, P->prm.m);
        else
            k_filter<T, true, false><<<nb, 256, 0, s>>>(P->g.nx, P->g.ny, P->g.nz, (const T*)x, (T*)y, Hs, P->stencil, w,
                                                        P->n_stencil, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0);
    } else {
        k_filter<T, false, false><<<nb, 256, 0, s>>>(P->g.nx, P->g.ny, P->g.nz, (const T*)x, (T*)y, Hs, P->stencil, w,
                                                     P->n_stencil, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0);
    }
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

int launch_filter(to_problem* P, const void* x, void* y, int transpose, cudaStream_t s) {
    return P->prec == TO_FP64 ? filter_t<double>(P, x, y, transpose, 0, s) : filter_t<float>(P, x, y, transpose, 0, s);
}

int launch_sens_filter_T(to_problem* P, cudaStream_t s) {
    return P->prec == TO_FP64 ? filter_t<double>(P, P->gt, P->grad, 1, 1, s) : filter_t<float>(P, P->gt, P->grad, 1, 1, s);
}

template <typename T>
static int moduli_t(to_problem* P, cudaStream_t s) {
    int rc = filter_t<T>(P, P->rho, P->rhot, 0, 0, s);
    if (rc) return rc;
    const int nb = grid_for(P->n_elem, 256, P->num_sms);
    k_moduli<T><<<nb, 256, 0, s>>>(P->n_elem, (const T*)P->rhot, (T*)P->lv[0].E, (T*)P->Ed, P->mat.E0, P->mat.Emin,
                                   P->mat.p, &P->sc->err);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

int launch_moduli(to_problem* P, cudaStream_t s) {
    return P->prec == TO_FP64 ? moduli_t<double>(P, s) : moduli_t<float>(P, s);
}

template <typename T>
static int diag_t(to_problem* P, int level, cudaStream_t s) {
    const Level& L = P->lv[level];
    const int nb = grid_for(L.n_node, 256, P->num_sms);
    k_diag<T><<<nb, 256, 0, s>>>(L.nx, L.ny, L.nz, (const T*)L.E, L.mask, (T*)L.d, L.kdiag);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

int launch_diag(to_problem* P, int level, cudaStream_t s) {
    return P->prec == TO_FP64 ? diag_t<double>(P, level, s) : diag_t<float>(P, level, s);
}

int launch_rowsum(to_problem* P, cudaStream_t s) {
    const int nb = grid_for(P->n_elem, 256, P->num_sms);
    if (P->prec == TO_FP64)
        k_filter_rowsum<double><<<nb, 256, 0, s>>>(P->g.nx, P->g.ny, P->g.nz, (double*)P->Hs, P->stencil,
                                                   (const double*)P->stencil_w, P->n_stencil);
    else
        k_filter_rowsum<float><<<nb, 256, 0, s>>>(P->g.nx, P->g.ny, P->g.nz, (float*)P->Hs, P->stencil,
                                                  (const float*)P->stencil_w, P->n_stencil);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

// ----------------------------------------------------------------------------- element energy
// gt_e = -E'_e u_e^T k_e u_e  (Sec. III exact-gradient formula applied to u, J = f^T u)
template <typename T>
__global__ void __launch_bounds__(256) k_energy(int nx, int ny, int nz, const T* __restrict__ u, const uint8_t* mask,
                                                const T* __restrict__ Ed, T* __restrict__ gt, HaarK<T> kh) {
    const long long n = (long long)nx * ny * nz;
    const int nxn = nx + 1, nyn = ny + 1;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((long long)nx * ny));
        T nv[2][2][2][3];
        for (int c2 = 0; c2 < 2; ++c2)
            for (int b2 = 0; b2 < 2; ++b2)
                for (int a2 = 0; a2 < 2; ++a2) {
                    const long long node = (i + a2) + (long long)nxn * ((j + b2) + (long long)nyn * (k + c2));
                    const uint8_t mk = mask[node];
                    for (int c = 0; c < 3; ++c) nv[c2][b2][a2][c] = ((mk >> c) & 1) ? T(0) : u[3 * node + c];
                }
        T uh[24];
        for (int c = 0; c < 3; ++c) {
            T F[2][4];
            for (int c2 = 0; c2 < 2; ++c2) {
                const T sx0 = nv[c2][0][1][c] + nv[c2][0][0][c], dx0 = nv[c2][0][1][c] - nv[c2][0][0][c];
                const T sx1 = nv[c2][1][1][c] + nv[c2][1][0][c], dx1 = nv[c2][1][1][c] - nv[c2][1][0][c];
                F[c2][0] = sx1 + sx0;
                F[c2][1] = dx1 + dx0;
                F[c2][2] = sx1 - sx0;
                F[c2][3] = dx1 - dx0;
            }
            for (int f = 0; f < 4; ++f) {
                uh[3 * f + c] = F[1][f] + F[0][f];
                uh[12 + 3 * f + c] = F[1][f] - F[0][f];
            }
        }
        // v = K^ u (same 45 positions as the operator)
        const T* kk = kh.v;
        T en = T(0);
        en += uh[3] * (kk[0] * uh[3] + kk[1] * uh[7] + kk[2] * uh[14]);
        en += uh[7] * (kk[3] * uh[3] + kk[4] * uh[7] + kk[5] * uh[14]);
        en += uh[14] * (kk[6] * uh[3] + kk[7] * uh[7] + kk[8] * uh[14]);
        en += uh[4] * (kk[9] * uh[4] + kk[10] * uh[6]) + uh[6] * (kk[11] * uh[4] + kk[12] * uh[6]);
        en += uh[5] * (kk[13] * uh[5] + kk[14] * uh[12]) + uh[12] * (kk[15] * uh[5] + kk[16] * uh[12]);
        en += uh[8] * (kk[17] * uh[8] + kk[18] * uh[13]) + uh[13] * (kk[19] * uh[8] + kk[20] * uh[13]);
        en += uh[9] * (kk[21] * uh[9] + kk[22] * uh[20]) + uh[20] * (kk[23] * uh[9] + kk[24] * uh[20]);
        en += uh[10] * (kk[25] * uh[10] + kk[26] * uh[17]) + uh[17] * (kk[27] * uh[10] + kk[28] * uh[17]);
        en += uh[15] * (kk[29] * uh[15] + kk[30] * uh[19]) + uh[19] * (kk[31] * uh[15] + kk[32] * uh[19]);
        en += uh[11] * (kk[33] * uh[11] + kk[34] * uh[16] + kk[35] * uh[18]);
        en += uh[16] * (kk[36] * uh[11] + kk[37] * uh[16] + kk[38] * uh[18]);
        en += uh[18] * (kk[39] * uh[11] + kk[40] * uh[16] + kk[41] * uh[18]);
        en += uh[21] * kk[42] * uh[21] + uh[22] * kk[43] * uh[22] + uh[23] * kk[44] * uh[23];
        gt[e] = -Ed[e] * en;
    }
}

int launch_energy(to_problem* P, const void* u, cudaStream_t s) {
    const int nb = grid_for(P->n_elem, 256, P->num_sms);
    if (P->prec == TO_FP64) {
        HaarK<double> kh;
        for (int i = 0; i < kHaarNnz; ++i) kh.v[i] = P->haar[i];
        k_energy<double><<<nb, 256, 0, s>>>(P->g.nx, P->g.ny, P->g.nz, (const double*)u, P->lv[0].mask,
                                            (const double*)P->Ed, (double*)P->gt, kh);
    } else {
        HaarK<float> kh;
        for (int i = 0; i < kHaarNnz; ++i) kh.v[i] = (float)P->haar[i];
        k_energy<float><<<nb, 256, 0, s>>>(P->g.nx, P->g.ny, P->g.nz, (const float*)u, P->lv[0].mask,
                                           (const float*)P->Ed, (float*)P->gt, kh);
    }
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

}  // namespace to
