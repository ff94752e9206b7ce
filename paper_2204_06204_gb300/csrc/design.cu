// Design-side kernels: the density filter of Remark 3.1 (a linear cone of
// radius rmin), the power-law moduli of Sec. III, the Jacobi diagonal, and the
// chain rule of the sensitivity through the filter.
#include <cmath>

#include "device.cuh"

namespace to {

// ----------------------------------------------------------------------------- filter
// forward:   y_e = sum_s w_s x_{e+s} / Hs_e
// transpose: y_i = sum_s w_s x_{i+s} / Hs_{i+s}   (the stencil is symmetric)
// PRESCALED: the input already carries the 1 / Hs factor (the fused sensitivity
// writes g~ / Hs), so the transpose is a plain weighted sum.
// STATS also reports max |y| and sum y and fixes the step size alpha_k.
template <typename T, bool TRANSPOSE, bool STATS, bool PRESCALED, bool MODULI = false>
__global__ void __launch_bounds__(256) k_filter(int nx, int ny, int nz, const T* __restrict__ x, T* __restrict__ y,
                                                const T* __restrict__ Hs, const int4* __restrict__ st,
                                                const T* __restrict__ w, int ns, int R, double* red, unsigned* counter,
                                                DevScalars* sc, double alpha0_param, double alpha_scale, double m_exp,
                                                T* Eout = nullptr, T* Edout = nullptr, SimpT<T> simp = SimpT<T>{}) {
    __shared__ double sh[32 * kRedQ];
    // the stencil, padded to a multiple of 8 with zero-weight copies of the centre
    extern __shared__ __align__(16) unsigned char fsm[];
    const int nsp = (ns + 7) & ~7;
    int4* s_st = reinterpret_cast<int4*>(fsm);
    T* s_w = reinterpret_cast<T*>(fsm + (size_t)nsp * sizeof(int4));
    for (int q = threadIdx.x + 32 * threadIdx.y; q < nsp; q += 256) {
        s_st[q] = q < ns ? st[q] : make_int4(0, 0, 0, 0);
        s_w[q] = q < ns ? w[q] : T(0);
    }
    __syncthreads();
    T amax = T(0), sum = T(0);   // per-thread partials in the element precision
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    const bool ij_in = i >= R && i < nx - R && j >= R && j < ny - R;
    for (int k = blockIdx.z; k < nz && i < nx && j < ny; k += gridDim.z) {
        const long long e = i + (long long)nx * (j + (long long)ny * k);
        const bool interior = ij_in && k >= R && k < nz - R;
        T acc = T(0);
        // eight stencil points per round, all loads issued before the sums
        for (int s0 = 0; s0 < nsp; s0 += 8) {
            T xv[8], hv[8];
            if (interior) {   // no bounds checks: the linear offsets stay inside the grid
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const long long m = e + s_st[s0 + q].w;
                    xv[q] = x[m];
                    hv[q] = (TRANSPOSE && !PRESCALED) ? Hs[m] : T(1);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int4 o = s_st[s0 + q];
                    const int ii = i + o.x, jj = j + o.y, kk = k + o.z;
                    const bool ok = ii >= 0 && ii < nx && jj >= 0 && jj < ny && kk >= 0 && kk < nz;
                    const long long m = e + o.w;
                    xv[q] = ok ? x[m] : T(0);
                    hv[q] = (TRANSPOSE && !PRESCALED) ? (ok ? Hs[m] : T(1)) : T(1);
                }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const T wq = s_w[s0 + q];
                if (TRANSPOSE && !PRESCALED)
                    acc += wq * xv[q] / hv[q];
                else
                    acc += wq * xv[q];
            }
        }
        const T hs_e = TRANSPOSE ? T(1) : Hs[e];
        const T out = TRANSPOSE ? acc : acc / hs_e;
        y[e] = out;
        if (MODULI) {   // E and E' / Hs (the sensitivity's prescaled factor)
            T Ee, Ed;
            simp_moduli(simp, out, Ee, Ed);
            Eout[e] = Ee;
            Edout[e] = Ed / hs_e;
            if (!tfinite(out)) set_err(&sc->err, TO_ERR_NONFINITE);
        }
        if (STATS) {
            amax = tmax(amax, tabs(out));
            sum += out;
        }
    }
    if (STATS) {
        T v[2] = {amax, sum};
        const int kind[2] = {1, 0};
        double tot[2];
        block_reduce<T, 2>(v, kind, reinterpret_cast<T*>(sh));
        if (finish_reduction<T, 2>(v, kind, red, counter, tot, sh, linear_block(), grid_blocks()) && threadIdx.x == 0 && threadIdx.y == 0) {
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

// dynamic shared memory of k_filter: the padded stencil
template <typename T>
static size_t filter_smem(int ns) {
    const int nsp = (ns + 7) & ~7;
    return (size_t)nsp * (sizeof(int4) + sizeof(T));
}

template <typename T>
SimpT<T> simp_params(const to_material& m) {
    SimpT<T> s;
    s.emin = (T)m.Emin;
    s.dE = (T)(m.E0 - m.Emin);
    s.p = (T)m.p;
    s.cubic = m.p == 3.0;
    return s;
}
template SimpT<float> simp_params<float>(const to_material&);
template SimpT<double> simp_params<double>(const to_material&);

template <typename T>
__global__ void k_filter_rowsum(int nx, int ny, int nz, T* Hs, const int4* st, const T* w, int ns) {
    const Idx3 t = idx3(nx, ny, nz);
    if (t.ok) {
        const int i = t.i, j = t.j, k = t.k;
        const long long e = i + (long long)nx * (j + (long long)ny * k);
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

// diag(K^): kdiag * sum of the moduli of the (up to 8) elements around a node; 1 on fixed DOFs
template <typename T>
__global__ void k_diag(int nx, int ny, int nz, const T* E, const uint8_t* mask, T* d, double kdiag) {
    const Idx3 t = idx3(nx + 1, ny + 1, nz + 1);
    if (t.ok) {
        const int i = t.i, j = t.j, k = t.k;
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
static int filter_t(to_problem* P, const void* x, void* y, int transpose, int stats, int prescaled, cudaStream_t s) {
    const T* Hs = (const T*)P->Hs;
    const T* w = (const T*)P->stencil_w;
    const int nx = P->g.nx, ny = P->g.ny, nz = P->g.nz;
    const int R = (int)std::ceil(P->mat.rmin);
    dim3 grid = grid3(nx, ny, nz);
    if (stats) {
        // one reduction slot per block: fold z into the kernel's loop when the grid would exceed the slots
        const long long per_z = (long long)grid.x * grid.y;
        long long gz = kMaxRedBlocks / per_z;
        if (gz < 1) return fail(TO_ERR_ARG, "filter grid exceeds the reduction scratch");
        if (gz < nz) grid.z = (unsigned)gz;
    }
#define TO_FILTER_ARGS nx, ny, nz, (const T*)x, (T*)y, Hs, P->stencil, w, P->n_stencil, R
    const size_t fs = filter_smem<T>(P->n_stencil);
    if (transpose && stats && prescaled)
        k_filter<T, true, true, true><<<grid, block3(), fs, s>>>(TO_FILTER_ARGS, P->red, P->counters + 2, P->sc,
                                                                  P->prm.alpha0, P->prm.alpha_scale, P->prm.m);
    else if (transpose && prescaled)
        k_filter<T, true, false, true><<<grid, block3(), fs, s>>>(TO_FILTER_ARGS, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0);
    else if (transpose)
        k_filter<T, true, false, false><<<grid, block3(), fs, s>>>(TO_FILTER_ARGS, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0);
    else
        k_filter<T, false, false, false><<<grid, block3(), fs, s>>>(TO_FILTER_ARGS, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0);
#undef TO_FILTER_ARGS
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

int launch_filter(to_problem* P, const void* x, void* y, int transpose, cudaStream_t s) {
    return P->prec == TO_FP64 ? filter_t<double>(P, x, y, transpose, 0, 0, s) : filter_t<float>(P, x, y, transpose, 0, 0, s);
}

// g = C^T g~ from the prescaled g~ / Hs that the sensitivity kernels write
int launch_filter_prescaled_T(to_problem* P, const void* x, void* y, cudaStream_t s) {
    return P->prec == TO_FP64 ? filter_t<double>(P, x, y, 1, 0, 1, s) : filter_t<float>(P, x, y, 1, 0, 1, s);
}

int launch_sens_filter_T(to_problem* P, cudaStream_t s) {
    return P->prec == TO_FP64 ? filter_t<double>(P, P->gt, P->grad, 1, 1, 1, s)
                              : filter_t<float>(P, P->gt, P->grad, 1, 1, 1, s);
}

template <typename T>
static int moduli_t(to_problem* P, cudaStream_t s) {
    // rho~ = C(rho) and the moduli in one pass
    const int nx = P->g.nx, ny = P->g.ny, nz = P->g.nz;
    k_filter<T, false, false, false, true><<<grid3(nx, ny, nz), block3(), filter_smem<T>(P->n_stencil), s>>>(
        nx, ny, nz, (const T*)P->rho, (T*)P->rhot, (const T*)P->Hs, P->stencil, (const T*)P->stencil_w, P->n_stencil,
        (int)std::ceil(P->mat.rmin), nullptr, nullptr, P->sc, 0.0, 0.0, 0.0, (T*)P->lv[0].E, (T*)P->Ed,
        simp_params<T>(P->mat));
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
    (void)nb;
    k_diag<T><<<grid3(L.nx + 1, L.ny + 1, L.nz + 1), block3(), 0, s>>>(L.nx, L.ny, L.nz, (const T*)L.E, L.mask,
                                                                      (T*)L.d, L.kdiag);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

int launch_diag(to_problem* P, int level, cudaStream_t s) {
    return P->prec == TO_FP64 ? diag_t<double>(P, level, s) : diag_t<float>(P, level, s);
}

int launch_rowsum(to_problem* P, cudaStream_t s) {
    const dim3 nb = grid3(P->g.nx, P->g.ny, P->g.nz);
    const dim3 b3 = block3();
    if (P->prec == TO_FP64)
        k_filter_rowsum<double><<<nb, b3, 0, s>>>(P->g.nx, P->g.ny, P->g.nz, (double*)P->Hs, P->stencil,
                                                   (const double*)P->stencil_w, P->n_stencil);
    else
        k_filter_rowsum<float><<<nb, b3, 0, s>>>(P->g.nx, P->g.ny, P->g.nz, (float*)P->Hs, P->stencil,
                                                  (const float*)P->stencil_w, P->n_stencil);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

// ----------------------------------------------------------------------------- element energy
// gt_e = -E'_e u_e^T k_e u_e / Hs_e (Sec. III exact-gradient formula applied to u, J = f^T u;
// the 1 / Hs factor of the filter transpose is carried by the stored E' / Hs)
template <typename T>
__global__ void __launch_bounds__(256) k_energy(int nx, int ny, int nz, const T* __restrict__ u, const uint8_t* mask,
                                                const T* __restrict__ Ed, T* __restrict__ gt, HaarK<T> kh) {
    const int nxn = nx + 1, nyn = ny + 1;
    const Idx3 t = idx3(nx, ny, nz);
    if (t.ok) {
        const int i = t.i, j = t.j, k = t.k;
        const long long e = i + (long long)nx * (j + (long long)ny * k);
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
    const dim3 nb = grid3(P->g.nx, P->g.ny, P->g.nz);
    const dim3 b3 = block3();
    if (P->prec == TO_FP64) {
        HaarK<double> kh;
        for (int i = 0; i < kHaarNnz; ++i) kh.v[i] = P->haar[i];
        k_energy<double><<<nb, b3, 0, s>>>(P->g.nx, P->g.ny, P->g.nz, (const double*)u, P->lv[0].mask,
                                            (const double*)P->Ed, (double*)P->gt, kh);
    } else {
        HaarK<float> kh;
        for (int i = 0; i < kHaarNnz; ++i) kh.v[i] = (float)P->haar[i];
        k_energy<float><<<nb, b3, 0, s>>>(P->g.nx, P->g.ny, P->g.nz, (const float*)u, P->lv[0].mask,
                                           (const float*)P->Ed, (float*)P->gt, kh);
    }
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

}  // namespace to
