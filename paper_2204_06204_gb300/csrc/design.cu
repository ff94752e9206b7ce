// Design-side kernels: the density filter of Remark 3.1 (a linear cone of
// radius rmin), the power-law moduli of Sec. III, the Jacobi diagonal, and the
// chain rule of the sensitivity through the filter.
#include <cmath>

#include "device.cuh"
#include "transfer.cuh"

namespace to {

// ----------------------------------------------------------------------------- filter
// forward:   y_e = sum_s w_s x_{e+s} / Hs_e
// transpose: y_i = sum_s w_s x_{i+s} / Hs_{i+s}   (the stencil is symmetric)
// PRESCALED: the input already carries the 1 / Hs factor (the fused sensitivity
// writes g~ / Hs), so the transpose is a plain weighted sum.
// STATS also reports max |y| and sum y and fixes the step size alpha_k.
// MODULI also writes E(y) and E'(y) / Hs (the forward filter of the design).
//
// A CTA of 32 x 8 threads owns a 32 x 8 column of elements over a chunk of kc z
// planes.  Its whole input box, kc + 2R planes of (32 + 2R) x (8 + 2R) values
// (R = the stencil's extent, zeros outside the grid), is copied to shared memory
// in one asynchronous batch, so that a CTA waits for memory once.  Each tap is a
// (weight, box offset) pair read as one shared-memory broadcast and applied to
// four z planes of the thread's column at once; the taps keep the stencil's
// order, so each output is summed in that order.  The transpose without
// PRESCALED stages x / Hs.
constexpr int kFilterPlanes = 4;     // z planes per thread and tap pass

template <typename T>
struct alignas(2 * sizeof(T)) FTap {
    T w;
    int off;   // dz * plane + dy * row + dx in the shared-memory box
};

// box planes a chunk of kc planes needs: kc rounded up to the tap pass, plus the halo
__host__ __device__ inline int filter_box_planes(int kchunk, int R) {
    return (kchunk + kFilterPlanes - 1) / kFilterPlanes * kFilterPlanes + 2 * R;
}

// one filter pass of one problem
template <typename T>
struct FilterArgs {
    int nx, ny, nz, kchunk;
    const T* x;
    T* y;
    const T* Hs;
    const int4* st;      // the stencil (dx, dy, dz, -) in ascending dz
    const T* w;          // its weights
    int ns, R;           // taps, extent
    double* red;         // STATS: reduction slots and counter
    unsigned* counter;
    DevScalars* sc;
    double alpha0_param, alpha_scale, m_exp;
    int mean_proj;       // STATS: ||g||_inf of the mean-projected g - 1 1^T g / E (Sec. IV-B)
    T* Eout;             // MODULI: E and E' / Hs
    T* Edout;
    SimpT<T> simp;
    const unsigned* gate;   // single-problem launch: nothing is done where gate[0] != gate[1] (nullptr: always)
};

// the CTA tile (bx, by, bz) of one problem; bid / nblocks place it among the problem's
// tiles for the STATS reduction
template <typename T, bool TRANSPOSE, bool STATS, bool PRESCALED, bool MODULI>
__device__ __forceinline__ void filter_body(const FilterArgs<T>& a, int bx, int by, int bz, unsigned bid, unsigned nblocks,
                                            unsigned char* fsm) {
    constexpr bool DIV = TRANSPOSE && !PRESCALED;   // the staged value is x / Hs
    __shared__ double sh[32 * kRedQ];
    const int nx = a.nx, ny = a.ny, nz = a.nz, kchunk = a.kchunk, ns = a.ns, R = a.R;
    const T* __restrict__ x = a.x;
    const T* __restrict__ Hs = a.Hs;
    const int4* __restrict__ st = a.st;
    const T* __restrict__ w = a.w;
    const int TW = 32 + 2 * R, TH = 8 + 2 * R, PS = TW * TH, NS = filter_box_planes(kchunk, R);
    FTap<T>* s_tap = reinterpret_cast<FTap<T>*>(fsm);
    T* box = reinterpret_cast<T*>(fsm + (size_t)ns * sizeof(FTap<T>));   // NS planes of the input
    T* hbox = box + (size_t)NS * PS;                                     // NS planes of Hs (DIV only)
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int i0 = bx * 32, j0 = by * 8;
    const int k0 = bz * kchunk, k1 = min(k0 + kchunk, nz);
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    const bool ij_ok = i < nx && j < ny;
    const long long plane = (long long)nx * ny;

    // planes k0 - R .. k1 + R - 1 into box planes 0 .. k1 - k0 + 2R - 1 (zeros outside the grid)
    for (int q = tid; q < PS; q += 256) {
        const int gi = i0 - R + q % TW, gj = j0 - R + q / TW;
        const bool okij = gi >= 0 && gi < nx && gj >= 0 && gj < ny;
        const long long base = okij ? gi + (long long)nx * gj : 0;
        for (int p = k0 - R, b = q; p < k1 + R; ++p, b += PS) {
            const bool v = okij && p >= 0 && p < nz;
            const long long e = v ? base + (long long)p * plane : 0;
            cp_async_t<T>(box + b, x + e, v);
            if (DIV) cp_async_t<T>(hbox + b, Hs + e, v);
        }
    }
    cp_commit();
    for (int q = tid; q < ns; q += 256) {   // the taps, while the copies are in flight
        const int4 o = st[q];
        s_tap[q].w = w[q];
        s_tap[q].off = o.z * PS + o.y * TW + o.x;
    }
    cp_wait<0>();
    if (DIV)   // x / Hs in place for the words this thread copied
        for (int q = tid; q < PS; q += 256) {
            const int gi = i0 - R + q % TW, gj = j0 - R + q / TW;
            const bool okij = gi >= 0 && gi < nx && gj >= 0 && gj < ny;
            for (int p = k0 - R, b = q; p < k1 + R; ++p, b += PS)
                if (okij && p >= 0 && p < nz) box[b] = box[b] / hbox[b];
        }
    __syncthreads();

    T vmax = T(-INFINITY), vmin = T(INFINITY), sum = T(0);   // per-thread partials in the element precision
    const T* col = box + (size_t)R * PS + (threadIdx.y + R) * TW + threadIdx.x + R;   // (i, j, k0) in the box
    for (int kb = k0; kb < k1; kb += kFilterPlanes) {
        T acc[kFilterPlanes];
#pragma unroll
        for (int c = 0; c < kFilterPlanes; ++c) acc[c] = T(0);
        const T* b0 = col + (size_t)(kb - k0) * PS;
        T hsv[kFilterPlanes];   // Hs of the outputs, loaded ahead of the taps
#pragma unroll
        for (int c = 0; c < kFilterPlanes; ++c)
            hsv[c] = (!TRANSPOSE && ij_ok && kb + c < k1) ? Hs[i + (long long)nx * (j + (long long)ny * (kb + c))] : T(1);
#pragma unroll 2
        for (int q = 0; q < ns; ++q) {
            const FTap<T> tp = s_tap[q];
            const T* pp = b0 + tp.off;
#pragma unroll
            for (int c = 0; c < kFilterPlanes; ++c) acc[c] += tp.w * pp[c * PS];   // planes past k1: discarded
        }
#pragma unroll
        for (int c = 0; c < kFilterPlanes; ++c) {
            const int k = kb + c;
            if (!ij_ok || k >= k1) continue;
            const long long e = i + (long long)nx * (j + (long long)ny * k);
            const T hs_e = hsv[c];
            const T out = TRANSPOSE ? acc[c] : acc[c] / hs_e;
            a.y[e] = out;
            if (MODULI) {   // E and E' / Hs (the sensitivity's prescaled factor)
                T Ee, Ed;
                simp_moduli(a.simp, out, Ee, Ed);
                a.Eout[e] = Ee;
                a.Edout[e] = Ed / hs_e;
                if (!tfinite(out)) set_err(&a.sc->err, TO_ERR_NONFINITE);
            }
            if (STATS) {
                vmax = tmax(vmax, out);
                vmin = tmin(vmin, out);
                sum += out;
            }
        }
    }
    if (STATS) {
        T v[3] = {vmax, -vmin, sum};
        const int kind[3] = {1, 1, 0};
        double tot[3];
        block_reduce<T, 3>(v, kind, reinterpret_cast<T*>(sh));
        if (finish_reduction<T, 3>(v, kind, a.red, a.counter, tot, sh, bid, nblocks) && tid == 0) {
            DevScalars* sc = a.sc;
            // ||g||_inf of the step direction: g itself, or g - mean(g) with the mean projection
            const double shift = a.mean_proj ? tot[2] / ((double)nx * ny * nz) : 0.0;
            const double gmax = fmax(tot[0] - shift, tot[1] + shift);
            sc->gmax = gmax;
            sc->gsum = tot[2];
            if (!isfinite(gmax) || !isfinite(tot[2])) set_err(&sc->err, TO_ERR_NONFINITE);
            // high-level step alpha_k = alpha0 k^-m; alpha0 fixed at the first k with g != 0
            double a0 = a.alpha0_param > 0.0 ? a.alpha0_param : sc->alpha0;
            if (!(a0 > 0.0) && gmax > 0.0) a0 = a.alpha_scale / gmax;
            sc->alpha0 = a0 > 0.0 ? a0 : 0.0;
            sc->alpha = a0 > 0.0 ? a0 * pow((double)sc->k, -a.m_exp) : 0.0;
        }
    }
}

template <typename T, bool TRANSPOSE, bool STATS, bool PRESCALED, bool MODULI = false>
__global__ void __launch_bounds__(256) k_filter(const FilterArgs<T> a) {
    extern __shared__ __align__(16) unsigned char fsm[];
    if (a.gate && a.gate[0] != a.gate[1]) return;   // the whole grid: no CTA reaches a barrier
    filter_body<T, TRANSPOSE, STATS, PRESCALED, MODULI>(a, blockIdx.x, blockIdx.y, blockIdx.z, linear_block(),
                                                         grid_blocks(), fsm);
}

// Many problems in one launch: blockIdx.y selects the problem, blockIdx.x its tile
template <typename T, bool TRANSPOSE, bool STATS, bool PRESCALED, bool MODULI>
__global__ void __launch_bounds__(256) k_filter_batch(const FilterArgs<T>* __restrict__ tab) {
    extern __shared__ __align__(16) unsigned char fsm[];
    const FilterArgs<T>& a = tab[blockIdx.y];
    const int gx = (a.nx + 31) / 32, gy = (a.ny + 7) / 8, gz = (a.nz + a.kchunk - 1) / a.kchunk;
    const int t = blockIdx.x;
    if (t >= gx * gy * gz) return;
    filter_body<T, TRANSPOSE, STATS, PRESCALED, MODULI>(a, t % gx, (t / gx) % gy, t / (gx * gy), (unsigned)t,
                                                         (unsigned)(gx * gy * gz), fsm);
}

// dynamic shared memory of k_filter: the taps, the input box (and the Hs box)
template <typename T>
static size_t filter_smem(int ns, int R, int kchunk, bool div) {
    const size_t PS = (size_t)(32 + 2 * R) * (8 + 2 * R), NS = filter_box_planes(kchunk, R);
    return (size_t)ns * sizeof(FTap<T>) + (div ? 2 : 1) * NS * PS * sizeof(T);
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

template <typename T>
__global__ void k_diag(int nx, int ny, int nz, const T* E, const uint8_t* mask, T* dinv, double kdiag, const unsigned* gate) {
    if (gate && gate[0] != gate[1]) return;
    const Idx3 t = idx3(nx + 1, ny + 1, nz + 1);
    if (t.ok) diag_node<T>(nx, ny, nz, t.i, t.j, t.k, E, mask, dinv, kdiag);
}

template <typename T>
static FilterArgs<T> filter_args(const to_problem* P, const T* x, T* y, int kchunk, bool stats, T* Eout, T* Edout) {
    FilterArgs<T> a;
    a.nx = P->g.nx;
    a.ny = P->g.ny;
    a.nz = P->g.nz;
    a.kchunk = kchunk;
    a.x = x;
    a.y = y;
    a.Hs = (const T*)P->Hs;
    a.st = P->stencil;
    a.w = (const T*)P->stencil_w;
    a.ns = P->n_stencil;
    a.R = P->filter_ext;
    a.red = stats ? P->red_d : nullptr;
    a.counter = stats ? P->counters + 2 : nullptr;
    a.sc = P->sc;
    a.alpha0_param = P->prm.alpha0;
    a.alpha_scale = P->prm.alpha_scale;
    a.m_exp = P->prm.m;
    a.mean_proj = P->prm.mean_proj;
    a.Eout = Eout;
    a.Edout = Edout;
    a.simp = simp_params<T>(P->mat);
    a.gate = nullptr;
    return a;
}

// the filter's launch shape: 32 x 8 element columns, each CTA a chunk of z planes
// (about four CTAs per SM), and its shared memory
template <typename T, bool TRANSPOSE, bool STATS, bool PRESCALED, bool MODULI>
static int filter_launch(to_problem* P, const T* x, T* y, cudaStream_t s, T* Eout = nullptr, T* Edout = nullptr,
                         const unsigned* gate = nullptr) {
    const int nx = P->g.nx, ny = P->g.ny, nz = P->g.nz, R = P->filter_ext;
    constexpr bool DIV = TRANSPOSE && !PRESCALED;
    const int gx = (nx + 31) / 32, gy = (ny + 7) / 8;
    long long chunks = (4LL * P->num_sms + (long long)gx * gy - 1) / ((long long)gx * gy);
    if (chunks > nz) chunks = nz;
    if (chunks < 1) chunks = 1;
    int kchunk = (int)((nz + chunks - 1) / chunks);
    while (kchunk > 1 && filter_smem<T>(P->n_stencil, R, kchunk, DIV) > 96 * 1024) --kchunk;   // the box fits
    chunks = (nz + kchunk - 1) / kchunk;
    if (STATS && (long long)gx * gy * chunks > kMaxRedBlocks) {
        kchunk = (int)((nz + kMaxRedBlocks / ((long long)gx * gy) - 1) / (kMaxRedBlocks / ((long long)gx * gy)));
        chunks = (nz + kchunk - 1) / kchunk;
        if ((long long)gx * gy * chunks > kMaxRedBlocks) return fail(TO_ERR_ARG, "filter grid exceeds the reduction scratch");
    }
    const size_t fs = filter_smem<T>(P->n_stencil, R, kchunk, DIV);
    if (fs > 227 * 1024) return fail(TO_ERR_ARG, "filter tile exceeds shared memory (radius too large for this grid)");
    auto kern = k_filter<T, TRANSPOSE, STATS, PRESCALED, MODULI>;
    // the opt-in is per kernel and shared by every problem (and by graphs captured
    // earlier): it only ever grows
    static size_t opted = 48 * 1024;
    if (fs > opted) {
        TO_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs));
        opted = fs;
    }
    const dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)chunks);
    FilterArgs<T> a = filter_args<T>(P, x, y, kchunk, STATS, Eout, Edout);
    a.gate = gate;
    kern<<<grid, block3(), fs, s>>>(a);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

// Batched filters: one table entry per problem and one launch for all of them (the
// design pass rho -> rho~, E, E'/Hs, and the gradient pass C^T g~ with the step-size
// statistics).  Each problem walks chunks of up to 8 planes; the launch's shared
// memory is the largest problem's box.
template <typename T>
static int filter_table_t(to_problem* const* probs, int n, int mode, void** dev, int* max_tiles, size_t* smem) {
    std::vector<FilterArgs<T>> h(n);
    int mt = 0;
    size_t fs = 0;
    for (int i = 0; i < n; ++i) {
        to_problem* P = probs[i];
        const int kchunk = std::min(P->g.nz, 8);
        if (mode == 0)
            h[i] = filter_args<T>(P, (const T*)P->rho, (T*)P->rhot, kchunk, false, (T*)P->lv[0].E, (T*)P->Ed);
        else
            h[i] = filter_args<T>(P, (const T*)P->gt, (T*)P->grad, kchunk, true, nullptr, nullptr);
        const int tiles = ((P->g.nx + 31) / 32) * ((P->g.ny + 7) / 8) * ((P->g.nz + kchunk - 1) / kchunk);
        if (tiles > kMaxRedBlocks) return fail(TO_ERR_ARG, "batched filter grid exceeds the reduction scratch");
        mt = std::max(mt, tiles);
        fs = std::max(fs, filter_smem<T>(P->n_stencil, P->filter_ext, kchunk, false));
    }
    if (fs > 227 * 1024) return fail(TO_ERR_ARG, "batched filter tile exceeds shared memory");
    if (cudaMalloc(dev, sizeof(FilterArgs<T>) * (size_t)n) != cudaSuccess) return fail(TO_ERR_CUDA, "table allocation");
    if (cudaMemcpy(*dev, h.data(), sizeof(FilterArgs<T>) * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(TO_ERR_CUDA, "table upload");
    if (fs > 48 * 1024) {
        if (mode == 0)
            TO_CUDA(cudaFuncSetAttribute(k_filter_batch<T, false, false, false, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        else
            TO_CUDA(cudaFuncSetAttribute(k_filter_batch<T, true, true, true, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    }
    *max_tiles = mt;
    *smem = fs;
    return TO_OK;
}

int filter_table_build(to_problem* const* probs, int n, int mode, void** dev, int* max_tiles, size_t* smem) {
    return probs[0]->prec == TO_FP64 ? filter_table_t<double>(probs, n, mode, dev, max_tiles, smem)
                                     : filter_table_t<float>(probs, n, mode, dev, max_tiles, smem);
}

int filter_batch_launch(int prec, int mode, const void* tab, int max_tiles, int n, size_t smem, cudaStream_t s) {
    const dim3 grid(max_tiles, n);
    if (prec == TO_FP64) {
        if (mode == 0) k_filter_batch<double, false, false, false, true><<<grid, block3(), smem, s>>>((const FilterArgs<double>*)tab);
        else k_filter_batch<double, true, true, true, false><<<grid, block3(), smem, s>>>((const FilterArgs<double>*)tab);
    } else {
        if (mode == 0) k_filter_batch<float, false, false, false, true><<<grid, block3(), smem, s>>>((const FilterArgs<float>*)tab);
        else k_filter_batch<float, true, true, true, false><<<grid, block3(), smem, s>>>((const FilterArgs<float>*)tab);
    }
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

template <typename T>
static int filter_t(to_problem* P, const void* x, void* y, int transpose, int stats, int prescaled, cudaStream_t s) {
    const T* xi = (const T*)x;
    T* yo = (T*)y;
    if (transpose && stats && prescaled) return filter_launch<T, true, true, true, false>(P, xi, yo, s);
    if (transpose && prescaled) return filter_launch<T, true, false, true, false>(P, xi, yo, s);
    if (transpose) return filter_launch<T, true, false, false, false>(P, xi, yo, s);
    return filter_launch<T, false, false, false, false>(P, xi, yo, s);
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
static int moduli_t(to_problem* P, cudaStream_t s, const unsigned* gate) {
    // rho~ = C(rho) and the moduli in one pass
    return filter_launch<T, false, false, false, true>(P, (const T*)P->rho, (T*)P->rhot, s, (T*)P->lv[0].E, (T*)P->Ed,
                                                       gate);
}

int launch_moduli(to_problem* P, cudaStream_t s, const unsigned* gate) {
    return P->prec == TO_FP64 ? moduli_t<double>(P, s, gate) : moduli_t<float>(P, s, gate);
}

template <typename T>
static int diag_t(to_problem* P, int level, cudaStream_t s, const unsigned* gate) {
    const Level& L = P->lv[level];
    k_diag<T><<<grid3(L.nx + 1, L.ny + 1, L.nz + 1), block3(), 0, s>>>(L.nx, L.ny, L.nz, (const T*)L.E, L.mask,
                                                                      (T*)L.dinv, L.kdiag, gate);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

int launch_diag(to_problem* P, int level, cudaStream_t s, const unsigned* gate) {
    return P->prec == TO_FP64 ? diag_t<double>(P, level, s, gate) : diag_t<float>(P, level, s, gate);
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
