// Projection onto X = {lo <= rho <= hi, 1^T rho <= vbar} (Sec. IV-B).
//
// The KKT conditions give rho = clamp(w - lambda, lo, hi) with lambda = 0 when
// the clamp already meets the volume bound, else the root of the piecewise-
// linear, non-increasing volume function of Eq. (piecewiseLinearEQ)
//   S(lambda) = sum_e clamp(w_e - lambda, lo, hi) = vbar.
// The paper finds the root by sorting the 2E breakpoints (Algorithm 4; on a GPU
// with a radix sort and a scan).  Here one cooperative kernel runs a
// safeguarded Newton iteration on S instead: each pass classifies every element
// as at-upper / at-lower / free for the current lambda (one grid reduction of
// the counts and of the free elements' sum), S is then known exactly on the
// current linear piece and the Newton step lands on the root of that piece;
// a bracket [lambda_lo, lambda_hi] with S(lambda_lo) > vbar >= S(lambda_hi)
// falls back to bisection whenever the step leaves it.  Once the pass sees the
// same piece twice the root is exact (up to rounding), typically in a handful
// of passes (one, when the previous multiplier is a good start).  The body of
// the search and its arithmetic are in projection.cuh.
#include <cooperative_groups.h>

#include <cmath>
#include <cstddef>
#include <mutex>

#include "projection.cuh"

namespace to {

template <typename T>
struct ProjArgs {
    long long n;
    const T* w_in;       // plain mode
    const T* rho_in;     // fused mode: w = rho - alpha (g - mean)
    const T* g;
    T* wbuf;             // scratch (n), used when a block's chunk does not fit in shared memory
    T* rho_out;
    double vbar, lo, hi;
    int fused, mean_proj;
    int wdirect;         // plain mode without a cache: read w from w_in, store nothing (wbuf == w_in)
    long long chunk;     // elements per block (contiguous)
    double* part;        // 2 * nblocks * kProjSlot words
    unsigned* bar;       // barrier words
    DevScalars* sc;
};

// Pass totals across the blocks of a cooperative launch: thread 0 publishes the
// block's partial in global memory, the grid barrier orders it, and warp 0 of
// every block folds all partials (L2 reads) in the same order.
struct GridComm {
    double* part;
    unsigned nb, bid;
    unsigned* bar;
    int* err;
    __device__ bool exchange(const ProjPart& mine, int parity, ProjPart& tot) {
        double* base = part + (size_t)parity * nb * kProjSlot;
        if (threadIdx.x == 0) *reinterpret_cast<ProjPart*>(base + (size_t)bid * kProjSlot) = mine;
        if (!grid_barrier(bar, err)) return false;
        if (threadIdx.x < 32) {
            const ProjPart t = proj_fold(nb, [&](unsigned b) {
                const ProjPart* p = reinterpret_cast<const ProjPart*>(base + (size_t)b * kProjSlot);
                ProjPart r;
#pragma unroll
                for (int q = 0; q < 6; ++q) r.n[q] = __ldcg(&p->n[q]);
                r.s[0] = __ldcg(&p->s[0]);
                r.s[1] = __ldcg(&p->s[1]);
                r.wmin = __ldcg(&p->wmin);
                r.wmax = __ldcg(&p->wmax);
                return r;
            });
            if (threadIdx.x == 0) tot = t;
        }
        return true;
    }
};

// One cooperative kernel: each block takes a contiguous chunk of the elements
// (cached in shared memory when it fits) and runs the shared projection body.
template <typename T, bool CACHE>
__global__ void __launch_bounds__(256) k_project(const ProjArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GridComm comm{a.part, gridDim.x, blockIdx.x, a.bar, &a.sc->err};
    ProjIO io;
    io.n = a.n;
    io.b0 = (long long)blockIdx.x * a.chunk;
    io.b1 = min(io.b0 + a.chunk, a.n);
    io.vbar = a.vbar;
    io.lo = a.lo;
    io.hi = a.hi;
    io.fused = a.fused;
    io.mean_proj = a.mean_proj;
    io.writer = blockIdx.x == 0;
    io.wdirect = a.wdirect;
    projection_body<T, CACHE>(comm, io, a.w_in, a.rho_in, a.g, reinterpret_cast<T*>(smem_raw), a.wbuf, a.rho_out,
                              a.sc);
}

constexpr size_t kProjSmem = 96 * 1024;

// ----------------------------------------------------------------------------- the problem's projection
// Three launches: a first pass over the whole GPU (w, the sets at lambda = 0 and
// at the warm start, min / max; its last block folds the partials and starts the
// search), the remaining search passes on one thread-block cluster (hardware
// barrier between passes; usually one pass, often none), and a final pass over
// the whole GPU (the clamp, ||drho||_inf, the volume).  The search state moves
// between them in DevScalars.

// thread 0 of the folding block: S0, the bracket, Newton from 0, the warm start;
// stores the state (and the multiplier when the search already ended)
__device__ __forceinline__ void proj_search_start(const ProjPart& tot, double lam_s, double vbar, double lo, double hi,
                                                  DevScalars* sc) {
    ProjSearch st;
    const double S0 = (double)tot.n[0] * hi + (double)tot.n[1] * lo + tot.s[0];
    if (!isfinite(S0)) set_err(&sc->err, TO_ERR_NONFINITE);
    sc->proj_active = S0 > vbar && isfinite(S0);
    st.done = !(S0 > vbar) || !isfinite(S0);
    st.have_prev = false;
    st.pU = st.pL = st.pF = 0.0;
    st.lam = 0.0;
    st.lo_b = 0.0;
    st.hi_b = 0.0;
    if (!st.done) {
        st.lo_b = fmax(0.0, tot.wmin - hi);
        st.hi_b = tot.wmax - lo;
        const double t0[4] = {(double)tot.n[0], (double)tot.n[1], (double)tot.n[2], tot.s[0]};
        proj_search_step(st, t0, vbar, lo, hi);
        if (!st.done && lam_s > st.lo_b && lam_s < st.hi_b) {
            const double ts[4] = {(double)tot.n[3], (double)tot.n[4], (double)tot.n[5], tot.s[1]};
            st.lam = lam_s;
            st.have_prev = false;
            proj_search_step(st, ts, vbar, lo, hi);
        }
        if (st.done) sc->lambda = st.lam;
    } else {
        sc->lambda = 0.0;   // the box clamp meets the volume bound
    }
    sc->proj_iters = 0;
    sc->ps = st;
}

template <typename T>
struct ProjPipe {
    long long n;
    const T* w_in;       // plain mode
    const T* rho_in;     // fused mode: w = rho - alpha (g - mean)
    const T* g;
    T* wbuf;             // w of the fused mode, read by the later passes
    T* rho_out;
    double vbar, lo, hi;
    int fused, mean_proj;
    double* part;        // kProjSlot words per block of the first pass
    double* red;         // kRedQ words per block of the final pass
    unsigned* counter;   // [0] first pass, [1] final pass
    DevScalars* sc;
};

template <typename T>
__global__ void __launch_bounds__(512) k_proj_first(const ProjPipe<T> a) {
    __shared__ float shf[128];
    __shared__ double shd[64];
    __shared__ unsigned shu[32 * 6];
    __shared__ T sht[32 * 2];
    __shared__ T s_alpha, s_gmean, s_tu0, s_tl0, s_tus, s_tls;
    __shared__ double s_lam;
    __shared__ int s_last;
    const int tid = threadIdx.x;
    DevScalars* sc = a.sc;
    if (tid == 0) {
        const double alpha = a.fused ? sc->alpha : 0.0;
        const double gmean = (a.fused && a.mean_proj) ? sc->gsum / (double)a.n : 0.0;
        s_alpha = (T)alpha;
        s_gmean = (T)gmean;
        s_lam = sc->lambda > 0.0 ? sc->lambda : 0.0;   // the warm start: the previous multiplier
        proj_thresholds<T>(0.0, a.lo, a.hi, s_tu0, s_tl0);
        proj_thresholds<T>(s_lam, a.lo, a.hi, s_tus, s_tls);
    }
    __syncthreads();
    const T alpha_t = s_alpha, gmean_t = s_gmean, tu0 = s_tu0, tl0 = s_tl0, tus = s_tus, tls = s_tls;
    unsigned cnt[6] = {0u, 0u, 0u, 0u, 0u, 0u};
    ProjSum<T> sum[2];
    T wmn = T(INFINITY), wmx = T(-INFINITY);
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long e0 = (long long)blockIdx.x * blockDim.x + tid; e0 < a.n; e0 += 4 * step) {
        T rv[4], gv[4];   // four elements per round: their loads are in flight together
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long e = e0 + q * step;
            rv[q] = e < a.n ? (a.fused ? a.rho_in[e] : a.w_in[e]) : T(0);
            gv[q] = (a.fused && e < a.n) ? a.g[e] : T(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long e = e0 + q * step;
            if (e < a.n) {
                const T w = a.fused ? rv[q] - alpha_t * (gv[q] - gmean_t) : rv[q];
                if (a.fused) a.wbuf[e] = w;
                if (w >= tu0) ++cnt[0];
                else if (w <= tl0) ++cnt[1];
                else { ++cnt[2]; sum[0].add(w); }
                if (w >= tus) ++cnt[3];
                else if (w <= tls) ++cnt[4];
                else { ++cnt[5]; sum[1].add(w); }
                wmn = tmin(wmn, w);
                wmx = tmax(wmx, w);
            }
        }
    }
    const int ksum[6] = {0, 0, 0, 0, 0, 0};
    block_reduce<unsigned, 6>(cnt, ksum, shu);
    double sums[2];
    proj_block_sums(sum, sums, shf, shd);
    T mm[2] = {-wmn, wmx};
    const int kmax[2] = {1, 1};
    block_reduce<T, 2>(mm, kmax, sht);
    if (tid == 0) {
        ProjPart* mine = reinterpret_cast<ProjPart*>(a.part + (size_t)blockIdx.x * kProjSlot);
#pragma unroll
        for (int q = 0; q < 6; ++q) mine->n[q] = cnt[q];
        mine->s[0] = sums[0];
        mine->s[1] = sums[1];
        mine->wmin = -(double)mm[0];
        mine->wmax = (double)mm[1];
        __threadfence();
        const unsigned t = atomicAdd(a.counter, 1u);
        s_last = (t == gridDim.x - 1);
        if (s_last) atomicExch(a.counter, 0u);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (tid < 32) {
        const ProjPart tot = proj_fold(gridDim.x, [&](unsigned b) {
            const ProjPart* p = reinterpret_cast<const ProjPart*>(a.part + (size_t)b * kProjSlot);
            ProjPart r;
#pragma unroll
            for (int q = 0; q < 6; ++q) r.n[q] = __ldcg(&p->n[q]);
            r.s[0] = __ldcg(&p->s[0]);
            r.s[1] = __ldcg(&p->s[1]);
            r.wmin = __ldcg(&p->wmin);
            r.wmax = __ldcg(&p->wmax);
            return r;
        });
        if (tid == 0) proj_search_start(tot, s_lam, a.vbar, a.lo, a.hi, sc);
    }
}

// the remaining passes of the search over [b0, b1) of w, with pass totals from `comm`
template <typename T, class Comm>
__device__ __forceinline__ void proj_search_passes(Comm& comm, long long b0, long long b1, const T* w, double vbar,
                                                   double lo, double hi, DevScalars* sc, bool writer) {
    __shared__ float shf[128];
    __shared__ double shd[64];
    __shared__ unsigned shu[32 * 3];
    __shared__ ProjSearch st;
    __shared__ ProjPart tot, mine;
    __shared__ T s_tu, s_tl;
    __shared__ int s_done, s_iters;
    const int tid = threadIdx.x;
    const int nthreads = blockDim.x;
    if (tid == 0) {
        st = sc->ps;
        s_done = st.done;
        s_iters = 0;
        proj_thresholds<T>(st.lam, lo, hi, s_tu, s_tl);
    }
    __syncthreads();
    if (s_done) return;   // every block reads the same state: all leave together
    int parity = 0;
    while (!s_done && s_iters < kProjMaxIter) {
        const T tu = s_tu, tl = s_tl;
        unsigned cnt[3] = {0u, 0u, 0u};
        ProjSum<T> sum[2];
        const long long step = nthreads;
        for (long long e0 = b0 + tid; e0 < b1; e0 += 4 * step) {
            T wv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const long long e = e0 + q * step;
                wv[q] = e < b1 ? w[e] : T(0);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const long long e = e0 + q * step;
                if (e < b1) {
                    const T x = wv[q];
                    if (x >= tu) ++cnt[0];
                    else if (x <= tl) ++cnt[1];
                    else { ++cnt[2]; sum[0].add(x); }
                }
            }
        }
        const int ksum[3] = {0, 0, 0};
        block_reduce<unsigned, 3>(cnt, ksum, shu);
        double sums[2];
        proj_block_sums(sum, sums, shf, shd);
        if (tid == 0) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                mine.n[q] = cnt[q];
                mine.n[q + 3] = 0ull;
            }
            mine.s[0] = sums[0];
            mine.s[1] = 0.0;
            mine.wmin = INFINITY;
            mine.wmax = -INFINITY;
        }
        if (!comm.exchange(mine, parity, tot)) return;
        parity ^= 1;
        if (tid == 0) {
            const double t4[4] = {(double)tot.n[0], (double)tot.n[1], (double)tot.n[2], tot.s[0]};
            proj_search_step(st, t4, vbar, lo, hi);
            s_done = st.done;
            s_iters += 1;
            proj_thresholds<T>(st.lam, lo, hi, s_tu, s_tl);
        }
        __syncthreads();
    }
    if (tid == 0 && writer) {
        sc->lambda = st.lam;
        sc->proj_iters = s_iters;
        st.done = true;
        sc->ps = st;
    }
}

// search passes on one cluster: each CTA takes a contiguous chunk of w
template <typename T>
__global__ void __launch_bounds__(1024) k_proj_search_cluster(const T* __restrict__ w, long long n, double vbar,
                                                              double lo, double hi, DevScalars* sc) {
    namespace cg = cooperative_groups;
    __shared__ ProjPart slots[2];
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank(), cs = cl.num_blocks();
    const long long chunk = (n + cs - 1) / cs;
    const long long b0 = (long long)rank * chunk, b1 = min(b0 + chunk, n);
    ClusterComm comm{slots};
    proj_search_passes<T>(comm, b0, b1, w, vbar, lo, hi, sc, rank == 0);
    cl.sync();   // no CTA leaves while another may still read its slots
}

// search passes on a cooperative grid (when no cluster of 16 can be placed)
template <typename T>
__global__ void __launch_bounds__(256) k_proj_search_grid(const T* __restrict__ w, long long n, double vbar, double lo,
                                                          double hi, DevScalars* sc, double* part, unsigned* bar) {
    const long long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long long b0 = (long long)blockIdx.x * chunk, b1 = min(b0 + chunk, n);
    GridComm comm{part, gridDim.x, blockIdx.x, bar, &sc->err};
    proj_search_passes<T>(comm, b0, b1, w, vbar, lo, hi, sc, blockIdx.x == 0);
}

// rho = clamp(w - lambda), ||drho||_inf (fused mode), the volume
template <typename T>
__global__ void __launch_bounds__(512) k_proj_final(const ProjPipe<T> a) {
    __shared__ float shf[128];
    __shared__ double shd[64];
    __shared__ T sht[32];
    __shared__ double shr[32 * kRedQ];
    __shared__ T s_lh, s_ll;
    const int tid = threadIdx.x;
    if (tid == 0) {
        const double lam = a.sc->lambda;
        if (sizeof(T) == 4) {
            const float lh = (float)lam;
            s_lh = (T)lh;
            s_ll = (T)(float)(lam - (double)lh);
        } else {
            s_lh = (T)lam;
            s_ll = T(0);
        }
    }
    __syncthreads();
    const T lh = s_lh, ll = s_ll, lo = (T)a.lo, hi = (T)a.hi;
    const T* w = a.fused ? a.wbuf : a.w_in;
    T dmax = T(0);
    ProjSum<T> vol[2];
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long e0 = (long long)blockIdx.x * blockDim.x + tid; e0 < a.n; e0 += 4 * step) {
        T wv[4], rv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long e = e0 + q * step;
            wv[q] = e < a.n ? w[e] : T(0);
            rv[q] = (a.fused && e < a.n) ? a.rho_in[e] : T(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long e = e0 + q * step;
            if (e < a.n) {
                const T rt = tmin(tmax((wv[q] - lh) - ll, lo), hi);
                if (a.fused) dmax = tmax(dmax, tabs(rt - rv[q]));
                vol[0].add(rt);
                a.rho_out[e] = rt;
            }
        }
    }
    double sums[2];
    proj_block_sums(vol, sums, shf, shd);
    T mm[1] = {dmax};
    const int kmax[1] = {1};
    block_reduce<T, 1>(mm, kmax, sht);
    double v[2] = {(double)mm[0], sums[0]};
    const int kind[2] = {1, 0};
    double tot[2];
    if (finish_reduction<double, 2>(v, kind, a.red, a.counter + 1, tot, shr, blockIdx.x, gridDim.x) && tid == 0) {
        a.sc->drho_inf = tot[0];
        a.sc->volume = tot[1];
    }
}

template <typename T>
static int project_t(to_problem* P, const void* w, const void* rho_in, const void* g, void* rho_out, int fused,
                     cudaStream_t s) {
    ProjPipe<T> a{};
    a.n = P->n_elem;
    a.w_in = (const T*)w;
    a.rho_in = (const T*)rho_in;
    a.g = (const T*)g;
    a.wbuf = (T*)P->tmp_e;
    a.rho_out = (T*)rho_out;
    a.vbar = P->mat.volfrac * (double)P->n_elem;
    a.lo = P->mat.rho_min;
    a.hi = P->mat.rho_max;
    a.fused = fused;
    a.mean_proj = P->prm.mean_proj;
    a.part = P->red_d + (size_t)kMaxRedBlocks * kRedQ;
    a.red = P->red_d;
    a.counter = P->counters + 10;   // [10] first pass, [11] final pass
    a.sc = P->sc;
    // the streaming passes: 512 threads, four elements per thread and round, at most
    // one block per SM (few partials keep the folding block's tail short)
    long long nb = (P->n_elem + 2047) / 2048;
    if (nb > P->num_sms) nb = P->num_sms;
    if (nb < 1) nb = 1;
    k_proj_first<T><<<(unsigned)nb, 512, 0, s>>>(a);
    TO_CUDA(cudaGetLastError());
    const T* wsrc = fused ? (const T*)P->tmp_e : (const T*)w;
    const double vbar = a.vbar, lo = a.lo, hi = a.hi;
    long long n = a.n;
    DevScalars* sc = P->sc;
    if (P->prm.proj_sort) {
        int rc = projsort_lambda(P, wsrc, s);   // the paper's sort-and-scan form of Algorithm 4
        if (rc) return rc;
    } else if (P->cluster16) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(1024);
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        TO_CUDA(cudaLaunchKernelEx(&cfg, k_proj_search_cluster<T>, wsrc, n, vbar, lo, hi, sc));
    } else {
        double* part = a.part;
        unsigned* bar = P->counters + 8;
        void* args[] = {(void*)&wsrc, (void*)&n, (void*)&vbar, (void*)&lo, (void*)&hi, (void*)&sc, (void*)&part,
                        (void*)&bar};
        TO_CUDA(cudaLaunchCooperativeKernel((const void*)k_proj_search_grid<T>, dim3((unsigned)P->coop_blocks), dim3(256),
                                            args, 0, s));
    }
    k_proj_final<T><<<(unsigned)nb, 512, 0, s>>>(a);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

// Self-test of the bounded grid barrier: every block but `absent` waits at the
// barrier with the given spin limit; with a block absent nobody releases it, so
// the waiting blocks give up, record TO_ERR_TIMEOUT and return.
__global__ void __launch_bounds__(256) k_barrier_selftest(unsigned* bar, int* err, int absent,
                                                          unsigned long long spin_limit) {
    if ((int)blockIdx.x == absent) return;
    grid_barrier(bar, err, spin_limit);
}

int barrier_selftest(to_problem* P, int absent, long long spin_limit, cudaStream_t s) {
    const int nb = P->coop_blocks > 1 ? (P->coop_blocks < 8 ? P->coop_blocks : 8) : 1;
    if (absent >= nb) return fail(TO_ERR_ARG, "absent block index beyond the launch");
    unsigned* bar = P->counters + 8;
    int* err = &P->sc->err;
    unsigned long long lim = (unsigned long long)spin_limit;
    void* args[] = {(void*)&bar, (void*)&err, (void*)&absent, (void*)&lim};
    TO_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
    TO_CUDA(cudaLaunchCooperativeKernel((const void*)k_barrier_selftest, dim3((unsigned)nb), dim3(256), args, 0, s));
    DevScalars h;
    TO_CUDA(cudaMemcpyAsync(&h, P->sc, sizeof h, cudaMemcpyDeviceToHost, s));
    TO_CUDA(cudaStreamSynchronize(s));
    // the barrier words of an abandoned barrier are not reusable: clear them and the flag
    TO_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
    TO_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(P->sc) + offsetof(DevScalars, err), 0, sizeof(int), s));
    TO_CUDA(cudaStreamSynchronize(s));
    if (h.err) return fail(h.err, "grid barrier self-test: a block did not arrive and the waiting blocks gave up");
    return TO_OK;
}

// can one 16-CTA cluster of the search kernel be placed on this device?
int project_cluster_setup(to_problem* P) {
    cudaError_t e;
    const void* f = P->prec == TO_FP64 ? (const void*)k_proj_search_cluster<double> : (const void*)k_proj_search_cluster<float>;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    int ncl = 0;
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(1024);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaOccupancyMaxActiveClusters(&ncl, f, &cfg);
    }
    if (e != cudaSuccess) cudaGetLastError();
    P->cluster16 = (e == cudaSuccess && ncl >= 1) ? 1 : 0;
    return TO_OK;
}

int launch_project(to_problem* P, const void* w, const void* rho_in, const void* g, void* rho_out, int fused,
                   cudaStream_t s) {
    return P->prec == TO_FP64 ? project_t<double>(P, w, rho_in, g, rho_out, fused, s)
                              : project_t<float>(P, w, rho_in, g, rho_out, fused, s);
}

int project_coop_blocks(int prec, int num_sms, int* out) {
    // co-residency with the largest shared-memory request: one block per SM is
    // always possible; take two when the occupancy query allows it
    int per_sm = 0;
    cudaError_t e;
    if (prec == TO_FP64) {
        e = cudaFuncSetAttribute(k_project<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProjSmem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_project<double, true>, 256, kProjSmem);
    } else {
        e = cudaFuncSetAttribute(k_project<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProjSmem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_project<float, true>, 256, kProjSmem);
    }
    if (e != cudaSuccess) return fail(TO_ERR_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
    if (per_sm > 2) per_sm = 2;
    *out = per_sm * num_sms;
    if (*out > kMaxRedBlocks) *out = kMaxRedBlocks;
    return TO_OK;
}

}  // namespace to

// ----------------------------------------------------------------------------- allocation-free variant
// The same projection kernel, for callers that must not allocate device
// memory: its reduction slots, barrier words and result scalars live in one
// file-scope device array instead of a problem's buffers.  Every GPU that
// loads this library holds the array (about 200 KB) until the process exits.
namespace to {
namespace {

constexpr int kNoAllocMaxBlocks = 1024;           // co-resident blocks the scratch has slots for
constexpr long long kNoAllocMaxN = 1LL << 21;     // 2,097,152 design variables per call

struct NoAllocScratch {
    DevScalars sc;                                  // lambda, volume, error flag of the last call
    unsigned words[64];                             // [8], [9] grid barrier
    double part[2 * kNoAllocMaxBlocks * kProjSlot];
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

struct NoAllocDevice {
    bool ready = false;
    NoAllocScratch* ptr = nullptr;   // device address of g_noalloc_scratch on this device
    int coop[2] = {0, 0};            // co-resident blocks: [0] double, [1] float
};
std::mutex g_noalloc_mtx;
NoAllocDevice g_noalloc_dev[64];

// Once per device, with that device current: the symbol's device address, the
// shared-memory opt-in and the co-residency limit of the kernel.  None of these
// calls allocates device memory.
int noalloc_setup(int dev, NoAllocDevice** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mtx);
    if (dev < 0 || dev >= 64) return fail(TO_ERR_ARG, "device index out of range for the allocation-free path");
    NoAllocDevice& D = g_noalloc_dev[dev];
    if (!D.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fail(TO_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fail(TO_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
        int per_sm[2] = {0, 0};
        e = cudaFuncSetAttribute(k_project<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProjSmem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], k_project<double, true>, 256, kProjSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_project<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProjSmem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], k_project<float, true>, 256, kProjSmem);
        if (e != cudaSuccess) return fail(TO_ERR_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
        for (int i = 0; i < 2; ++i) {
            const int ps = per_sm[i] > 2 ? 2 : per_sm[i];
            D.coop[i] = ps * sms > kNoAllocMaxBlocks ? kNoAllocMaxBlocks : ps * sms;
        }
        D.ptr = reinterpret_cast<NoAllocScratch*>(p);
        D.ready = true;
    }
    *out = &D;
    return TO_OK;
}

template <typename T>
int project_noalloc_t(NoAllocDevice& D, const void* w, void* rho, long long n, double vbar, double lo, double hi,
                      double* lambda_out, cudaStream_t s) {
    NoAllocScratch* S = D.ptr;
    // the last call's contents stay in the array: reset what must start at zero,
    // except the error word, which is sticky until a synchronising call reports it
    const size_t e0 = offsetof(NoAllocScratch, sc) + offsetof(DevScalars, err);
    const size_t e1 = e0 + sizeof(int);
    TO_CUDA(cudaMemsetAsync(S, 0, e0, s));
    TO_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(S) + e1, 0, offsetof(NoAllocScratch, part) - e1, s));
    ProjArgs<T> a{};
    a.n = n;
    a.w_in = (const T*)w;
    a.wbuf = nullptr;          // only the shared-memory variant runs here
    a.rho_out = (T*)rho;
    a.vbar = vbar;
    a.lo = lo;
    a.hi = hi;
    a.fused = 0;
    a.mean_proj = 0;
    a.part = S->part;
    a.bar = S->words + 8;
    a.sc = &S->sc;
    long long nb = (n + 255) / 256;
    const int coop = D.coop[sizeof(T) == 4 ? 1 : 0];
    if (nb > coop) nb = coop;
    if (nb < 1) nb = 1;
    a.chunk = (n + nb - 1) / nb;
    nb = (n + a.chunk - 1) / a.chunk;
    const size_t smem = (size_t)a.chunk * sizeof(T);
    void* args[] = {(void*)&a};
    if (smem <= kProjSmem) {   // each block keeps its chunk of w in shared memory
        TO_CUDA(cudaLaunchCooperativeKernel((const void*)k_project<T, true>, dim3((unsigned)nb), dim3(256), args, smem,
                                            s));
    } else {                   // the search passes re-read w from the input (nothing is stored)
        a.wbuf = const_cast<T*>(a.w_in);
        a.wdirect = 1;
        TO_CUDA(cudaLaunchCooperativeKernel((const void*)k_project<T, false>, dim3((unsigned)nb), dim3(256), args, 0,
                                            s));
    }
    if (lambda_out) {
        DevScalars h;
        TO_CUDA(cudaMemcpyAsync(&h, &S->sc, sizeof h, cudaMemcpyDeviceToHost, s));
        TO_CUDA(cudaStreamSynchronize(s));
        *lambda_out = h.lambda;
        if (h.err) {
            // report once: clear the sticky word so that the next call starts clean
            TO_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(S) + e0, 0, sizeof(int), s));
            TO_CUDA(cudaStreamSynchronize(s));
            return fail(h.err, "device-side error in the allocation-free projection (this call or an earlier "
                               "call made without lambda_out)");
        }
    }
    return TO_OK;
}

}  // namespace
}  // namespace to

extern "C" int to_project_noalloc(const void* w_dev, void* rho_dev, int64_t n, int32_t precision, double vbar,
                                  double lo, double hi, double* lambda_out, void* stream) {
    using namespace to;
    if (!w_dev || !rho_dev) return fail(TO_ERR_ARG, "null vector");
    if (n < 1 || n > kNoAllocMaxN)
        return fail(TO_ERR_ARG, "n must lie in [1, 2097152] for the allocation-free projection");
    if (precision != TO_FP64 && precision != TO_FP32_MIXED) return fail(TO_ERR_ARG, "bad precision");
    if (!(lo >= 0.0 && hi > lo) || !std::isfinite(vbar)) return fail(TO_ERR_ARG, "need 0 <= lo < hi and a finite vbar");
    if (vbar < (double)n * lo) return fail(TO_ERR_INFEASIBLE, "vbar < n * lo: X is empty");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(TO_ERR_CUDA, "no current CUDA device");
    NoAllocDevice* D = nullptr;
    int rc = noalloc_setup(dev, &D);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    return precision == TO_FP64 ? project_noalloc_t<double>(*D, w_dev, rho_dev, n, vbar, lo, hi, lambda_out, s)
                                : project_noalloc_t<float>(*D, w_dev, rho_dev, n, vbar, lo, hi, lambda_out, s);
}
