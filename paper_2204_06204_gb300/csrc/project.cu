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
// of passes.  lambda and every sum are double; the element values are the
// problem's precision.
#include <cmath>
#include <cstddef>
#include <mutex>

#include "device.cuh"

namespace to {

constexpr int kProjSlot = 12;     // doubles per block per pass in the projection scratch
constexpr int kProjMaxIter = 100;

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
    long long chunk;     // elements per block (contiguous)
    double* part;        // 2 * nblocks * kProjSlot doubles
    double* red;         // final reduction scratch (kRedQ per block)
    unsigned* bar;       // barrier words
    unsigned* counter;   // final reduction counter
    DevScalars* sc;
};

// element classification for the current lambda: at upper bound, at lower bound or free.
// For float w the thresholds are rounded outward once (w >= t exactly iff w >= RU(t)
// for a float w), so the per-element test needs no double arithmetic.
__device__ __forceinline__ float round_up_f(double t) {
    float f = (float)t;
    if ((double)f < t) f = nextafterf(f, INFINITY);
    return f;
}
__device__ __forceinline__ float round_down_f(double t) {
    float f = (float)t;
    if ((double)f > t) f = nextafterf(f, -INFINITY);
    return f;
}
template <typename T> struct Thresh;
template <> struct Thresh<float> {
    float tu, tl;
    __device__ Thresh(double lam, double lo, double hi) : tu(round_up_f(lam + hi)), tl(round_down_f(lam + lo)) {}
    __device__ int cls(float w) const { return w >= tu ? 0 : (w <= tl ? 1 : 2); }
};
template <> struct Thresh<double> {
    double tu, tl;
    __device__ Thresh(double lam, double lo, double hi) : tu(lam + hi), tl(lam + lo) {}
    __device__ int cls(double w) const { return w >= tu ? 0 : (w <= tl ? 1 : 2); }
};

// Totals of the per-block partials of one pass: warp 0 folds a lane-strided
// subset in block order and reduces in a fixed tree, then broadcasts through
// shared memory (identical, deterministic totals in every block).
template <int NQ>
__device__ __forceinline__ void combine_partials(const double* part, unsigned nb, const int (&kind)[NQ], double (&tot)[NQ],
                                                 double* shb) {
    if (threadIdx.x < 32) {
        double acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = kind[q] ? -INFINITY : 0.0;
        for (unsigned b = threadIdx.x; b < nb; b += 32)
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const double t = __ldcg(part + b * kProjSlot + q);
                acc[q] = kind[q] ? fmax(acc[q], t) : acc[q] + t;
            }
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = kind[q] ? warp_max(acc[q]) : warp_sum(acc[q]);
        if (threadIdx.x == 0)
#pragma unroll
            for (int q = 0; q < NQ; ++q) shb[q] = acc[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NQ; ++q) tot[q] = shb[q];
    __syncthreads();
}

template <typename T, bool CACHE>
__global__ void __launch_bounds__(256) k_project(const ProjArgs<T> a) {
    extern __shared__ unsigned char smem_raw[];
    T* wloc = reinterpret_cast<T*>(smem_raw);
    __shared__ double sh[32 * kRedQ];
    __shared__ double sh10[32 * 10];
    __shared__ double shb[10];
    const unsigned nb = gridDim.x, bid = blockIdx.x;
    const long long b0 = (long long)bid * a.chunk;
    const long long b1 = min(b0 + a.chunk, a.n);
    const int tid = threadIdx.x;
    DevScalars* sc = a.sc;

    const double alpha = a.fused ? sc->alpha : 0.0;
    const double gmean = (a.fused && a.mean_proj) ? sc->gsum / (double)a.n : 0.0;
    const T alpha_t = (T)alpha, gmean_t = (T)gmean;
    auto wat = [&](long long e) -> T { return CACHE ? wloc[e - b0] : a.wbuf[e]; };

    // pass 0: w; the piece at lambda = 0 (box-clamp volume), the piece at the warm
    // start lambda_s (the previous multiplier), min / max of w
    const double lam_s = sc->lambda;
    double tot[10];
    int parity = 0;
    {
        double v[10] = {0.0, 0.0, 0.0, 0.0, INFINITY, -INFINITY, 0.0, 0.0, 0.0, 0.0};
        T sF = T(0), sFs = T(0), wmn = T(INFINITY), wmx = T(-INFINITY);
        const Thresh<T> th0(0.0, a.lo, a.hi), ths(lam_s > 0.0 ? lam_s : 0.0, a.lo, a.hi);
        for (long long e = b0 + tid; e < b1; e += blockDim.x) {
            const T w = a.fused ? a.rho_in[e] - alpha_t * (a.g[e] - gmean_t) : a.w_in[e];
            if (CACHE) wloc[e - b0] = w;
            else a.wbuf[e] = w;
            int c = th0.cls(w);
            if (c == 0) v[0] += 1.0;
            else if (c == 1) v[1] += 1.0;
            else { v[2] += 1.0; sF += w; }
            c = ths.cls(w);
            if (c == 0) v[6] += 1.0;
            else if (c == 1) v[7] += 1.0;
            else { v[8] += 1.0; sFs += w; }
            wmn = fmin(wmn, w);
            wmx = fmax(wmx, w);
        }
        double mv[10] = {v[0], v[1], v[2], (double)sF, -(double)wmn, (double)wmx, v[6], v[7], v[8], (double)sFs};
        const int kind[10] = {0, 0, 0, 0, 1, 1, 0, 0, 0, 0};
        block_reduce<10>(mv, kind, sh10);
        if (tid == 0)
            for (int q = 0; q < 10; ++q) a.part[(parity * nb + bid) * kProjSlot + q] = mv[q];
        if (!grid_barrier(a.bar, &sc->err)) return;
        combine_partials<10>(a.part + parity * nb * kProjSlot, nb, kind, tot, shb);
        parity ^= 1;
    }
    const double wmin = -tot[4], wmax = tot[5];
    const double S0 = tot[0] * a.hi + tot[1] * a.lo + tot[3];
    double lambda = 0.0;
    int iters = 0;
    if (!isfinite(S0)) set_err(&sc->err, TO_ERR_NONFINITE);
    ProjSearch st;
    st.done = !(S0 > a.vbar) || !isfinite(S0);
    st.have_prev = false;
    st.pU = st.pL = st.pF = 0.0;
    if (!st.done) {
        st.lo_b = fmax(0.0, wmin - a.hi);
        st.hi_b = wmax - a.lo;
        const double t0[4] = {tot[0], tot[1], tot[2], tot[3]};
        st.lam = 0.0;
        proj_search_step(st, t0, a.vbar, a.lo, a.hi);          // Newton from lambda = 0
        if (!st.done && lam_s > st.lo_b && lam_s < st.hi_b) {           // the warm start tightens it
            const double ts[4] = {tot[6], tot[7], tot[8], tot[9]};
            st.lam = lam_s;
            st.have_prev = false;
            proj_search_step(st, ts, a.vbar, a.lo, a.hi);
        }
    }
    while (!st.done && iters < kProjMaxIter) {
        ++iters;
        const Thresh<T> th(st.lam, a.lo, a.hi);
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        T sF = T(0);
        for (long long e = b0 + tid; e < b1; e += blockDim.x) {
            const T w = wat(e);
            const int c = th.cls(w);
            if (c == 0) v[0] += 1.0;
            else if (c == 1) v[1] += 1.0;
            else { v[2] += 1.0; sF += w; }
        }
        v[3] = (double)sF;
        const int kind[4] = {0, 0, 0, 0};
        block_reduce<4>(v, kind, sh);
        if (tid == 0)
            for (int q = 0; q < 4; ++q) a.part[(parity * nb + bid) * kProjSlot + q] = v[q];
        if (!grid_barrier(a.bar, &sc->err)) return;
        double t4[4];
        combine_partials<4>(a.part + parity * nb * kProjSlot, nb, kind, t4, shb);
        parity ^= 1;
        proj_search_step(st, t4, a.vbar, a.lo, a.hi);
    }
    lambda = st.done && !(S0 > a.vbar) ? 0.0 : st.lam;

    // final pass: rho = clamp(w - lambda), ||drho||_inf, volume
    double dmax = 0.0, vol = 0.0;
    for (long long e = b0 + tid; e < b1; e += blockDim.x) {
        const double wd = (double)wat(e);
        const T rt = (T)fmin(fmax(wd - lambda, a.lo), a.hi);
        if (a.fused) dmax = fmax(dmax, fabs((double)rt - (double)a.rho_in[e]));
        vol += (double)rt;
        a.rho_out[e] = rt;
    }
    double v2[2] = {dmax, vol};
    const int kind2[2] = {1, 0};
    double tot2[2];
    block_reduce<2>(v2, kind2, sh);
    if (finish_reduction<2>(v2, kind2, a.red, a.counter, tot2, sh, linear_block(), grid_blocks()) && tid == 0) {
        sc->lambda = lambda;
        sc->drho_inf = tot2[0];
        sc->volume = tot2[1];
        sc->proj_iters = iters;
    }
}

constexpr size_t kProjSmem = 96 * 1024;

template <typename T>
static int project_t(to_problem* P, const void* w, const void* rho_in, const void* g, void* rho_out, int fused,
                     cudaStream_t s) {
    ProjArgs<T> a{};
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
    a.part = P->red + (size_t)kMaxRedBlocks * kRedQ;
    a.red = P->red;
    a.bar = P->counters + 8;
    a.counter = P->counters + 3;
    a.sc = P->sc;
    long long nb = (P->n_elem + 255) / 256;
    if (nb > P->coop_blocks) nb = P->coop_blocks;
    if (nb < 1) nb = 1;
    a.chunk = (P->n_elem + nb - 1) / nb;
    nb = (P->n_elem + a.chunk - 1) / a.chunk;
    if (nb < 1) nb = 1;
    void* args[] = {(void*)&a};
    const size_t smem = (size_t)a.chunk * sizeof(T);
    if (smem <= kProjSmem) {
        TO_CUDA(cudaLaunchCooperativeKernel((const void*)k_project<T, true>, dim3((unsigned)nb), dim3(256), args, smem, s));
    } else {
        TO_CUDA(cudaLaunchCooperativeKernel((const void*)k_project<T, false>, dim3((unsigned)nb), dim3(256), args, 0, s));
    }
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
// loads this library holds the array (about 230 KB) until the process exits.
namespace to {
namespace {

constexpr int kNoAllocMaxBlocks = 1024;           // co-resident blocks the scratch has slots for
constexpr long long kNoAllocMaxN = 1LL << 21;     // 2,097,152 design variables per call

struct NoAllocScratch {
    DevScalars sc;                                  // lambda, volume, error flag of the last call
    unsigned words[64];                             // [3] reduction counter, [8], [9] grid barrier
    double red[kNoAllocMaxBlocks * kRedQ];
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
    // the last call's contents stay in the array: reset what must start at zero
    TO_CUDA(cudaMemsetAsync(S, 0, offsetof(NoAllocScratch, red), s));
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
    a.red = S->red;
    a.bar = S->words + 8;
    a.counter = S->words + 3;
    a.sc = &S->sc;
    long long nb = (n + 255) / 256;
    const int coop = D.coop[sizeof(T) == 4 ? 1 : 0];
    if (nb > coop) nb = coop;
    if (nb < 1) nb = 1;
    a.chunk = (n + nb - 1) / nb;
    nb = (n + a.chunk - 1) / a.chunk;
    const size_t smem = (size_t)a.chunk * sizeof(T);
    if (smem > kProjSmem)
        return fail(TO_ERR_ARG, "n too large for the allocation-free projection on this device");
    void* args[] = {(void*)&a};
    TO_CUDA(cudaLaunchCooperativeKernel((const void*)k_project<T, true>, dim3((unsigned)nb), dim3(256), args, smem, s));
    if (lambda_out) {
        DevScalars h;
        TO_CUDA(cudaMemcpyAsync(&h, &S->sc, sizeof h, cudaMemcpyDeviceToHost, s));
        TO_CUDA(cudaStreamSynchronize(s));
        *lambda_out = h.lambda;
        if (h.err) return fail(h.err, "device-side error in the allocation-free projection");
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
