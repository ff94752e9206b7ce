// The multiplier of the projection onto X by the paper's parallel form of
// Algorithm 4 (Sec. IV-D): sort the 2E breakpoints of the piecewise-linear
// volume S(lambda) = sum_e clamp(w_e - lambda, lo, hi), scan, and solve on the
// segment where S crosses vbar.
//
//   breakpoints  w_e - hi (the element leaves hi: the slope loses 1) and
//                w_e - lo (the element reaches lo: the slope gains 1 back);
//   sort         a stable least-significant-digit radix sort of the breakpoints
//                (4-bit digits; keys are the breakpoints' bit patterns made
//                order-preserving, values their kinds); ranks inside a warp
//                come from __match_any_sync, so each pass is one count, one
//                scan and one scatter;
//   scan         slope_a = sum_{j <= a} kind_j (an integer scan), then
//                S(t_{a+1}) = S(t_a) + slope_a (t_{a+1} - t_a) from S = E hi
//                below every breakpoint (a double scan);
//   crossing     the first segment with S(t_a) >= vbar >= S(t_{a+1}) gives
//                lambda = t_a + (S(t_a) - vbar)(t_{a+1} - t_a) / (S(t_a) - S(t_{a+1}))
//                (t_a on a flat segment: the smallest multiplier, as the oracle).
//
// The first pass of the problem's projection (w, whether the bound is active)
// runs before, and its final pass (the clamp) after; this replaces the
// multiplier search between them.  It is slower than that search (2E keys are
// sorted every iteration) and exists as the paper's exact parallel method.
#include <cmath>

#include "device.cuh"

namespace to {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsBits = 4;
constexpr int kRsBins = 1 << kRsBits;

template <typename T> struct SortKey;
template <> struct SortKey<float> {
    using K = unsigned;
    static constexpr int bits = 32;
    __device__ static K enc(float x) {
        const unsigned u = __float_as_uint(x);
        return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    }
    __device__ static float dec(K k) { return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k); }
};
template <> struct SortKey<double> {
    using K = unsigned long long;
    static constexpr int bits = 64;
    __device__ static K enc(double x) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(x);
        return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
    }
    __device__ static double dec(K k) {
        return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
    }
};

// breakpoints of element e: 2e = w_e - hi (kind -1), 2e + 1 = w_e - lo (kind +1)
template <typename T>
__global__ void k_bp_make(const T* __restrict__ w, long long n, double lo, double hi,
                          typename SortKey<T>::K* __restrict__ keys, int* __restrict__ kinds) {
    const T tlo = (T)lo, thi = (T)hi;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const T x = w[e];
        keys[2 * e] = SortKey<T>::enc(x - thi);
        kinds[2 * e] = -1;
        keys[2 * e + 1] = SortKey<T>::enc(x - tlo);
        kinds[2 * e + 1] = 1;
    }
}

// digit counts per tile, digit-major: counts[d * nblocks + block]
template <typename K>
__global__ void __launch_bounds__(kRsThreads) k_rs_count(const K* __restrict__ keys, long long n, int shift,
                                                         unsigned* __restrict__ counts) {
    __shared__ unsigned c[kRsBins];
    if (threadIdx.x < kRsBins) c[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsItems; ++r) {
        const long long i = base + r * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&c[(unsigned)(keys[i] >> shift) & (kRsBins - 1)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kRsBins) counts[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = c[threadIdx.x];
}

// exclusive scan of m counts by one block (in place)
__global__ void __launch_bounds__(1024) k_rs_scan(unsigned* __restrict__ v, long long m) {
    __shared__ unsigned s[1024];
    __shared__ unsigned carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long b0 = 0; b0 < m; b0 += 1024) {
        const long long i = b0 + threadIdx.x;
        const unsigned x = i < m ? v[i] : 0u;
        s[threadIdx.x] = x;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {   // inclusive Hillis-Steele scan
            const unsigned t = threadIdx.x >= o ? s[threadIdx.x - o] : 0u;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < m) v[i] = carry + s[threadIdx.x] - x;
        __syncthreads();
        if (threadIdx.x == 0) carry += s[1023];
        __syncthreads();
    }
}

// stable scatter: positions in (round, warp, lane) order within the tile
template <typename K>
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const K* __restrict__ kin, const int* __restrict__ vin,
                                                           K* __restrict__ kout, int* __restrict__ vout, long long n,
                                                           int shift, const unsigned* __restrict__ offsets) {
    constexpr int NW = kRsThreads / 32;
    __shared__ unsigned run[kRsBins];
    __shared__ unsigned wcnt[NW][kRsBins];
    __shared__ unsigned wpre[NW][kRsBins];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x < kRsBins) run[threadIdx.x] = offsets[(size_t)threadIdx.x * gridDim.x + blockIdx.x];
    const long long base = (long long)blockIdx.x * kRsTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kRsItems; ++r) {
        const long long i = base + r * kRsThreads + threadIdx.x;
        const bool ok = i < n;
        K k = 0;
        int v = 0;
        unsigned d = kRsBins;   // out-of-range lanes get a digit of their own
        if (ok) {
            k = kin[i];
            v = vin[i];
            d = (unsigned)(k >> shift) & (kRsBins - 1);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned rank = __popc(peers & lt);
        if (threadIdx.x < NW * kRsBins) (&wcnt[0][0])[threadIdx.x] = 0;
        __syncthreads();
        if (ok && rank == 0) wcnt[wid][d] = __popc(peers);
        __syncthreads();
        if (threadIdx.x < kRsBins) {   // per digit: the warps' exclusive prefix, then the round total
            unsigned acc = 0;
            for (int q = 0; q < NW; ++q) {
                wpre[q][threadIdx.x] = acc;
                acc += wcnt[q][threadIdx.x];
            }
            wcnt[0][threadIdx.x] = acc;   // reuse: the round's total for digit threadIdx.x (read after the barrier)
        }
        __syncthreads();
        if (ok) {
            const unsigned pos = run[d] + wpre[wid][d] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        if (threadIdx.x < kRsBins) run[threadIdx.x] += wcnt[0][threadIdx.x];
        __syncthreads();
    }
}

// block-level inclusive scans with block totals: the kinds (int), then the segment
// volumes (double); a second launch adds the scanned block totals
template <typename V>
__global__ void __launch_bounds__(1024) k_scan_block(const V* __restrict__ in, V* __restrict__ out, long long n,
                                                     V* __restrict__ totals) {
    __shared__ V s[1024];
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    s[threadIdx.x] = i < n ? in[i] : V(0);
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const V t = threadIdx.x >= o ? s[threadIdx.x - o] : V(0);
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x];
    if (threadIdx.x == 1023) totals[blockIdx.x] = s[1023];
}

template <typename V>
__global__ void __launch_bounds__(1024) k_scan_totals(V* __restrict__ totals, long long m) {   // exclusive, one block
    __shared__ V s[1024];
    __shared__ V carry;
    if (threadIdx.x == 0) carry = V(0);
    __syncthreads();
    for (long long b0 = 0; b0 < m; b0 += 1024) {
        const long long i = b0 + threadIdx.x;
        const V x = i < m ? totals[i] : V(0);
        s[threadIdx.x] = x;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const V t = threadIdx.x >= o ? s[threadIdx.x - o] : V(0);
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < m) totals[i] = carry + s[threadIdx.x] - x;
        __syncthreads();
        if (threadIdx.x == 0) carry += s[1023];
        __syncthreads();
    }
}

template <typename V>
__global__ void k_scan_add(V* __restrict__ out, long long n, const V* __restrict__ totals) {
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    if (i < n) out[i] += totals[blockIdx.x];
}

// segment a = [t_a, t_{a+1}]: its volume change slope_a (t_{a+1} - t_a) (the last breakpoint
// has none)
template <typename T>
__global__ void k_seg_volume(const typename SortKey<T>::K* __restrict__ keys, const int* __restrict__ slope, long long m,
                             double* __restrict__ dv) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < m; a += (long long)gridDim.x * blockDim.x) {
        double d = 0.0;
        if (a + 1 < m) {
            const double ta = (double)SortKey<T>::dec(keys[a]), tb = (double)SortKey<T>::dec(keys[a + 1]);
            d = (double)slope[a] * (tb - ta);
        }
        dv[a] = d;
    }
}

// S(t_a) = E hi + sum_{j < a} dv_j (inclusive scan shifted by one); the first crossing
// segment (smallest index) wins
template <typename T>
__global__ void k_crossing(const typename SortKey<T>::K* __restrict__ keys, const double* __restrict__ cum, long long m,
                           double S_top, double vbar, unsigned long long* __restrict__ best) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a + 1 < m; a += (long long)gridDim.x * blockDim.x) {
        const double ra = S_top + (a > 0 ? cum[a - 1] : 0.0), rb = S_top + cum[a];
        if (ra >= vbar && vbar >= rb) atomicMin(best, (unsigned long long)a);
    }
}

template <typename T>
__global__ void k_pick_lambda(const typename SortKey<T>::K* __restrict__ keys, const double* __restrict__ cum, long long m,
                              double S_top, double vbar, const unsigned long long* __restrict__ best, DevScalars* sc) {
    if (!sc->proj_active) return;   // the box clamp is feasible: lambda = 0 from the first pass
    double lam;
    const unsigned long long a = *best;
    if (a < (unsigned long long)(m - 1)) {
        const double ta = (double)SortKey<T>::dec(keys[a]), tb = (double)SortKey<T>::dec(keys[a + 1]);
        const double ra = S_top + (a > 0 ? cum[a - 1] : 0.0), rb = S_top + cum[a];
        lam = ra == rb ? ta : ta + (ra - vbar) * (tb - ta) / (ra - rb);
    } else {
        lam = (double)SortKey<T>::dec(keys[m - 1]);   // vbar at E lo: every element at its lower bound
    }
    sc->lambda = lam > 0.0 ? lam : 0.0;
    sc->proj_iters = 0;
}

template <typename T>
static int projsort_t(to_problem* P, const void* w, cudaStream_t s) {
    using K = typename SortKey<T>::K;
    const long long n = P->n_elem, m = 2 * n;
    char* base = (char*)P->ps_buf;
    K* k0 = (K*)base;
    K* k1 = k0 + m;
    int* v0 = (int*)(k1 + m);
    int* v1 = v0 + m;
    double* cum = (double*)(v1 + m);
    unsigned* counts = (unsigned*)(cum + m);
    const long long nbt = (m + kRsTile - 1) / kRsTile;
    unsigned long long* best = (unsigned long long*)(counts + kRsBins * nbt);
    double* dtot = (double*)(best + 1);
    int* itot = (int*)(dtot + (m + 1023) / 1024 + 1);
    const int g1 = (int)std::min<long long>((n + 255) / 256, 8LL * P->num_sms);
    const double lo = P->mat.rho_min, hi = P->mat.rho_max, vbar = P->mat.volfrac * (double)n;
    k_bp_make<T><<<g1, 256, 0, s>>>((const T*)w, n, lo, hi, k0, v0);
    for (int shift = 0; shift < SortKey<T>::bits; shift += kRsBits) {
        k_rs_count<K><<<(unsigned)nbt, kRsThreads, 0, s>>>(k0, m, shift, counts);
        k_rs_scan<<<1, 1024, 0, s>>>(counts, kRsBins * nbt);
        k_rs_scatter<K><<<(unsigned)nbt, kRsThreads, 0, s>>>(k0, v0, k1, v1, m, shift, counts);
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    // slope_a = inclusive scan of the kinds (in v1), then the segment volumes and their scan
    const long long nb = (m + 1023) / 1024;
    k_scan_block<int><<<(unsigned)nb, 1024, 0, s>>>(v0, v1, m, itot);
    k_scan_totals<int><<<1, 1024, 0, s>>>(itot, nb);
    k_scan_add<int><<<(unsigned)nb, 1024, 0, s>>>(v1, m, itot);
    const int g2 = (int)std::min<long long>((m + 255) / 256, 8LL * P->num_sms);
    k_seg_volume<T><<<g2, 256, 0, s>>>(k0, v1, m, cum);
    k_scan_block<double><<<(unsigned)nb, 1024, 0, s>>>(cum, cum, m, dtot);
    k_scan_totals<double><<<1, 1024, 0, s>>>(dtot, nb);
    k_scan_add<double><<<(unsigned)nb, 1024, 0, s>>>(cum, m, dtot);
    TO_CUDA(cudaMemsetAsync(best, 0xff, sizeof(unsigned long long), s));
    const double S_top = (double)n * hi;
    k_crossing<T><<<g2, 256, 0, s>>>(k0, cum, m, S_top, vbar, best);
    k_pick_lambda<T><<<1, 1, 0, s>>>(k0, cum, m, S_top, vbar, best, P->sc);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

int projsort_lambda(to_problem* P, const void* w, cudaStream_t s) {
    return P->prec == TO_FP64 ? projsort_t<double>(P, w, s) : projsort_t<float>(P, w, s);
}

size_t projsort_bytes(const to_problem* P) {
    const long long m = 2 * P->n_elem;
    const size_t ks = P->prec == TO_FP64 ? 8 : 4;
    const long long nbt = (m + kRsTile - 1) / kRsTile, nb = (m + 1023) / 1024;
    return 2 * m * ks + 2 * m * sizeof(int) + m * sizeof(double) + kRsBins * nbt * sizeof(unsigned) + 8 +
           (nb + 1) * sizeof(double) + (nb + 1) * sizeof(int) + 64;
}

}  // namespace to
