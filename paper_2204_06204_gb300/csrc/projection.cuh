// The projection onto X = {lo <= rho <= hi, 1^T rho <= vbar} (Sec. IV-B) as a
// device body shared by the grid-wide kernel (cooperative launch, software grid
// barrier, partials in global memory) and the cluster kernel (one thread-block
// cluster per problem, hardware cluster barrier, partials in distributed shared
// memory).
//
// The KKT conditions give rho = clamp(w - lambda, lo, hi), lambda = 0 when the
// clamp already meets the volume bound, else the root of the piecewise-linear
// volume S(lambda) = sum_e clamp(w_e - lambda, lo, hi) (Eq. piecewiseLinearEQ).
// Each pass classifies every element at the current lambda (count at hi, count
// at lo, count and sum of the free ones); one thread then runs the search step
// (device.cuh: ProjSearch) on the totals and broadcasts the next lambda.
//
// Arithmetic: per element only the element precision (classification against
// thresholds rounded outward once per pass; the clamp with lambda as a float
// pair on the mixed path).  Counts are exact integers; the free-set and volume
// sums are float pairs (FF) on the mixed path, doubles on the FP64 path; the
// per-block partials meet in double, folded by one warp in a fixed order, so that
// every block sees bitwise the same totals and takes the same decisions.
#pragma once

#include <cooperative_groups.h>

#include "device.cuh"

namespace to {

constexpr int kProjSlot = 12;     // 8-byte words per block per pass in the projection scratch
constexpr int kProjMaxIter = 100;

// one block's contribution to a pass (fits kProjSlot words)
struct ProjPart {
    unsigned long long n[6];   // (at hi, at lo, free) at the pass lambda, then at the warm start (pass 0)
    double s[2];               // sums of w over the two free sets; final pass: volume
    double wmin, wmax;         // pass 0: min / max of w; final pass: wmax = max |rho_new - rho_old|
};
static_assert(sizeof(ProjPart) <= kProjSlot * sizeof(double), "projection slot");

// totals over `n` slots: lane l folds slots l, l + 32, ... in order, then a fixed
// shuffle tree; valid in lane 0 of the calling warp
template <typename Load>
__device__ __forceinline__ ProjPart proj_fold(unsigned n, Load load) {
    const unsigned lane = threadIdx.x & 31;
    ProjPart a;
#pragma unroll
    for (int q = 0; q < 6; ++q) a.n[q] = 0ull;
    a.s[0] = a.s[1] = 0.0;
    a.wmin = INFINITY;
    a.wmax = -INFINITY;
    for (unsigned b0 = lane; b0 < n; b0 += 4 * 32) {
        ProjPart p[4];   // four slots per round: their loads are in flight together
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (b0 + 32 * u < n) p[u] = load(b0 + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (b0 + 32 * u < n) {
#pragma unroll
                for (int q = 0; q < 6; ++q) a.n[q] += p[u].n[q];
                a.s[0] += p[u].s[0];
                a.s[1] += p[u].s[1];
                a.wmin = fmin(a.wmin, p[u].wmin);
                a.wmax = fmax(a.wmax, p[u].wmax);
            }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int q = 0; q < 6; ++q) a.n[q] += __shfl_xor_sync(0xffffffffu, a.n[q], o);
        a.s[0] += __shfl_xor_sync(0xffffffffu, a.s[0], o);
        a.s[1] += __shfl_xor_sync(0xffffffffu, a.s[1], o);
        a.wmin = fmin(a.wmin, __shfl_xor_sync(0xffffffffu, a.wmin, o));
        a.wmax = fmax(a.wmax, __shfl_xor_sync(0xffffffffu, a.wmax, o));
    }
    return a;
}

// thresholds of one pass in the element precision: w >= tu is "at hi", w <= tl
// "at lo".  For float w, rounding lambda + hi up and lambda + lo down once makes
// the float comparison agree with the exact one.
__device__ __forceinline__ float proj_round_up(double t) {
    float f = (float)t;
    if ((double)f < t) f = nextafterf(f, INFINITY);
    return f;
}
__device__ __forceinline__ float proj_round_down(double t) {
    float f = (float)t;
    if ((double)f > t) f = nextafterf(f, -INFINITY);
    return f;
}
template <typename T>
__device__ __forceinline__ void proj_thresholds(double lam, double lo, double hi, T& tu, T& tl) {
    if (sizeof(T) == 4) {
        tu = (T)proj_round_up(lam + hi);
        tl = (T)proj_round_down(lam + lo);
    } else {
        tu = (T)(lam + hi);
        tl = (T)(lam + lo);
    }
}

// per-thread sums: a float pair on the mixed path, a double on the FP64 path
template <typename T> struct ProjSum;
template <> struct ProjSum<float> {
    FF v{0.f, 0.f};
    __device__ __forceinline__ void add(float x) { v = ff_add(v, x); }
};
template <> struct ProjSum<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double x) { v += x; }
};
// block totals of two sums, valid in thread 0; `shf` holds 128 floats, `shd` 64 doubles
__device__ __forceinline__ void proj_block_sums(ProjSum<float> (&a)[2], double (&out)[2], float* shf, double*) {
    FF v[2] = {a[0].v, a[1].v};
    block_reduce_ff<2>(v, out, shf);
}
__device__ __forceinline__ void proj_block_sums(ProjSum<double> (&a)[2], double (&out)[2], float*, double* shd) {
    double v[2] = {a[0].v, a[1].v};
    const int kind[2] = {0, 0};
    block_reduce<double, 2>(v, kind, shd);
    out[0] = v[0];
    out[1] = v[1];
}

// what thread 0 broadcasts after each search step
template <typename T>
struct ProjCast {
    double lam;
    T tu, tl;       // thresholds at lam
    T lh, ll;       // lam as an element-precision pair (final clamp)
    int done, iters;
};

struct ProjIO {
    long long n, b0, b1;      // all elements; this block's range [b0, b1)
    double vbar, lo, hi;
    int fused, mean_proj, writer;   // writer: the block that stores the scalars
    int wdirect;                    // uncached plain mode: wbuf is the input w itself (read, never stored)
};

// Comm: exchange(const ProjPart& mine (thread 0), int parity, ProjPart& tot (thread 0)) -> false on a timeout;
// it is called by every thread of the block and synchronises the block.
template <typename T, bool CACHE, class Comm>
__device__ __forceinline__ void projection_body(Comm& comm, const ProjIO& io, const T* w_in, const T* rho_in, const T* g,
                                                T* wloc, T* wbuf, T* rho_out, DevScalars* sc) {
    __shared__ ProjCast<T> cast;
    __shared__ float shf[128];
    __shared__ double shd[64];
    __shared__ unsigned shu[32 * 6];
    __shared__ T sht[32 * 2];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const long long b0 = io.b0, b1 = io.b1;
    auto wat = [&](long long e) -> T { return CACHE ? wloc[e - b0] : wbuf[e]; };

    // thread 0: step size, mean shift, warm start and the thresholds of pass 0.  The
    // search state and the totals live in shared memory (used by thread 0 only),
    // so that they hold no registers in the element loops.
    __shared__ ProjSearch st;
    __shared__ ProjPart tot;
    __shared__ double S0, lam_s;
    __shared__ T s_alpha, s_gmean, s_tu0, s_tl0, s_tus, s_tls;
    if (tid == 0) {
        const double alpha = io.fused ? sc->alpha : 0.0;
        const double gmean = (io.fused && io.mean_proj) ? sc->gsum / (double)io.n : 0.0;
        s_alpha = (T)alpha;
        s_gmean = (T)gmean;
        lam_s = sc->lambda > 0.0 ? sc->lambda : 0.0;
        proj_thresholds<T>(0.0, io.lo, io.hi, s_tu0, s_tl0);
        proj_thresholds<T>(lam_s, io.lo, io.hi, s_tus, s_tls);
    }
    __syncthreads();

    // pass 0: w; the sets at lambda = 0 (box-clamp volume) and at the warm start, min / max of w
    int parity = 0;
    {
        const T alpha_t = s_alpha, gmean_t = s_gmean, tu0 = s_tu0, tl0 = s_tl0, tus = s_tus, tls = s_tls;
        unsigned cnt[6] = {0u, 0u, 0u, 0u, 0u, 0u};
        ProjSum<T> sum[2];
        T wmn = T(INFINITY), wmx = T(-INFINITY);
        const long long step = nthreads;
        for (long long e0 = b0 + tid; e0 < b1; e0 += 4 * step) {
            T rv[4], gv[4];   // four elements per round: their loads are in flight together
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const long long e = e0 + q * step;
                rv[q] = e < b1 ? (io.fused ? rho_in[e] : w_in[e]) : T(0);
                gv[q] = (io.fused && e < b1) ? g[e] : T(0);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const long long e = e0 + q * step;
                if (e < b1) {
                    const T w = io.fused ? rv[q] - alpha_t * (gv[q] - gmean_t) : rv[q];
                    if (CACHE) wloc[e - b0] = w;
                    else if (!io.wdirect) wbuf[e] = w;
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
        __shared__ ProjPart mine;
        if (tid == 0) {
#pragma unroll
            for (int q = 0; q < 6; ++q) mine.n[q] = cnt[q];
            mine.s[0] = sums[0];
            mine.s[1] = sums[1];
            mine.wmin = -(double)mm[0];
            mine.wmax = (double)mm[1];
        }
        if (!comm.exchange(mine, parity, tot)) return;
        parity ^= 1;
    }

    // thread 0: the search from lambda = 0, tightened by the warm start
    if (tid == 0) {
        S0 = (double)tot.n[0] * io.hi + (double)tot.n[1] * io.lo + tot.s[0];
        if (!isfinite(S0)) set_err(&sc->err, TO_ERR_NONFINITE);
        st.done = !(S0 > io.vbar) || !isfinite(S0);
        st.have_prev = false;
        st.pU = st.pL = st.pF = 0.0;
        st.lam = 0.0;
        if (!st.done) {
            st.lo_b = fmax(0.0, tot.wmin - io.hi);
            st.hi_b = tot.wmax - io.lo;
            const double t0[4] = {(double)tot.n[0], (double)tot.n[1], (double)tot.n[2], tot.s[0]};
            proj_search_step(st, t0, io.vbar, io.lo, io.hi);
            if (!st.done && lam_s > st.lo_b && lam_s < st.hi_b) {
                const double ts[4] = {(double)tot.n[3], (double)tot.n[4], (double)tot.n[5], tot.s[1]};
                st.lam = lam_s;
                st.have_prev = false;
                proj_search_step(st, ts, io.vbar, io.lo, io.hi);
            }
        }
        cast.lam = st.lam;
        cast.done = st.done;
        cast.iters = 0;
        proj_thresholds<T>(st.lam, io.lo, io.hi, cast.tu, cast.tl);
    }
    __syncthreads();

    while (!cast.done && cast.iters < kProjMaxIter) {
        const T tu = cast.tu, tl = cast.tl;
        unsigned cnt[3] = {0u, 0u, 0u};
        ProjSum<T> sum[2];
        for (long long e = b0 + tid; e < b1; e += nthreads) {
            const T w = wat(e);
            if (w >= tu) ++cnt[0];
            else if (w <= tl) ++cnt[1];
            else { ++cnt[2]; sum[0].add(w); }
        }
        const int ksum[3] = {0, 0, 0};
        block_reduce<unsigned, 3>(cnt, ksum, shu);
        double sums[2];
        proj_block_sums(sum, sums, shf, shd);
        __shared__ ProjPart mine;
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
            proj_search_step(st, t4, io.vbar, io.lo, io.hi);
            cast.lam = st.lam;
            cast.done = st.done;
            cast.iters += 1;
            proj_thresholds<T>(st.lam, io.lo, io.hi, cast.tu, cast.tl);
        }
        __syncthreads();
    }

    // final pass: rho = clamp(w - lambda), ||drho||_inf, volume
    if (tid == 0) {
        const double lambda = (st.done && !(S0 > io.vbar)) ? 0.0 : cast.lam;
        cast.lam = lambda;
        if (sizeof(T) == 4) {
            const float lh = (float)lambda;
            cast.lh = (T)lh;
            cast.ll = (T)(float)(lambda - (double)lh);
        } else {
            cast.lh = (T)lambda;
            cast.ll = T(0);
        }
    }
    __syncthreads();
    {
        const T lh = cast.lh, ll = cast.ll, lo = (T)io.lo, hi = (T)io.hi;
        T dmax = T(0);
        ProjSum<T> vol[2];
        const long long step = nthreads;
        for (long long e0 = b0 + tid; e0 < b1; e0 += 4 * step) {
            T rv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const long long e = e0 + q * step;
                rv[q] = (io.fused && e < b1) ? rho_in[e] : T(0);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const long long e = e0 + q * step;
                if (e < b1) {
                    const T rt = tmin(tmax((wat(e) - lh) - ll, lo), hi);
                    if (io.fused) dmax = tmax(dmax, tabs(rt - rv[q]));
                    vol[0].add(rt);
                    rho_out[e] = rt;
                }
            }
        }
        double sums[2];
        proj_block_sums(vol, sums, shf, shd);
        T mm[1] = {dmax};
        const int kmax[1] = {1};
        block_reduce<T, 1>(mm, kmax, sht);
        __shared__ ProjPart mine;
        if (tid == 0) {
#pragma unroll
            for (int q = 0; q < 6; ++q) mine.n[q] = 0ull;
            mine.s[0] = sums[0];
            mine.s[1] = 0.0;
            mine.wmin = INFINITY;
            mine.wmax = (double)mm[0];
        }
        if (!comm.exchange(mine, parity, tot)) return;
        if (tid == 0 && io.writer) {
            sc->lambda = cast.lam;
            sc->drho_inf = tot.wmax;
            sc->volume = tot.s[0];
            sc->proj_iters = cast.iters;
        }
    }
}

// Pass totals across the CTAs of a cluster: thread 0 publishes the CTA's partial
// in its shared memory, the cluster barrier orders it, and warp 0 of every CTA
// folds the CTAs' partials through distributed shared memory in rank order.
struct ClusterComm {
    ProjPart* slots;   // two per CTA (by pass parity)
    __device__ bool exchange(const ProjPart& mine, int parity, ProjPart& tot) {
        cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
        if (threadIdx.x == 0) slots[parity] = mine;
        cl.sync();
        if (threadIdx.x < 32) {
            const ProjPart t =
                proj_fold(cl.num_blocks(), [&](unsigned r) { return *cl.map_shared_rank(&slots[parity], r); });
            if (threadIdx.x == 0) tot = t;
        }
        return true;
    }
};

}  // namespace to
