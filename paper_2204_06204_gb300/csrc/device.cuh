// Device helpers shared by the kernels: deterministic block / grid reductions,
// float-pair sums, a bounded grid barrier, the projection's search step, the
// 3-D lattice launch shape and the asynchronous-copy wrappers.
#pragma once

#include "internal.cuh"

namespace to {

// Reductions are deterministic (fixed shuffle trees, fixed fold orders).  On GB300
// the FP64 rate is a small fraction of FP32, so the warp and block trees run in
// the element precision (float on the mixed path, exact integers for counts) and
// FP64 is used only where per-block partials meet, by a single warp.
template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename V>
__device__ __forceinline__ V vmax(V a, V b) { return a > b ? a : b; }
template <> __device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
template <> __device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
template <typename V>
__device__ __forceinline__ V warp_max(V v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = vmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename V> __device__ __forceinline__ V lowest();
template <> __device__ __forceinline__ float lowest<float>() { return -INFINITY; }
template <> __device__ __forceinline__ double lowest<double>() { return -INFINITY; }
template <> __device__ __forceinline__ unsigned lowest<unsigned>() { return 0u; }

// Reduce NQ values of type V over the block (kind[q] = 0: sum, 1: max): a shuffle
// tree per warp, then one over the warps' results.  The result is valid in
// thread 0.  `sh` must hold 32 * NQ values of type V.
template <typename V, int NQ>
__device__ __forceinline__ void block_reduce(V (&v)[NQ], const int (&kind)[NQ], V* sh) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, wid = tid >> 5, nw = (nthreads + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = kind[q] ? warp_max(v[q]) : warp_sum(v[q]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) sh[wid * NQ + q] = v[q];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const V t = lane < nw ? sh[lane * NQ + q] : (kind[q] ? lowest<V>() : V(0));
            v[q] = kind[q] ? warp_max(t) : warp_sum(t);
        }
    }
    __syncthreads();
}

// element-precision math: the float overloads are named explicitly so that no
// float value is ever widened to double (FP64 is scarce on GB300)
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float tabs(float a) { return fabsf(a); }
__device__ __forceinline__ double tabs(double a) { return fabs(a); }
__device__ __forceinline__ float tsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double tsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float tpow(float a, float b) { return powf(a, b); }
__device__ __forceinline__ double tpow(double a, double b) { return pow(a, b); }
__device__ __forceinline__ bool tfinite(float a) { return (__float_as_uint(a) & 0x7f800000u) != 0x7f800000u; }
__device__ __forceinline__ bool tfinite(double a) {
    return (__double_as_longlong(a) & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}

// SIMP moduli of Sec. III in the element precision: E = Emin + rho~^p (E0 - Emin),
// E' = p rho~^(p-1) (E0 - Emin); the constants are converted once on the host
template <typename T>
struct SimpT {
    T emin, dE, p;
    int cubic;   // p == 3: products instead of pow
};
template <typename T>
__device__ __forceinline__ void simp_moduli(const SimpT<T>& m, T rt, T& E, T& Ed) {
    T pw, pw1;
    if (m.cubic) {
        pw1 = rt * rt;
        pw = pw1 * rt;
    } else {
        pw1 = tpow(rt, m.p - T(1));
        pw = pw1 * rt;
    }
    E = m.emin + pw * m.dE;
    Ed = m.p * pw1 * m.dE;
}

// Float pair hi + lo carrying a sum to about twice float precision (two-sum
// error transformation; Knuth, TAOCP vol. 2, 4.2.2).  Used where a float sum
// over many elements must stay accurate (the projection's volume sums).
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF a, float x) {
    const float s = a.hi + x, bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (x - bb);
    return FF{s, a.lo + e};
}
__device__ __forceinline__ FF ff_merge(FF a, FF b) {
    FF r = ff_add(a, b.hi);
    r.lo += b.lo;
    return r;
}
__device__ __forceinline__ unsigned lane_id() {
    unsigned l;
    asm("mov.u32 %0, %%laneid;" : "=r"(l));
    return l;
}
// sum (two-sum merge) or max (of the high parts) of two pairs
__device__ __forceinline__ FF ff_op(FF a, FF b, bool mx) { return mx ? FF{fmaxf(a.hi, b.hi), 0.f} : ff_merge(a, b); }
__device__ __forceinline__ FF warp_red_ff(FF v, bool mx) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const FF u{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        // both lanes of a pair form the same result: order the operands by lane
        v = (lane & o) ? ff_op(u, v, mx) : ff_op(v, u, mx);
    }
    return v;
}
// block totals of NQ float pairs (kind[q] = 0: sum, 1: max), valid in thread 0 as
// doubles; `sh` holds 64 * NQ floats
template <int NQ>
__device__ __forceinline__ void block_reduce_ff(FF (&v)[NQ], const int (&kind)[NQ], double (&out)[NQ], float* sh) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, wid = tid >> 5, nw = (nthreads + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = warp_red_ff(v[q], kind[q] != 0);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            sh[2 * (wid * NQ + q)] = v[q].hi;
            sh[2 * (wid * NQ + q) + 1] = v[q].lo;
        }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const FF idn = kind[q] ? FF{-INFINITY, 0.f} : FF{0.f, 0.f};
            const FF t = lane < nw ? FF{sh[2 * (lane * NQ + q)], sh[2 * (lane * NQ + q) + 1]} : idn;
            const FF r = warp_red_ff(t, kind[q] != 0);
            if (lane == 0) out[q] = (double)r.hi + (double)r.lo;
        }
    }
    __syncthreads();
}
template <int NQ>
__device__ __forceinline__ void block_reduce_ff(FF (&v)[NQ], double (&out)[NQ], float* sh) {
    int kind[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) kind[q] = 0;
    block_reduce_ff<NQ>(v, kind, out, sh);
}

// Write this block's partials (slot `bid` of `nblocks` taking part; thread 0's
// block totals), then let the last block to finish combine all partials and
// return true (in every thread) only there, with the totals in `tot` valid in all
// its threads.  The last block's threads load the partials in batches (so that
// the loads are in flight together) and fold them in a fixed pattern followed by
// a fixed tree.  Float totals travel as float pairs (no FP64 arithmetic on the
// mixed path); double totals as doubles.  `sh` holds at least 32 * kRedQ doubles.
template <typename V, int NQ>
__device__ __forceinline__ bool finish_reduction(const V (&v)[NQ], const int (&kind)[NQ], double* partials,
                                                 unsigned* counter, double (&tot)[NQ], double* sh, unsigned bid,
                                                 unsigned nblocks) {
    static_assert(NQ <= kRedQ, "reduction slot");
    __shared__ int s_last;
    constexpr bool kF = sizeof(V) == 4;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            if (kF) reinterpret_cast<float2*>(partials)[bid * kRedQ + q] = make_float2((float)v[q], 0.f);
            else partials[bid * kRedQ + q] = (double)v[q];
        }
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        s_last = (t == nblocks - 1);
        if (s_last) atomicExch(counter, 0u);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double out[NQ];
    if (kF) {
        const float2* p2 = reinterpret_cast<const float2*>(partials);
        FF acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = kind[q] ? FF{-INFINITY, 0.f} : FF{0.f, 0.f};
        for (unsigned b0 = tid; b0 < nblocks; b0 += 4u * nthreads) {
            float2 t[4][NQ];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned b = b0 + u * nthreads;
#pragma unroll
                for (int q = 0; q < NQ; ++q)
                    t[u][q] = b < nblocks ? __ldcg(p2 + b * kRedQ + q) : make_float2(kind[q] ? -INFINITY : 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int q = 0; q < NQ; ++q) acc[q] = ff_op(acc[q], FF{t[u][q].x, t[u][q].y}, kind[q] != 0);
        }
        block_reduce_ff<NQ>(acc, kind, out, reinterpret_cast<float*>(sh));
    } else {
        double acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = kind[q] ? -INFINITY : 0.0;
        for (unsigned b0 = tid; b0 < nblocks; b0 += 4u * nthreads) {
            double t[4][NQ];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned b = b0 + u * nthreads;
#pragma unroll
                for (int q = 0; q < NQ; ++q) t[u][q] = b < nblocks ? __ldcg(partials + b * kRedQ + q) : (kind[q] ? -INFINITY : 0.0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int q = 0; q < NQ; ++q) acc[q] = kind[q] ? fmax(acc[q], t[u][q]) : acc[q] + t[u][q];
        }
        block_reduce<double, NQ>(acc, kind, sh);
#pragma unroll
        for (int q = 0; q < NQ; ++q) out[q] = acc[q];
    }
    __shared__ double s_tot[kRedQ];
    if (tid == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) s_tot[q] = out[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NQ; ++q) tot[q] = s_tot[q];
    __syncthreads();
    return true;
}

// Grid-wide barrier for a cooperative (co-resident) launch.  bar[0] counts
// arrivals, bar[1] is the generation.  Spins at most spin_limit times (about
// 1 s with the default); on timeout records TO_ERR_TIMEOUT in *err and returns
// false.
constexpr unsigned long long kBarrierSpins = 1ull << 24;
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err, unsigned long long spin_limit = kBarrierSpins) {
    __shared__ int s_ok;
    const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
        volatile unsigned* vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        s_ok = 1;
        if (arrived == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned long long spins = 0;
            while (*vgen == gen) {
                if (++spins > spin_limit) {
                    atomicCAS(err, 0, (int)TO_ERR_TIMEOUT);
                    s_ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void set_err(int* err, int code) { atomicCAS(err, 0, code); }

__device__ __forceinline__ unsigned linear_block() { return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z); }
__device__ __forceinline__ unsigned grid_blocks() { return gridDim.x * gridDim.y * gridDim.z; }

// Multiplier search of the projection onto X (Eq. piecewiseLinearEQ).  Each pass
// classifies the elements at lambda into n_U (at hi), n_L (at lo) and the free
// set (count n_F, sum s_F of w).  On that piece the volume is
// S = n_U hi + n_L lo + s_F - lambda n_F, whose root is
// lambda_N = (n_U hi + n_L lo + s_F - vbar) / n_F: a function of the sets alone.
// The search moves to lambda_N (or bisects the bracket when lambda_N leaves it)
// and stops when the sets at lambda_N are the sets lambda_N came from; the
// result is then lambda_N of the final sets, independent of the starting point
// (so a warm start from the previous multiplier changes the pass count only).
__device__ __forceinline__ void proj_search_step(ProjSearch& st, const double (&t)[4], double vbar, double lo,
                                                 double hi) {
    if (st.have_prev && t[0] == st.pU && t[1] == st.pL && t[2] == st.pF) {
        st.done = true;          // lam = lambda_N of these very sets
        return;
    }
    const double S = t[0] * hi + t[1] * lo + t[3] - st.lam * t[2];
    if (S > vbar) st.lo_b = fmax(st.lo_b, st.lam);
    else st.hi_b = fmin(st.hi_b, st.lam);
    const double ln = t[2] > 0.0 ? (t[0] * hi + t[1] * lo + t[3] - vbar) / t[2] : NAN;
    const bool newton = ln >= st.lo_b && ln <= st.hi_b;
    const double next = newton ? ln : 0.5 * (st.lo_b + st.hi_b);
    if (!newton && !(st.hi_b - st.lo_b > 1e-15 * fmax(1.0, fabs(st.lam)))) {
        st.lam = next;
        st.done = true;
        return;
    }
    st.pU = t[0];
    st.pL = t[1];
    st.pF = t[2];
    st.have_prev = newton;
    st.lam = next;
}

// 3-D lattice launches: block (32, 8), grid (ceil(X/32), ceil(Y/8), Z); no divisions per thread.
inline dim3 grid3(int X, int Y, int Z) { return dim3((unsigned)((X + 31) / 32), (unsigned)((Y + 7) / 8), (unsigned)Z); }
inline dim3 block3() { return dim3(32, 8, 1); }
struct Idx3 {
    int i, j, k;
    bool ok;
};
__device__ __forceinline__ Idx3 idx3(int X, int Y, int Z) {
    Idx3 r;
    r.i = blockIdx.x * 32 + threadIdx.x;
    r.j = blockIdx.y * 8 + threadIdx.y;
    r.k = blockIdx.z;
    r.ok = r.i < X && r.j < Y && r.k < Z;
    return r;
}

// ----------------------------------------------------------------------------- async copies
__device__ __forceinline__ void cp_async_4(void* smem, const void* gmem, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 8 : 0));
}
template <typename T>
__device__ __forceinline__ void cp_async_t(T* smem, const T* gmem, bool valid) {
    if (sizeof(T) == 8) cp_async_8(smem, gmem, valid);
    else cp_async_4(smem, gmem, valid);
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

}  // namespace to
