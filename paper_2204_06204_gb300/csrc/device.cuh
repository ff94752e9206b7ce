// Device helpers shared by the kernels: deterministic block / grid reductions
// and a bounded grid barrier.
#pragma once

#include "internal.cuh"

namespace to {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Reduce NQ values over the block (kind[q] = 0: sum, 1: max).  The result is
// valid in thread 0.  `sh` must hold 32 * NQ doubles.  Fixed order.
template <int NQ>
__device__ __forceinline__ void block_reduce(double (&v)[NQ], const int (&kind)[NQ], double* sh) {
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
            double t = lane < nw ? sh[lane * NQ + q] : (kind[q] ? -INFINITY : 0.0);
            v[q] = kind[q] ? warp_max(t) : warp_sum(t);
        }
    }
    __syncthreads();
}

// Write this block's partials (slot `bid` of `nblocks` taking part), then let the
// last block to finish combine all partials in block order.  Returns true (in every thread) only in that block,
// with the totals in `tot` valid in all its threads.
template <int NQ>
__device__ __forceinline__ bool finish_reduction(const double (&v)[NQ], const int (&kind)[NQ], double* partials,
                                                 unsigned* counter, double (&tot)[NQ], double* sh, unsigned bid,
                                                 unsigned nblocks) {
    __shared__ int s_last;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) partials[bid * kRedQ + q] = v[q];
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        s_last = (t == nblocks - 1);
        if (s_last) atomicExch(counter, 0u);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    // every thread folds a strided subset in order, then a fixed-order tree
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = kind[q] ? -INFINITY : 0.0;
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    for (unsigned b = tid; b < nblocks; b += nthreads)
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const double t = __ldcg(partials + b * kRedQ + q);
            acc[q] = kind[q] ? fmax(acc[q], t) : acc[q] + t;
        }
    block_reduce<NQ>(acc, kind, sh);
    if (tid == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) sh[q] = acc[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NQ; ++q) tot[q] = sh[q];
    __syncthreads();
    return true;
}

// Grid-wide barrier for a cooperative (co-resident) launch.  bar[0] counts
// arrivals, bar[1] is the generation.  Spins a bounded number of times; on
// timeout records TO_ERR_TIMEOUT in *err and returns false.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err) {
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
                if (++spins > (1ull << 24)) {
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
struct ProjSearch {
    double lam, lo_b, hi_b;
    double pU, pL, pF;   // sets that produced lam (when have_prev)
    bool have_prev, done;
};

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

}  // namespace to
