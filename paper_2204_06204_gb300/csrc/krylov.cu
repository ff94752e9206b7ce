// The Krylov preconditioner of Eq. (LSP) (Sec. IV-C): M^-1 b is the vector x of
// the Krylov space span{b, K b, ..., K^D b} whose K x is closest to b, i.e. the
// minimiser of ||b - sum_{i=1}^{D+1} c_{i-1} K^i b||.  Used with constant
// beta = 1 in the lower-level step it gives Algorithm CPFBTO.
//
// The space is spanned by an orthonormal Arnoldi basis q_0 .. q_D (classical
// Gram-Schmidt applied twice against the earlier q's, which keeps the float
// basis orthogonal to working precision), so that K Q_{D+1} = Q_{D+2} H with
// H upper Hessenberg and ||b - K Q y|| = || ||b|| e_1 - H y ||.  One thread
// solves that (D+2) x (D+1) least-squares problem by Givens rotations, and
// x = Q y.  (The paper solves the same problem on the power basis with a
// Householder QR; the power basis loses rank in floating point well before
// D = 20 on these problems, the Arnoldi basis does not.)
//
// Per basis vector j: w = K q_j (the operator kernel, on the still unnormalised
// q_j), then three streaming passes over the basis: q_j and w scaled by the
// previous column's norm, h = Q^T w; w -= Q h with the second Gram-Schmidt dots
// fused in (h' = Q^T w, element by element on the updated w); w -= Q h' with
// ||w||^2 fused in.  Dots: float products, float
// block trees, float-pair cross-block sums on the mixed path (double on the
// FP64 path), delivered as doubles; the coefficients are double.
#include <cmath>

#include "device.cuh"

namespace to {

constexpr int kKryThreads = 512;
constexpr int kKryMax = 30;   // largest Krylov dimension D

// device coefficients of one preconditioner application
struct KrylovScalars {
    double beta0;                       // ||b||
    double w2;                          // squared norm delivered by the last norm pass
    int m;                              // basis vectors in use (D + 1, or fewer after a breakdown)
    int breakdown;                      // the space became invariant: later steps are no-ops
    double H[(kKryMax + 2) * (kKryMax + 1)];   // column-major: H[i + (kKryMax + 2) j]
    double h[kKryMax + 1];              // Gram-Schmidt coefficients of the current pass
    double y[kKryMax + 1];              // least-squares solution
};
constexpr int kHld = kKryMax + 2;

// ----------------------------------------------------------------------------- streaming passes
// One kernel, four passes over the basis (columns of Q, leading dimension ld):
//   MODE 3 (start): beta0 = ||b||; one basis vector, H cleared.
//   MODE 0 (column j, first Gram-Schmidt pass): the column's candidate q_j (b for j = 0)
//          and w = K q_j are scaled by 1/sigma (sigma = beta0, or H[j, j-1]: the previous
//          column left q_j and its image unnormalised), then h = Q^T w -> H[0..j, j].
//   MODE 1 (second pass): w -= Q H[., j], then h' = Q^T w; H[., j] += h'.
//   MODE 2 (norm): w -= Q h', then H[j+1, j] = ||w||; w stays unnormalised in column j+1.
// Each thread loads the basis values of an element once (all loads in flight together);
// the last block to finish folds the per-block partials and does the column's bookkeeping.
template <typename T, int MODE>
__global__ void __launch_bounds__(kKryThreads) k_kry_pass(T* Q, long long n, long long ld, int j, const T* b,
                                                          double* part, unsigned* counter, KrylovScalars* ks, int m_full) {
    __shared__ T s_h[kKryMax + 1];
    __shared__ T sh[32 * (kKryMax + 1)];
    __shared__ T s_inv;
    __shared__ int s_skip, s_last;
    const int tid = threadIdx.x;
    constexpr int NQ = kKryMax + 1;
    const int m = MODE == 3 ? 0 : j + 1;   // basis vectors q_0 .. q_j
    if (tid == 0) {
        s_skip = MODE == 3 ? 0 : ks->breakdown;
        if (MODE == 0) {
            const double sg = j == 0 ? ks->beta0 : ks->H[j + kHld * (j - 1)];
            s_inv = sg > 0.0 ? (T)(1.0 / sg) : T(0);
        }
    }
    if (MODE == 1 && tid <= j) s_h[tid] = (T)ks->H[tid + kHld * j];
    if (MODE == 2 && tid <= j) s_h[tid] = (T)ks->h[tid];
    __syncthreads();
    if (s_skip) return;   // every block reads the same flag: all leave together
    T* w = Q + (size_t)(j + 1) * ld;
    T acc[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) acc[i] = T(0);
    for (long long e = (long long)blockIdx.x * blockDim.x + tid; e < n; e += (long long)gridDim.x * blockDim.x) {
        if constexpr (MODE == 3) {
            const T x = b[e];
            acc[0] = fma(x, x, acc[0]);
        } else {
        T qv[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) qv[i] = (i < m) ? Q[i * ld + e] : T(0);   // predicated, independent loads
        T we = w[e];
        if (MODE == 0) {
            const T inv = s_inv;
            T qraw = j == 0 ? b[e] : T(0);
#pragma unroll
            for (int i = 1; i < NQ; ++i)
                if (i == j) qraw = qv[i];   // compile-time register index: no local memory
            const T qj = qraw * inv;
            Q[(size_t)j * ld + e] = qj;
#pragma unroll
            for (int i = 0; i < NQ; ++i)
                if (i == j) qv[i] = qj;
            we *= inv;
            w[e] = we;
        } else {
#pragma unroll
            for (int i = 0; i < NQ; ++i) we = fma(-s_h[i < m ? i : 0], qv[i], we);   // qv = 0 beyond m
            w[e] = we;
        }
        if (MODE == 0 || MODE == 1) {
#pragma unroll
            for (int i = 0; i < NQ; ++i) acc[i] = fma(qv[i], we, acc[i]);
        } else {
            acc[0] = fma(we, we, acc[0]);
        }
        }
    }
    const int nq = (MODE == 0 || MODE == 1) ? m : 1;
    // block totals: a shuffle tree per warp, then the warps in order
    const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NQ; ++i)
        if (i < nq) {
            const T v = warp_sum(acc[i]);
            if (lane == 0) sh[wid * NQ + i] = v;
        }
    __syncthreads();
    if (tid < nq) {
        T t = T(0);
        for (int q = 0; q < nw; ++q) t += sh[q * NQ + tid];
        if (sizeof(T) == 4) reinterpret_cast<float2*>(part)[(size_t)blockIdx.x * NQ + tid] = make_float2((float)t, 0.f);
        else part[(size_t)blockIdx.x * NQ + tid] = (double)t;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned t = atomicAdd(counter, 1u);
        s_last = (t == gridDim.x - 1);
        if (s_last) atomicExch(counter, 0u);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last block: output i folded by threads i, i + 32, ... over chunks of the blocks
    // (loads batched), then the chunks in order
    __shared__ double s_chunk[16][NQ];
    __shared__ double s_tot[NQ];
    const int i = tid & 31, c = tid >> 5;
    const int nchunk = blockDim.x >> 5;
    if (i < nq) {
        FF accf{0.f, 0.f};
        double accd = 0.0;
        for (unsigned b0 = c; b0 < gridDim.x; b0 += 4u * nchunk) {
            float2 tf[4];
            double td[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned bb = b0 + u * nchunk;
                if (sizeof(T) == 4)
                    tf[u] = bb < gridDim.x ? __ldcg(reinterpret_cast<const float2*>(part) + (size_t)bb * NQ + i)
                                           : make_float2(0.f, 0.f);
                else
                    td[u] = bb < gridDim.x ? __ldcg(part + (size_t)bb * NQ + i) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (sizeof(T) == 4) accf = ff_merge(accf, FF{tf[u].x, tf[u].y});
                else accd += td[u];
            }
        }
        s_chunk[c][i] = sizeof(T) == 4 ? (double)accf.hi + (double)accf.lo : accd;
    }
    __syncthreads();
    if (tid < nq) {
        double t = 0.0;
        for (int q = 0; q < nchunk; ++q) t += s_chunk[q][tid];
        s_tot[tid] = t;
    }
    __syncthreads();
    if (tid != 0) return;
    // the column's bookkeeping (one thread)
    if (MODE == 3) {
        const double b2 = s_tot[0];
        ks->beta0 = b2 > 0.0 ? sqrt(b2) : 0.0;
        ks->breakdown = !(ks->beta0 > 0.0);
        ks->m = ks->breakdown ? 0 : 1;
        for (int q = 0; q < kHld * (kKryMax + 1); ++q) ks->H[q] = 0.0;
    } else if (MODE == 0) {
        for (int q = 0; q <= j; ++q) ks->H[q + kHld * j] = s_tot[q];
    } else if (MODE == 1) {
        for (int q = 0; q <= j; ++q) {
            ks->h[q] = s_tot[q];
            ks->H[q + kHld * j] += s_tot[q];
        }
    } else {
        const double w2 = s_tot[0];
        const double hn = w2 > 0.0 ? sqrt(w2) : 0.0;
        ks->H[(j + 1) + kHld * j] = hn;
        double col2 = w2;   // ||K q_j||^2 = sum_i H[i, j]^2 + H[j+1, j]^2
        for (int q = 0; q <= j; ++q) col2 += ks->H[q + kHld * j] * ks->H[q + kHld * j];
        if (!(hn > 1e-12 * sqrt(col2))) {
            ks->breakdown = 1;        // K q_j lies in span{q_0 .. q_j}: the space is complete
            ks->m = j + 1;
        } else {
            ks->m = (j + 2 < m_full) ? j + 2 : m_full;
        }
    }
}

// one warp: min || beta0 e_1 - H y || over the m columns in use, by Givens rotations
__global__ void __launch_bounds__(32) k_kry_lsq(KrylovScalars* ks, int m_full) {
    __shared__ double R[kKryMax + 2][kKryMax + 1];
    __shared__ double g[kKryMax + 2];
    __shared__ double y[kKryMax + 1];
    const int lane = threadIdx.x;
    const int m = ks->breakdown ? ks->m : m_full;
    for (int i = 0; i <= m; ++i)
        for (int k = lane; k < m; k += 32) R[i][k] = ks->H[i + kHld * k];
    if (lane <= m) g[lane] = lane == 0 ? ks->beta0 : 0.0;
    __syncwarp();
    for (int j = 0; j < m; ++j) {   // annihilate R[j+1][j]
        const double a = R[j][j], bb = R[j + 1][j];
        const double r = hypot(a, bb);
        const double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? bb / r : 0.0;
        __syncwarp();
        for (int k = j + lane; k < m; k += 32) {
            const double x = R[j][k], yv = R[j + 1][k];
            R[j][k] = c * x + s * yv;
            R[j + 1][k] = -s * x + c * yv;
        }
        if (lane == 0) {
            const double x = g[j], yv = g[j + 1];
            g[j] = c * x + s * yv;
            g[j + 1] = -s * x + c * yv;
        }
        __syncwarp();
    }
    for (int j = m - 1; j >= 0; --j) {
        double t = 0.0;
        for (int k = j + 1 + lane; k < m; k += 32) t += R[j][k] * y[k];
        t = warp_sum(t);
        if (lane == 0) y[j] = R[j][j] != 0.0 ? (g[j] - t) / R[j][j] : 0.0;
        __syncwarp();
    }
    if (lane <= kKryMax) ks->y[lane] = lane < m ? y[lane] : 0.0;
    if (lane == 0) {
        ks->m = m;
        ks->breakdown = 0;   // the combination uses all m columns
    }
}

// x = Q y over the m columns in use
template <typename T>
__global__ void __launch_bounds__(256) k_kry_combine(const T* __restrict__ Q, long long n, long long ld, T* __restrict__ x,
                                                     const KrylovScalars* ks) {
    __shared__ T s_y[kKryMax + 1];
    __shared__ int s_m;
    if (threadIdx.x == 0) s_m = ks->m;
    if (threadIdx.x < kKryMax + 1) s_y[threadIdx.x] = (T)ks->y[threadIdx.x];
    __syncthreads();
    const int m = s_m;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        T qv[kKryMax + 1];
#pragma unroll
        for (int i = 0; i < kKryMax + 1; ++i) qv[i] = (i < m) ? Q[i * ld + e] : T(0);
        T t = T(0);
#pragma unroll
        for (int i = 0; i < kKryMax + 1; ++i) t = fma(s_y[i], qv[i], t);
        x[e] = t;
    }
}

// ----------------------------------------------------------------------------- host side
template <typename T>
static int krylov_t(to_problem* P, const void* b, void* x, cudaStream_t s) {
    const int D = P->prm.krylov_dim, m_full = D + 1;
    const long long n = P->n_dof, ld = P->kry_ld;
    T* Q = (T*)P->kry_q;
    KrylovScalars* ks = (KrylovScalars*)P->kry_s;
    double* part = P->kry_part;
    unsigned* cnt = P->counters + 12;
    const int nb = P->kry_blocks;
    const int nbs = (int)std::min<long long>((n + 255) / 256, 4LL * P->num_sms);
    k_kry_pass<T, 3><<<nb, kKryThreads, 0, s>>>(Q, n, ld, -1, (const T*)b, part, cnt, ks, m_full);   // beta0
    for (int j = 0; j <= D; ++j) {
        // w = K q_j with q_j still unnormalised (b itself for j = 0): the next pass scales both
        const void* qj = j == 0 ? b : (const void*)(Q + (size_t)j * ld);
        int rc = launch_operator(P, 0, 0 /* OP_APPLY */, qj, Q + (size_t)(j + 1) * ld, nullptr, s, 0.0, 0);
        if (rc) return rc;
        k_kry_pass<T, 0><<<nb, kKryThreads, 0, s>>>(Q, n, ld, j, (const T*)b, part, cnt, ks, m_full);
        k_kry_pass<T, 1><<<nb, kKryThreads, 0, s>>>(Q, n, ld, j, (const T*)b, part, cnt, ks, m_full);
        k_kry_pass<T, 2><<<nb, kKryThreads, 0, s>>>(Q, n, ld, j, (const T*)b, part, cnt, ks, m_full);
    }
    k_kry_lsq<<<1, 32, 0, s>>>(ks, m_full);
    k_kry_combine<T><<<nbs, 256, 0, s>>>(Q, n, ld, (T*)x, ks);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

int krylov_apply(to_problem* P, const void* b, void* x, cudaStream_t s) {
    return P->prec == TO_FP64 ? krylov_t<double>(P, b, x, s) : krylov_t<float>(P, b, x, s);
}

int krylov_build(to_problem* P) {
    const int D = P->prm.krylov_dim;
    if (D < 0 || D > kKryMax) return fail(TO_ERR_ARG, "krylov_dim must lie in [0, 30]");
    P->kry_ld = (P->n_dof + 63) & ~63LL;   // 256-byte aligned columns
    if (cudaMalloc(&P->kry_q, (size_t)(D + 2) * P->kry_ld * P->esz) != cudaSuccess)
        return fail(TO_ERR_CUDA, "Krylov basis allocation");
    if (cudaMalloc(&P->kry_s, sizeof(KrylovScalars)) != cudaSuccess) return fail(TO_ERR_CUDA, "Krylov scalars");
    cudaMemset(P->kry_s, 0, sizeof(KrylovScalars));
    P->kry_blocks = P->num_sms;
    if (cudaMalloc(&P->kry_part, sizeof(double) * (size_t)P->kry_blocks * (kKryMax + 1)) != cudaSuccess)
        return fail(TO_ERR_CUDA, "Krylov reduction scratch");
    return TO_OK;
}

}  // namespace to
