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
// Per basis vector j: w = K q_j (the operator kernel), then three streaming
// passes over the basis: h = Q^T w; w -= Q h with the second Gram-Schmidt dots
// fused in (h' = Q^T w, element by element on the updated w); w -= Q h' with
// ||w||^2 fused in; then q_{j+1} = w / ||w||.  Dots: float products, float
// block trees, float-pair cross-block sums on the mixed path (double on the
// FP64 path), delivered as doubles; the coefficients are double.
#include <cmath>

#include "device.cuh"

namespace to {

int launch_operator(to_problem* P, int level, int mode, const void* x, void* y, const void* b, cudaStream_t s,
                    double omega, int first);

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
// MODE 0: out = Q^T w (the first m basis vectors)
// MODE 1: w -= Q h_in, then out = Q^T w (fused second Gram-Schmidt dots)
// MODE 2: w -= Q h_in, then out[0] = w^T w
// MODE 3: out[0] = w^T w
// Partials of each block (one per output) are combined by the last block; `add` adds the
// totals to `dst` (dst[i] += t_i) instead of storing them.
template <typename T, int MODE>
__global__ void __launch_bounds__(kKryThreads) k_kry_pass(const T* __restrict__ Q, long long n, long long ld, T* w,
                                                          const double* h_in, double* part, unsigned* counter,
                                                          double* dst, int add, KrylovScalars* ks) {
    __shared__ T s_h[kKryMax + 1];
    __shared__ T sh[32 * (kKryMax + 1)];
    __shared__ int s_m, s_last;
    const int tid = threadIdx.x;
    if (tid == 0) s_m = MODE == 3 ? 1 : (ks->breakdown ? 0 : ks->m);
    __syncthreads();
    const int m = s_m;
    if (m == 0) return;   // every block reads the same flag: all leave together
    if (MODE == 1 || MODE == 2) {
        if (tid < m) s_h[tid] = (T)h_in[tid];
        __syncthreads();
    }
    constexpr int NQ = (MODE == 0 || MODE == 1) ? kKryMax + 1 : 1;
    T acc[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) acc[i] = T(0);
    for (long long e = (long long)blockIdx.x * blockDim.x + tid; e < n; e += (long long)gridDim.x * blockDim.x) {
        T we = w[e];
        if (MODE == 1 || MODE == 2) {
#pragma unroll
            for (int i = 0; i < kKryMax + 1; ++i)
                if (i < m) we -= s_h[i] * Q[i * ld + e];
            w[e] = we;
        }
        if (MODE == 0 || MODE == 1) {
#pragma unroll
            for (int i = 0; i < NQ; ++i)
                if (i < m) acc[i] = fma(Q[i * ld + e], we, acc[i]);
        } else {
            acc[0] = fma(we, we, acc[0]);
        }
    }
    const int nq = (MODE == 0 || MODE == 1) ? m : 1;
    // block totals: a shuffle tree per warp, then one over the warps (fixed order)
    const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NQ; ++i)
        if (i < nq) {
            const T v = warp_sum(acc[i]);
            if (lane == 0) sh[wid * (kKryMax + 1) + i] = v;
        }
    __syncthreads();
    if (tid < nq) {
        T t = T(0);
        for (int q = 0; q < nw; ++q) t += sh[q * (kKryMax + 1) + tid];
        if (sizeof(T) == 4) reinterpret_cast<float2*>(part)[(size_t)blockIdx.x * (kKryMax + 1) + tid] = make_float2((float)t, 0.f);
        else part[(size_t)blockIdx.x * (kKryMax + 1) + tid] = (double)t;
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
    // the last block: output i is folded by threads i, i + 32, ... over block chunks, then
    // the chunks in order (fixed pattern)
    __shared__ double s_chunk[16][kKryMax + 1];
    const int i = tid & 31, c = tid >> 5;   // up to 16 chunks of the blocks
    const int nchunk = blockDim.x >> 5;
    if (i < nq) {
        FF accf{0.f, 0.f};
        double accd = 0.0;
        for (unsigned b0 = c; b0 < gridDim.x; b0 += 4u * nchunk) {
            float2 tf[4];
            double td[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned b = b0 + u * nchunk;
                if (sizeof(T) == 4)
                    tf[u] = b < gridDim.x ? __ldcg(reinterpret_cast<const float2*>(part) + (size_t)b * (kKryMax + 1) + i)
                                          : make_float2(0.f, 0.f);
                else
                    td[u] = b < gridDim.x ? __ldcg(part + (size_t)b * (kKryMax + 1) + i) : 0.0;
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
        if (add) dst[tid] += t;
        else dst[tid] = t;
    }
}

// beta0 = ||b||, q_0 = b / beta0 (the first column) -- the scale step of any column:
// q_{j+1} = w / H[j+1, j]; a vanishing norm marks the space invariant
template <typename T>
__global__ void __launch_bounds__(256) k_kry_scale(const T* w, T* q, long long n, KrylovScalars* ks, int j) {
    __shared__ T s_inv;
    __shared__ int s_skip;
    if (threadIdx.x == 0) {
        double nrm;
        if (j < 0) {
            nrm = ks->beta0;
        } else {
            nrm = ks->H[(j + 1) + kHld * j];
        }
        const bool dead = ks->breakdown || !(nrm > 1e-30 * (ks->beta0 > 0.0 ? ks->beta0 : 1.0));
        s_skip = dead;
        s_inv = dead ? T(0) : (T)(1.0 / nrm);
    }
    __syncthreads();
    if (s_skip) return;
    const T inv = s_inv;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        q[e] = w[e] * inv;
}

// one thread: bookkeeping between the passes of column j
//   stage 0: beta0 = sqrt(w2) at the start of an application; one basis vector
//   stage 1: H[0..j, j] = h (first Gram-Schmidt pass)
//   stage 3: H[0..j, j] += h (second pass)
//   stage 2: H[j+1, j] = sqrt(w2); the space is invariant when it vanishes relative
//            to the column, else one more basis vector is in use
__global__ void k_kry_book(KrylovScalars* ks, int j, int stage, int m_full) {
    if (stage == 0) {
        const double b2 = ks->w2;
        ks->beta0 = b2 > 0.0 ? sqrt(b2) : 0.0;
        ks->breakdown = !(ks->beta0 > 0.0);
        ks->m = 1;
        for (int q = 0; q < kHld * (kKryMax + 1); ++q) ks->H[q] = 0.0;
        return;
    }
    if (ks->breakdown) return;
    if (stage == 1 || stage == 3) {
        for (int i = 0; i <= j; ++i) ks->H[i + kHld * j] = (stage == 1 ? 0.0 : ks->H[i + kHld * j]) + ks->h[i];
        return;
    }
    double colmax = 0.0;
    for (int i = 0; i <= j; ++i) colmax = fmax(colmax, fabs(ks->H[i + kHld * j]));
    const double w2 = ks->w2;
    const double hn = w2 > 0.0 ? sqrt(w2) : 0.0;
    ks->H[(j + 1) + kHld * j] = hn;
    if (!(hn > 1e-12 * colmax)) {
        ks->breakdown = 1;        // K q_j lies in the span of q_0 .. q_j: the space is complete
        ks->m = j + 1;
    } else {
        ks->m = (j + 2 < m_full) ? j + 2 : m_full;
    }
}

// one thread: min || beta0 e_1 - H y || over the m columns in use, by Givens rotations
__global__ void k_kry_lsq(KrylovScalars* ks, int m_full) {
    const int m = ks->breakdown ? ks->m : m_full;
    double R[kKryMax + 2][kKryMax + 1];
    double g[kKryMax + 2];
    for (int i = 0; i <= m; ++i) {
        g[i] = i == 0 ? ks->beta0 : 0.0;
        for (int j = 0; j < m; ++j) R[i][j] = ks->H[i + kHld * j];
    }
    for (int j = 0; j < m; ++j) {   // annihilate R[j+1][j]
        const double a = R[j][j], b = R[j + 1][j];
        const double r = hypot(a, b);
        const double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? b / r : 0.0;
        for (int k = j; k < m; ++k) {
            const double x = R[j][k], y = R[j + 1][k];
            R[j][k] = c * x + s * y;
            R[j + 1][k] = -s * x + c * y;
        }
        const double x = g[j], y = g[j + 1];
        g[j] = c * x + s * y;
        g[j + 1] = -s * x + c * y;
    }
    for (int j = m - 1; j >= 0; --j) {
        double t = g[j];
        for (int k = j + 1; k < m; ++k) t -= R[j][k] * ks->y[k];
        ks->y[j] = R[j][j] != 0.0 ? t / R[j][j] : 0.0;
    }
    for (int j = m; j <= kKryMax; ++j) ks->y[j] = 0.0;
    ks->m = m;
    ks->breakdown = 0;   // the combination uses all m columns
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
        T t = T(0);
#pragma unroll
        for (int i = 0; i < kKryMax + 1; ++i)
            if (i < m) t = fma(s_y[i], Q[i * ld + e], t);
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
    // beta0 = ||b||, q_0 = b / beta0
    k_kry_pass<T, 3><<<nb, kKryThreads, 0, s>>>(Q, n, ld, (T*)b, nullptr, part, cnt, &ks->w2, 0, ks);
    k_kry_book<<<1, 1, 0, s>>>(ks, 0, 0, m_full);
    k_kry_scale<T><<<nbs, 256, 0, s>>>((const T*)b, Q, n, ks, -1);
    for (int j = 0; j <= D; ++j) {
        T* qj = Q + (size_t)j * ld;
        T* w = Q + (size_t)(j + 1) * ld;
        int rc = launch_operator(P, 0, 0 /* OP_APPLY */, qj, w, nullptr, s, 0.0, 0);
        if (rc) return rc;
        // h = Q^T w over the j+1 basis vectors (ks->m = j + 1 here)
        k_kry_pass<T, 0><<<nb, kKryThreads, 0, s>>>(Q, n, ld, w, nullptr, part, cnt, ks->h, 0, ks);
        k_kry_book<<<1, 1, 0, s>>>(ks, j, 1, m_full);
        // w -= Q h, then the second pass's h' = Q^T w
        k_kry_pass<T, 1><<<nb, kKryThreads, 0, s>>>(Q, n, ld, w, ks->h, part, cnt, ks->h, 0, ks);
        k_kry_book<<<1, 1, 0, s>>>(ks, j, 3, m_full);
        // w -= Q h', then ||w||^2
        k_kry_pass<T, 2><<<nb, kKryThreads, 0, s>>>(Q, n, ld, w, ks->h, part, cnt, &ks->w2, 0, ks);
        k_kry_book<<<1, 1, 0, s>>>(ks, j, 2, m_full);
        if (j < D) k_kry_scale<T><<<nbs, 256, 0, s>>>(w, w, n, ks, j);
    }
    k_kry_lsq<<<1, 1, 0, s>>>(ks, m_full);
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
