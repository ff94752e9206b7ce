// Geometric-multigrid V-cycle used as the lower-level preconditioner M
// (Algorithm 3 with a non-Krylov M; the paper cites multigrid as prior art in
// Sec. II and IV-A/D and leaves its design open).  Definition:
//   level l+1 halves every grid dimension and doubles the element edge; its
//   element moduli are the mean of the 8 children, its operator is the hex8
//   operator of that grid (K_e scales with the edge length in 3-D); a coarse
//   DOF is fixed when any fine DOF of the same component at the fine nodes
//   {2I-1, 2I, 2I+1}^3 is; transfer is trilinear prolongation P (restriction
//   P^T) with fixed DOFs masked on both sides; smoothing is damped Jacobi with
//   weight omega, nu_pre sweeps before and nu_post after the coarse
//   correction; the coarsest grid is solved exactly.
// Coarsest solve: the dense operator is assembled on the device, scaled to a
// unit diagonal (S A S, S = diag(A)^-1/2, so that the 1e9 stiffness contrast of
// void regions does not reach the factorisation) and inverted by Gauss-Jordan
// elimination: by one CTA with the entries in registers up to 160 DOFs, above
// that by 32-blocks over many CTAs; each V-cycle then applies S A^-1 S.  The
// levels below about a thousand elements run as one CTA (the coarse tail), and
// the last part of the file batches all of it over many problems.
#include <algorithm>
#include <cmath>

#include <type_traits>

#include "device.cuh"
#include "haar.cuh"
#include "transfer.cuh"

namespace to {

constexpr int kMaxCoarseDof = 1024;  // dense coarsest solve; in shared memory while n^2 entries fit
// dynamic shared memory left for the matrix next to the static row / column / scale arrays

static int grid1(long long n, int num_sms) {
    long long b = (n + 255) / 256;
    if (b > 8LL * num_sms) b = 8LL * num_sms;
    return (int)(b < 1 ? 1 : b);
}

// coarse modulus = mean of the 8 fine children (coarse element (I, J, K))
template <typename T>
__device__ __forceinline__ void coarsen_elem(int cx, int cy, int I, int J, int K, const T* __restrict__ Ef,
                                             T* __restrict__ Ec) {
    const int fx = 2 * cx, fy = 2 * cy;
    const long long e = I + (long long)cx * (J + (long long)cy * K);
    T s = T(0);
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a)
                s += Ef[(2 * I + a) + (long long)fx * ((2 * J + b) + (long long)fy * (2 * K + c))];
    Ec[e] = T(0.125) * s;
}

template <typename T>
__global__ void k_coarsen_E(int cx, int cy, int cz, const T* __restrict__ Ef, T* __restrict__ Ec, const unsigned* gate) {
    if (gate && gate[0] != gate[1]) return;   // (gate: to_set_state found the design unchanged)
    const Idx3 t = idx3(cx, cy, cz);
    if (t.ok) coarsen_elem<T>(cx, cy, t.i, t.j, t.k, Ef, Ec);
}

// b_c = m_c P^T (m_f t), optionally with the coarse level's first sweep (IX: 32-bit indices
// while the fine level has fewer than 2^31 DOFs)
template <typename T, typename IX>
__global__ void k_restrict(int cx, int cy, int cz, const T* __restrict__ tf, const uint8_t* __restrict__ mf,
                           const uint8_t* __restrict__ mc, T* __restrict__ bc, const T* __restrict__ dinvc,
                           T* __restrict__ xc, T omega) {
    const Idx3 t = idx3(cx + 1, cy + 1, cz + 1);
    if (t.ok) restrict_node<T, IX, true>(cx, cy, cz, t.i, t.j, t.k, tf, mf, mc, bc, dinvc, xc, omega);
}

// x_f += m_f P (m_c x_c)
template <typename T, typename IX>
__global__ void k_prolong_add(int cx, int cy, int cz, const T* __restrict__ xc, const uint8_t* __restrict__ mc,
                              const uint8_t* __restrict__ mf, T* __restrict__ xf) {
    const Idx3 t = idx3(2 * cx + 1, 2 * cy + 1, 2 * cz + 1);
    if (t.ok) prolong_node<T, IX>(cx, cy, cz, t.i, t.j, t.k, xc, mc, mf, xf);
}

// x = omega D^-1 b  (first Jacobi sweep from x = 0; dinv = D^-1)
template <typename T>
__global__ void k_jacobi_first(long long n, const T* __restrict__ b, const T* __restrict__ dinv, T* __restrict__ x, T omega) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = omega * b[i] * dinv[i];
}

// dense coarsest operator (fixed rows / columns = identity)
template <typename T>
__device__ __forceinline__ T dense_entry(int nx, int ny, int nz, const T* __restrict__ E, const uint8_t* __restrict__ mask,
                                         const double* __restrict__ ke, double hscale, int n, long long idx) {
    const int nxn = nx + 1, nyn = ny + 1;
    {
        const int a = (int)(idx / n), b = (int)(idx % n);
        const int na = a / 3, ca = a % 3, nb = b / 3, cb = b % 3;
        const int ia = na % nxn, ja = (na / nxn) % nyn, kka = na / (nxn * nyn);
        const int ib = nb % nxn, jb = (nb / nxn) % nyn, kkb = nb / (nxn * nyn);
        const bool fa = (mask[na] >> ca) & 1, fbb = (mask[nb] >> cb) & 1;
        double v = 0.0;
        if (fa || fbb) {
            v = (a == b) ? 1.0 : 0.0;
        } else if (abs(ia - ib) <= 1 && abs(ja - jb) <= 1 && abs(kka - kkb) <= 1) {
            for (int dk = -1; dk <= 0; ++dk)
                for (int dj = -1; dj <= 0; ++dj)
                    for (int di = -1; di <= 0; ++di) {
                        const int ei = ia + di, ej = ja + dj, ek = kka + dk;
                        if (ei < 0 || ei >= nx || ej < 0 || ej >= ny || ek < 0 || ek >= nz) continue;
                        const int ob_i = ib - ei, ob_j = jb - ej, ob_k = kkb - ek;
                        if (ob_i < 0 || ob_i > 1 || ob_j < 0 || ob_j > 1 || ob_k < 0 || ob_k > 1) continue;
                        // local node numbering (0,0,0),(1,0,0),(1,1,0),(0,1,0),(0,0,1),(1,0,1),(1,1,1),(0,1,1)
                        const int oa_i = -di, oa_j = -dj, oa_k = -dk;
                        const int la = 4 * oa_k + (oa_j ? (oa_i ? 2 : 3) : oa_i);
                        const int lb = 4 * ob_k + (ob_j ? (ob_i ? 2 : 3) : ob_i);
                        v += (double)E[ei + nx * (ej + ny * ek)] * hscale * ke[(3 * la + ca) * 24 + 3 * lb + cb];
                    }
        }
        return (T)v;
    }
}

template <typename T>
__global__ void k_dense_assemble(int nx, int ny, int nz, const T* __restrict__ E, const uint8_t* __restrict__ mask,
                                 const double* __restrict__ ke, double hscale, T* __restrict__ A, int n,
                                 const unsigned* gate) {
    if (gate && gate[0] != gate[1]) return;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)n * n;
         idx += (long long)gridDim.x * blockDim.x)
        A[idx] = dense_entry<T>(nx, ny, nz, E, mask, ke, hscale, n, idx);
}

// Register-blocked variant for n <= 160: thread (tx, ty) of a 32 x 32 block keeps
// entries (ty + 32a, tx + 32b), a, b < 5, in registers; each elimination step
// publishes the pivot row and column through double-buffered shared memory
// (one barrier per step) and updates the held entries in place.
constexpr int kRegDof = 160;

template <typename T>
__device__ __forceinline__ void dense_invert_reg_body(const T* __restrict__ A, T* __restrict__ Ainv,
                                                      T* __restrict__ sc, int n, int* err) {
    __shared__ T rowb[2][kRegDof];
    __shared__ T colb[2][kRegDof];
    __shared__ T s[kRegDof];
    __shared__ int bad;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int i = tid; i < n; i += 1024) {
        const T d = A[(long long)i * n + i];
        s[i] = d > T(0) ? T(1) / tsqrt(d) : T(0);
        if (!(d > T(0))) bad = 1;
    }
    __syncthreads();
    if (bad) {
        if (tid == 0) set_err(err, TO_ERR_SINGULAR);
        return;
    }
    T R[5][5];
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            const int i = ty + 32 * a, j = tx + 32 * b;
            R[a][b] = (i < n && j < n) ? s[i] * A[(long long)i * n + j] * s[j] : T(0);
        }
    for (int k = 0; k < n; ++k) {
        const int buf = k & 1, ka = k >> 5, kr = k & 31;
        // publish the pivot row (old values) and column
        if (ty == kr) {
#pragma unroll
            for (int b = 0; b < 5; ++b)
                if (ka == 0) rowb[buf][tx + 32 * b] = R[0][b];
                else if (ka == 1) rowb[buf][tx + 32 * b] = R[1][b];
                else if (ka == 2) rowb[buf][tx + 32 * b] = R[2][b];
                else if (ka == 3) rowb[buf][tx + 32 * b] = R[3][b];
                else rowb[buf][tx + 32 * b] = R[4][b];
        }
        if (tx == kr) {
#pragma unroll
            for (int a = 0; a < 5; ++a)
                if (ka == 0) colb[buf][ty + 32 * a] = R[a][0];
                else if (ka == 1) colb[buf][ty + 32 * a] = R[a][1];
                else if (ka == 2) colb[buf][ty + 32 * a] = R[a][2];
                else if (ka == 3) colb[buf][ty + 32 * a] = R[a][3];
                else colb[buf][ty + 32 * a] = R[a][4];
        }
        __syncthreads();
        const T piv = rowb[buf][k];
        if (!(piv > T(0))) {
            if (tid == 0) set_err(err, TO_ERR_SINGULAR);
            return;
        }
        const T ip = T(1) / piv;
        T rn[5], co[5];
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            const int j = tx + 32 * b;
            rn[b] = (j == k ? T(1) : rowb[buf][j]) * ip;        // the new pivot row
        }
#pragma unroll
        for (int a = 0; a < 5; ++a) co[a] = colb[buf][ty + 32 * a];
        // the pivot column is eliminated: its entries enter the update as 0
        if (tx == kr) {
#pragma unroll
            for (int a = 0; a < 5; ++a)
                if (ka == 0) R[a][0] = T(0);
                else if (ka == 1) R[a][1] = T(0);
                else if (ka == 2) R[a][2] = T(0);
                else if (ka == 3) R[a][3] = T(0);
                else R[a][4] = T(0);
        }
#pragma unroll
        for (int a = 0; a < 5; ++a)
#pragma unroll
            for (int b = 0; b < 5; ++b) R[a][b] = fma(-co[a], rn[b], R[a][b]);
        // the pivot row is the scaled old row
        if (ty == kr) {
#pragma unroll
            for (int b = 0; b < 5; ++b)
                if (ka == 0) R[0][b] = rn[b];
                else if (ka == 1) R[1][b] = rn[b];
                else if (ka == 2) R[2][b] = rn[b];
                else if (ka == 3) R[3][b] = rn[b];
                else R[4][b] = rn[b];
        }
    }
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            const int i = ty + 32 * a, j = tx + 32 * b;
            if (i < n && j < n) Ainv[(long long)i * n + j] = R[a][b];
        }
    for (int i = tid; i < n; i += 1024) sc[i] = s[i];
}

template <typename T>
__global__ void __launch_bounds__(1024) k_dense_invert_reg(const T* __restrict__ A, T* __restrict__ Ainv,
                                                           T* __restrict__ sc, int n, int* err, const unsigned* gate) {
    if (gate && gate[0] != gate[1]) return;
    dense_invert_reg_body<T>(A, Ainv, sc, n, err);
}

// Blocked Gauss-Jordan inversion for the larger coarsest operators (n > 160): the
// scaled matrix S A S (s = diag(A)^-1/2), padded with the identity to N = 32 nb, in
// a global work matrix W; per 32-block k, the same in-place elimination as the
// scalar form, by blocks:
//   W_kk <- W_kk^-1 = P;  W_kj <- P W_kj (j != k);
//   W_ij <- W_ij - W_ik W_kj (i, j != k, W_ik before this step);  W_ik <- -W_ik P (i != k).
// One launch for the pivot block, one for the block row (which also saves the old
// block column), one for every other block: many CTAs per step instead of one CTA
// sweeping the whole matrix n times.  Tables hold one entry per problem.
constexpr int kGjB = 32;

template <typename T>
struct GjArgs {
    int n, nb;      // order, 32-blocks (N = 32 nb)
    const T* A;     // n x n operator
    T* W;           // N x N work matrix
    T* C;           // N x 32: the block column of W before the current step
    T* P;           // 32 x 32: the current pivot block's inverse
    T* inv;         // n x n inverse of S A S, then the n scale factors s
    int* err;
};

template <typename T>
__global__ void __launch_bounds__(256) k_gj_init(const GjArgs<T>* __restrict__ tab) {
    const GjArgs<T>& a = tab[blockIdx.y];
    const int n = a.n, N = a.nb * kGjB;
    const long long NN = (long long)N * N;
    for (long long q = blockIdx.x * 256LL + threadIdx.x; q < NN; q += (long long)gridDim.x * 256) {
        const int i = (int)(q / N), j = (int)(q % N);
        T v = i == j ? T(1) : T(0);
        if (i < n && j < n) {
            const T di = a.A[(long long)i * n + i], dj = a.A[(long long)j * n + j];
            const T si = di > T(0) ? T(1) / tsqrt(di) : T(0), sj = dj > T(0) ? T(1) / tsqrt(dj) : T(0);
            v = si * a.A[(long long)i * n + j] * sj;
            if (j == 0) {
                a.inv[(long long)n * n + i] = si;
                if (!(di > T(0))) set_err(a.err, TO_ERR_SINGULAR);
            }
        }
        a.W[q] = v;
    }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_gj_pivot(const GjArgs<T>* __restrict__ tab, int k) {
    const GjArgs<T>& a = tab[blockIdx.x];
    if (k >= a.nb) return;
    __shared__ T M[kGjB][kGjB + 1];
    __shared__ T row[kGjB], col[kGjB];
    const int tx = threadIdx.x, ty = threadIdx.y, N = a.nb * kGjB;
    T* Wkk = a.W + (size_t)(k * kGjB) * N + k * kGjB;
    M[ty][tx] = Wkk[(size_t)ty * N + tx];
    __syncthreads();
    for (int p = 0; p < kGjB; ++p) {
        const T piv = M[p][p];
        if (!(piv > T(0)) && tx == 0 && ty == 0) set_err(a.err, TO_ERR_SINGULAR);
        const T ip = piv > T(0) ? T(1) / piv : T(0);
        if (ty == 0) row[tx] = (tx == p ? T(1) : M[p][tx]) * ip;
        if (ty == 1) col[tx] = M[tx][p];
        __syncthreads();
        M[ty][tx] = ty == p ? row[tx] : (tx == p ? T(0) : M[ty][tx]) - col[ty] * row[tx];
        __syncthreads();
    }
    const T v = M[ty][tx];
    Wkk[(size_t)ty * N + tx] = v;
    a.P[ty * kGjB + tx] = v;
}

// block tiles below: 32 x 8 threads, thread (tx, ty) owns rows ty + 8 m (m < 4) of column tx
constexpr int kGjRows = kGjB / 8;

template <typename T>
__global__ void __launch_bounds__(256) k_gj_row(const GjArgs<T>* __restrict__ tab, int k) {
    const GjArgs<T>& a = tab[blockIdx.y];
    const int r = blockIdx.x;
    if (k >= a.nb || r >= a.nb || r == k) return;
    __shared__ T Ps[kGjB][kGjB + 1], Rs[kGjB][kGjB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y, N = a.nb * kGjB;
    T* Wkr = a.W + (size_t)(k * kGjB) * N + r * kGjB;
#pragma unroll
    for (int m = 0; m < kGjRows; ++m) {
        const int y = ty + 8 * m;
        Ps[y][tx] = a.P[y * kGjB + tx];
        Rs[y][tx] = Wkr[(size_t)y * N + tx];
        a.C[(size_t)(r * kGjB + y) * kGjB + tx] = a.W[(size_t)(r * kGjB + y) * N + k * kGjB + tx];   // block (r, k)
    }
    __syncthreads();
    T acc[kGjRows];
#pragma unroll
    for (int m = 0; m < kGjRows; ++m) acc[m] = T(0);
#pragma unroll 8
    for (int t = 0; t < kGjB; ++t) {
        const T b = Rs[t][tx];
#pragma unroll
        for (int m = 0; m < kGjRows; ++m) acc[m] = fma(Ps[ty + 8 * m][t], b, acc[m]);
    }
#pragma unroll
    for (int m = 0; m < kGjRows; ++m) Wkr[(size_t)(ty + 8 * m) * N + tx] = acc[m];
}

template <typename T>
__global__ void __launch_bounds__(256) k_gj_update(const GjArgs<T>* __restrict__ tab, int k, int nbmax) {
    const GjArgs<T>& a = tab[blockIdx.y];
    const int i = blockIdx.x / nbmax, j = blockIdx.x % nbmax;
    if (k >= a.nb || i >= a.nb || j >= a.nb || i == k) return;
    __shared__ T Cs[kGjB][kGjB + 1], Bs[kGjB][kGjB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y, N = a.nb * kGjB;
#pragma unroll
    for (int m = 0; m < kGjRows; ++m) {
        const int y = ty + 8 * m;
        Cs[y][tx] = a.C[(size_t)(i * kGjB + y) * kGjB + tx];
        Bs[y][tx] = j == k ? a.P[y * kGjB + tx] : a.W[(size_t)(k * kGjB + y) * N + j * kGjB + tx];
    }
    __syncthreads();
    T acc[kGjRows];
#pragma unroll
    for (int m = 0; m < kGjRows; ++m) acc[m] = T(0);
#pragma unroll 8
    for (int t = 0; t < kGjB; ++t) {
        const T b = Bs[t][tx];
#pragma unroll
        for (int m = 0; m < kGjRows; ++m) acc[m] = fma(Cs[ty + 8 * m][t], b, acc[m]);
    }
#pragma unroll
    for (int m = 0; m < kGjRows; ++m) {
        T* w = a.W + (size_t)(i * kGjB + ty + 8 * m) * N + j * kGjB + tx;
        *w = j == k ? -acc[m] : *w - acc[m];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_gj_final(const GjArgs<T>* __restrict__ tab) {
    const GjArgs<T>& a = tab[blockIdx.y];
    const int n = a.n, N = a.nb * kGjB;
    const long long nn = (long long)n * n;
    for (long long q = blockIdx.x * 256LL + threadIdx.x; q < nn; q += (long long)gridDim.x * 256)
        a.inv[q] = a.W[(size_t)(q / n) * N + q % n];
}

// The same block steps for a batch, over compact tile maps: the problems are ordered
// by block count (largest first) so that step k's pivots are the first m_k of them,
// and each step's block-row and rank-32-update tiles are listed as (problem, tile)
// pairs, so that no CTA is launched for a problem that has no block left.
template <typename T>
__global__ void __launch_bounds__(256) k_gj_row_map(const GjArgs<T>* __restrict__ tab, const int2* __restrict__ map,
                                                    int k) {
    const int2 m = map[blockIdx.x];
    const GjArgs<T>& a = tab[m.x];
    const int r = m.y;
    __shared__ T Ps[kGjB][kGjB + 1], Rs[kGjB][kGjB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y, N = a.nb * kGjB;
    T* Wkr = a.W + (size_t)(k * kGjB) * N + r * kGjB;
#pragma unroll
    for (int mm = 0; mm < kGjRows; ++mm) {
        const int y = ty + 8 * mm;
        Ps[y][tx] = a.P[y * kGjB + tx];
        Rs[y][tx] = Wkr[(size_t)y * N + tx];
        a.C[(size_t)(r * kGjB + y) * kGjB + tx] = a.W[(size_t)(r * kGjB + y) * N + k * kGjB + tx];   // block (r, k)
    }
    __syncthreads();
    T acc[kGjRows];
#pragma unroll
    for (int mm = 0; mm < kGjRows; ++mm) acc[mm] = T(0);
#pragma unroll 8
    for (int t = 0; t < kGjB; ++t) {
        const T b = Rs[t][tx];
#pragma unroll
        for (int mm = 0; mm < kGjRows; ++mm) acc[mm] = fma(Ps[ty + 8 * mm][t], b, acc[mm]);
    }
#pragma unroll
    for (int mm = 0; mm < kGjRows; ++mm) Wkr[(size_t)(ty + 8 * mm) * N + tx] = acc[mm];
}

template <typename T>
__global__ void __launch_bounds__(256) k_gj_update_map(const GjArgs<T>* __restrict__ tab, const int2* __restrict__ map,
                                                       int k) {
    const int2 m = map[blockIdx.x];
    const GjArgs<T>& a = tab[m.x];
    const int i = m.y >> 16, j = m.y & 0xffff;
    __shared__ T Cs[kGjB][kGjB + 1], Bs[kGjB][kGjB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y, N = a.nb * kGjB;
#pragma unroll
    for (int mm = 0; mm < kGjRows; ++mm) {
        const int y = ty + 8 * mm;
        Cs[y][tx] = a.C[(size_t)(i * kGjB + y) * kGjB + tx];
        Bs[y][tx] = j == k ? a.P[y * kGjB + tx] : a.W[(size_t)(k * kGjB + y) * N + j * kGjB + tx];
    }
    __syncthreads();
    T acc[kGjRows];
#pragma unroll
    for (int mm = 0; mm < kGjRows; ++mm) acc[mm] = T(0);
#pragma unroll 8
    for (int t = 0; t < kGjB; ++t) {
        const T b = Bs[t][tx];
#pragma unroll
        for (int mm = 0; mm < kGjRows; ++mm) acc[mm] = fma(Cs[ty + 8 * mm][t], b, acc[mm]);
    }
#pragma unroll
    for (int mm = 0; mm < kGjRows; ++mm) {
        T* w = a.W + (size_t)(i * kGjB + ty + 8 * mm) * N + j * kGjB + tx;
        *w = j == k ? -acc[mm] : *w - acc[mm];
    }
}

// per block step k: pivots over the first piv[k] problems, rows map[row_off[k] ..] (row_n[k]
// entries), updates map[upd_off[k] ..] (upd_n[k] entries)
struct GjMaps {
    const int2* map = nullptr;
    std::vector<int> piv, row_off, row_n, upd_off, upd_n;
};

// tile maps for problems sorted by block count (descending); returns the host map
static std::vector<int2> gj_build_maps(const std::vector<int>& nbs, GjMaps& g) {
    std::vector<int2> h;
    const int nbmax = nbs.empty() ? 0 : nbs[0];
    for (int k = 0; k < nbmax; ++k) {
        int m = 0;
        while (m < (int)nbs.size() && nbs[m] > k) ++m;
        g.piv.push_back(m);
        g.row_off.push_back((int)h.size());
        for (int p = 0; p < m; ++p)
            for (int r = 0; r < nbs[p]; ++r)
                if (r != k) h.push_back(make_int2(p, r));
        g.row_n.push_back((int)h.size() - g.row_off.back());
        g.upd_off.push_back((int)h.size());
        for (int p = 0; p < m; ++p)
            for (int i = 0; i < nbs[p]; ++i)
                if (i != k)
                    for (int j = 0; j < nbs[p]; ++j) h.push_back(make_int2(p, (i << 16) | j));
        g.upd_n.push_back((int)h.size() - g.upd_off.back());
    }
    return h;
}

template <typename T>
static int gj_launch_maps(const void* tab, int nprob, const GjMaps& g, int num_sms, cudaStream_t s) {
    const GjArgs<T>* t = (const GjArgs<T>*)tab;
    const int nbmax = (int)g.piv.size();
    const long long NN = (long long)nbmax * kGjB * nbmax * kGjB;
    const int gx = (int)std::max<long long>(1, std::min<long long>((NN + 255) / 256, (8LL * num_sms + nprob - 1) / nprob));
    k_gj_init<T><<<dim3(gx, nprob), 256, 0, s>>>(t);
    for (int k = 0; k < nbmax; ++k) {
        k_gj_pivot<T><<<g.piv[k], dim3(kGjB, kGjB), 0, s>>>(t, k);
        if (g.row_n[k] > 0) k_gj_row_map<T><<<g.row_n[k], dim3(kGjB, 8), 0, s>>>(t, g.map + g.row_off[k], k);
        if (g.upd_n[k] > 0) k_gj_update_map<T><<<g.upd_n[k], dim3(kGjB, 8), 0, s>>>(t, g.map + g.upd_off[k], k);
    }
    k_gj_final<T><<<dim3(gx, nprob), 256, 0, s>>>(t);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

// the blocked inversion of nprob problems' coarsest operators (largest nbmax blocks)
template <typename T>
static int gj_launch(const void* tab, int nprob, int nbmax, int num_sms, cudaStream_t s) {
    const GjArgs<T>* t = (const GjArgs<T>*)tab;
    const long long NN = (long long)nbmax * kGjB * nbmax * kGjB;
    const int gx = (int)std::max<long long>(1, std::min<long long>((NN + 255) / 256, (8LL * num_sms + nprob - 1) / nprob));
    k_gj_init<T><<<dim3(gx, nprob), 256, 0, s>>>(t);
    for (int k = 0; k < nbmax; ++k) {
        k_gj_pivot<T><<<nprob, dim3(kGjB, kGjB), 0, s>>>(t, k);
        k_gj_row<T><<<dim3(nbmax, nprob), dim3(kGjB, 8), 0, s>>>(t, k);
        k_gj_update<T><<<dim3(nbmax * nbmax, nprob), dim3(kGjB, 8), 0, s>>>(t, k, nbmax);
    }
    k_gj_final<T><<<dim3(gx, nprob), 256, 0, s>>>(t);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

// one problem's blocked-inversion table entry (work buffers from gj_work)
template <typename T>
static GjArgs<T> gj_args(const to_problem* P) {
    GjArgs<T> g;
    g.n = P->n_coarse;
    g.nb = (P->n_coarse + kGjB - 1) / kGjB;
    const size_t N = (size_t)g.nb * kGjB;
    g.A = (const T*)P->coarse_A;
    g.W = (T*)P->gj_work;
    g.C = g.W + N * N;
    g.P = g.C + N * kGjB;
    g.inv = (T*)P->coarse_L;
    g.err = &P->sc->err;
    return g;
}

// x = S Ainv S b   (one CTA per row block)
template <typename T>
__global__ void k_dense_solve(const T* __restrict__ Ainv, const T* __restrict__ sc, const T* __restrict__ b,
                              T* __restrict__ x, int n) {
    const int i = blockIdx.x * blockDim.y + threadIdx.y;
    if (i >= n) return;
    T acc = T(0);
    for (int j = threadIdx.x; j < n; j += 32) acc += Ainv[(long long)i * n + j] * sc[j] * b[j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) x[i] = sc[i] * acc;
}

// ----------------------------------------------------------------------------- the coarse tail on one CTA
// Below about a thousand elements a level's sweep costs far less than a kernel
// launch.  The V-cycle from the first such level down (its smoothing, residual,
// restriction, the dense coarsest solve, prolongation and post-smoothing) then
// runs in one CTA, with a barrier between steps.  Its operator is element-
// parallel: each thread applies the element matrix of its elements (the same
// Haar factorisation as the operator kernel) into shared memory, then each node
// adds the contributions of its (up to 8) elements in a fixed order.
constexpr int kTailMaxLevels = 8;
template <typename T>
constexpr int tail_threads() { return 512; }   // measured: 1024 FP32 threads are no faster (longer start-up)
constexpr int kTailMaxElems = 1024;
constexpr size_t kTailSmem = 220 * 1024;

// q = n / d without a divide: q = mulhi(n, m) with m = ceil(2^32 / d), exact
// whenever n * d < 2^32 (division by invariant integers using multiplication,
// Granlund and Montgomery 1994: with n = q d + r and m d = 2^32 + e, 0 <= e < d,
// n m / 2^32 = q + (r + n e / 2^32) / d and r + n e / 2^32 < r + 1 <= d).
// m = 0 stands for d = 1.
struct FastDiv {
    unsigned d, m;
};
inline FastDiv make_fast_div(unsigned d) {
    FastDiv f;
    f.d = d;
    f.m = d > 1 ? (unsigned)(((1ull << 32) + d - 1) / d) : 0u;
    return f;
}
__device__ __forceinline__ unsigned fdiv(unsigned n, FastDiv f) { return f.m ? __umulhi(n, f.m) : n; }

// one level of the tail: its arrays live in shared memory for the whole kernel
template <typename T>
struct TailLevel {
    int nx, ny, nz;
    FastDiv ex, exy, nxd, nxyd;   // element and node index divisors: nx, nx ny, nx+1, (nx+1)(ny+1)
    const T* E;
    const T* dinv;   // 1 / diag(K^) of the level
    const uint8_t* mask;
    T* x;
    T* b;
    T* t;
    T escale;   // h_level / h_0 = 2^level (exact): the level's K_e is escale times the finest one
};

// global arrays of a level and the byte offsets of its shared-memory copies
template <typename T>
struct TailGlobal {
    int nx, ny, nz;
    FastDiv ex, exy, nxd, nxyd;
    const T* E;
    const T* dinv;
    const uint8_t* mask;
    T* x;              // level 0 of the tail: the result goes back here
    const T* b;        // level 0: the right-hand side
    const T* first;    // level 0: its first sweep (written with the restriction)
    unsigned oE, od, omask, ox, ot, ob;
    T escale;
};

template <typename T>
struct TailArgs {
    int nlev;            // levels in the tail, the last one the coarsest (dense solve)
    int nu1, nu2;
    T omega;
    const T* inv;        // n_c x n_c scaled inverse, then the n_c scale factors
    int n_c;
    int inv_smem;        // the inverse (and scale factors) fit in the contribution buffer
    unsigned ocontrib;   // byte offset of the element contributions
    TailGlobal<T> lv[kTailMaxLevels];
};

// copy `bytes` from global to shared memory: 16-byte asynchronous copies where
// both ends allow, the rest by plain loads; completed by cp_async_wait_all()
__device__ __forceinline__ void tail_stage(void* dst, const void* src, unsigned bytes) {
    unsigned done = 0;
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
        const unsigned n16 = bytes >> 4;
        const unsigned base = (unsigned)__cvta_generic_to_shared(dst);
        for (unsigned q = threadIdx.x; q < n16; q += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(base + 16 * q),
                         "l"(static_cast<const char*>(src) + 16 * (size_t)q));
        done = n16 << 4;
    }
    for (unsigned q = done + threadIdx.x; q < bytes; q += blockDim.x)
        static_cast<unsigned char*>(dst)[q] = static_cast<const unsigned char*>(src)[q];
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// y = x + omega D^-1 (b - K^ x) (smooth) or y = b - K^ x on one level; `contrib`
// holds 24 values per element (component-major: [24][ne]).  Inside the tail x is
// zero on every fixed DOF (the restricted right-hand sides are, each sweep maps
// (x, b) = (0, 0) there to 0, and the prolongation skips those DOFs), so
// K^ x = K x on the free DOFs and the element gather needs no mask.
template <typename T>
__device__ __forceinline__ void tail_operator(const TailLevel<T>& Lv, const HaarK<T>& kh, const T* x, T* y, bool smooth,
                                              T omega, T* contrib) {
    const int nx = Lv.nx, ny = Lv.ny, nz = Lv.nz, nxn = nx + 1, nyn = ny + 1;
    const int ne = nx * ny * nz, nn = nxn * nyn * (nz + 1);
    const int pl = nxn * nyn;
    const int off[8] = {0, 1, 1 + nxn, nxn, pl, 1 + pl, 1 + nxn + pl, nxn + pl};   // local node -> node offset
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        const int q = (int)fdiv((unsigned)e, Lv.ex), k = (int)fdiv((unsigned)e, Lv.exy);
        const int i = e - q * nx, j = q - k * ny;
        const int n0 = i + nxn * (j + nyn * k);
        T u[24];
#pragma unroll
        for (int l = 0; l < 8; ++l)
#pragma unroll
            for (int c = 0; c < 3; ++c) u[3 * l + c] = x[3 * (n0 + off[l]) + c];
        T yv[24];
        elem_apply_haar(kh.v, Lv.E[e] * Lv.escale, u, yv);
#pragma unroll
        for (int r = 0; r < 24; ++r) contrib[r * ne + e] = yv[r];
    }
    __syncthreads();
    constexpr int kNode[2][2][2] = {{{0, 4}, {3, 7}}, {{1, 5}, {2, 6}}};
    for (int n = threadIdx.x; n < nn; n += blockDim.x) {
        const int q = (int)fdiv((unsigned)n, Lv.nxd), k = (int)fdiv((unsigned)n, Lv.nxyd);
        const int i = n - q * nxn, j = q - k * nyn;
        const int e0 = (i - 1) + nx * ((j - 1) + ny * (k - 1));   // element (i-1, j-1, k-1)
        T kx[3] = {T(0), T(0), T(0)};
        // the elements (i-1+a, j-1+b, k-1+c) around the node, in a fixed order
#pragma unroll
        for (int cc = 0; cc < 2; ++cc)
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                for (int aa = 0; aa < 2; ++aa) {
                    const bool in = (aa ? i < nx : i > 0) && (bb ? j < ny : j > 0) && (cc ? k < nz : k > 0);
                    if (!in) continue;
                    const int e = e0 + aa + nx * (bb + ny * cc);
                    const int l = kNode[1 - aa][1 - bb][1 - cc];
#pragma unroll
                    for (int c = 0; c < 3; ++c) kx[c] += contrib[(3 * l + c) * ne + e];
                }
        const uint8_t m = Lv.mask[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T xv = x[3 * n + c], bv = Lv.b[3 * n + c];
            const T K = ((m >> c) & 1) ? xv : kx[c];   // K^ is the identity on fixed DOFs
            y[3 * n + c] = smooth ? xv + omega * (bv - K) * Lv.dinv[3 * n + c] : bv - K;
        }
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void tail_body(const TailArgs<T>& a, const HaarK<T>& kh, unsigned char* tsm) {
    T* contrib = reinterpret_cast<T*>(tsm + a.ocontrib);
    TailLevel<T> lv[kTailMaxLevels];
    T* cur[kTailMaxLevels];
    // stage every level's moduli, inverse diagonal and mask (and the top level's right-hand side
    // and first sweep) in shared memory: all copies in flight at once
    const bool even = (a.nu1 - 1 + a.nu2) % 2 == 0;   // the first target, so that the last sweep writes x
    for (int t = 0; t < a.nlev; ++t) {
        const TailGlobal<T>& G = a.lv[t];
        TailLevel<T>& L = lv[t];
        L.nx = G.nx;
        L.ny = G.ny;
        L.nz = G.nz;
        L.ex = G.ex;
        L.exy = G.exy;
        L.nxd = G.nxd;
        L.nxyd = G.nxyd;
        L.escale = G.escale;
        T* E = reinterpret_cast<T*>(tsm + G.oE);
        T* d = reinterpret_cast<T*>(tsm + G.od);
        uint8_t* m = tsm + G.omask;
        L.E = E;
        L.dinv = d;
        L.mask = m;
        L.x = reinterpret_cast<T*>(tsm + G.ox);
        L.t = reinterpret_cast<T*>(tsm + G.ot);
        L.b = reinterpret_cast<T*>(tsm + G.ob);
        const unsigned ne = G.nx * G.ny * G.nz, nn = (G.nx + 1) * (G.ny + 1) * (G.nz + 1);
        if (t + 1 < a.nlev) {
            tail_stage(E, G.E, ne * sizeof(T));
            tail_stage(d, G.dinv, 3 * nn * sizeof(T));
        }
        tail_stage(m, G.mask, nn);
        if (t == 0) {
            tail_stage(L.b, G.b, 3 * nn * sizeof(T));
            tail_stage(even ? L.x : L.t, G.first, 3 * nn * sizeof(T));
        }
    }
    cp_async_wait_all();
    __syncthreads();
    const TailLevel<T>* tl = lv;
    // down: the first sweep of lv[0] came with its restriction, later ones come from ours
    for (int t = 0; t + 1 < a.nlev; ++t) {
        const TailLevel<T>& F = tl[t];
        const TailLevel<T>& C = tl[t + 1];
        T* c = even ? F.x : F.t;
        T* o = even ? F.t : F.x;
        for (int it = 1; it < a.nu1; ++it) {
            tail_operator<T>(F, kh, c, o, true, a.omega, contrib);
            T* sw = c;
            c = o;
            o = sw;
        }
        tail_operator<T>(F, kh, c, o, false, a.omega, contrib);
        // before the last restriction: the coarsest inverse starts its way into the
        // (now idle) contribution buffer
        if (t + 2 == a.nlev && a.inv_smem) tail_stage(contrib, a.inv, (unsigned)((a.n_c + 1) * a.n_c * sizeof(T)));
        T* xc = t + 2 < a.nlev ? (even ? C.x : C.t) : nullptr;
        const int X = C.nx + 1, nnc = X * (C.ny + 1) * (C.nz + 1);
        for (int n = threadIdx.x; n < nnc; n += blockDim.x) {
            const int q = (int)fdiv((unsigned)n, C.nxd), K = (int)fdiv((unsigned)n, C.nxyd);
            restrict_node<T, int, true>(C.nx, C.ny, C.nz, n - q * X, q - K * (C.ny + 1), K, o, F.mask, C.mask, C.b, C.dinv,
                                        xc, a.omega);
        }
        __syncthreads();
        cur[t] = c;
    }
    // the coarsest level: x = S A^-1 S b, one warp per row (lane-strided sums, shuffle tree);
    // s_j b_j first, then eight columns per lane in flight
    {
        const TailLevel<T>& Cst = tl[a.nlev - 1];
        const int n = a.n_c, lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        if (a.inv_smem) cp_async_wait_all();
        const T* inv = a.inv_smem ? contrib : a.inv;
        const T* sc = inv + (size_t)n * n;
        T* sb = Cst.t;
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) sb[j] = sc[j] * Cst.b[j];
        __syncthreads();
        for (int i = wid; i < n; i += nw) {
            const T* row = inv + (size_t)i * n;
            T acc = T(0);
            for (int j0 = 0; j0 < n; j0 += 8 * 32) {
                T v[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int j = j0 + 32 * r + lane;
                    v[r] = j < n ? row[j] : T(0);
                }
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int j = j0 + 32 * r + lane;
                    acc += j < n ? v[r] * sb[j] : T(0);
                }
            }
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) Cst.x[i] = sc[i] * acc;
        }
        __syncthreads();
    }
    // up
    for (int t = a.nlev - 2; t >= 0; --t) {
        const TailLevel<T>& F = tl[t];
        const TailLevel<T>& C = tl[t + 1];
        T* c = cur[t];
        T* o = c == F.x ? F.t : F.x;
        const int X = F.nx + 1, nnf = X * (F.ny + 1) * (F.nz + 1);
        for (int n = threadIdx.x; n < nnf; n += blockDim.x) {
            const int q = (int)fdiv((unsigned)n, F.nxd), k = (int)fdiv((unsigned)n, F.nxyd);
            prolong_node<T, int>(C.nx, C.ny, C.nz, n - q * X, q - k * (F.ny + 1), k, C.x, C.mask, F.mask, c);
        }
        __syncthreads();
        for (int it = 0; it < a.nu2; ++it) {
            tail_operator<T>(F, kh, c, o, true, a.omega, contrib);
            T* sw = c;
            c = o;
            o = sw;
        }
    }
    // the top level's correction back to global memory
    const TailGlobal<T>& G = a.lv[0];
    const int nn = (G.nx + 1) * (G.ny + 1) * (G.nz + 1);
    for (int q = threadIdx.x; q < 3 * nn; q += blockDim.x) G.x[q] = tl[0].x[q];
}

template <typename T>
__global__ void __launch_bounds__(tail_threads<T>()) k_mg_tail(const TailArgs<T> a, const HaarK<T> kh) {
    extern __shared__ __align__(16) unsigned char tsm[];
    tail_body<T>(a, kh, tsm);
}

// ----------------------------------------------------------------------------- host side

// shared-memory layout of the tail from level l0: per level E, d, mask, x, t, b, then
// the element contributions of level l0; returns the total bytes
template <typename T>
static size_t tail_layout(const to_problem* P, int l0, TailArgs<T>* a) {
    const int L = (int)P->lv.size();
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 15) & ~(size_t)15;
        return (unsigned)o;
    };
    for (int t = 0; t < L - l0 && t < kTailMaxLevels; ++t) {
        const Level& F = P->lv[l0 + t];
        const size_t nn = (size_t)F.n_node, ne = (size_t)F.n_elem;
        const unsigned oE = take(ne * sizeof(T)), od = take(3 * nn * sizeof(T)), om = take(nn),
                       ox = take(3 * nn * sizeof(T)), ot = take(3 * nn * sizeof(T)), ob = take(3 * nn * sizeof(T));
        if (a) {
            TailGlobal<T>& g = a->lv[t];
            g.nx = F.nx;
            g.ny = F.ny;
            g.nz = F.nz;
            g.ex = make_fast_div((unsigned)F.nx);
            g.exy = make_fast_div((unsigned)(F.nx * F.ny));
            g.nxd = make_fast_div((unsigned)(F.nx + 1));
            g.nxyd = make_fast_div((unsigned)((F.nx + 1) * (F.ny + 1)));
            g.E = (const T*)F.E;
            g.dinv = (const T*)F.dinv;
            g.mask = F.mask;
            g.x = (T*)F.x;
            g.b = (const T*)F.b;
            g.first = (const T*)((((P->prm.mg_nu_pre - 1 + P->prm.mg_nu_post) % 2) == 0) ? F.x : F.t);
            g.oE = oE;
            g.od = od;
            g.omask = om;
            g.ox = ox;
            g.ot = ot;
            g.ob = ob;
            g.escale = (T)(F.h / P->g.h);
        }
    }
    const unsigned oc = take((size_t)24 * P->lv[l0].n_elem * sizeof(T));
    if (a) a->ocontrib = oc;
    return off;
}



static int auto_levels(int nx, int ny, int nz) {
    int t = 0;
    while (nx % (2 << t) == 0 && ny % (2 << t) == 0 && nz % (2 << t) == 0 && std::min(nx, std::min(ny, nz)) / (2 << t) >= 2)
        ++t;
    return t + 1;
}

int mg_build(to_problem* P) {
    const int Lmax = auto_levels(P->g.nx, P->g.ny, P->g.nz);
    int L = P->prm.mg_levels > 0 ? P->prm.mg_levels : Lmax;
    if (L > Lmax) return fail(TO_ERR_ARG, "mg_levels exceeds the number of times the grid can be halved");
    if (P->prm.mg_nu_pre < 1 || P->prm.mg_nu_post < 0 || !(P->prm.mg_omega > 0.0))
        return fail(TO_ERR_ARG, "multigrid needs nu_pre >= 1, nu_post >= 0, omega > 0");
    const size_t es = P->esz;
    // coarse masks on the host (conservative rule, see the file comment)
    std::vector<uint8_t> mf((size_t)P->n_node);
    if (cudaMemcpy(mf.data(), P->lv[0].mask, mf.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(TO_ERR_CUDA, "mask download");
    for (int l = 1; l < L; ++l) {
        const Level& F = P->lv[l - 1];
        Level C{};
        C.nx = F.nx / 2; C.ny = F.ny / 2; C.nz = F.nz / 2;
        C.n_elem = (int64_t)C.nx * C.ny * C.nz;
        C.n_node = (int64_t)(C.nx + 1) * (C.ny + 1) * (C.nz + 1);
        C.n_dof = 3 * C.n_node;
        C.h = F.h * 2.0;
        C.kdiag = F.kdiag * 2.0;
        std::vector<uint8_t> mc((size_t)C.n_node, 0);
        for (int K = 0; K <= C.nz; ++K)
            for (int J = 0; J <= C.ny; ++J)
                for (int I = 0; I <= C.nx; ++I) {
                    uint8_t m = 0;
                    for (int k = std::max(2 * K - 1, 0); k <= std::min(2 * K + 1, F.nz); ++k)
                        for (int j = std::max(2 * J - 1, 0); j <= std::min(2 * J + 1, F.ny); ++j)
                            for (int i = std::max(2 * I - 1, 0); i <= std::min(2 * I + 1, F.nx); ++i)
                                m |= mf[(size_t)i + (size_t)(F.nx + 1) * ((size_t)j + (size_t)(F.ny + 1) * k)];
                    mc[(size_t)I + (size_t)(C.nx + 1) * ((size_t)J + (size_t)(C.ny + 1) * K)] = m;
                }
        void *E = nullptr, *d = nullptr, *mk = nullptr, *x = nullptr, *b = nullptr, *t = nullptr;
        cudaError_t e = cudaMalloc(&E, C.n_elem * es);
        if (e == cudaSuccess) e = cudaMalloc(&d, C.n_dof * es);
        if (e == cudaSuccess) e = cudaMalloc(&mk, ((size_t)C.n_node + 7) & ~(size_t)3);   // read as 4-byte words
        if (e == cudaSuccess) e = cudaMemset(mk, 0, ((size_t)C.n_node + 7) & ~(size_t)3);
        if (e == cudaSuccess) e = cudaMalloc(&x, C.n_dof * es);
        if (e == cudaSuccess) e = cudaMalloc(&b, C.n_dof * es);
        if (e == cudaSuccess) e = cudaMalloc(&t, C.n_dof * es);
        C.E = E; C.dinv = d; C.mask = (uint8_t*)mk; C.x = x; C.b = b; C.t = t;
        P->lv.push_back(C);
        if (e != cudaSuccess) return fail(TO_ERR_CUDA, std::string("multigrid allocation: ") + cudaGetErrorString(e));
        if (cudaMemcpy(mk, mc.data(), mc.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(TO_ERR_CUDA, "mask upload");
        if (int rc2 = build_tile_mask(P->lv.back(), mc.data())) return rc2;
        mf.swap(mc);
    }
    const Level& Cst = P->lv.back();
    const int n = (int)Cst.n_dof;
    if (n > kMaxCoarseDof)
        return fail(TO_ERR_ARG, "coarsest multigrid grid too large for the dense solve (" + std::to_string(n) +
                                    " DOFs > " + std::to_string(kMaxCoarseDof) + "): use a grid that halves more often");
    P->n_coarse = n;
    if (cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&P->ev_ljoin, cudaEventDisableTiming) != cudaSuccess)
        return fail(TO_ERR_CUDA, "multigrid stream / event creation failed");
    if (cudaMalloc(&P->coarse_A, (size_t)n * n * es) != cudaSuccess ||
        cudaMalloc(&P->coarse_L, (size_t)n * n * es + (size_t)n * es) != cudaSuccess)
        return fail(TO_ERR_CUDA, "coarse allocation");
    void* ked = nullptr;
    if (cudaMalloc(&ked, 576 * sizeof(double)) != cudaSuccess ||
        cudaMemcpy(ked, P->ke, 576 * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(TO_ERR_CUDA, "element matrix upload");
    P->ke_dev = (double*)ked;
    // level-0 V-cycle scratch
    if (cudaMalloc(&P->lv[0].t, P->n_dof * es) != cudaSuccess) return fail(TO_ERR_CUDA, "scratch allocation");
    if (n > kRegDof) {   // the blocked inversion's work matrix, block column and pivot block, and its table
        const size_t N = (size_t)((n + kGjB - 1) / kGjB) * kGjB;
        if (cudaMalloc(&P->gj_work, (N * N + N * kGjB + (size_t)kGjB * kGjB) * es) != cudaSuccess ||
            cudaMalloc(&P->gj_tab, P->prec == TO_FP64 ? sizeof(GjArgs<double>) : sizeof(GjArgs<float>)) != cudaSuccess)
            return fail(TO_ERR_CUDA, "coarse inversion scratch allocation");
        cudaError_t e;
        if (P->prec == TO_FP64) {
            const GjArgs<double> g = gj_args<double>(P);
            e = cudaMemcpy(P->gj_tab, &g, sizeof(g), cudaMemcpyHostToDevice);
        } else {
            const GjArgs<float> g = gj_args<float>(P);
            e = cudaMemcpy(P->gj_tab, &g, sizeof(g), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return fail(TO_ERR_CUDA, "coarse inversion table upload");
    }
    // the coarse tail: from the first level (>= 1, above the coarsest) with at most
    // kTailMaxElems elements whose levels fit in shared memory
    P->mg_tail = 0;
    for (int l = 1; l + 1 < L && L - l <= kTailMaxLevels; ++l) {
        if (P->lv[l].n_elem > kTailMaxElems) continue;
        if ((unsigned long long)P->lv[l].n_node * (unsigned long long)P->lv[l].n_node >= (1ull << 32)) continue;   // FastDiv range
        const size_t tsm = P->prec == TO_FP64 ? tail_layout<double>(P, l, nullptr) : tail_layout<float>(P, l, nullptr);
        if (tsm > kTailSmem) continue;   // FP64 at ~1024 elements: start one level coarser
        cudaError_t e = P->prec == TO_FP64
                            ? cudaFuncSetAttribute(k_mg_tail<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmem)
                            : cudaFuncSetAttribute(k_mg_tail<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmem);
        // (the attribute is per kernel, shared by every problem: the cap, not this problem's size)
        if (e != cudaSuccess) return fail(TO_ERR_CUDA, std::string("shared memory opt-in: ") + cudaGetErrorString(e));
        P->mg_tail = l;
        break;
    }
    return TO_OK;
}

// every coarse level's moduli and 1 / d, and the coarsest level's dense operator (gate:
// each kernel returns at once where gate[0] != gate[1])
template <typename T>
static int refresh_levels_t(to_problem* P, cudaStream_t s, const unsigned* gate) {
    const int L = (int)P->lv.size();
    for (int l = 1; l < L; ++l) {
        const Level& C = P->lv[l];
        k_coarsen_E<T><<<grid3(C.nx, C.ny, C.nz), block3(), 0, s>>>(C.nx, C.ny, C.nz, (const T*)P->lv[l - 1].E, (T*)C.E,
                                                                    gate);
        TO_CUDA(cudaGetLastError());
        int rc = launch_diag(P, l, s, gate);
        if (rc) return rc;
    }
    const Level& Cst = P->lv.back();
    const int n = P->n_coarse;
    k_dense_assemble<T><<<grid1((long long)n * n, P->num_sms), 256, 0, s>>>(
        Cst.nx, Cst.ny, Cst.nz, (const T*)Cst.E, Cst.mask, P->ke_dev, Cst.h, (T*)P->coarse_A, n, gate);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

// the inverse of the coarsest operator (a gate only for the one-CTA register inverse)
template <typename T>
static int refresh_inverse_t(to_problem* P, cudaStream_t s, const unsigned* gate) {
    const int n = P->n_coarse;
    T* inv = (T*)P->coarse_L;
    if (n <= kRegDof) {
        k_dense_invert_reg<T><<<1, dim3(32, 32), 0, s>>>((const T*)P->coarse_A, inv, inv + (size_t)n * n, n, &P->sc->err,
                                                        gate);
        TO_CUDA(cudaGetLastError());
        return TO_OK;
    }
    if (gate) return fail(TO_ERR_STATE, "the blocked coarsest inversion has no gate");
    return gj_launch<T>(P->gj_tab, 1, (n + kGjB - 1) / kGjB, P->num_sms, s);
}

template <typename T>
static int refresh_t(to_problem* P, cudaStream_t s, bool join, bool inline_inv) {
    if (int rc = refresh_levels_t<T>(P, s, nullptr)) return rc;
    // the inverse runs on a branch; the first coarse solve joins it (it is needed only
    // there) -- unless s is itself a branch that the caller joins (inline_inv)
    cudaStream_t main_s = s;
    if (!inline_inv) {
        TO_CUDA(cudaEventRecord(P->ev_fork, s));
        TO_CUDA(cudaStreamWaitEvent(P->side, P->ev_fork, 0));
        s = P->side;
    }
    if (int rc = refresh_inverse_t<T>(P, s, nullptr)) return rc;
    if (inline_inv) return TO_OK;
    TO_CUDA(cudaEventRecord(P->ev_join, s));
    // outside the outer iteration nothing else joins the branch: without this a later
    // refresh could rewrite coarse_A / coarse_L while this inverse still runs
    if (join) TO_CUDA(cudaStreamWaitEvent(main_s, P->ev_join, 0));
    P->coarse_wait = join ? 0 : 1;   // the coarse solves on main_s join it
    return TO_OK;
}

int mg_refresh_levels(to_problem* P, cudaStream_t s, const unsigned* gate) {
    return P->prec == TO_FP64 ? refresh_levels_t<double>(P, s, gate) : refresh_levels_t<float>(P, s, gate);
}

int mg_refresh_inverse(to_problem* P, cudaStream_t s, const unsigned* gate) {
    return P->prec == TO_FP64 ? refresh_inverse_t<double>(P, s, gate) : refresh_inverse_t<float>(P, s, gate);
}

bool mg_refresh_gatable(const to_problem* P) { return P->n_coarse <= kRegDof; }

int mg_refresh(to_problem* P, cudaStream_t s, bool join, bool inline_inv) {
    return P->prec == TO_FP64 ? refresh_t<double>(P, s, join, inline_inv) : refresh_t<float>(P, s, join, inline_inv);
}

// The second set of design-dependent buffers: rho~, E', every level's moduli and 1 / d,
// the coarsest inverse (with its own inversion table; the work matrix is shared, as only
// one inversion runs at a time).  Allocated on the first pipelined outer iteration.
int pipe_alloc(to_problem* P) {
    if (P->alt_alloc) return TO_OK;
    const size_t es = P->esz;
    const int L = (int)P->lv.size();
    P->alt_E.assign(L, nullptr);
    P->alt_dinv.assign(L, nullptr);
    bool ok = cudaMalloc(&P->alt_rhot, P->n_elem * es) == cudaSuccess && cudaMalloc(&P->alt_Ed, P->n_elem * es) == cudaSuccess;
    for (int l = 0; l < L && ok; ++l)
        ok = cudaMalloc(&P->alt_E[l], P->lv[l].n_elem * es) == cudaSuccess &&
             cudaMalloc(&P->alt_dinv[l], P->lv[l].n_dof * es) == cudaSuccess;
    const size_t n = (size_t)P->n_coarse;
    if (ok && P->coarse_L) ok = cudaMalloc(&P->alt_coarse_L, (n * n + n) * es) == cudaSuccess;
    if (ok && P->gj_tab) {
        std::swap(P->coarse_L, P->alt_coarse_L);   // the table of the other set's inverse
        if (P->prec == TO_FP64) {
            const GjArgs<double> g = gj_args<double>(P);
            ok = cudaMalloc(&P->alt_gj_tab, sizeof g) == cudaSuccess &&
                 cudaMemcpy(P->alt_gj_tab, &g, sizeof g, cudaMemcpyHostToDevice) == cudaSuccess;
        } else {
            const GjArgs<float> g = gj_args<float>(P);
            ok = cudaMalloc(&P->alt_gj_tab, sizeof g) == cudaSuccess &&
                 cudaMemcpy(P->alt_gj_tab, &g, sizeof g, cudaMemcpyHostToDevice) == cudaSuccess;
        }
        std::swap(P->coarse_L, P->alt_coarse_L);
    }
    P->alt_alloc = 1;   // whatever was allocated is freed with the problem
    if (!ok) {
        P->alt_alloc = 2;   // unusable: the pipelined iteration stays off
        return fail(TO_ERR_CUDA, "allocation of the second design set");
    }
    return TO_OK;
}

void pipe_swap(to_problem* P) {
    std::swap(P->rhot, P->alt_rhot);
    std::swap(P->Ed, P->alt_Ed);
    for (size_t l = 0; l < P->lv.size(); ++l) {
        std::swap(P->lv[l].E, P->alt_E[l]);
        std::swap(P->lv[l].dinv, P->alt_dinv[l]);
    }
    std::swap(P->coarse_L, P->alt_coarse_L);
    std::swap(P->gj_tab, P->alt_gj_tab);
    P->set_parity ^= 1;
}

// levels mg_tail .. L-1 in one launch (after the coarsest inverse is ready)
template <typename T>
static int tail_args(to_problem* P, int l0, TailArgs<T>* a);

template <typename T>
static int tail_t(to_problem* P, cudaStream_t s) {
    TailArgs<T> a;
    const size_t tsm = (size_t)tail_args<T>(P, P->mg_tail, &a);
    HaarK<T> kh;
    for (int q = 0; q < kHaarNnz; ++q) kh.v[q] = (T)P->haar[q];
    if (P->coarse_wait) TO_CUDA(cudaStreamWaitEvent(s, P->ev_join, 0));   // the inverse of this design is ready
    k_mg_tail<T><<<1, tail_threads<T>(), tsm, s>>>(a, kh);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

template <typename T>
static int coarse_solve_t(to_problem* P, const void* b, void* x, cudaStream_t s) {
    const int n = P->n_coarse;
    if (P->coarse_wait) TO_CUDA(cudaStreamWaitEvent(s, P->ev_join, 0));   // the inverse of this design is ready
    const T* inv = (const T*)P->coarse_L;
    k_dense_solve<T><<<(n + 7) / 8, dim3(32, 8), 0, s>>>(inv, inv + (size_t)n * n, (const T*)b, (T*)x, n);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

// x_l = V(l, b_l); the result lands in `x`, `t` is scratch of the same size
template <typename T>
static int vcycle_t(to_problem* P, int l, const void* b, void* x, void* t, cudaStream_t s, bool first_done = false) {
    const int L = (int)P->lv.size();
    const Level& F = P->lv[l];
    if (l == L - 1) return coarse_solve_t<T>(P, b, x, s);
    const int nu1 = P->prm.mg_nu_pre, nu2 = P->prm.mg_nu_post;
    const double om = P->prm.mg_omega;
    int rc;
    // choose the first target so that the last sweep writes into x
    void* cur = ((nu1 - 1 + nu2) % 2 == 0) ? x : t;
    void* oth = cur == x ? t : x;
    if (std::is_same<T, float>::value && first_done && mg_cluster_applicable(P, l)) {
        // this level (just above the tail) in one cluster: the down leg from the first sweep
        // in cur, the tail, the up leg into x; the buffers end as in the launched steps
        const int npre = nu1 - 1;
        void* it_buf = (npre % 2 == 0) ? cur : oth;   // the iterate after the pre-smoothing
        void* other = it_buf == cur ? oth : cur;
        void* fin = (nu2 % 2 == 0) ? it_buf : other;
        if (fin != x) return fail(TO_ERR_STATE, "V-cycle buffer parity");
        const Level& C = P->lv[l + 1];
        void* cfirst = ((nu1 - 1 + nu2) % 2 == 0) ? C.x : C.t;
        if ((rc = mg_cluster_down(P, l, cur, it_buf, l + 1 < L - 1 ? cfirst : nullptr, s))) return rc;
        if ((rc = tail_t<T>(P, s))) return rc;
        return mg_cluster_up(P, l, it_buf, x, s);
    }
    if (!first_done) {
        k_jacobi_first<T><<<grid1(F.n_dof, P->num_sms), 256, 0, s>>>(F.n_dof, (const T*)b, (const T*)F.dinv, (T*)cur, (T)om);
        TO_CUDA(cudaGetLastError());
    }
    for (int it = 1; it < nu1; ++it) {
        if ((rc = launch_operator(P, l, OP_SMOOTH, cur, oth, b, s, om))) return rc;
        std::swap(cur, oth);
    }
    // residual into oth, restrict to the coarse right-hand side
    if ((rc = launch_operator(P, l, OP_BMINUS, cur, oth, b, s))) return rc;
    if (P->levels_wait) TO_CUDA(cudaStreamWaitEvent(s, P->ev_ljoin, 0));   // the coarse levels of this design are ready
    if (l == 0 && P->legs_grid > 0) {
        // levels 1 .. tail - 1 as two cooperative launches around the coarse tail
        if ((rc = mg_legs_launch(P, 0, oth, s))) return rc;
        if ((rc = tail_t<T>(P, s))) return rc;
        if ((rc = mg_legs_launch(P, 1, cur, s))) return rc;
        for (int it = 0; it < nu2; ++it) {
            const int flag = it == nu2 - 1 ? 2 : 0;   // r^T z of the lower-level step
            if ((rc = launch_operator(P, l, OP_SMOOTH, cur, oth, b, s, om, flag))) return rc;
            std::swap(cur, oth);
        }
        if (cur != x) return fail(TO_ERR_STATE, "V-cycle buffer parity");
        return TO_OK;
    }
    const Level& C = P->lv[l + 1];
    // above the coarsest level the restriction also takes the coarse level's first sweep
    const bool fuse = l + 1 < L - 1;
    void* cfirst = ((nu1 - 1 + nu2) % 2 == 0) ? C.x : C.t;
    const dim3 gr = grid3(C.nx + 1, C.ny + 1, C.nz + 1);
    if (F.n_dof < (1LL << 31))
        k_restrict<T, int><<<gr, block3(), 0, s>>>(C.nx, C.ny, C.nz, (const T*)oth, F.mask, C.mask, (T*)C.b,
                                                   (const T*)C.dinv, fuse ? (T*)cfirst : nullptr, (T)om);
    else
        k_restrict<T, long long><<<gr, block3(), 0, s>>>(C.nx, C.ny, C.nz, (const T*)oth, F.mask, C.mask, (T*)C.b,
                                                         (const T*)C.dinv, fuse ? (T*)cfirst : nullptr, (T)om);
    TO_CUDA(cudaGetLastError());
    if (P->mg_tail == l + 1) {
        if ((rc = tail_t<T>(P, s))) return rc;   // levels l+1 .. L-1 in one CTA
    } else if ((rc = vcycle_t<T>(P, l + 1, C.b, C.x, C.t, s, fuse))) {
        return rc;
    }
    const dim3 gp = grid3(F.nx + 1, F.ny + 1, F.nz + 1);
    if (F.n_dof < (1LL << 31))
        k_prolong_add<T, int><<<gp, block3(), 0, s>>>(C.nx, C.ny, C.nz, (const T*)C.x, C.mask, F.mask, (T*)cur);
    else
        k_prolong_add<T, long long><<<gp, block3(), 0, s>>>(C.nx, C.ny, C.nz, (const T*)C.x, C.mask, F.mask, (T*)cur);
    TO_CUDA(cudaGetLastError());
    for (int it = 0; it < nu2; ++it) {
        // on the fine level the last sweep also reduces b^T x (= r^T z of the lower-level step)
        const int flag = (l == 0 && it == nu2 - 1) ? 2 : 0;
        if ((rc = launch_operator(P, l, OP_SMOOTH, cur, oth, b, s, om, flag))) return rc;
        std::swap(cur, oth);
    }
    if (cur != x) return fail(TO_ERR_STATE, "V-cycle buffer parity");
    return TO_OK;
}

int mg_vcycle(to_problem* P, const void* r, void* z, cudaStream_t s) {
    return P->prec == TO_FP64 ? vcycle_t<double>(P, 0, r, z, P->lv[0].t, s)
                              : vcycle_t<float>(P, 0, r, z, P->lv[0].t, s);
}

// kernel launches of one V-cycle (for launch accounting)
int mg_launches(const to_problem* P) {
    const int L = (int)P->lv.size();
    const int nu1 = P->prm.mg_nu_pre, nu2 = P->prm.mg_nu_post;
    if (L == 1) return 1;
    const int host_levels = P->mg_tail > 0 ? P->mg_tail : L - 1;
    return 1 + host_levels * ((nu1 - 1) + 1 + 1 + 1 + nu2) + 1;   // + the dense solve or the tail kernel
}

// ----------------------------------------------------------------------------- batched multigrid
// The V-cycle and the per-iteration refresh of many problems, one launch per
// step: every batched kernel reads a table of per-problem arguments (blockIdx.y,
// or blockIdx.x for the one-CTA kernels) and grid-strides over that problem's
// nodes or elements.  The launch sequence replays the single-problem V-cycle
// (the same buffers, sweep order and reductions): levels above each problem's
// coarse tail one launch per step and level (problems whose tail starts higher
// sit those launches out), then every problem's tail in one launch, one CTA each.

int op_table_level(to_problem* const* probs, int n, int level, int mode, const void* const* x, void* const* y,
                   const void* const* b, double omega, int first, int kchunk, void** dev, int* max_tiles);
void* level_haar(const to_problem* P, int level);
int batch_operator_launch(int prec, int mode, const void* tab, const void* kh, int max_tiles, int n, cudaStream_t s);

template <typename T>
struct BmJac {          // x = omega b / d
    long long n;
    const T* b;
    const T* dinv;
    T* x;
    T omega;
};
template <typename T>
struct BmRestrict {     // b_c = m_c P^T (m_f t) and the coarse first sweep
    int cx, cy, cz;
    const T* tf;
    const uint8_t* mf;
    const uint8_t* mc;
    T* bc;
    const T* dinvc;
    T* xc;
    T omega;
};
template <typename T>
struct BmProlong {      // x_f += m_f P (m_c x_c)
    int cx, cy, cz;
    const T* xc;
    const uint8_t* mc;
    const uint8_t* mf;
    T* xf;
};
template <typename T>
struct BmLevel {        // a coarse level's moduli and inverse diagonal
    int nx, ny, nz;
    const T* Ef;
    T* E;
    const uint8_t* mask;
    T* dinv;
    double kdiag;
};
template <typename T>
struct BmDense {        // the coarsest level's dense operator and its inverse
    int nx, ny, nz, n;
    const T* E;
    const uint8_t* mask;
    const double* ke;
    double hscale;
    T* A;
    T* inv;             // n x n, then the n scale factors
    int* err;
};

template <typename T>
__global__ void __launch_bounds__(256) k_bm_jacobi_first(const BmJac<T>* __restrict__ tab) {
    const BmJac<T>& a = tab[blockIdx.y];
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < a.n; i += (long long)gridDim.x * 256)
        a.x[i] = a.omega * a.b[i] * a.dinv[i];
}

template <typename T>
__global__ void __launch_bounds__(256) k_bm_restrict(const BmRestrict<T>* __restrict__ tab) {
    const BmRestrict<T>& a = tab[blockIdx.y];
    const long long X = a.cx + 1, Y = a.cy + 1, nn = X * Y * (a.cz + 1);
    for (long long q = blockIdx.x * 256LL + threadIdx.x; q < nn; q += (long long)gridDim.x * 256)
        restrict_node<T, long long, true>(a.cx, a.cy, a.cz, (int)(q % X), (int)((q / X) % Y), (int)(q / (X * Y)), a.tf,
                                          a.mf, a.mc, a.bc, a.dinvc, a.xc, a.omega);
}

template <typename T>
__global__ void __launch_bounds__(256) k_bm_prolong(const BmProlong<T>* __restrict__ tab) {
    const BmProlong<T>& a = tab[blockIdx.y];
    const long long X = 2 * a.cx + 1, Y = 2 * a.cy + 1, nn = X * Y * (2 * a.cz + 1);
    for (long long q = blockIdx.x * 256LL + threadIdx.x; q < nn; q += (long long)gridDim.x * 256)
        prolong_node<T>(a.cx, a.cy, a.cz, (int)(q % X), (int)((q / X) % Y), (int)(q / (X * Y)), a.xc, a.mc, a.mf, a.xf);
}

template <typename T>
__global__ void __launch_bounds__(256) k_bm_coarsen(const BmLevel<T>* __restrict__ tab) {
    const BmLevel<T>& a = tab[blockIdx.y];
    const long long X = a.nx, Y = a.ny, ne = X * Y * a.nz;
    for (long long q = blockIdx.x * 256LL + threadIdx.x; q < ne; q += (long long)gridDim.x * 256)
        coarsen_elem<T>(a.nx, a.ny, (int)(q % X), (int)((q / X) % Y), (int)(q / (X * Y)), a.Ef, a.E);
}

template <typename T>
__global__ void __launch_bounds__(256) k_bm_diag(const BmLevel<T>* __restrict__ tab) {
    const BmLevel<T>& a = tab[blockIdx.y];
    const long long X = a.nx + 1, Y = a.ny + 1, nn = X * Y * (a.nz + 1);
    for (long long q = blockIdx.x * 256LL + threadIdx.x; q < nn; q += (long long)gridDim.x * 256)
        diag_node<T>(a.nx, a.ny, a.nz, (int)(q % X), (int)((q / X) % Y), (int)(q / (X * Y)), a.E, a.mask, a.dinv, a.kdiag);
}

template <typename T>
__global__ void __launch_bounds__(256) k_bm_assemble(const BmDense<T>* __restrict__ tab) {
    const BmDense<T>& a = tab[blockIdx.y];
    const long long nn = (long long)a.n * a.n;
    for (long long q = blockIdx.x * 256LL + threadIdx.x; q < nn; q += (long long)gridDim.x * 256)
        a.A[q] = dense_entry<T>(a.nx, a.ny, a.nz, a.E, a.mask, a.ke, a.hscale, a.n, q);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_bm_invert_reg(const BmDense<T>* __restrict__ tab) {
    const BmDense<T>& a = tab[blockIdx.x];
    dense_invert_reg_body<T>(a.A, a.inv, a.inv + (size_t)a.n * a.n, a.n, a.err);
}

template <typename T>
__global__ void __launch_bounds__(tail_threads<T>()) k_mg_tail_batch(const TailArgs<T>* __restrict__ tab, const HaarK<T> kh) {
    extern __shared__ __align__(16) unsigned char tsm[];
    tail_body<T>(tab[blockIdx.x], kh, tsm);
}

enum BmKind { BM_JAC, BM_OPER, BM_RESTRICT, BM_PROLONG, BM_TAIL, BM_COARSEN, BM_DIAG, BM_ASSEMBLE, BM_INVERT_REG,
              BM_INVERT_GJ };

struct BmOp {
    int kind = 0, mode = 0, n = 0, grid_x = 1, max_tiles = 0;
    void* tab = nullptr;        // device table
    const void* kh = nullptr;   // host element constants (operator and tail launches)
    size_t smem = 0;
    GjMaps gj;                  // BM_INVERT_GJ: the compact tile maps of its block steps
};

struct BatchMG {
    int prec = TO_FP32_MIXED, n = 0, num_sms = 1;
    std::vector<BmOp> refresh, vcycle;
    std::vector<void*> dev, host;
    // the coarsest operators' assembly and inversion run on a forked branch that the first
    // coarse tail joins, overlapping the fine-level work before it
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    mutable bool join_pending = false;
};

static int grid_x_for(long long items, int num_sms, int n) {
    // enough CTAs for the largest problem, about 8 per SM over the whole batch
    long long g = (items + 255) / 256;
    const long long cap = std::max<long long>(1, (8LL * num_sms + n - 1) / n);
    return (int)std::max<long long>(1, std::min(g, cap));
}

template <typename S>
static int upload_table(BatchMG* M, const std::vector<S>& h, void** out) {
    void* d = nullptr;
    if (cudaMalloc(&d, sizeof(S) * h.size()) != cudaSuccess) return fail(TO_ERR_CUDA, "batched multigrid table allocation");
    M->dev.push_back(d);
    if (cudaMemcpy(d, h.data(), sizeof(S) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(TO_ERR_CUDA, "batched multigrid table upload");
    *out = d;
    return TO_OK;
}

template <typename T>
static int tail_args(to_problem* P, int l0, TailArgs<T>* a) {
    const int L = (int)P->lv.size();
    *a = TailArgs<T>{};
    a->nlev = L - l0;
    a->nu1 = P->prm.mg_nu_pre;
    a->nu2 = P->prm.mg_nu_post;
    a->omega = (T)P->prm.mg_omega;
    a->inv = (const T*)P->coarse_L;
    a->n_c = P->n_coarse;
    a->inv_smem = (size_t)(a->n_c + 1) * a->n_c <= (size_t)24 * P->lv[l0].n_elem;
    return (int)tail_layout<T>(P, l0, a);
}

template <typename T>
static int batch_mg_build_t(to_problem* const* probs, int n, int kchunk, BatchMG* M) {
    const int nu1 = probs[0]->prm.mg_nu_pre, nu2 = probs[0]->prm.mg_nu_post;
    const double om = probs[0]->prm.mg_omega;
    const int num_sms = probs[0]->num_sms;
    const bool even = (nu1 - 1 + nu2) % 2 == 0;
    // each problem's tail: its one-CTA coarse tail, or (where none fits) the dense coarsest solve alone
    std::vector<int> tail(n);
    int maxH = 0, maxL = 0;
    for (int i = 0; i < n; ++i) {
        const int L = (int)probs[i]->lv.size();
        tail[i] = probs[i]->mg_tail > 0 ? probs[i]->mg_tail : L - 1;
        maxH = std::max(maxH, tail[i]);
        maxL = std::max(maxL, L);
    }
    // V-cycle vectors of problem p on level l: (b, x, t)
    auto vb = [&](int p, int l) -> void* { return l == 0 ? probs[p]->r : probs[p]->lv[l].b; };
    auto vx = [&](int p, int l) -> void* { return l == 0 ? probs[p]->z : probs[p]->lv[l].x; };
    auto vt = [&](int p, int l) -> void* { return probs[p]->lv[l].t; };
    auto cur0 = [&](int p, int l) { return even ? vx(p, l) : vt(p, l); };
    auto oth0 = [&](int p, int l) { return even ? vt(p, l) : vx(p, l); };
    auto members = [&](int l) {   // problems with a host-side level l
        std::vector<int> m;
        for (int i = 0; i < n; ++i)
            if (tail[i] > l) m.push_back(i);
        return m;
    };
    auto oper = [&](int l, int mode, const std::vector<int>& m, bool cur_is_0, int first) -> int {
        std::vector<to_problem*> ps;
        std::vector<const void*> xs, bs;
        std::vector<void*> ys;
        for (int p : m) {
            ps.push_back(probs[p]);
            xs.push_back(cur_is_0 ? cur0(p, l) : oth0(p, l));
            ys.push_back(cur_is_0 ? oth0(p, l) : cur0(p, l));
            bs.push_back(vb(p, l));
        }
        BmOp op;
        op.kind = BM_OPER;
        op.mode = mode;
        op.n = (int)m.size();
        int rc = op_table_level(ps.data(), op.n, l, mode, xs.data(), ys.data(), bs.data(), om, first, kchunk, &op.tab,
                                &op.max_tiles);
        if (op.tab) M->dev.push_back(op.tab);
        if (rc) return rc;
        void* kh = level_haar(probs[m[0]], l);
        if (!kh) return fail(TO_ERR_CUDA, "host allocation");
        M->host.push_back(kh);
        op.kh = kh;
        M->vcycle.push_back(op);
        return TO_OK;
    };
    int rc;
    // ---- down
    std::vector<bool> cur_is_0(maxH, true);   // after the pre-sweeps: the current iterate is cur0 (else oth0)
    for (int l = 0; l < maxH; ++l) {
        const std::vector<int> m = members(l);
        if (l == 0) {
            std::vector<BmJac<T>> h;
            long long mx = 0;
            for (int p : m) {
                const Level& F = probs[p]->lv[0];
                h.push_back(BmJac<T>{F.n_dof, (const T*)vb(p, 0), (const T*)F.dinv, (T*)cur0(p, 0), (T)om});
                mx = std::max<long long>(mx, F.n_dof);
            }
            BmOp op;
            op.kind = BM_JAC;
            op.n = (int)m.size();
            op.grid_x = grid_x_for(mx, num_sms, op.n);
            if ((rc = upload_table(M, h, &op.tab))) return rc;
            M->vcycle.push_back(op);
        }
        bool c0 = true;
        for (int it = 1; it < nu1; ++it) {
            if ((rc = oper(l, OP_SMOOTH, m, c0, 0))) return rc;
            c0 = !c0;
        }
        if ((rc = oper(l, OP_BMINUS, m, c0, 0))) return rc;   // b - K x into the other buffer
        cur_is_0[l] = c0;
        std::vector<BmRestrict<T>> h;
        long long mx = 0;
        for (int p : m) {
            const Level& F = probs[p]->lv[l];
            const Level& C = probs[p]->lv[l + 1];
            // above the coarsest level the restriction also takes the coarse level's first sweep
            const bool fuse = l + 1 < (int)probs[p]->lv.size() - 1;
            h.push_back(BmRestrict<T>{C.nx, C.ny, C.nz, (const T*)(c0 ? oth0(p, l) : cur0(p, l)), F.mask, C.mask, (T*)C.b,
                                      (const T*)C.dinv, fuse ? (T*)(even ? C.x : C.t) : (T*)nullptr, (T)om});
            mx = std::max<long long>(mx, C.n_node);
        }
        BmOp op;
        op.kind = BM_RESTRICT;
        op.n = (int)m.size();
        op.grid_x = grid_x_for(mx, num_sms, op.n);
        if ((rc = upload_table(M, h, &op.tab))) return rc;
        M->vcycle.push_back(op);
    }
    // ---- the tails, one CTA per problem
    {
        std::vector<TailArgs<T>> h(n);
        size_t smem = 0;
        for (int p = 0; p < n; ++p) smem = std::max<size_t>(smem, (size_t)tail_args<T>(probs[p], tail[p], &h[p]));
        if (smem > kTailSmem) return fail(TO_ERR_ARG, "batched multigrid: a coarse tail exceeds shared memory");
        BmOp op;
        op.kind = BM_TAIL;
        op.n = n;
        op.smem = smem;
        if ((rc = upload_table(M, h, &op.tab))) return rc;
        HaarK<T>* kh = (HaarK<T>*)malloc(sizeof(HaarK<T>));
        if (!kh) return fail(TO_ERR_CUDA, "host allocation");
        M->host.push_back(kh);
        for (int q = 0; q < kHaarNnz; ++q) kh->v[q] = (T)probs[0]->haar[q];
        op.kh = kh;
        // per kernel, shared by every batch: the cap, not this batch's size
        TO_CUDA(cudaFuncSetAttribute(k_mg_tail_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmem));
        M->vcycle.push_back(op);
    }
    // ---- up
    for (int l = maxH - 1; l >= 0; --l) {
        const std::vector<int> m = members(l);
        std::vector<BmProlong<T>> h;
        long long mx = 0;
        for (int p : m) {
            const Level& F = probs[p]->lv[l];
            const Level& C = probs[p]->lv[l + 1];
            h.push_back(BmProlong<T>{C.nx, C.ny, C.nz, (const T*)C.x, C.mask, F.mask,
                                     (T*)(cur_is_0[l] ? cur0(p, l) : oth0(p, l))});
            mx = std::max<long long>(mx, F.n_node);
        }
        BmOp op;
        op.kind = BM_PROLONG;
        op.n = (int)m.size();
        op.grid_x = grid_x_for(mx, num_sms, op.n);
        if ((rc = upload_table(M, h, &op.tab))) return rc;
        M->vcycle.push_back(op);
        bool c0 = cur_is_0[l];
        for (int it = 0; it < nu2; ++it) {
            if ((rc = oper(l, OP_SMOOTH, m, c0, (l == 0 && it == nu2 - 1) ? 2 : 0))) return rc;
            c0 = !c0;
        }
        // the last sweep lands in x (the buffer parity chosen at the first sweep): cur0 = x exactly when even
        if (c0 != even) return fail(TO_ERR_STATE, "batched V-cycle buffer parity");
    }
    // ---- refresh: coarse moduli and diagonals, the dense coarsest operators and their inverses
    for (int l = 1; l < maxL; ++l) {
        std::vector<BmLevel<T>> h;
        long long mxe = 0, mxn = 0;
        for (int p = 0; p < n; ++p) {
            if ((int)probs[p]->lv.size() <= l) continue;
            const Level& F = probs[p]->lv[l - 1];
            const Level& C = probs[p]->lv[l];
            h.push_back(BmLevel<T>{C.nx, C.ny, C.nz, (const T*)F.E, (T*)C.E, C.mask, (T*)C.dinv, C.kdiag});
            mxe = std::max<long long>(mxe, C.n_elem);
            mxn = std::max<long long>(mxn, C.n_node);
        }
        BmOp op;
        op.kind = BM_COARSEN;
        op.n = (int)h.size();
        op.grid_x = grid_x_for(mxe, num_sms, op.n);
        if ((rc = upload_table(M, h, &op.tab))) return rc;
        M->refresh.push_back(op);
        op.kind = BM_DIAG;
        op.grid_x = grid_x_for(mxn, num_sms, op.n);
        M->refresh.push_back(op);
    }
    {
        std::vector<BmDense<T>> h;
        long long mx = 0;
        int nmax = 0;
        for (int p = 0; p < n; ++p) {
            to_problem* P = probs[p];
            const Level& C = P->lv.back();
            h.push_back(BmDense<T>{C.nx, C.ny, C.nz, P->n_coarse, (const T*)C.E, C.mask, P->ke_dev, C.h,
                                   (T*)P->coarse_A, (T*)P->coarse_L, &P->sc->err});
            mx = std::max<long long>(mx, (long long)P->n_coarse * P->n_coarse);
            nmax = std::max(nmax, P->n_coarse);
        }
        BmOp op;
        op.kind = BM_ASSEMBLE;
        op.n = n;
        op.grid_x = grid_x_for(mx, num_sms, n);
        if ((rc = upload_table(M, h, &op.tab))) return rc;
        M->refresh.push_back(op);
        // the inverses: register-blocked for n <= 160, blocked Gauss-Jordan over many CTAs above
        std::vector<BmDense<T>> hr;
        std::vector<GjArgs<T>> hg;
        int nbmax = 0;
        for (int p = 0; p < n; ++p) {
            if (probs[p]->n_coarse <= kRegDof) {
                hr.push_back(h[p]);
            } else {
                hg.push_back(gj_args<T>(probs[p]));
                nbmax = std::max(nbmax, hg.back().nb);
            }
        }
        (void)nmax;
        if (!hr.empty()) {
            BmOp r;
            r.kind = BM_INVERT_REG;
            r.n = (int)hr.size();
            if ((rc = upload_table(M, hr, &r.tab))) return rc;
            M->refresh.push_back(r);
        }
        if (!hg.empty()) {
            BmOp g;
            g.kind = BM_INVERT_GJ;
            g.n = (int)hg.size();
            g.max_tiles = nbmax;
            // largest first, so that every block step's pivots are a prefix of the table
            std::stable_sort(hg.begin(), hg.end(), [](const GjArgs<T>& x, const GjArgs<T>& y) { return x.nb > y.nb; });
            std::vector<int> nbs;
            for (const GjArgs<T>& x : hg) nbs.push_back(x.nb);
            const std::vector<int2> hm = gj_build_maps(nbs, g.gj);
            void* dm = nullptr;
            if ((rc = upload_table(M, hm, &dm))) return rc;
            g.gj.map = (const int2*)dm;
            if ((rc = upload_table(M, hg, &g.tab))) return rc;
            M->refresh.push_back(g);
        }
        return TO_OK;
    }
    return TO_OK;
}

template <typename T>
static int batch_mg_run(const BatchMG* M, const std::vector<BmOp>& ops, cudaStream_t s_main, bool fork = false) {
    cudaStream_t s = s_main;
    for (const BmOp& op : ops) {
        const dim3 g2(op.grid_x, op.n);
        const bool dense = op.kind == BM_ASSEMBLE || op.kind == BM_INVERT_REG || op.kind == BM_INVERT_GJ;
        if (fork && dense && s == s_main) {   // the rest of the refresh on the side branch
            TO_CUDA(cudaEventRecord(M->ev_fork, s_main));
            TO_CUDA(cudaStreamWaitEvent(M->side, M->ev_fork, 0));
            s = M->side;
        }
        if (op.kind == BM_TAIL && M->join_pending) {   // the coarse solves need the inverses
            TO_CUDA(cudaStreamWaitEvent(s, M->ev_join, 0));
            M->join_pending = false;
        }
        switch (op.kind) {
            case BM_JAC: k_bm_jacobi_first<T><<<g2, 256, 0, s>>>((const BmJac<T>*)op.tab); break;
            case BM_OPER: {
                const int rc = batch_operator_launch(M->prec, op.mode, op.tab, op.kh, op.max_tiles, op.n, s);
                if (rc) return rc;
                break;
            }
            case BM_RESTRICT: k_bm_restrict<T><<<g2, 256, 0, s>>>((const BmRestrict<T>*)op.tab); break;
            case BM_PROLONG: k_bm_prolong<T><<<g2, 256, 0, s>>>((const BmProlong<T>*)op.tab); break;
            case BM_TAIL:
                k_mg_tail_batch<T><<<op.n, tail_threads<T>(), op.smem, s>>>((const TailArgs<T>*)op.tab, *(const HaarK<T>*)op.kh);
                break;
            case BM_COARSEN: k_bm_coarsen<T><<<g2, 256, 0, s>>>((const BmLevel<T>*)op.tab); break;
            case BM_DIAG: k_bm_diag<T><<<g2, 256, 0, s>>>((const BmLevel<T>*)op.tab); break;
            case BM_ASSEMBLE: k_bm_assemble<T><<<g2, 256, 0, s>>>((const BmDense<T>*)op.tab); break;
            case BM_INVERT_REG: k_bm_invert_reg<T><<<op.n, dim3(32, 32), 0, s>>>((const BmDense<T>*)op.tab); break;
            default: {
                const int rc = gj_launch_maps<T>(op.tab, op.n, op.gj, M->num_sms, s);
                if (rc) return rc;
                break;
            }
        }
        TO_CUDA(cudaGetLastError());
    }
    if (s != s_main) {
        TO_CUDA(cudaEventRecord(M->ev_join, s));
        M->join_pending = true;
    }
    return TO_OK;
}

void batch_mg_free(BatchMG* M) {
    if (!M) return;
    if (M->side) cudaStreamSynchronize(M->side);
    for (void* d : M->dev) cudaFree(d);
    for (void* h : M->host) free(h);
    if (M->ev_fork) cudaEventDestroy(M->ev_fork);
    if (M->ev_join) cudaEventDestroy(M->ev_join);
    if (M->side) cudaStreamDestroy(M->side);
    delete M;
}

// tables of the batched V-cycle and refresh; every problem has a multigrid hierarchy
// of at least two levels and the same smoothing parameters
int batch_mg_build(to_problem* const* probs, int n, int kchunk, BatchMG** out) {
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (probs[i]->lv.size() < 2)
            return fail(TO_ERR_ARG, "batched multigrid needs every grid to halve at least once");
    BatchMG* M = new BatchMG();
    M->prec = probs[0]->prec;
    M->n = n;
    M->num_sms = probs[0]->num_sms;
    if (cudaStreamCreateWithFlags(&M->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&M->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&M->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        batch_mg_free(M);
        return fail(TO_ERR_CUDA, "batched multigrid stream / events");
    }
    const int rc = M->prec == TO_FP64 ? batch_mg_build_t<double>(probs, n, kchunk, M) : batch_mg_build_t<float>(probs, n, kchunk, M);
    if (rc) {
        batch_mg_free(M);
        return rc;
    }
    *out = M;
    return TO_OK;
}

int batch_mg_refresh(const BatchMG* M, cudaStream_t s) {
    return M->prec == TO_FP64 ? batch_mg_run<double>(M, M->refresh, s, true) : batch_mg_run<float>(M, M->refresh, s, true);
}

// the whole refresh on s (a branch that its caller joins)
int batch_mg_refresh_inline(const BatchMG* M, cudaStream_t s) {
    return M->prec == TO_FP64 ? batch_mg_run<double>(M, M->refresh, s, false) : batch_mg_run<float>(M, M->refresh, s, false);
}

// make s wait for a pending refresh branch, leaving it pending for the coarse tails
int batch_mg_wait(const BatchMG* M, cudaStream_t s) {
    if (M->join_pending) TO_CUDA(cudaStreamWaitEvent(s, M->ev_join, 0));
    return TO_OK;
}

// make s wait for a refresh branch that no coarse tail has joined yet
int batch_mg_join(const BatchMG* M, cudaStream_t s) {
    if (M->join_pending) {
        TO_CUDA(cudaStreamWaitEvent(s, M->ev_join, 0));
        M->join_pending = false;
    }
    return TO_OK;
}

int batch_mg_vcycle(const BatchMG* M, cudaStream_t s) {
    return M->prec == TO_FP64 ? batch_mg_run<double>(M, M->vcycle, s) : batch_mg_run<float>(M, M->vcycle, s);
}

int batch_mg_launches(const BatchMG* M, int* refresh, int* vcycle) {
    *refresh = (int)M->refresh.size();
    *vcycle = (int)M->vcycle.size();
    return TO_OK;
}

}  // namespace to
