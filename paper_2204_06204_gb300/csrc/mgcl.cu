// Multigrid: the level just above the one-CTA coarse tail, run in one 16-CTA thread-block
// cluster instead of one launch per step (FP32).  The level's smoothing, residual and
// grid transfers are the damped-Jacobi V-cycle steps of the launched form (Sec. IV: M is
// one V-cycle; the same steps and buffers, results up to the order of the sums).
//
// Each CTA of the cluster owns one element layer c of the level (the level has at most 16
// layers and at most 512 elements per layer: one thread per element) and node plane c (the
// last layer's CTA also plane nz).  The owned planes' values (x, b, 1 / d, the fixture
// mask), a copy of plane c + 1 and the layer's moduli stay in shared memory for the whole
// leg.  Every read in a sweep is from the CTA's own shared memory; what a neighbour needs
// is pushed to it with remote stores (distributed shared memory), which do not stall the
// writer the way remote loads stall a reader.  A sweep:
//   1. cluster barrier (the planes of this sweep, own and pushed, are in place);
//   2. every thread applies its element's matrix (elem_apply_haar) to the element's 24
//      values (fixed components zeroed), keeps the lower face's 12 results and pushes the
//      upper face's 12 to the CTA of the layer above (plane nz's: kept);
//   3. cluster barrier;
//   4. every owned node adds the upper corners of the layer below (pushed) and the lower
//      corners of its own layer, in a fixed order, applies the damped-Jacobi or b - K x
//      epilogue (K^ is the identity on fixed DOFs) and pushes plane c's new values to the
//      copy of the CTA below.
// 640 threads: one per node of a plane in step 4, one per element in step 2.
//
// Down leg: the first sweep (fused into the restriction from the finer level) is loaded,
// the remaining pre-smoothing sweeps and b - K x run, the iterate is written out, and the
// residual is restricted to the tail's level: every CTA sums the in-plane terms of
// restrict_node for its own planes and pushes the partial sums to the CTA that owns the
// coarse plane, which adds the three planes' partials and writes the coarse right-hand side
// (and the coarse first sweep).  Up leg: every CTA stages the two coarse planes its planes
// interpolate from, adds the prolongation (prolong_node's terms in its order) in shared
// memory and runs the post-smoothing sweeps; the result goes to the V-cycle's output.
//
// A cluster barrier costs about 0.2 us against about 0.5 us between two graph launches,
// and the data never leave the SMs; against that, the level runs on 16 SMs instead of
// all of them.  Measured on the 128x64x64 cantilever the two legs take the time of the
// six launches they replace (the same outer iterations per second), so the path is off
// unless asked for.
#include <cooperative_groups.h>

#include "device.cuh"
#include "haar.cuh"
#include "transfer.cuh"

namespace to {

namespace cg = cooperative_groups;

namespace {

constexpr int kMcQ = 16;     // CTAs in the cluster (non-portable size)
constexpr int kMcE = 512;    // element slots per layer: one thread each in the element phase
constexpr int kMcNP = 640;   // node slots per plane: one thread each in the node phase
constexpr int kMcT = kMcNP;  // threads per CTA
constexpr int kMcCP = 192;   // node slots per coarse plane

struct McArgs {
    int nx, ny, nz;          // the level
    int nsweep;              // down: pre-smoothing sweeps after the first; up: post-smoothing sweeps
    float omega;
    const uint8_t* mask;
    const float* E;
    const float* b;
    const float* dinv;
    float* xin;              // down: the first sweep; up: the iterate (the prolongation is added here)
    float* xout;             // down: the iterate after the pre-smoothing; up: the V-cycle's result
    // the coarse level (restriction on the way down, prolongation on the way up)
    int cx, cy, cz;
    const uint8_t* cmask;
    float* cb;               // down: coarse right-hand side
    const float* cdinv;
    float* cfirst;           // down: the coarse first sweep (nullptr: none)
    const float* cxv;        // up: the coarse correction
};

struct McSmem {
    float x[2][2][kMcNP][3];   // [ping-pong][owned plane][node][component], raw values
    float xu[2][kMcNP][3];     // [ping-pong] plane c + 1, pushed by the CTA that owns it
    float b[2][kMcNP][3];
    float d[2][kMcNP][3];
    uint8_t m[2][kMcNP];
    uint8_t mu[kMcNP];         // the fixture mask of plane c + 1
    float e[kMcE];             // moduli of the owned element layer
    float lo[12][kMcE];        // the layer's results at its lower face (local nodes 0-3)
    float in[12][kMcE];        // layer c - 1's results at its upper face, pushed by CTA c - 1
    float top[12][kMcE];       // the last layer's results at its upper face (plane nz)
    float cx[2][kMcCP][3];     // up leg: the two coarse planes the owned fine planes interpolate from
    uint8_t cm[2][kMcCP];
    float rp[3][kMcCP][3];     // down leg: the partial restriction sums of fine planes 2K - 1, 2K, 2K + 1
};

// local node of elem_apply_haar for corner (a, b) of face z
__device__ __forceinline__ int mc_local(int a, int b, int z) {
    return z * 4 + (b ? (a ? 2 : 3) : (a ? 1 : 0));
}

}  // namespace

template <bool UP>
__global__ void __launch_bounds__(kMcT, 1) k_mg_cluster(const McArgs a, const HaarK<float> kh) {
    extern __shared__ __align__(16) unsigned char mc_smem_raw[];
    McSmem& sm = *reinterpret_cast<McSmem*>(mc_smem_raw);
    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank();
    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int nxn = nx + 1, np = (nx + 1) * (ny + 1), nxy = nx * ny;
    const int nown = c < nz ? (c == nz - 1 ? 2 : 1) : 0;   // owned node planes c (and nz)

    // the owned planes and the layer's moduli into shared memory (flat, coalesced copies:
    // a plane's 3 np values are contiguous in global memory and in shared memory)
    for (int q = 0; q < nown; ++q) {
        const long long p0 = (long long)(c + q) * np;
        const float* xs = a.xin + 3 * p0;
        const float* bs = a.b + 3 * p0;
        const float* ds = a.dinv + 3 * p0;
        float* xd = &sm.x[0][q][0][0];
        float* bd = &sm.b[q][0][0];
        float* dd = &sm.d[q][0][0];
        for (int f = tid; f < 3 * np; f += kMcT) {
            xd[f] = xs[f];
            bd[f] = bs[f];
            dd[f] = ds[f];
        }
        for (int n = tid; n < np; n += kMcT) sm.m[q][n] = a.mask[p0 + n];
    }
    if (c < nz)
        for (int e = tid; e < nxy; e += kMcT) sm.e[e] = a.E[(long long)c * nxy + e];
    if (c < nz - 1)
        for (int n = tid; n < np; n += kMcT) sm.mu[n] = a.mask[(long long)(c + 1) * np + n];
    const int ncx = a.cx + 1, ncp = (a.cx + 1) * (a.cy + 1);
    if (UP && nown > 0) {
        // the two coarse planes the owned fine planes interpolate from (K0 = c / 2, K0 + 1)
        const int K0 = c >> 1;
        for (int h = 0; h < 2; ++h) {
            const int K = K0 + h;
            if (K > a.cz) continue;
            const long long c0 = (long long)K * ncp;
            for (int f = tid; f < 3 * ncp; f += kMcT) (&sm.cx[h][0][0])[f] = a.cxv[3 * c0 + f];
            for (int n = tid; n < ncp; n += kMcT) sm.cm[h][n] = a.cmask[c0 + n];
        }
        __syncthreads();
        // x_f += m_f P (m_c x_c) at the owned fine nodes: prolong_node's terms in its order
        for (int q = 0; q < nown; ++q) {
            const int k = c + q;
            for (int n = tid; n < np; n += kMcT) {
                const int i = n % nxn, j = n / nxn;
                const uint8_t m = sm.m[q][n];
                if (m == 7) continue;
                const int i0 = i >> 1, i1 = (i + 1) >> 1, j0 = j >> 1, j1 = (j + 1) >> 1, k0 = k >> 1, k1 = (k + 1) >> 1;
                float acc[3] = {0.f, 0.f, 0.f};
                const float w = ((i & 1) ? 0.5f : 1.f) * ((j & 1) ? 0.5f : 1.f) * ((k & 1) ? 0.5f : 1.f);
#pragma unroll
                for (int qq = 0; qq < 8; ++qq) {
                    const int ic = (qq & 1) ? i1 : i0, jc = (qq & 2) ? j1 : j0, kc = (qq & 4) ? k1 : k0;
                    const bool use = (!(qq & 1) || i1 != i0) && (!(qq & 2) || j1 != j0) && (!(qq & 4) || k1 != k0);
                    const int cn = ic + ncx * jc, h = kc - K0;
                    const uint8_t mcn = use ? sm.cm[h][cn] : 7;
                    const float v0 = use ? sm.cx[h][cn][0] : 0.f, v1 = use ? sm.cx[h][cn][1] : 0.f,
                                v2 = use ? sm.cx[h][cn][2] : 0.f;
                    acc[0] += (mcn & 1) ? 0.f : w * v0;
                    acc[1] += (mcn & 2) ? 0.f : w * v1;
                    acc[2] += (mcn & 4) ? 0.f : w * v2;
                }
                for (int cc = 0; cc < 3; ++cc)
                    if (!((m >> cc) & 1)) sm.x[0][q][n][cc] += acc[cc];
            }
        }
    }

    // plane c goes to the copy of CTA c - 1 (plane c + 1 there) by remote stores; the
    // first barrier also makes sure that every CTA of the cluster has started
    McSmem* below = c > 0 ? cl.map_shared_rank(&sm, c - 1) : nullptr;
    McSmem* above = c < nz - 1 ? cl.map_shared_rank(&sm, c + 1) : nullptr;
    cl.sync();
    if (below && nown > 0)
        for (int f = tid; f < 3 * np; f += kMcT) (&below->xu[0][0][0])[f] = (&sm.x[0][0][0][0])[f];

    // one sweep from ping buffer `cur` into `cur ^ 1`: damped Jacobi, or b - K x (bminus);
    // every read is from the CTA's own shared memory, what a neighbour needs is pushed to it
    auto sweep = [&](int cur, bool bminus) {
        cl.sync();   // planes `cur` (own and pushed) are in place; the last sweep's results are consumed
        if (c < nz && tid < nxy) {
            const int i = tid % nx, j = tid / nx;
            // plane c: own; plane c + 1: own second plane (last layer) or the pushed copy
            const bool last = c == nz - 1;
            float u[24];
#pragma unroll
            for (int z = 0; z < 2; ++z)
#pragma unroll
                for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                    for (int aa = 0; aa < 2; ++aa) {
                        const int n = (i + aa) + nxn * (j + bb);
                        const float* xv = z ? (last ? sm.x[cur][1][n] : sm.xu[cur][n]) : sm.x[cur][0][n];
                        const unsigned mk = z ? (last ? sm.m[1][n] : sm.mu[n]) : sm.m[0][n];
                        const int l = mc_local(aa, bb, z);
#pragma unroll
                        for (int k = 0; k < 3; ++k) u[3 * l + k] = ((mk >> k) & 1u) ? 0.f : xv[k];
                    }
            float y[24];
            elem_apply_haar<float>(kh.v, sm.e[tid], u, y);
#pragma unroll
            for (int k = 0; k < 12; ++k) sm.lo[k][tid] = y[k];
            // the upper face: to the CTA of the layer above (its plane c + 1), or kept (plane nz)
            float (*up)[kMcE] = last ? sm.top : above->in;
#pragma unroll
            for (int k = 0; k < 12; ++k) up[k][tid] = y[12 + k];
        }
        cl.sync();   // every layer's element results are in place
        for (int q = 0; q < nown; ++q) {
            const int p = c + q;
            // the layer below plane p (upper corners): pushed by the previous CTA, or own (plane nz)
            const float (*lower)[kMcE] = q == 1 ? sm.top : sm.in;
            const int n = tid;
            if (n >= np) continue;
            const int i = n % nxn, j = n / nxn;
            float kx[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int zz = 0; zz < 2; ++zz) {   // 0: layer p - 1 (upper corners), 1: layer p (lower corners)
                const bool has = zz ? (p < nz) : (p > 0);
                if (!has) continue;
                const float (*src)[kMcE] = zz ? sm.lo : lower;
#pragma unroll
                for (int db = 0; db < 2; ++db)
#pragma unroll
                    for (int da = 0; da < 2; ++da) {
                        const int ei = i - 1 + da, ej = j - 1 + db;   // element (ei, ej) of the layer
                        if (ei < 0 || ei >= nx || ej < 0 || ej >= ny) continue;
                        const int l = mc_local(1 - da, 1 - db, 0);   // the face's corner (0-3)
                        const int e = ei + nx * ej;
#pragma unroll
                        for (int k = 0; k < 3; ++k) kx[k] += src[3 * l + k][e];
                    }
            }
            const unsigned mk = sm.m[q][n];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float xv = sm.x[cur][q][n][k];
                const float Kx = ((mk >> k) & 1u) ? xv : kx[k];   // K^ is the identity on fixed DOFs
                const float bv = sm.b[q][n][k];
                const float v = bminus ? bv - Kx : xv + a.omega * (bv - Kx) * sm.d[q][n][k];
                sm.x[cur ^ 1][q][n][k] = v;
                if (q == 0 && below && !bminus) below->xu[cur ^ 1][n][k] = v;
            }
        }
    };

    int cur = 0;
    for (int it = 0; it < a.nsweep; ++it) {
        sweep(cur, false);
        cur ^= 1;
    }
    if (UP) {
        cl.sync();   // the last pushes have landed: no CTA's shared memory is written after this
        for (int q = 0; q < nown; ++q) {
            float* xo = a.xout + 3 * (long long)(c + q) * np;
            const float* xs = &sm.x[cur][q][0][0];
            for (int f = tid; f < 3 * np; f += kMcT) xo[f] = xs[f];
        }
        return;
    }
    sweep(cur, true);   // the residual into cur ^ 1 (own planes only: nothing is pushed)
    __syncthreads();
    for (int q = 0; q < nown; ++q) {
        float* xo = a.xout + 3 * (long long)(c + q) * np;
        const float* xs = &sm.x[cur][q][0][0];
        for (int f = tid; f < 3 * np; f += kMcT) xo[f] = xs[f];
    }
    // the restriction to the coarse level, b_c = m_c P^T (m_f r): every CTA sums the 9 in-plane
    // terms of each owned fine plane k for every coarse plane K with |2K - k| <= 1 and pushes
    // the partial sum to the CTA that owns coarse plane K (the owner of fine plane 2K), which
    // adds the partials of planes 2K - 1, 2K, 2K + 1 in that order
    const int rb = cur ^ 1;
    const int fx = 2 * a.cx, fy = 2 * a.cy;
    {
        // tasks: (owned plane q, target K, coarse node) -> at most 2 x 2 x kMcCP / 2 of them
        int task = tid;
        for (int q = 0; q < nown; ++q) {
            const int k = c + q;
            const int nK = (k & 1) ? 2 : 1;   // an odd plane feeds K = (k - 1) / 2 and (k + 1) / 2
            for (int h = 0; h < nK; ++h) {
                const int K = (k & 1) ? (k - 1) / 2 + h : k / 2;
                const int dk = k - 2 * K;   // -1, 0 or +1
                if (task >= 0 && task < ncp) {
                    const int I = task % ncx, J = task / ncx;
                    const float wk = dk ? 0.5f : 1.f;
                    float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
                    for (int dj = -1; dj <= 1; ++dj) {
                        const int j = 2 * J + dj;
                        const float wj = dj ? 0.5f : 1.f;
#pragma unroll
                        for (int di = -1; di <= 1; ++di) {
                            const int i = 2 * I + di;
                            if (j < 0 || j > fy || i < 0 || i > fx) continue;
                            const int fn = i + nxn * j;
                            const float w = (di ? 0.5f : 1.f) * wj * wk;
                            const uint8_t m = sm.m[q][fn];
#pragma unroll
                            for (int cc = 0; cc < 3; ++cc)
                                acc[cc] += ((m >> cc) & 1) ? 0.f : w * sm.x[rb][q][fn][cc];
                        }
                    }
                    const int owner = 2 * K < nz ? 2 * K : nz - 1;
                    McSmem* dst = owner == c ? &sm : cl.map_shared_rank(&sm, owner);
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) dst->rp[dk + 1][task][cc] = acc[cc];
                }
                task -= ncp;
            }
        }
    }
    cl.sync();   // the partials have landed; no CTA's shared memory is written after this
    for (int K = 0; K <= a.cz; ++K) {
        if ((2 * K < nz ? 2 * K : nz - 1) != c) continue;
        for (int t = tid; t < ncp; t += kMcT) {
            const long long n = t + (long long)ncp * K;
            const uint8_t mcv = a.cmask[n];
            for (int cc = 0; cc < 3; ++cc) {
                // planes 2K - 1 and 2K + 1 exist unless K is the first or the last coarse plane
                float v = K > 0 ? sm.rp[0][t][cc] : 0.f;
                v += sm.rp[1][t][cc];
                v += K < a.cz ? sm.rp[2][t][cc] : 0.f;
                v = ((mcv >> cc) & 1) ? 0.f : v;
                a.cb[3 * n + cc] = v;
                if (a.cfirst) a.cfirst[3 * n + cc] = a.omega * v * a.cdinv[3 * n + cc];
            }
        }
    }
}

// ----------------------------------------------------------------------------- host side
namespace {

constexpr size_t kMcSmem = sizeof(McSmem);

template <bool UP>
int mc_attrs() {
    TO_CUDA(cudaFuncSetAttribute(k_mg_cluster<UP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMcSmem));
    TO_CUDA(cudaFuncSetAttribute(k_mg_cluster<UP>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    return TO_OK;
}

template <bool UP>
int mc_launch(const McArgs& a, const HaarK<float>& kh, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kMcQ);
    cfg.blockDim = dim3(kMcT);
    cfg.dynamicSmemBytes = kMcSmem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kMcQ;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    TO_CUDA(cudaLaunchKernelEx(&cfg, k_mg_cluster<UP>, a, kh));
    return TO_OK;
}

}  // namespace

// the one-time set-up (before any capture): shared-memory opt-in, the 16-CTA cluster, and
// whether one such cluster can be resident at all
int mg_cluster_init(to_problem* P) {
    P->mgc_ok = 0;
    if (P->prec != TO_FP32_MIXED) return TO_OK;
    if (mc_attrs<false>() || mc_attrs<true>()) {
        cudaGetLastError();
        return TO_OK;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kMcQ);
    cfg.blockDim = dim3(kMcT);
    cfg.dynamicSmemBytes = kMcSmem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kMcQ;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_mg_cluster<false>, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        return TO_OK;
    }
    P->mgc_ok = 1;
    return TO_OK;
}

// can level l (the level above the coarse tail) run in the cluster
bool mg_cluster_applicable(const to_problem* P, int l) {
    if (!P->mgc_ok || P->prec != TO_FP32_MIXED || P->prm.mg_cluster == 0) return false;
    if (l < 1 || P->mg_tail != l + 1) return false;
    const Level& F = P->lv[l];
    const Level& C = P->lv[l + 1];
    return F.nz <= kMcQ && F.nx * F.ny <= kMcE && (F.nx + 1) * (F.ny + 1) <= kMcNP &&
           (C.nx + 1) * (C.ny + 1) <= kMcCP && C.nx * 2 == F.nx && C.ny * 2 == F.ny && C.nz * 2 == F.nz &&
           P->prm.mg_nu_pre >= 1;
}

static void mc_level_args(const to_problem* P, int l, McArgs& a, HaarK<float>& kh) {
    const Level& F = P->lv[l];
    const Level& C = P->lv[l + 1];
    a = McArgs{};
    a.nx = F.nx;
    a.ny = F.ny;
    a.nz = F.nz;
    a.omega = (float)P->prm.mg_omega;
    a.mask = F.mask;
    a.E = (const float*)F.E;
    a.b = (const float*)F.b;
    a.dinv = (const float*)F.dinv;
    a.cx = C.nx;
    a.cy = C.ny;
    a.cz = C.nz;
    a.cmask = C.mask;
    for (int n = 0; n < kHaarNnz; ++n) kh.v[n] = (float)(P->haar[n] * (F.h / P->g.h));
}

// the down leg on level l: from the first sweep in x_first, the remaining pre-smoothing
// sweeps and b - K x; the iterate into x_iter; the restriction of the residual
// to the tail's level into its right-hand side and (cfirst) its first sweep
int mg_cluster_down(const to_problem* P, int l, void* x_first, void* x_iter, void* cfirst, cudaStream_t s) {
    McArgs a;
    HaarK<float> kh;
    mc_level_args(P, l, a, kh);
    const Level& C = P->lv[l + 1];
    a.nsweep = P->prm.mg_nu_pre - 1;
    a.xin = (float*)x_first;
    a.xout = (float*)x_iter;
    a.cb = (float*)C.b;
    a.cdinv = (const float*)C.dinv;
    a.cfirst = (float*)cfirst;
    return mc_launch<false>(a, kh, s);
}

// the up leg on level l: the tail's correction prolongated into x_iter, then the
// post-smoothing sweeps; the result into x_out
int mg_cluster_up(const to_problem* P, int l, void* x_iter, void* x_out, cudaStream_t s) {
    McArgs a;
    HaarK<float> kh;
    mc_level_args(P, l, a, kh);
    a.nsweep = P->prm.mg_nu_post;
    a.xin = (float*)x_iter;
    a.xout = (float*)x_out;
    a.cxv = (const float*)P->lv[l + 1].x;
    return mc_launch<true>(a, kh, s);
}

}  // namespace to
