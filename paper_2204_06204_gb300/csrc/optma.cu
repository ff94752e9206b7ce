// Matrix-free hex8 operator y = K^(E) x in FP32 with TMA staging, persistent CTAs
// and element pairs in packed FP32x2 (Sec. III: K = sum_e E_e K_e, fixtures
// eliminated), with the same fused epilogues as the general operator kernel
// (lower-level steps of Algorithms 1 / 3, the multigrid smoother).
//
// Tiles.  A tile owns the node columns x in [64 t + 1, 64 t + 64] (node 0 too when
// t = 0) and the node rows y in [j0, j0 + TYW) (row ny too when j0 + TYW = ny), every
// node plane, so grids whose element counts are multiples of 64 and TYW are covered
// exactly.  Its warps:
//   * TYW + 1 pair warps: warp w walks element row j0 - 1 + w (w = 0 is the halo row
//     whose top corners complete node row j0); lane l takes the element pair
//     (64 t + 2l, 64 t + 2l + 1) and keeps both elements in the two halves of FP32x2
//     registers, so every butterfly, product and scaling is one packed instruction
//     for two elements;
//   * one column warp: lane i takes the single element (64 t + 64, j0 - 1 + i), the
//     element beyond the tile that node column 64 t + 64 also touches, and its lanes
//     issue the TMA copies.
// Per element layer k (bottom node plane k, top plane k + 1), each element's 24
// nodal values are brought to the sum/difference (Haar) basis by x, y and z
// butterflies, the 45 non-zeros of the unit element matrix are applied, the result
// is scaled by E_e and split into its bottom-plane part (added to the top-plane part
// carried from layer k - 1: node plane k is then complete for this element column)
// and its top-plane part (carried), and inverse butterflies return corner values.
// Corners meet at the owned nodes in a fixed order: x neighbours by a shuffle, the
// column warp's corner through shared memory, y neighbours through shared memory
// (one barrier per layer).  No atomics: bitwise reproducible.
//
// Staging.  Each node plane (rows j0 - 1 .. j0 + TYW of x, rows of E, the fixture
// mask, the epilogue's right-hand side and inverse diagonal) arrives by 1-D bulk
// tensor copies, one per row, into a ring of NS shared-memory slots completed on
// mbarriers.  Rows start at a 16-byte boundary below the first needed value (the
// offset is recomputed by the readers); values outside the vectors arrive as zeros
// and out-of-grid elements get E = 0.
//
// Persistence.  The grid is one CTA per SM; the tile columns x planes of the level
// are split into equal contiguous ranges, one per CTA, each walked as segments of
// consecutive planes of one column (one recomputed halo layer per segment).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <mutex>

#include "device.cuh"
#include "tma.cuh"

namespace to {

// ----------------------------------------------------------------------------- packed arithmetic
// V = float2: two elements (the pair); V = float: one element (the column warp).
// Explicitly rounded operations (no contraction), identical for both widths.
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fmaf_rn(b, -1.f, a); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <typename V> __device__ __forceinline__ V vsplat(float k);
template <> __device__ __forceinline__ float2 vsplat<float2>(float k) { return make_float2(k, k); }
template <> __device__ __forceinline__ float vsplat<float>(float k) { return k; }
template <typename V> __device__ __forceinline__ V vzero() { return vsplat<V>(0.f); }

// The 45 non-zeros of the unit element matrix in the sum/difference basis (order of
// kHaarRow / kHaarCol) take only eight distinct values: the cube's symmetries map the
// entries of each group below onto one another for every Poisson ratio (the host checks
// this for the problem before it picks this kernel).  The eight values stay in registers
// as (k, k) pairs, so every packed product has register operands only.
//   group 0: 0 4 8             group 4: 22 23 26 27 30 31
//   group 1: 1 2 3 5 6 7       group 5: 33 37 41
//   group 2: 9 .. 20           group 6: 34 35 36 38 39 40
//   group 3: 21 24 25 28 29 32 group 7: 42 43 44
__host__ __device__ constexpr int haar_group(int i) {
    return (i == 0 || i == 4 || i == 8) ? 0
         : (i <= 7) ? 1
         : (i <= 20) ? 2
         : (i == 21 || i == 24 || i == 25 || i == 28 || i == 29 || i == 32) ? 3
         : (i <= 32) ? 4
         : (i == 33 || i == 37 || i == 41) ? 5
         : (i <= 41) ? 6
         : 7;
}

// v = K^ uh in the sum/difference basis
template <typename V>
__device__ __forceinline__ void haar_apply_v(const V (&g)[8], const V (&u)[24], V (&v)[24]) {
#define KS(i) g[haar_group(i)]
    v[3] = vfma(KS(2), u[14], vfma(KS(1), u[7], vmul(KS(0), u[3])));
    v[7] = vfma(KS(5), u[14], vfma(KS(4), u[7], vmul(KS(3), u[3])));
    v[14] = vfma(KS(8), u[14], vfma(KS(7), u[7], vmul(KS(6), u[3])));
    v[4] = vfma(KS(10), u[6], vmul(KS(9), u[4]));
    v[6] = vfma(KS(12), u[6], vmul(KS(11), u[4]));
    v[5] = vfma(KS(14), u[12], vmul(KS(13), u[5]));
    v[12] = vfma(KS(16), u[12], vmul(KS(15), u[5]));
    v[8] = vfma(KS(18), u[13], vmul(KS(17), u[8]));
    v[13] = vfma(KS(20), u[13], vmul(KS(19), u[8]));
    v[9] = vfma(KS(22), u[20], vmul(KS(21), u[9]));
    v[20] = vfma(KS(24), u[20], vmul(KS(23), u[9]));
    v[10] = vfma(KS(26), u[17], vmul(KS(25), u[10]));
    v[17] = vfma(KS(28), u[17], vmul(KS(27), u[10]));
    v[15] = vfma(KS(30), u[19], vmul(KS(29), u[15]));
    v[19] = vfma(KS(32), u[19], vmul(KS(31), u[15]));
    v[11] = vfma(KS(35), u[18], vfma(KS(34), u[16], vmul(KS(33), u[11])));
    v[16] = vfma(KS(38), u[18], vfma(KS(37), u[16], vmul(KS(36), u[11])));
    v[18] = vfma(KS(41), u[18], vfma(KS(40), u[16], vmul(KS(39), u[11])));
    v[21] = vmul(KS(42), u[21]);
    v[22] = vmul(KS(43), u[22]);
    v[23] = vmul(KS(44), u[23]);
    v[0] = v[1] = v[2] = vzero<V>();
#undef KS
}

// Face butterflies of one plane's 2 x 2 nodes per component: F[c][f], f = 0 sum-sum,
// 1 x-difference, 2 y-difference, 3 both (the x / y sums and differences)
template <typename V>
__device__ __forceinline__ void face4(V a00, V a10, V a01, V a11, V (&F)[4]) {
    const V sx0 = vadd(a10, a00), dx0 = vsub(a10, a00), sx1 = vadd(a11, a01), dx1 = vsub(a11, a01);
    F[0] = vadd(sx1, sx0);
    F[1] = vadd(dx1, dx0);
    F[2] = vsub(sx1, sx0);
    F[3] = vsub(dx1, dx0);
}

// One element layer: face coefficients of the top (Ft) and bottom (Fb) planes, the
// modulus E, the carried top-plane part Gc of the layer below (updated to this
// layer's); corner values cor[c] = (x0y0, x1y0, x0y1, x1y1) of node plane k; the
// unit-modulus energy u^T k_e u (ENERGY)
template <typename V, bool ENERGY>
__device__ __forceinline__ void elem_layer(const V (&kh)[8], const V (&Ft)[3][4], const V (&Fb)[3][4], V E,
                                           V (&Gc)[3][4], V (&cor)[3][4], V& en) {
    V uh[24];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            uh[3 * f + c] = vadd(Ft[c][f], Fb[c][f]);
            uh[12 + 3 * f + c] = vsub(Ft[c][f], Fb[c][f]);
        }
    V v[24];
    haar_apply_v<V>(kh, uh, v);
    if (ENERGY) {
        V e = vmul(uh[3], v[3]);
#pragma unroll
        for (int i = 4; i < 24; ++i) e = vfma(uh[i], v[i], e);
        en = e;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        V S[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const V vs = v[3 * f + c], vd = v[12 + 3 * f + c];
            S[f] = vfma(E, vsub(vs, vd), Gc[c][f]);
            Gc[c][f] = vmul(E, vadd(vs, vd));
        }
        const V sx0 = vsub(S[0], S[2]), sx1 = vadd(S[0], S[2]), dx0 = vsub(S[1], S[3]), dx1 = vadd(S[1], S[3]);
        cor[c][0] = vsub(sx0, dx0);
        cor[c][1] = vadd(sx0, dx0);
        cor[c][2] = vsub(sx1, dx1);
        cor[c][3] = vadd(sx1, dx1);
    }
}

// ----------------------------------------------------------------------------- layout
constexpr int kTX = 64;                    // element columns per tile (32 lanes x 2)
constexpr int kUBox = 204;                 // floats per x / b / d row copy: 66 nodes + alignment slack
constexpr int kUPitch = 224;               // floats per staged row (896 B, 128-byte aligned rows)
constexpr int kEBox = 68;                  // floats per E row copy: 65 elements + slack
constexpr int kEPitch = 96;
constexpr int kMBox = 96;                  // bytes per mask row copy: 66 nodes + slack
constexpr int kMPitch = 128;

template <int TYW, bool BD>
struct TmaLayout {
    static constexpr int NUR = TYW + 2;    // node rows j0 - 1 .. j0 + TYW
    static constexpr int NER = TYW + 1;    // element rows j0 - 1 .. j0 + TYW - 1
    static constexpr int NBR = TYW + 1;    // owned node rows j0 .. j0 + TYW (epilogue operands)
    static constexpr int U = 0;
    static constexpr int E = U + NUR * kUPitch * 4;
    static constexpr int M = E + NER * kEPitch * 4;
    static constexpr int B = M + NUR * kMPitch;
    static constexpr int D = B + NBR * kUPitch * 4;
    static constexpr int SLOT = ((BD ? D + NBR * kUPitch * 4 : B) + 127) / 128 * 128;
};

struct TOpArgs {
    int nx, ny, nz;
    int tiles_x, tiles_y;
    long long units;               // tile columns x (nz + 1) planes
    float* y;
    float* z;                      // RESID: r / d (optional)
    const float* Ed;               // RESID: E' / Hs (with gt)
    float* gt;                     // RESID: -E'_e u_e^T k_e u_e / Hs_e (optional)
    const uint8_t* tmask;          // per tile column: any fixed node in its footprint
    float kg[8];                   // the element matrix's eight distinct values (for the level's edge)
    float omega;
    double* red;
    unsigned* counter;
    DevScalars* sc;
    int first_step;
    int load_d;                    // the inverse diagonal is staged (SMOOTH; RESID with z)
};

// the CTA's walk: contiguous units [u, u_end) of (tile column, plane), in segments
struct Walk {
    long long u, u_end;
    int P;                         // planes per column (nz + 1)
    __device__ bool seg(int& col, int& p0, int& p1) const {
        if (u >= u_end) return false;
        col = (int)(u / P);
        p0 = (int)(u - (long long)col * P);
        const long long e = min(u_end, (long long)(col + 1) * P);
        p1 = p0 + (int)(e - u);
        return true;
    }
};

// plane-load cursor of the producer: load index q runs over every segment's planes p0 - 1 .. p1
struct LoadCursor {
    Walk w;
    int col, p0, p1, p;
    bool ok;
    __device__ void init(const Walk& w0) {
        w = w0;
        ok = w.seg(col, p0, p1);
        p = p0 - 1;
    }
    __device__ void next() {
        if (++p > p1) {
            w.u += p1 - p0;
            ok = w.seg(col, p0, p1);
            p = p0 - 1;
        }
    }
};

template <int TYW, int MODE, int NS>
__global__ void __launch_bounds__((TYW + 3) * 32, 1)
    k_op_tma(const TOpArgs a, const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_E,
             const __grid_constant__ CUtensorMap tm_m, const __grid_constant__ CUtensorMap tm_b,
             const __grid_constant__ CUtensorMap tm_d) {
    constexpr bool NEED_B = MODE == OP_RESID || MODE == OP_SMOOTH || MODE == OP_BMINUS;
    constexpr bool NEED_D = MODE == OP_RESID || MODE == OP_SMOOTH;
    constexpr bool BD = NEED_B;
    using LY = TmaLayout<TYW, BD>;
    constexpr int NPW = TYW + 1;                 // pair warps
    constexpr int CW = TYW + 1;                  // the column warp
    constexpr int PW = TYW + 2;                  // the producer warp (TMA copies)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the ring starts at the first 128-byte boundary (the request carries 128 bytes of slack)
    unsigned char* const smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t full[NS];
    __shared__ float2 xbuf[2][NPW][3][32];       // y0-row corner sums of the owned nodes (A, B halves), per parity
    __shared__ float xb0[2][NPW][3];             // node 0 (t = 0): y0-row corner
    __shared__ float colbuf[2][NPW][6];          // column warp: x0 corners of rows y0 (0..2) and y1 (3..5)
    __shared__ double red_sh[32 * kRedQ];
    __shared__ float2 s_kg[8];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int nxn = nx + 1, nyn = ny + 1;
    const int P = nz + 1;
    const unsigned NPn = (unsigned)nxn * (unsigned)nyn;   // node plane stride, modulo 2^32
    const unsigned NPe = (unsigned)nx * (unsigned)ny;     // element plane stride, modulo 2^32
    const long long NPl = (long long)nxn * nyn;
    const bool dz = MODE == OP_RESID && a.z != nullptr;
    int* err = &a.sc->err;

    Walk walk;
    walk.P = P;
    {
        const long long G = gridDim.x, b = blockIdx.x;
        walk.u = a.units * b / G;
        walk.u_end = a.units * (b + 1) / G;
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    if (threadIdx.x < 8) s_kg[threadIdx.x] = make_float2(a.kg[threadIdx.x], a.kg[threadIdx.x]);
    if (warp == PW && lane == 0) {
        tma_prefetch_map(&tm_x);
        tma_prefetch_map(&tm_E);
        tma_prefetch_map(&tm_m);
        if (NEED_B) tma_prefetch_map(&tm_b);
        if (NEED_D && a.load_d) tma_prefetch_map(&tm_d);
    }
    __syncthreads();

    // ---- producer (column warp): the copies of load q (cursor at q) into slot q % NS
    LoadCursor cur;
    int issued = 0;
    auto issue_one = [&]() {
        const int slot = issued % NS;
        unsigned char* base = smem + (size_t)slot * LY::SLOT;
        const int t = cur.col % a.tiles_x, s = cur.col / a.tiles_x;
        const int X0 = kTX * t, j0 = TYW * s, p = cur.p;
        const bool masked = a.tmask == nullptr || a.tmask[cur.col] != 0;
        if (lane == 0) {
            unsigned bytes = LY::NUR * kUBox * 4 + LY::NER * kEBox * 4;
            if (masked) bytes += LY::NUR * kMBox;
            if (NEED_B) bytes += LY::NBR * kUBox * 4;
            if (NEED_D && a.load_d) bytes += LY::NBR * kUBox * 4;
            mbar_arrive_expect_tx(&full[slot], bytes);
        }
        __syncwarp();
        const int r = lane;
        if (r < LY::NUR) {   // x (and mask) row: node row j0 - 1 + r
            const long long n0 = (long long)X0 + (long long)nxn * ((long long)(j0 - 1 + r) + (long long)nyn * p);
            tma_load_1d(base + LY::U + r * kUPitch * 4, &tm_x, (int)((3 * n0) & ~3LL), &full[slot]);
            if (masked) tma_load_1d(base + LY::M + r * kMPitch, &tm_m, (int)(n0 & ~15LL), &full[slot]);
        }
        if (r < LY::NER) {   // E row: element row j0 - 1 + r of layer p
            const long long e0 = (long long)X0 + (long long)nx * ((long long)(j0 - 1 + r) + (long long)ny * p);
            tma_load_1d(base + LY::E + r * kEPitch * 4, &tm_E, (int)(e0 & ~3LL), &full[slot]);
        }
        if (NEED_B && r < LY::NBR) {   // epilogue operands: node row j0 + r
            const long long n0 = (long long)X0 + (long long)nxn * ((long long)(j0 + r) + (long long)nyn * p);
            const int x = (int)((3 * n0) & ~3LL);
            tma_load_1d(base + LY::B + r * kUPitch * 4, &tm_b, x, &full[slot]);
            if (NEED_D && a.load_d) tma_load_1d(base + LY::D + r * kUPitch * 4, &tm_d, x, &full[slot]);
        }
        ++issued;
        cur.next();
    };
    int total_loads = 0;   // planes loaded by this CTA (p1 - p0 + 2 per segment)
    {
        Walk w2 = walk;
        int c_, a_, b_;
        while (w2.seg(c_, a_, b_)) {
            total_loads += b_ - a_ + 2;
            w2.u += b_ - a_;
        }
    }
    if (warp == PW) {
        cur.init(walk);
        const int first = min(total_loads, NS);
        while (issued < first) issue_one();
    }
    // the element matrix's values in registers (read once: volatile keeps them from being re-read)
    float2 kg[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        const volatile float2* vp = &s_kg[g];
        kg[g] = make_float2(vp->x, vp->y);
    }

    // ---- consumers.  Pair warp w, lane l: elements A = X0 + l and B = X0 + 32 + l of
    // element row j0 - 1 + w (the .x and .y halves); it owns nodes X0 + l + 1 (A) and
    // X0 + l + 33 (B) of node row j0 + w.  Column warp lane i: element X0 + 64 of row
    // j0 - 1 + i (in the .x halves).
    const bool is_pair = warp < NPW;
    const bool is_comp = warp <= CW;             // pair and column warps compute; the producer only copies
    const int w = warp;                          // pair warp index
    // staged row of the thread's y0 nodes (y1: rlo + 1); column-warp lanes past the tile's
    // element rows compute on the last row and their results are discarded, so that every
    // shared-memory read stays inside the staged rows
    const int rlo = is_pair ? w : min(lane, TYW);
    const int xA = is_pair ? lane : kTX;         // node offset (in the tile) of the A / single element's x0 node
    float acc0 = 0.f, acc1 = 0.f, accmax = 0.f, acc3 = 0.f;
    int q_base = 0;      // load index of the current segment's first plane
    int qslot = 0;       // ring slot of the current layer's bottom load
    unsigned qphase = 0; // its phase parity
    int layer = 0;       // layers walked by this CTA (shared-buffer parity)
    int col, p0, p1;
    Walk wk = walk;

    // One segment: tile column col, emitted planes [p0, p1).  FAST: a tile with no fixed node
    // in its footprint, not the first tile column, and every element column (and the column
    // warp's element) inside the grid, so that no mask, node-0 or x-validity work is needed.
    auto segment = [&](auto fast_c) {
        constexpr bool FAST = decltype(fast_c)::value;
        const int t = col % a.tiles_x, s = col / a.tiles_x;
        const int X0 = kTX * t, j0 = TYW * s;
        const bool masked = !FAST && (a.tmask == nullptr || a.tmask[col] != 0);
        const bool last_row_tile = j0 + TYW == ny;
        const int je = j0 - 1 + rlo;             // the thread's element row
        const bool row_in = je >= 0 && je < ny && (is_pair || lane < NPW);
        const bool vA = FAST ? row_in : (row_in && X0 + xA < nx);
        const bool vB = is_pair && (FAST ? row_in : (row_in && X0 + 32 + lane < nx));
        // staged-row offsets (floats / bytes) of node X0 of rows je, je + 1 at plane 0; a plane
        // adds 3 NPn (floats) or NPn (bytes), all modulo the copy alignment
        const unsigned u0 = 3u * ((unsigned)X0 + (unsigned)nxn * (unsigned)je);
        const unsigned u1 = u0 + 3u * (unsigned)nxn;
        const unsigned m0 = (unsigned)X0 + (unsigned)nxn * (unsigned)je;
        const unsigned m1 = m0 + (unsigned)nxn;
        const unsigned e0 = (unsigned)X0 + (unsigned)nx * (unsigned)je;
        const unsigned uo = 3u * ((unsigned)X0 + (unsigned)nxn * (unsigned)(j0 + w));   // the owned row (pair warps)
        const unsigned mo = (unsigned)X0 + (unsigned)nxn * (unsigned)(j0 + w);
        // byte offsets of the thread's rows in slot 0 (a slot adds s * SLOT bytes)
        const unsigned ur0 = LY::U + (rlo * kUPitch + 3 * xA) * 4;
        const unsigned er0 = LY::E + (rlo * kEPitch + xA) * 4;
        const unsigned mr0 = LY::M + rlo * kMPitch + xA;
        const int jn = j0 + w;                   // pair warps: the owned node row
        const bool has_next = w < TYW;
        const bool owner = is_pair && (has_next || last_row_tile) && jn <= ny;
        const unsigned uo_r = LY::U + ((w + 1) * kUPitch + 3 * (lane + 1)) * 4;
        const unsigned bo_r = LY::B + (w * kUPitch + 3 * (lane + 1)) * 4;
        const unsigned mo_r = LY::M + (w + 1) * kMPitch + lane + 1;
        const bool v1 = FAST || X0 + lane + 1 <= nx, v2 = FAST || X0 + lane + 33 <= nx;
        const float2 vm = make_float2(v1 ? 1.f : 0.f, v2 ? 1.f : 0.f);   // reductions: owned, in-grid nodes

        // face coefficients of this thread's element(s) on the plane pl staged at slot byte offset so
        auto load_face = [&](unsigned so, int pl, float2 (&F)[3][4]) {
            const unsigned pp = (unsigned)pl;
            const float* r0 = reinterpret_cast<const float*>(smem + so + ur0) + ((u0 + 3u * NPn * pp) & 3u);
            const float* r1 = reinterpret_cast<const float*>(smem + so + ur0 + kUPitch * 4) + ((u1 + 3u * NPn * pp) & 3u);
            float a0[3], a1[3], b0[3], b1[3], c0[3], c1[3], d0[3], d1[3];   // A: x0, x1 of rows y0, y1; B likewise
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                a0[c] = r0[c];
                a1[c] = r0[3 + c];
                c0[c] = r1[c];
                c1[c] = r1[3 + c];
                b0[c] = r0[96 + c];
                b1[c] = r0[99 + c];
                d0[c] = r1[96 + c];
                d1[c] = r1[99 + c];
            }
            if (!FAST && masked) {   // fixed components of x enter K as zeros
                const unsigned char* q0 = smem + so + mr0 + ((m0 + NPn * pp) & 15u);
                const unsigned char* q1 = smem + so + mr0 + kMPitch + ((m1 + NPn * pp) & 15u);
                const unsigned fa0 = q0[0], fa1 = q0[1], fc0 = q1[0], fc1 = q1[1];
                const unsigned fb0 = q0[32], fb1 = q0[33], fd0 = q1[32], fd1 = q1[33];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    a0[c] = ((fa0 >> c) & 1u) ? 0.f : a0[c];
                    a1[c] = ((fa1 >> c) & 1u) ? 0.f : a1[c];
                    c0[c] = ((fc0 >> c) & 1u) ? 0.f : c0[c];
                    c1[c] = ((fc1 >> c) & 1u) ? 0.f : c1[c];
                    b0[c] = ((fb0 >> c) & 1u) ? 0.f : b0[c];
                    b1[c] = ((fb1 >> c) & 1u) ? 0.f : b1[c];
                    d0[c] = ((fd0 >> c) & 1u) ? 0.f : d0[c];
                    d1[c] = ((fd1 >> c) & 1u) ? 0.f : d1[c];
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c)
                face4<float2>(make_float2(a0[c], b0[c]), make_float2(a1[c], b1[c]), make_float2(c0[c], d0[c]),
                              make_float2(c1[c], d1[c]), F[c]);
        };

        float2 Gp[3][4];   // carried top-plane part (the column warp uses the .x halves)
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int f = 0; f < 4; ++f) Gp[c][f] = make_float2(0.f, 0.f);

        // one element layer k (bottom plane k, top plane k + 1)
        auto layer_step = [&](int k) {
            const int qb = q_base + (k - p0 + 1);
            const int sb = qslot, st = qslot + 1 == NS ? 0 : qslot + 1;
            const unsigned ptp = qslot + 1 == NS ? qphase ^ 1u : qphase;
            if (is_comp) {
                mbar_wait(&full[sb], qphase, err);
                mbar_wait(&full[st], ptp, err);
            }
            const unsigned sob = (unsigned)sb * LY::SLOT, sot = (unsigned)st * LY::SLOT;
            const int par = layer & 1;
            const bool lay_ok = k >= 0 && k < nz;
            const unsigned kk = (unsigned)k;
            float2 Kr[3];      // pair warp: own y1-row corner sums at the owned nodes (A, B halves)
            float n0y1[3];     // lane 0 of the first tile column: node 0's y1-row corner
            if (is_comp) {
                float2 E2 = make_float2(0.f, 0.f);
                {
                    const float* er = reinterpret_cast<const float*>(smem + sob + er0) + ((e0 + NPe * kk) & 3u);
                    if (vA && lay_ok) E2.x = er[0];
                    if (vB && lay_ok) E2.y = er[32];
                }
                float2 Fbot[3][4], Ftop[3][4];
                load_face(sob, k, Fbot);
                load_face(sot, k + 1, Ftop);
                float2 cor[3][4], en2;
                const bool want_en = MODE == OP_RESID && a.gt != nullptr && is_pair;
                if (want_en) elem_layer<float2, true>(kg, Ftop, Fbot, E2, Gp, cor, en2);
                else elem_layer<float2, false>(kg, Ftop, Fbot, E2, Gp, cor, en2);
                if (is_pair) {
                    if (want_en && w >= 1 && k >= p0 && lay_ok) {   // each element once: its tile, its segment
                        const long long e = (long long)X0 + lane + (long long)nx * ((long long)je + (long long)ny * k);
                        if (vA) a.gt[e] = -a.Ed[e] * en2.x;
                        if (vB) a.gt[e + 32] = -a.Ed[e + 32] * en2.y;
                    }
                    // x neighbours: node l+1 = A(l) x1 + A(l+1) x0, node l+33 = B(l) x1 + B(l+1) x0; lane 31:
                    // A(31) x1 + B(0) x0, and B(31) x1 + the column warp's x0 (added after the barrier)
                    const int src = (lane + 1) & 31;
                    const bool l31 = lane == 31;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float sa0 = __shfl_sync(0xffffffffu, cor[c][0].x, src);
                        const float sb0 = __shfl_sync(0xffffffffu, cor[c][0].y, src);
                        const float sa2 = __shfl_sync(0xffffffffu, cor[c][2].x, src);
                        const float sb2 = __shfl_sync(0xffffffffu, cor[c][2].y, src);
                        xbuf[par][w][c][lane] = vadd(cor[c][1], make_float2(l31 ? sb0 : sa0, l31 ? 0.f : sb0));
                        Kr[c] = vadd(cor[c][3], make_float2(l31 ? sb2 : sa2, l31 ? 0.f : sb2));
                        n0y1[c] = cor[c][2].x;
                    }
                    if (!FAST && lane == 0)
#pragma unroll
                        for (int c = 0; c < 3; ++c) xb0[par][w][c] = cor[c][0].x;
                } else if (lane < NPW) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        colbuf[par][lane][c] = cor[c][0].x;       // x0 corner, row y0 (node row je)
                        colbuf[par][lane][3 + c] = cor[c][2].x;   // x0 corner, row y1 (node row je + 1)
                    }
                }
            }
            __syncthreads();
            if (owner && k >= p0) {
                // ------------------------------------------------------------ epilogue: node row jn, plane k
                float2 Kx[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float2 v = Kr[c];
                    if (has_next) v = vadd(v, xbuf[par][w + 1][c][lane]);
                    if (lane == 31) v.y += colbuf[par][w][3 + c] + (has_next ? colbuf[par][w + 1][c] : 0.f);
                    Kx[c] = v;
                }
                const int ob = (int)((uo + 3u * NPn * kk) & 3u);
                const float* xr = reinterpret_cast<const float*>(smem + sob + uo_r) + ob;
                float2 xv[3], bv[3], dv[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) xv[c] = make_float2(xr[c], xr[96 + c]);
                if (NEED_B) {
                    const float* br = reinterpret_cast<const float*>(smem + sob + bo_r) + ob;
#pragma unroll
                    for (int c = 0; c < 3; ++c) bv[c] = make_float2(br[c], br[96 + c]);
                }
                if (NEED_D && (MODE == OP_SMOOTH || dz)) {
                    const float* dr = reinterpret_cast<const float*>(smem + sob + bo_r + (LY::D - LY::B)) + ob;
#pragma unroll
                    for (int c = 0; c < 3; ++c) dv[c] = make_float2(dr[c], dr[96 + c]);
                }
                if (!FAST && masked) {   // K^ is the identity on fixed DOFs
                    const unsigned char* mr = smem + sob + mo_r + ((mo + NPn * kk) & 15u);
                    const unsigned f1 = mr[0], f2 = mr[32];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        Kx[c].x = ((f1 >> c) & 1u) ? xv[c].x : Kx[c].x;
                        Kx[c].y = ((f2 >> c) & 1u) ? xv[c].y : Kx[c].y;
                    }
                }
                float2 out[3], zo[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (MODE == OP_APPLY) {
                        out[c] = Kx[c];
                    } else if (MODE == OP_Q) {
                        out[c] = Kx[c];
                        const float2 pr = vmul(vm, vmul(xv[c], Kx[c]));
                        acc0 += pr.x + pr.y;
                    } else if (MODE == OP_BMINUS) {
                        out[c] = vsub(bv[c], Kx[c]);
                    } else if (MODE == OP_SMOOTH) {
                        out[c] = vfma(vmul(vsplat<float2>(a.omega), vsub(bv[c], Kx[c])), dv[c], xv[c]);
                        const float2 pr = vmul(vm, vmul(bv[c], out[c]));
                        acc0 += pr.x + pr.y;
                    } else {   // OP_RESID
                        const float2 rr = vsub(bv[c], Kx[c]);
                        out[c] = rr;
                        const float2 rm = vmul(vm, rr);
                        if (dz) {
                            zo[c] = vmul(rr, dv[c]);
                            const float2 pz = vmul(rm, zo[c]);
                            acc0 += pz.x + pz.y;
                        }
                        const float2 r2 = vmul(rm, rr);
                        acc1 += r2.x + r2.y;
                        accmax = fmaxf(accmax, fmaxf(fabsf(rm.x), fabsf(rm.y)));
                        const float2 bx = vmul(vm, vmul(bv[c], xv[c]));
                        acc3 += bx.x + bx.y;
                    }
                }
                const long long nd = (long long)X0 + lane + 1 + (long long)nxn * jn + NPl * k;
                auto store = [&](float* base, const float2 (&o)[3]) {
                    float* pa = base + 3 * nd;
                    if (v1) {
                        pa[0] = o[0].x;
                        pa[1] = o[1].x;
                        pa[2] = o[2].x;
                    }
                    if (v2) {
                        pa[96] = o[0].y;
                        pa[97] = o[1].y;
                        pa[98] = o[2].y;
                    }
                };
                store(a.y, out);
                if (dz) store(a.z, zo);
                // node 0 of the first tile column: the A element's x0 corners alone
                if (!FAST && t == 0 && lane == 0) {
                    float K0[3], x0v[3], b0v[3], d0v[3];
                    const float* ub = reinterpret_cast<const float*>(smem + sob + LY::U);
                    const float* bb = reinterpret_cast<const float*>(smem + sob + LY::B);
                    const float* db = reinterpret_cast<const float*>(smem + sob + LY::D);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        K0[c] = n0y1[c] + (has_next ? xb0[par][w + 1][c] : 0.f);
                        x0v[c] = ub[(w + 1) * kUPitch + ob + c];
                        b0v[c] = NEED_B ? bb[w * kUPitch + ob + c] : 0.f;
                        d0v[c] = (NEED_D && (MODE == OP_SMOOTH || dz)) ? db[w * kUPitch + ob + c] : 0.f;
                    }
                    if (masked) {
                        const unsigned f0 = smem[sob + LY::M + (w + 1) * kMPitch + ((mo + NPn * kk) & 15u)];
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            if ((f0 >> c) & 1u) K0[c] = x0v[c];
                    }
                    const long long nd0 = (long long)nxn * jn + NPl * k;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float o;
                        if (MODE == OP_APPLY) {
                            o = K0[c];
                        } else if (MODE == OP_Q) {
                            o = K0[c];
                            acc0 = fmaf(x0v[c], K0[c], acc0);
                        } else if (MODE == OP_BMINUS) {
                            o = b0v[c] - K0[c];
                        } else if (MODE == OP_SMOOTH) {
                            o = fmaf(a.omega * (b0v[c] - K0[c]), d0v[c], x0v[c]);
                            acc0 = fmaf(b0v[c], o, acc0);
                        } else {
                            o = b0v[c] - K0[c];
                            if (dz) {
                                const float zz = o * d0v[c];
                                a.z[3 * nd0 + c] = zz;
                                acc0 = fmaf(o, zz, acc0);
                            }
                            acc1 = fmaf(o, o, acc1);
                            accmax = fmaxf(accmax, fabsf(o));
                            acc3 = fmaf(b0v[c], x0v[c], acc3);
                        }
                        a.y[3 * nd0 + c] = o;
                    }
                }
            }
            if (warp == PW) {
                // refill: loads [0, qb + NS) may now be in flight (every load below qb is consumed)
                const int target = min(total_loads, qb + NS);
                while (issued < target) issue_one();
            }
            // the next layer's bottom load is qb + 1
            if (++qslot == NS) {
                qslot = 0;
                qphase ^= 1u;
            }
            ++layer;
        };

        for (int k = p0 - 1; k < p1; ++k) layer_step(k);
        // the next segment's bottom load is this one's last top load + 1
        if (++qslot == NS) {
            qslot = 0;
            qphase ^= 1u;
        }
    };

    while (wk.seg(col, p0, p1)) {
        const int t = col % a.tiles_x;
        const bool fast = t > 0 && kTX * t + kTX < nx && a.tmask != nullptr && a.tmask[col] == 0;
        if (fast) segment(std::true_type{});
        else segment(std::false_type{});
        q_base += p1 - p0 + 2;
        wk.u += p1 - p0;
    }

    // ---- fused reductions (deterministic: block tree, then the last CTA folds in CTA order)
    const unsigned bid = blockIdx.x, nblocks = gridDim.x;
    if (MODE == OP_SMOOTH && a.first_step == 2) {
        float v[1] = {acc0};
        const int kind[1] = {0};
        double tot[1];
        block_reduce<float, 1>(v, kind, reinterpret_cast<float*>(red_sh));
        if (finish_reduction<float, 1>(v, kind, a.red, a.counter, tot, red_sh, bid, nblocks) && threadIdx.x == 0) {
            a.sc->rz = tot[0];
            if (!isfinite(tot[0])) set_err(&a.sc->err, TO_ERR_NONFINITE);
        }
    }
    if (MODE == OP_Q) {
        float v[1] = {acc0};
        const int kind[1] = {0};
        double tot[1];
        block_reduce<float, 1>(v, kind, reinterpret_cast<float*>(red_sh));
        if (finish_reduction<float, 1>(v, kind, a.red, a.counter, tot, red_sh, bid, nblocks) && threadIdx.x == 0) {
            DevScalars* sc = a.sc;
            sc->zq = tot[0];
            const double rz = sc->rz;
            double beta = (tot[0] > 0.0 && rz != 0.0) ? rz / tot[0] : 0.0;
            if (!isfinite(beta)) {
                set_err(&sc->err, TO_ERR_NONFINITE);
                beta = 0.0;
            }
            sc->beta = beta;
            if (a.first_step) sc->beta_first = beta;
            sc->n_inner_done += 1;
        }
    } else if (MODE == OP_RESID) {
        float v[4] = {acc0, acc1, accmax, acc3};
        const int kind[4] = {0, 0, 1, 0};
        double tot[4];
        block_reduce<float, 4>(v, kind, reinterpret_cast<float*>(red_sh));
        if (finish_reduction<float, 4>(v, kind, a.red, a.counter, tot, red_sh, bid, nblocks) && threadIdx.x == 0) {
            DevScalars* sc = a.sc;
            sc->rz = tot[0];
            if (a.first_step) {
                sc->res2 = sqrt(tot[1]);
                sc->res_inf = tot[2];
                sc->J = tot[3];
            }
            if (!isfinite(tot[1]) || !isfinite(tot[0])) set_err(&sc->err, TO_ERR_NONFINITE);
        }
    }
}

// ----------------------------------------------------------------------------- host
namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
}  // namespace

int encode_map_1d(CUtensorMap* out, const void* base, unsigned long long n, CUtensorMapDataType dtype, unsigned esize,
                  unsigned box) {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    });
    if (!g_encode) return fail(TO_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0) return fail(TO_ERR_ARG, "TMA source not 16-byte aligned");
    if ((box * esize) % 16 != 0 || box > 256) return fail(TO_ERR_ARG, "bad TMA box");
    // the vector as a 2-D tensor of one row (n x 1): a rank-2 map with an explicit row
    // stride (the byte length rounded up to 16), boxes of box x 1
    const unsigned long long row = (n * esize + 15ull) & ~15ull;
    cuuint64_t dims[2] = {(cuuint64_t)n, 1};
    cuuint64_t strides[1] = {(cuuint64_t)row};
    cuuint32_t bx[2] = {box, 1};
    cuuint32_t es[2] = {1, 1};
    const CUresult r = g_encode(out, dtype, 2, const_cast<void*>(base), dims, strides, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(TO_ERR_CUDA, "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ", n " +
                                     std::to_string(n) + ", box " + std::to_string(box) + ", element " +
                                     std::to_string(esize) + " B)");
    return TO_OK;
}

constexpr int kTmaTYW = kTmaTileY;

template <int MODE>
constexpr int tma_ns() {
    return (MODE == OP_RESID || MODE == OP_SMOOTH || MODE == OP_BMINUS) ? 5 : 6;
}

// the ring plus 128 bytes of slack for aligning its start to 128 bytes
template <int MODE>
static size_t tma_smem() {
    return (size_t)tma_ns<MODE>() * TmaLayout<kTmaTYW, (MODE == OP_RESID || MODE == OP_SMOOTH || MODE == OP_BMINUS)>::SLOT +
           128;
}

template <int MODE>
static const void* tma_fn() {
    return (const void*)k_op_tma<kTmaTYW, MODE, tma_ns<MODE>()>;
}

// the dynamic shared-memory opt-in of every mode (on the problem's device, before any capture)
int operator_tma_init(to_problem* P) {
    const void* fns[5] = {tma_fn<OP_APPLY>(), tma_fn<OP_RESID>(), tma_fn<OP_Q>(), tma_fn<OP_SMOOTH>(),
                          tma_fn<OP_BMINUS>()};
    const size_t sm[5] = {tma_smem<OP_APPLY>(), tma_smem<OP_RESID>(), tma_smem<OP_Q>(), tma_smem<OP_SMOOTH>(),
                          tma_smem<OP_BMINUS>()};
    for (int m = 0; m < 5; ++m) {
        TO_CUDA(cudaFuncSetAttribute(fns[m], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm[m]));
        int occ = 0;
        TO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fns[m], (kTmaTYW + 3) * 32, sm[m]));
        P->tma_occ[m] = occ;
    }
    P->tma_ready = 1;
    for (int m = 0; m < 5; ++m)
        if (P->tma_occ[m] < 1) P->tma_ready = 0;
    return TO_OK;
}

// can this launch take the TMA kernel: FP32, 32-bit copy coordinates, aligned vectors
bool operator_tma_applicable(const to_problem* P, int level, const void* x, const void* y, const void* b) {
    if (P->prec != TO_FP32_MIXED || !P->tma_ready || P->prm.op_kernel != 1) return false;
    const Level& L = P->lv[level];
    // every copy coordinate (planes -1 .. nz + 1 included) fits a signed 32-bit int
    if (3.0 * ((double)L.n_node + 2.0 * (L.nx + 1.0) * (L.ny + 1.0)) + 1024.0 > 2147483647.0) return false;
    // a tensor map's box may not exceed the vector it spans
    if (L.n_dof < kUBox || L.n_elem < kEBox || L.n_node < kMBox) return false;
    // the element matrix's non-zeros take the eight group values the kernel keeps in registers
    double rep[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    bool seen[8] = {false, false, false, false, false, false, false, false};
    for (int n = 0; n < kHaarNnz; ++n) {
        const int g = haar_group(n);
        if (!seen[g]) {
            seen[g] = true;
            rep[g] = P->haar[n];
        } else if (std::fabs(P->haar[n] - rep[g]) > 1e-12 * std::fabs(rep[g])) {
            return false;
        }
    }
    auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    auto al8 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; };
    if (!al16(x) || !al8(y) || (b && !al16(b)) || !al16(L.E) || !al16(L.mask) || !al16(L.dinv)) return false;
    return L.tmask64 != nullptr;
}

int launch_operator_tma(to_problem* P, int level, int mode, const void* x, void* y, const void* b, cudaStream_t s,
                        double omega, int first, const OpOut* out) {
    const Level& L = P->lv[level];
    TOpArgs a{};
    a.nx = L.nx;
    a.ny = L.ny;
    a.nz = L.nz;
    a.tiles_x = (L.nx + kTX - 1) / kTX;
    a.tiles_y = (L.ny + kTmaTYW - 1) / kTmaTYW;
    a.units = (long long)a.tiles_x * a.tiles_y * (L.nz + 1);
    a.y = (float*)y;
    a.tmask = L.tmask64;
    const double hs = L.h / P->g.h;
    for (int n = 0; n < kHaarNnz; ++n) a.kg[haar_group(n)] = (float)(P->haar[n] * hs);
    a.omega = (float)omega;
    a.red = P->red;
    a.sc = P->sc;
    a.first_step = first;
    const void* dinv = L.dinv;
    a.load_d = 0;
    if (mode == OP_RESID) {
        a.counter = P->counters + 0;
        a.z = (P->prm.precond == TO_PRECOND_JACOBI && level == 0) ? (float*)P->z : nullptr;
        a.Ed = (const float*)P->Ed;
        a.gt = (float*)P->gt;
        if (out) {
            a.z = (float*)out->z;
            a.gt = (float*)out->gt;
        }
        if (a.z && (reinterpret_cast<uintptr_t>(a.z) & 7u)) return fail(TO_ERR_ARG, "z not 8-byte aligned");
        a.load_d = a.z != nullptr;
    } else if (mode == OP_Q) {
        a.counter = P->counters + 1;
    } else if (mode == OP_SMOOTH) {
        a.counter = P->counters + 6;
        a.load_d = 1;
    }
    CUtensorMap mx, mE, mm, mb, md;
    std::memset(&mb, 0, sizeof mb);
    std::memset(&md, 0, sizeof md);
    int rc;
    if ((rc = encode_map_1d(&mx, x, (unsigned long long)L.n_dof, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, kUBox)) ||
        (rc = encode_map_1d(&mE, L.E, (unsigned long long)L.n_elem, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, kEBox)) ||
        (rc = encode_map_1d(&mm, L.mask, (unsigned long long)L.n_node, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, kMBox)))
        return rc;
    const bool need_b = mode == OP_RESID || mode == OP_SMOOTH || mode == OP_BMINUS;
    const bool need_d = a.load_d != 0;
    if (need_b && (rc = encode_map_1d(&mb, b, (unsigned long long)L.n_dof, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, kUBox)))
        return rc;
    if (need_d && (rc = encode_map_1d(&md, dinv, (unsigned long long)L.n_dof, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, kUBox)))
        return rc;
    long long grid = (long long)P->num_sms * std::max(1, P->tma_occ[mode]);
    if (grid > a.units) grid = a.units;
    if (grid > kMaxRedBlocks) grid = kMaxRedBlocks;
    const dim3 blk((kTmaTYW + 3) * 32);
    switch (mode) {
        case OP_APPLY:
            k_op_tma<kTmaTYW, OP_APPLY, tma_ns<OP_APPLY>()><<<(unsigned)grid, blk, tma_smem<OP_APPLY>(), s>>>(a, mx, mE, mm, mb, md);
            break;
        case OP_RESID:
            k_op_tma<kTmaTYW, OP_RESID, tma_ns<OP_RESID>()><<<(unsigned)grid, blk, tma_smem<OP_RESID>(), s>>>(a, mx, mE, mm, mb, md);
            break;
        case OP_Q:
            k_op_tma<kTmaTYW, OP_Q, tma_ns<OP_Q>()><<<(unsigned)grid, blk, tma_smem<OP_Q>(), s>>>(a, mx, mE, mm, mb, md);
            break;
        case OP_SMOOTH:
            k_op_tma<kTmaTYW, OP_SMOOTH, tma_ns<OP_SMOOTH>()><<<(unsigned)grid, blk, tma_smem<OP_SMOOTH>(), s>>>(a, mx, mE, mm, mb, md);
            break;
        case OP_BMINUS:
            k_op_tma<kTmaTYW, OP_BMINUS, tma_ns<OP_BMINUS>()><<<(unsigned)grid, blk, tma_smem<OP_BMINUS>(), s>>>(a, mx, mE, mm, mb, md);
            break;
        default:
            return fail(TO_ERR_ARG, "bad operator mode");
    }
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

// per tile column of the 64 x kTmaTileY tiling: does its node footprint (x from 64 t to
// 64 t + 65, y from j0 - 1 to j0 + kTmaTileY, every z) hold a fixed DOF?
int build_tile_mask64(Level& L, const uint8_t* mask_host) {
    const int nxn = L.nx + 1, nyn = L.ny + 1, nzn = L.nz + 1;
    std::vector<uint8_t> colm((size_t)nxn * nyn, 0);
    for (int k = 0; k < nzn; ++k)
        for (int j = 0; j < nyn; ++j)
            for (int i = 0; i < nxn; ++i)
                if (mask_host[(size_t)i + (size_t)nxn * ((size_t)j + (size_t)nyn * k)]) colm[(size_t)i + (size_t)nxn * j] = 1;
    const int tx = (L.nx + kTX - 1) / kTX, ty = (L.ny + kTmaTileY - 1) / kTmaTileY;
    std::vector<uint8_t> t((size_t)tx * ty, 0);
    for (int s = 0; s < ty; ++s)
        for (int c = 0; c < tx; ++c) {
            uint8_t f = 0;
            for (int j = std::max(kTmaTileY * s - 1, 0); j <= std::min(kTmaTileY * s + kTmaTileY, nyn - 1) && !f; ++j)
                for (int i = kTX * c; i <= std::min(kTX * c + kTX + 1, nxn - 1); ++i)
                    if (colm[(size_t)i + (size_t)nxn * j]) {
                        f = 1;
                        break;
                    }
            t[(size_t)c + (size_t)tx * s] = f;
        }
    void* d = nullptr;
    TO_CUDA(cudaMalloc(&d, t.size()));
    TO_CUDA(cudaMemcpy(d, t.data(), t.size(), cudaMemcpyHostToDevice));
    L.tmask64 = (uint8_t*)d;
    return TO_OK;
}

}  // namespace to
