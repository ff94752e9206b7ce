// Matrix-free hex8 operator y = K^(E) x in FP32 with the element contraction on the
// fifth-generation tensor cores (Sec. III: K = sum_e E_e K_e, fixtures eliminated),
// with the fused epilogues of the general operator kernel (the lower-level steps of
// Algorithms 1 / 3 and the multigrid smoother).
//
// Contraction.  Per element layer, the 24 nodal values of each of a CTA's 256 element
// columns are a row of A; the element matrix of the level (the unit matrix scaled by
// the element edge) is B; tcgen05.mma computes D = A B^T for two groups of 128 rows
// into tensor memory (M 128, N 32: the 24 outputs padded, K 32: two faces of 12 inputs
// each padded to 16), accumulating in FP32.  A and B enter as split BF16 pairs,
// v = v_hi + v_lo with v_hi = RN(v), v_lo = RN(v - v_hi), and D = A_hi B_hi + A_lo B_hi
// + A_hi B_lo: three passes, a relative error of about 2^-16 per product term (the
// dropped A_lo B_lo and the pieces' rounding).  Each thread reads its element's row
// of D back with tcgen05.ld, scales it by E_e and adds it into the node sums.
//
// Faces.  A row is [bottom face | top face] of the element, where a face is the
// element column's 2 x 2 nodes on one node plane: 12 values in the K order
// (x, y) of corners 00, 10, 01, 11, then their z, then four zeros.  The top face of
// layer k is the bottom face of layer k + 1, so each face is split and stored once:
// three face planes of A live in shared memory (canonical K-major layout without
// swizzle, 8-row x 16-byte core matrices), and the two MMAs of a pass read faces k and
// k + 1 through their own descriptors.  D's columns follow the same order per face:
// 0-7 (x, y) and 8-11 z of the bottom corners, 12-19 and 20-23 of the top corners.
//
// Work decomposition and node sums as in the general kernel: a CTA of 32 x 8 threads
// owns 31 x 7 node columns and a range of planes, walks element layers upwards, carries
// the top-face part of each layer's result to the next, sums x neighbours by shuffles
// and y neighbours through shared memory, in a fixed order (no atomics).
//
// Pipeline, one barrier per layer.  In the iteration of layer k: copies of plane k + 4
// are issued (cp.async ring of six planes), the face of plane k + 2 is split and stored,
// the product of layer k (issued one iteration earlier) is waited for and read back,
// plane k + 3 lands; after the barrier one thread issues the product of layer k + 1 into
// the other tensor-memory buffer while every thread finishes node plane k.  Waits on the
// products are bounded: after kMbarSpins polls the kernel records TO_ERR_TIMEOUT, stops
// walking, waits once more (bounded) for its last product and frees its tensor memory.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>

#include "device.cuh"
#include "tma.cuh"

namespace to {

namespace {

constexpr int kTcTX = 32, kTcTY = 8, kTcNT = kTcTX * kTcTY;
constexpr int kTcPN = (kTcTX + 1) * (kTcTY + 1);      // staged nodes per plane (33 x 9)
constexpr int kTcSR = (kTcPN + kTcNT - 1) / kTcNT;    // staged nodes per thread
constexpr int kTcRing = 6;                            // staged planes
constexpr int kTcFaces = 3;                           // face planes of A
constexpr unsigned kTcCols = 128;                     // tensor-memory columns: 2 buffers x 2 groups x 32
// instruction descriptor: D F32, A and B BF16, both K-major, N = 32, M = 128
constexpr unsigned kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

struct TcSmem {
    unsigned char face[kTcFaces][2][2][4096];   // [face plane][row group][hi, lo]: 128 rows x 16 BF16
    unsigned char bmat[2][2][1024];             // [hi, lo][bottom, top face]: 32 rows x 16 BF16
    float4 plane[kTcRing][kTcPN];               // node values (x, y, z, pad), fixed components zeroed
    uint32_t mword[kTcRing][kTcPN];             // 4-byte word holding each node's mask byte
    float ebuf[kTcRing][kTcTY][kTcTX];          // element moduli of the CTA's columns, per layer
    float4 ybuf[2][kTcTY][kTcTX];               // y-neighbour corner sums, two layers
    double red[32 * kRedQ];
    uint64_t mbar[2];                           // product of the layer in tensor-memory buffer 0 / 1 done
    unsigned tmem;                              // tensor-memory base address
    int abort;                                  // a bounded wait gave up: stop walking
};
constexpr size_t kTcSmemBytes = sizeof(TcSmem) + 128;   // slack to align the start to 128 bytes

// shared-memory matrix descriptor: canonical K-major layout without swizzle, core
// matrices 8 rows x 16 bytes, K-adjacent core matrices 128 bytes apart, 8-row groups
// 256 bytes apart (a 16-wide BF16 face per row)
__device__ __forceinline__ uint64_t tc_desc(unsigned addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(256u >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void tc_mma(unsigned d, uint64_t da, uint64_t db, unsigned acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(da), "l"(db), "r"(kTcIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// the warp's 32 lanes of tensor memory, 24 columns from taddr: one row of D per thread
__device__ __forceinline__ void tc_ld24(unsigned taddr, float (&d)[24]) {
    uint32_t r[24];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
                   "=r"(r[23])
                 : "r"(taddr + 16u)
                 : "memory");
    // the registers are operands of the wait, so no use of them moves above it
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23])
                 :
                 : "memory");
#pragma unroll
    for (int i = 0; i < 24; ++i) d[i] = __uint_as_float(r[i]);
}

// (a, b) -> BF16 pairs: hi = RN(a), RN(b); lo = RN(a - hi_a), RN(b - hi_b) (low half a)
__device__ __forceinline__ void tc_split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const uint32_t hw = *reinterpret_cast<const uint32_t*>(&h);
    const float ah = __uint_as_float(hw << 16), bh = __uint_as_float(hw & 0xffff0000u);
    const __nv_bfloat162 l = __floats2bfloat162_rn(__fsub_rn(a, ah), __fsub_rn(b, bh));
    hi = hw;
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}

__device__ __forceinline__ float2 tc_padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 tc_pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 tc_pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ bool tc_wait(uint64_t* bar, unsigned parity) {
    for (unsigned long long i = 0; i < kMbarSpins; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

}  // namespace

// launch arguments (the general operator kernel's, without its element constants)
struct TcArgs {
    int nx, ny, nz, kchunk;
    const float* x;
    float* y;
    const float* b;        // f (RESID) or right-hand side (SMOOTH / BMINUS)
    const float* dinv;     // 1 / diag(K^) (RESID with Jacobi z, SMOOTH)
    float* z;              // RESID: z = r / d (optional)
    const float* E;
    const float* Ed;       // RESID: dE/drho~ for the fused sensitivity (optional)
    float* gt;             // RESID: -E'_e u_e^T k_e u_e (optional)
    const uint8_t* mask;
    const uint8_t* tmask;  // per CTA tile column: any fixed node in its footprint (nullptr = assume yes)
    float omega;
    double* red;
    unsigned* counter;
    DevScalars* sc;
    int first_step;
};

template <int MODE>
__global__ void __launch_bounds__(kTcNT, 2) k_op_tc(const TcArgs a, const uint4* __restrict__ bglob) {
    constexpr int TX = kTcTX, TY = kTcTY, NT = kTcNT, PN = kTcPN, SR = kTcSR;
    constexpr bool NEED_B = MODE == OP_RESID || MODE == OP_SMOOTH || MODE == OP_BMINUS;
    constexpr bool NEED_D = MODE == OP_SMOOTH || MODE == OP_RESID;
    using P = float2;
    extern __shared__ __align__(16) unsigned char tc_smem_raw[];
    TcSmem& sm = *reinterpret_cast<TcSmem*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 127) & ~uintptr_t(127));

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + TX * ty;
    const int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
    const int X0 = bx * (TX - 1), Y0 = by * (TY - 1);
    const int kb = bz * a.kchunk;
    const int ke = min(kb + a.kchunk, a.nz + 1);
    const int nxn = a.nx + 1, nyn = a.ny + 1;
    const long long nplane = (long long)nxn * nyn;
    const long long eplane = (long long)a.nx * a.ny;
    const int ie = X0 - 1 + tx, je = Y0 - 1 + ty;
    const bool col_in = ie >= 0 && ie < a.nx && je >= 0 && je < a.ny;
    const int ni = X0 + tx, nj = Y0 + ty;
    const bool owner = tx < TX - 1 && ty < TY - 1 && ni < nxn && nj < nyn;
    const unsigned own_n = owner ? (unsigned)ni + (unsigned)nxn * (unsigned)nj : 0u;
    const unsigned own3 = 3u * own_n;
    const unsigned ecol = col_in ? (unsigned)ie + (unsigned)a.nx * (unsigned)je : 0u;
    const bool dz = NEED_D && a.dinv != nullptr && (MODE != OP_RESID || a.z != nullptr);
    const bool hm = a.tmask == nullptr || a.tmask[bx + ((a.nx + 1 + TX - 2) / (TX - 1)) * by] != 0;
    // this thread's row of A (element column) in its group of 128, and its lanes of D
    const int grp = ty >> 2;
    const int row = tx + 32 * (ty & 3);
    const unsigned frow = (unsigned)((row >> 3) * 256 + (row & 7) * 16);
    const int fidx = ty * (TX + 1) + tx;   // corner (0, 0) of the thread's face in a staged plane

    unsigned st_node[SR];
    bool st_ok[SR];
#pragma unroll
    for (int r = 0; r < SR; ++r) {
        const int sidx = tid + r * NT;
        const int px = sidx % (TX + 1), py = sidx / (TX + 1);
        const int gi = X0 - 1 + px, gj = Y0 - 1 + py;
        st_ok[r] = sidx < PN && gi >= 0 && gi < nxn && gj >= 0 && gj < nyn;
        st_node[r] = st_ok[r] ? (unsigned)gi + (unsigned)nxn * (unsigned)gj : 0u;
    }

    // every asynchronous copy that plane p (and element layer p - 1) needs, into ring slot SP
    auto issue = [&](int p, auto SPc) {
        constexpr int SP = decltype(SPc)::value;
        const bool pin = p >= 0 && p <= a.nz;
        const long long pn = pin ? (long long)p * nplane : 0;
        const float* xp = a.x + 3 * pn;
#pragma unroll
        for (int r = 0; r < SR; ++r) {
            const int sidx = tid + r * NT;
            if (sidx < PN) {
                const bool v = st_ok[r] && pin;
                const float* src = xp + 3u * st_node[r];
                float* dst = reinterpret_cast<float*>(&sm.plane[SP][sidx]);
                cp_async_4(dst + 0, src + 0, v);
                cp_async_4(dst + 1, src + 1, v);
                cp_async_4(dst + 2, src + 2, v);
                if (hm)
                    cp_async_4(&sm.mword[SP][sidx], reinterpret_cast<const uint32_t*>(a.mask) + ((st_node[r] + pn) >> 2),
                               v);
            }
        }
        const int L = p - 1;
        const bool ev = col_in && L >= 0 && L < a.nz;
        cp_async_4(&sm.ebuf[SP][ty][tx], a.E + (ev ? (long long)L * eplane : 0) + ecol, ev);
        cp_commit();
    };
    // fixed components of this thread's staged nodes of plane p set to zero
    auto patch = [&](int p, auto SPc) {
        constexpr int SP = decltype(SPc)::value;
        if (!hm || p < 0 || p > a.nz) return;
        const long long pn = (long long)p * nplane;
#pragma unroll
        for (int r = 0; r < SR; ++r) {
            const int sidx = tid + r * NT;
            if (sidx < PN && st_ok[r]) {
                const unsigned node = st_node[r] + (unsigned)pn;   // low bits only
                const uint32_t m = (sm.mword[SP][sidx] >> (8 * (node & 3u))) & 0xffu;
                if (m) {
                    float* dst = reinterpret_cast<float*>(&sm.plane[SP][sidx]);
                    if (m & 1) dst[0] = 0.f;
                    if (m & 2) dst[1] = 0.f;
                    if (m & 4) dst[2] = 0.f;
                }
            }
        }
    };
    // the thread's face of the staged plane in slot SP as its row of A in face plane FP
    auto write_face = [&](auto SPc, auto FPc) {
        constexpr int SP = decltype(SPc)::value;
        constexpr int FP = decltype(FPc)::value;
        const float4 n00 = sm.plane[SP][fidx], n10 = sm.plane[SP][fidx + 1];
        const float4 n01 = sm.plane[SP][fidx + TX + 1], n11 = sm.plane[SP][fidx + TX + 2];
        uint32_t h[6], l[6];
        tc_split2(n00.x, n00.y, h[0], l[0]);
        tc_split2(n10.x, n10.y, h[1], l[1]);
        tc_split2(n01.x, n01.y, h[2], l[2]);
        tc_split2(n11.x, n11.y, h[3], l[3]);
        tc_split2(n00.z, n10.z, h[4], l[4]);
        tc_split2(n01.z, n11.z, h[5], l[5]);
        unsigned char* fh = sm.face[FP][grp][0] + frow;
        unsigned char* fl = sm.face[FP][grp][1] + frow;
        *reinterpret_cast<uint4*>(fh) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(fh + 128) = make_uint4(h[4], h[5], 0u, 0u);
        *reinterpret_cast<uint4*>(fl) = make_uint4(l[0], l[1], l[2], l[3]);
        *reinterpret_cast<uint4*>(fl + 128) = make_uint4(l[4], l[5], 0u, 0u);
    };
    // one thread: the product of the layer whose faces are in FB (bottom) and FT (top),
    // both row groups, into tensor-memory buffer BUF; completion arrives on mbar[BUF]
    auto issue_mma = [&](unsigned tbase, auto FBc, auto FTc, auto BUFc) {
        constexpr int FB = decltype(FBc)::value;
        constexpr int FT = decltype(FTc)::value;
        constexpr int BUF = decltype(BUFc)::value;
        tc_fence_after();
        const uint64_t bhb = tc_desc(smem_u32(sm.bmat[0][0])), bht = tc_desc(smem_u32(sm.bmat[0][1]));
        const uint64_t blb = tc_desc(smem_u32(sm.bmat[1][0])), blt = tc_desc(smem_u32(sm.bmat[1][1]));
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            const unsigned d = tbase + (unsigned)(BUF * 64 + g * 32);
            const uint64_t ahb = tc_desc(smem_u32(sm.face[FB][g][0])), alb = tc_desc(smem_u32(sm.face[FB][g][1]));
            const uint64_t aht = tc_desc(smem_u32(sm.face[FT][g][0])), alt = tc_desc(smem_u32(sm.face[FT][g][1]));
            tc_mma(d, ahb, bhb, 0u);
            tc_mma(d, aht, bht, 1u);
            tc_mma(d, alb, bhb, 1u);
            tc_mma(d, alt, bht, 1u);
            tc_mma(d, ahb, blb, 1u);
            tc_mma(d, aht, blt, 1u);
        }
        tc_commit(&sm.mbar[BUF]);
    };

    // ---- set-up: the element matrix pieces, the barriers, tensor memory
    cp_async_16(reinterpret_cast<unsigned char*>(&sm.bmat[0][0][0]) + 16 * tid, bglob + tid);
    cp_commit();
    if (tid == 0) {
        mbar_init(&sm.mbar[0], 1);
        mbar_init(&sm.mbar[1], 1);
        sm.abort = 0;
        fence_mbar_init();
    }
    if (ty == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using I3 = std::integral_constant<int, 3>;
    issue(kb - 1, I0{});
    issue(kb, I1{});
    issue(kb + 1, I2{});
    issue(kb + 2, I3{});
    cp_wait<1>();   // the matrix pieces and planes kb - 1 .. kb + 1
    patch(kb - 1, I0{});
    patch(kb, I1{});
    patch(kb + 1, I2{});
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tbase = sm.tmem;
    const unsigned tlane = tbase + ((unsigned)(32 * (ty & 3)) << 16) + (unsigned)(grp * 32);
    write_face(I0{}, I0{});
    write_face(I1{}, I1{});
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) issue_mma(tbase, I0{}, I1{}, I0{});

    float acc0 = 0.f, acc1 = 0.f, acc3 = 0.f, accmax = 0.f;
    P cxy[4];        // carried top-face part of the previous layer: (x, y) of corners 00, 10, 01, 11
    float cz[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        cxy[q] = P{0.f, 0.f};
        cz[q] = 0.f;
    }
    unsigned ph0 = 0, ph1 = 0;   // phase parity of mbar[0] / mbar[1]
    bool aborted = false;
    int pend_buf = -1;           // a product whose bounded wait gave up (its buffer and parity)
    unsigned pend_par = 0;

    // the iteration of layer k; J = (k - kb + 1) mod 6 fixes every slot at compile time
    auto layer = [&](int k, auto Jc) {
        constexpr int J = decltype(Jc)::value;
        constexpr int S0 = J % 6, S1 = (J + 1) % 6, S2 = (J + 2) % 6, S3 = (J + 3) % 6, S4 = (J + 4) % 6;
        constexpr int F1 = (J + 1) % 3, F2 = (J + 2) % 3;
        constexpr int BUF = J & 1;
        // (a) copies of plane k + 4; the epilogue's right-hand side and 1 / d at the owned node of plane k
        issue(k + 4, std::integral_constant<int, S4>{});
        const bool outp = owner && k >= kb;
        float ebv[3] = {0.f, 0.f, 0.f}, edv[3] = {0.f, 0.f, 0.f};
        const long long pofs = 3 * (long long)k * nplane;
        if (NEED_B && outp)
#pragma unroll
            for (int c = 0; c < 3; ++c) ebv[c] = __ldg(a.b + pofs + own3 + c);
        if (NEED_D && dz && outp)
#pragma unroll
            for (int c = 0; c < 3; ++c) edv[c] = __ldg(a.dinv + pofs + own3 + c);
        // (b) the face of plane k + 2 (the top of layer k + 1)
        if (k + 2 <= ke) write_face(std::integral_constant<int, S2>{}, std::integral_constant<int, F2>{});
        // (c) layer k's product: scaled by E_e, bottom part plus the carry = the column's share of plane k
        const unsigned par = BUF ? ph1 : ph0;
        const bool ok = tc_wait(&sm.mbar[BUF], par);
        if (BUF) ph1 ^= 1u;
        else ph0 ^= 1u;
        if (!ok) {
            set_err(&a.sc->err, TO_ERR_TIMEOUT);
            sm.abort = 1;
            pend_buf = BUF;
            pend_par = par;
        }
        tc_fence_after();
        float d[24];
        tc_ld24(tlane + (unsigned)(BUF * 64), d);
        if (MODE == OP_RESID) {
            if (a.gt && owner && col_in && k >= 0 && k < a.nz && k + 1 >= kb && k + 1 < ke) {
                const float4* pb = sm.plane[S0];
                const float4* pt = sm.plane[S1];
                const float4 u[8] = {pb[fidx], pb[fidx + 1], pb[fidx + TX + 1], pb[fidx + TX + 2],
                                     pt[fidx], pt[fidx + 1], pt[fidx + TX + 1], pt[fidx + TX + 2]};
                float en = 0.f;
#pragma unroll
                for (int f = 0; f < 2; ++f)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        en = fmaf(u[4 * f + q].x, d[12 * f + 2 * q], en);
                        en = fmaf(u[4 * f + q].y, d[12 * f + 2 * q + 1], en);
                        en = fmaf(u[4 * f + q].z, d[12 * f + 8 + q], en);
                    }
                const long long e = (long long)k * eplane + ecol;
                a.gt[e] = -a.Ed[e] * en;
            }
        }
        const float Ee = sm.ebuf[S1][ty][tx];
        const P E2{Ee, Ee};
        P sxy[4];
        float sz[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            sxy[q] = tc_pfma(E2, P{d[2 * q], d[2 * q + 1]}, cxy[q]);
            sz[q] = fmaf(Ee, d[8 + q], cz[q]);
            cxy[q] = tc_pmul(E2, P{d[12 + 2 * q], d[13 + 2 * q]});
            cz[q] = Ee * d[20 + q];
        }
        // node (X0 + tx, Y0 + ty): corner 11 of this column, 01 of column tx + 1; the
        // row above adds corners 10 and 00 of its columns through shared memory
        P n01, n00;
        n01.x = __shfl_down_sync(0xffffffffu, sxy[2].x, 1);
        n01.y = __shfl_down_sync(0xffffffffu, sxy[2].y, 1);
        n00.x = __shfl_down_sync(0xffffffffu, sxy[0].x, 1);
        n00.y = __shfl_down_sync(0xffffffffu, sxy[0].y, 1);
        const float m01 = __shfl_down_sync(0xffffffffu, sz[2], 1);
        const float m00 = __shfl_down_sync(0xffffffffu, sz[0], 1);
        const P Xp = tc_padd(sxy[3], n01);
        const float Xz = sz[3] + m01;
        const P Yp = tc_padd(sxy[1], n00);
        const float Yz = sz[1] + m00;
        if (k >= kb) sm.ybuf[BUF][ty][tx] = make_float4(Yp.x, Yp.y, Yz, 0.f);
        // (d) plane k + 3 landed (this thread's copies), fixed components zeroed
        cp_wait<1>();
        patch(k + 3, std::integral_constant<int, S3>{});
        // (e) one barrier: the new face, plane k + 3, the y sums and tensor-memory reads
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (sm.abort) {
            aborted = true;
            return;
        }
        // (f) the product of layer k + 1 into the other buffer
        if (tid == 0 && k + 1 < ke)
            issue_mma(tbase, std::integral_constant<int, F1>{}, std::integral_constant<int, F2>{},
                      std::integral_constant<int, BUF ^ 1>{});
        // (g) node plane k at the owned node
        if (outp) {
            const float4 yb = sm.ybuf[BUF][ty + 1][tx];
            const float Kx3[3] = {Xp.x + yb.x, Xp.y + yb.y, Xz + yb.z};
            const int oidx = (ty + 1) * (TX + 1) + tx + 1;
            const float4 xs = sm.plane[S0][oidx];
            const float xv3[3] = {xs.x, xs.y, xs.z};
            uint32_t mk = 0;
            if (hm) mk = (sm.mword[S0][oidx] >> (8 * ((own_n + (unsigned)((long long)k * nplane)) & 3u))) & 0xffu;
            float* yo = a.y + pofs + own3;
            const float* xo = a.x + pofs + own3;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float Kx = Kx3[c], xv = xv3[c];
                if ((mk >> c) & 1) {   // K^ is the identity on fixed DOFs
                    xv = xo[c];
                    Kx = xv;
                }
                if (MODE == OP_APPLY) {
                    yo[c] = Kx;
                } else if (MODE == OP_Q) {
                    yo[c] = Kx;
                    acc0 = fmaf(xv, Kx, acc0);
                } else if (MODE == OP_BMINUS) {
                    yo[c] = ebv[c] - Kx;
                } else if (MODE == OP_SMOOTH) {
                    const float bv = ebv[c];
                    const float yv = xv + a.omega * (bv - Kx) * edv[c];
                    yo[c] = yv;
                    acc0 = fmaf(bv, yv, acc0);
                } else if (MODE == OP_RESID) {
                    const float bv = ebv[c];
                    const float rv2 = bv - Kx;
                    yo[c] = rv2;
                    if (a.z) {
                        const float zv = rv2 * edv[c];
                        a.z[pofs + own3 + c] = zv;
                        acc0 = fmaf(rv2, zv, acc0);
                    }
                    acc1 = fmaf(rv2, rv2, acc1);
                    accmax = fmaxf(accmax, fabsf(rv2));
                    acc3 = fmaf(bv, xv, acc3);
                }
            }
        }
    };

    // six layers per trip with every slot a compile-time constant; the remainder one at a time
    int j = 0;
    const int nlayers = ke - kb + 1;   // layers kb - 1 .. ke - 1
    while (j + 6 <= nlayers && !aborted) {
        const int k = kb - 1 + j;
        layer(k, I0{});
        if (aborted) break;
        layer(k + 1, I1{});
        if (aborted) break;
        layer(k + 2, I2{});
        if (aborted) break;
        layer(k + 3, I3{});
        if (aborted) break;
        layer(k + 4, std::integral_constant<int, 4>{});
        if (aborted) break;
        layer(k + 5, std::integral_constant<int, 5>{});
        j += 6;
    }
    for (; j < nlayers && !aborted; ++j) {
        const int k = kb - 1 + j;
        switch (j % 6) {
            case 0: layer(k, I0{}); break;
            case 1: layer(k, I1{}); break;
            case 2: layer(k, I2{}); break;
            case 3: layer(k, I3{}); break;
            case 4: layer(k, std::integral_constant<int, 4>{}); break;
            default: layer(k, std::integral_constant<int, 5>{}); break;
        }
    }
    cp_wait<0>();
    // a product whose wait gave up may still run: wait once more (bounded) before the
    // tensor memory is freed (every other product issued was waited for)
    if (pend_buf >= 0) tc_wait(&sm.mbar[pend_buf], pend_par);
    tc_fence_before();
    __syncthreads();
    if (ty == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTcCols) : "memory");
    }
    if (aborted) return;

    double* sh_red = sm.red;
    const unsigned bid = linear_block(), nblocks = grid_blocks();
    if (MODE == OP_SMOOTH && a.first_step == 2) {
        float v[1] = {acc0};
        const int kind[1] = {0};
        double tot[1];
        block_reduce<float, 1>(v, kind, reinterpret_cast<float*>(sh_red));
        if (finish_reduction<float, 1>(v, kind, a.red, a.counter, tot, sh_red, bid, nblocks) && tid == 0) {
            a.sc->rz = tot[0];
            if (!isfinite(tot[0])) set_err(&a.sc->err, TO_ERR_NONFINITE);
        }
    }
    if (MODE == OP_Q) {
        float v[1] = {acc0};
        const int kind[1] = {0};
        double tot[1];
        block_reduce<float, 1>(v, kind, reinterpret_cast<float*>(sh_red));
        if (finish_reduction<float, 1>(v, kind, a.red, a.counter, tot, sh_red, bid, nblocks) && tid == 0) {
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
        block_reduce<float, 4>(v, kind, reinterpret_cast<float*>(sh_red));
        if (finish_reduction<float, 4>(v, kind, a.red, a.counter, tot, sh_red, bid, nblocks) && tid == 0) {
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

// ----------------------------------------------------------------------------- host side
namespace {

uint16_t bf16_rn(float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float bf16_val(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float v;
    std::memcpy(&v, &u, 4);
    return v;
}

template <int MODE>
const void* tc_fn() {
    return (const void*)k_op_tc<MODE>;
}

}  // namespace

// the dynamic shared-memory opt-in and residency of every mode (before any capture)
int operator_tc_init(to_problem* P) {
    const void* fns[5] = {tc_fn<OP_APPLY>(), tc_fn<OP_RESID>(), tc_fn<OP_Q>(), tc_fn<OP_SMOOTH>(), tc_fn<OP_BMINUS>()};
    P->tc_ready = 0;
    for (int m = 0; m < 5; ++m) {
        TO_CUDA(cudaFuncSetAttribute(fns[m], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBytes));
        int occ = 0;
        TO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fns[m], kTcNT, kTcSmemBytes));
        // tensor memory: every resident CTA holds kTcCols of the SM's 512 columns
        if (occ < 1 || occ * kTcCols > 512) return TO_OK;
        P->tc_occ[m] = occ;
    }
    P->tc_ready = 1;
    return TO_OK;
}

// Per level: the element matrix of edge h (unit matrix x h) as split BF16 pieces in
// the B layout the kernel copies to shared memory: [hi, lo][bottom, top face] blocks
// of 32 output rows x 16 inputs, output n / input kk in the face order (x, y) of
// corners 00, 10, 01, 11, then their z; zero beyond 24 outputs and 12 inputs.
int operator_tc_build(to_problem* P) {
    if (P->prec != TO_FP32_MIXED || P->prm.op_kernel != 2 || !P->tc_ready) return TO_OK;
    // local node of the element matrix for corner (a, b) of face z
    auto node = [](int a, int b, int z) {
        static const int off[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0}, {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
        for (int l = 0; l < 8; ++l)
            if (off[l][0] == a && off[l][1] == b && off[l][2] == z) return l;
        return -1;
    };
    // position within a face (0 .. 11) -> (corner q = 2b + a, component)
    auto face_pos = [](int kk, int& q, int& c) {
        if (kk < 8) {
            q = kk / 2;
            c = kk % 2;
        } else {
            q = kk - 8;
            c = 2;
        }
    };
    for (Level& L : P->lv) {
        std::vector<uint16_t> buf(2 * 2 * 32 * 16, 0);
        for (int f = 0; f < 2; ++f)
            for (int n = 0; n < 24; ++n)
                for (int kk = 0; kk < 12; ++kk) {
                    int qo, co, qi, ci;
                    face_pos(n % 12, qo, co);
                    face_pos(kk, qi, ci);
                    const int lo = node(qo & 1, qo >> 1, n / 12), li = node(qi & 1, qi >> 1, f);
                    const double v = L.h * P->ke[(3 * lo + co) * 24 + 3 * li + ci];
                    const uint16_t h = bf16_rn((float)v);
                    const uint16_t l = bf16_rn((float)(v - (double)bf16_val(h)));
                    const size_t off = (size_t)(n / 8) * 128 + (size_t)(kk / 8) * 64 + (size_t)(n % 8) * 8 + (kk % 8);
                    buf[(0 * 2 + f) * 512 + off] = h;
                    buf[(1 * 2 + f) * 512 + off] = l;
                }
        if (!L.tcb) TO_CUDA(cudaMalloc(&L.tcb, buf.size() * sizeof(uint16_t)));
        TO_CUDA(cudaMemcpy(L.tcb, buf.data(), buf.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    }
    return TO_OK;
}

bool operator_tc_applicable(const to_problem* P, int level) {
    return P->prec == TO_FP32_MIXED && P->prm.op_kernel == 2 && P->tc_ready && P->lv[level].tcb != nullptr;
}

int choose_kchunk(long long columns, int planes, long long slots);

int launch_operator_tc(to_problem* P, int level, int mode, const void* x, void* y, const void* b, cudaStream_t s,
                       double omega, int first, const OpOut* out) {
    const Level& L = P->lv[level];
    if (3LL * (L.nx + 1) * (L.ny + 1) >= (1LL << 31)) return fail(TO_ERR_ARG, "grid plane too large for the operator kernel");
    TcArgs a{};
    a.nx = L.nx;
    a.ny = L.ny;
    a.nz = L.nz;
    a.x = (const float*)x;
    a.y = (float*)y;
    a.b = (const float*)b;
    a.dinv = (const float*)L.dinv;
    a.E = (const float*)L.E;
    a.mask = L.mask;
    a.tmask = L.tmask;
    a.omega = (float)omega;
    a.red = P->red;
    a.sc = P->sc;
    a.first_step = first;
    if (mode == OP_RESID) {
        a.counter = P->counters + 0;
        a.z = (P->prm.precond == TO_PRECOND_JACOBI && level == 0) ? (float*)P->z : nullptr;
        a.Ed = (const float*)P->Ed;
        a.gt = (float*)P->gt;
        if (out) {
            a.z = (float*)out->z;
            a.gt = (float*)out->gt;
        }
    } else if (mode == OP_Q) {
        a.counter = P->counters + 1;
    } else if (mode == OP_SMOOTH) {
        a.counter = P->counters + 6;
    }
    const int gx = (L.nx + 1 + kTcTX - 2) / (kTcTX - 1);
    const int gy = (L.ny + 1 + kTcTY - 2) / (kTcTY - 1);
    int kchunk = P->tile_z > 0 ? P->tile_z : L.kchunk;
    if (kchunk <= 0) kchunk = choose_kchunk((long long)gx * gy, L.nz + 1, (long long)P->tc_occ[mode] * P->num_sms);
    if (kchunk > L.nz + 1) kchunk = L.nz + 1;
    a.kchunk = kchunk;
    const int gz = (L.nz + 1 + kchunk - 1) / kchunk;
    if ((long long)gx * gy * gz > kMaxRedBlocks && (mode == OP_RESID || mode == OP_Q || mode == OP_SMOOTH))
        return fail(TO_ERR_ARG, "operator grid exceeds the reduction scratch; raise tile_z");
    const dim3 grid(gx, gy, gz), block(kTcTX, kTcTY);
    const uint4* bm = (const uint4*)L.tcb;
    switch (mode) {
        case OP_APPLY: k_op_tc<OP_APPLY><<<grid, block, kTcSmemBytes, s>>>(a, bm); break;
        case OP_RESID: k_op_tc<OP_RESID><<<grid, block, kTcSmemBytes, s>>>(a, bm); break;
        case OP_Q: k_op_tc<OP_Q><<<grid, block, kTcSmemBytes, s>>>(a, bm); break;
        case OP_SMOOTH: k_op_tc<OP_SMOOTH><<<grid, block, kTcSmemBytes, s>>>(a, bm); break;
        case OP_BMINUS: k_op_tc<OP_BMINUS><<<grid, block, kTcSmemBytes, s>>>(a, bm); break;
        default: return fail(TO_ERR_ARG, "bad operator mode");
    }
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

}  // namespace to
