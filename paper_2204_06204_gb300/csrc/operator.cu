// Matrix-free hex8 operator  y = K^(E) x  on a voxel grid (Sec. III:
// K = sum_e E_e K_e, fixtures eliminated), with fused epilogues for the
// lower-level steps (Algorithms 1 / 3, line 1) and the multigrid smoother.
//
// Work decomposition.  A CTA of TX x TY threads owns a (TX-1) x (TY-1) block of
// node columns and a range of node planes [kb, ke); thread (tx, ty) walks the
// element column (X0-1+tx, Y0-1+ty) upwards in z through element layers
// kb-1 .. ke-1 (one halo column / layer of recomputed elements per tile).
// Per element layer:
//   1. the CTA stages the (TX+1) x (TY+1) node plane k+1 in shared memory
//      (coalesced: consecutive threads read consecutive xyz words);
//   2. each thread forms the sum/difference coefficients of its element's top
//      face (2 x 12 butterfly adds); the bottom face is carried in registers
//      from the previous layer, so a z butterfly completes the 24 coefficients;
//   3. the element matrix is applied in that basis (45 products), scaled by E_e;
//   4. the inverse z butterfly splits the result into bottom-face and top-face
//      parts; the top part is carried to the next layer, the bottom part plus
//      the carry of the previous layer is the column's complete contribution
//      to node plane k, brought back to nodes by the inverse face butterflies;
//   5. the four columns around each owned node add their corner contributions
//      in a fixed order (no atomics: bitwise reproducible).
#include <algorithm>
#include <type_traits>
#include <vector>

#include "device.cuh"
#include "haar.cuh"
#include "transfer.cuh"

namespace to {

template <typename T>
struct OpArgs {
    int nx, ny, nz, kchunk;
    const T* x;
    T* y;
    const T* b;       // f (RESID) or right-hand side (SMOOTH / BMINUS)
    const T* dinv;    // 1 / diag(K^) (RESID with Jacobi z, SMOOTH)
    T* z;             // RESID: z = r / d (optional)
    const T* E;
    const T* Ed;      // RESID: dE/drho~ for the fused sensitivity (optional)
    T* gt;            // RESID: -E'_e u_e^T k_e u_e (optional)
    const uint8_t* mask;
    HaarK<T> kh;
    T omega;
    double* red;
    unsigned* counter;
    DevScalars* sc;
    const uint8_t* tmask;   // per CTA tile column: any fixed node in its footprint (nullptr = assume yes)
    int first_step;   // Q: record beta as the first step size of the iteration;
                      // RESID: this is the residual at u_k (record norms and J)
};

// ----------------------------------------------------------------------------- pairs
// (x, y) components travel as a pair: packed FP32x2 arithmetic for float,
// two scalar operations for double.
template <typename T> struct PairT;
template <> struct PairT<float> { using t = float2; };
template <> struct PairT<double> { using t = double2; };

__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) {   // one packed subtract (no -1 operand pair)
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 psub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) { return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)); }

template <typename T> struct Node4;
template <> struct Node4<float> { using t = float4; };
struct alignas(16) Dbl4 {
    double x, y, z, w;
};
template <> struct Node4<double> { using t = Dbl4; };

// 12 face coefficients (ss, sd, ds, dd) x (x, y, z): xy pairs and z scalars
template <typename T>
struct Face {
    typename PairT<T>::t p[4];
    T z[4];
};

template <typename T, typename N4>
__device__ __forceinline__ void face_forward4(const N4& a00, const N4& a10, const N4& a01, const N4& a11, Face<T>& F) {
    using P = typename PairT<T>::t;
    const P p00{a00.x, a00.y}, p10{a10.x, a10.y}, p01{a01.x, a01.y}, p11{a11.x, a11.y};
    const P sx0 = padd(p10, p00), dx0 = psub(p10, p00), sx1 = padd(p11, p01), dx1 = psub(p11, p01);
    F.p[0] = padd(sx1, sx0);
    F.p[1] = padd(dx1, dx0);
    F.p[2] = psub(sx1, sx0);
    F.p[3] = psub(dx1, dx0);
    const T zs0 = a10.z + a00.z, zd0 = a10.z - a00.z, zs1 = a11.z + a01.z, zd1 = a11.z - a01.z;
    F.z[0] = zs1 + zs0;
    F.z[1] = zd1 + zd0;
    F.z[2] = zs1 - zs0;
    F.z[3] = zd1 - zd0;
}

// Shared-memory layout of the operator kernel (NB-deep ring of staged planes).
template <typename T, int TX, int TY, int NB>
struct OpSmem {
    using N4 = typename Node4<T>::t;
    static constexpr int PN = (TX + 1) * (TY + 1);
    N4 plane[NB][PN];          // node values (xyz, pad), fixed components zeroed after landing
    uint32_t mword[NB][PN];    // 4-byte word holding each node's mask byte
    T ebuf[NB][TY][TX];        // element moduli of the CTA's columns, per layer
    T eb[NB][TY][TX][3];       // epilogue right-hand side at the owned node
    T ed[NB][TY][TX][3];       // epilogue inverse diagonal at the owned node
    N4 ybuf[TY][TX];
    double red[32 * kRedQ];
};

constexpr int kDepth = 2;                  // planes in flight ahead of the one being consumed
constexpr int kRing = kDepth + 2;

// The operator for one CTA tile (bx, by, bz) of one problem; `bid` / `nblocks` place
// the tile among the problem's tiles for the fused reductions.
template <typename T, int TX, int TY, int MODE>
__device__ __forceinline__ void op_body(const OpArgs<T>& a, const HaarK<T>& kh, int bx, int by, int bz, unsigned bid,
                                        unsigned nblocks) {
    static_assert(TX == 32, "one warp per row of element columns");
    static_assert(kRing == 4, "the ring phase is dispatched at compile time");
    using P = typename PairT<T>::t;
    using N4 = typename Node4<T>::t;
    using SM = OpSmem<T, TX, TY, kRing>;
    constexpr int NT = TX * TY;
    constexpr int PN = SM::PN;
    constexpr int SR = (PN + NT - 1) / NT;
    constexpr bool NEED_B = MODE == OP_RESID || MODE == OP_SMOOTH || MODE == OP_BMINUS;
    constexpr bool NEED_D = MODE == OP_SMOOTH || MODE == OP_RESID;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SM& sm = *reinterpret_cast<SM*>(smem_raw);

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + TX * ty;
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
    // in-plane offsets are 32-bit (the launch checks 3 (nx + 1)(ny + 1) < 2^31); plane
    // bases are 64-bit and formed once per layer
    const unsigned own_n = owner ? (unsigned)ni + (unsigned)nxn * (unsigned)nj : 0u;   // owned node in its plane
    const unsigned own3 = 3u * own_n;
    const unsigned ecol = col_in ? (unsigned)ie + (unsigned)a.nx * (unsigned)je : 0u;   // element column in its layer
    const bool dz = NEED_D && a.dinv != nullptr && (MODE != OP_RESID || a.z != nullptr);
    // tiles whose footprint holds no fixed node skip every mask operation
    const bool hm = a.tmask == nullptr || a.tmask[bx + ((a.nx + 1 + TX - 2) / (TX - 1)) * by] != 0;

    // per-thread staging pointers (advanced by whole planes)
    unsigned st_node[SR];   // staged node in its plane
    bool st_ok[SR];
#pragma unroll
    for (int r = 0; r < SR; ++r) {
        const int sidx = tid + r * NT;
        const int px = sidx % (TX + 1), py = sidx / (TX + 1);
        const int gi = X0 - 1 + px, gj = Y0 - 1 + py;
        st_ok[r] = sidx < PN && gi >= 0 && gi < nxn && gj >= 0 && gj < nyn;
        st_node[r] = st_ok[r] ? (unsigned)gi + (unsigned)nxn * (unsigned)gj : 0u;
    }

    // all asynchronous copies that plane p (and element layer p-1) needs, into ring slot SP
    auto issue = [&](int p, auto SPc) {
        constexpr int SP = decltype(SPc)::value;
        const bool pin = p >= 0 && p <= a.nz;
        const long long pn = pin ? (long long)p * nplane : 0;
        const T* xp = a.x + 3 * pn;
#pragma unroll
        for (int r = 0; r < SR; ++r) {
            const int sidx = tid + r * NT;
            if (sidx < PN) {
                const bool v = st_ok[r] && pin;
                const T* src = xp + 3u * st_node[r];
                T* dst = reinterpret_cast<T*>(&sm.plane[SP][sidx]);
                cp_async_t<T>(dst + 0, src + 0, v);
                cp_async_t<T>(dst + 1, src + 1, v);
                cp_async_t<T>(dst + 2, src + 2, v);
                if (hm)
                    cp_async_4(&sm.mword[SP][sidx],
                               reinterpret_cast<const uint32_t*>(a.mask) + ((st_node[r] + pn) >> 2), v);
            }
        }
        const int L = p - 1;
        const bool ev = col_in && L >= 0 && L < a.nz;
        cp_async_t<T>(&sm.ebuf[SP][ty][tx], a.E + (ev ? (long long)L * eplane : 0) + ecol, ev);
        if (NEED_B || dz) {
            const bool ov = owner && p >= kb && p < ke;
            if (NEED_B)
#pragma unroll
                for (int c = 0; c < 3; ++c) cp_async_t<T>(&sm.eb[SP][ty][tx][c], a.b + 3 * pn + own3 + c, ov);
            if (dz)
#pragma unroll
                for (int c = 0; c < 3; ++c) cp_async_t<T>(&sm.ed[SP][ty][tx][c], a.dinv + 3 * pn + own3 + c, ov);
        }
        cp_commit();
    };
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
                    T* dst = reinterpret_cast<T*>(&sm.plane[SP][sidx]);
                    if (m & 1) dst[0] = T(0);
                    if (m & 2) dst[1] = T(0);
                    if (m & 4) dst[2] = T(0);
                }
            }
        }
    };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using I3 = std::integral_constant<int, 3>;
    // ring slot of plane p is p & 3 (p >= -1, so use (p + 4) & 3)
    auto issue_p = [&](int p) {
        switch ((p + 4) & 3) {
            case 0: issue(p, I0{}); break;
            case 1: issue(p, I1{}); break;
            case 2: issue(p, I2{}); break;
            default: issue(p, I3{}); break;
        }
    };
    auto patch_p = [&](int p) {
        switch ((p + 4) & 3) {
            case 0: patch(p, I0{}); break;
            case 1: patch(p, I1{}); break;
            case 2: patch(p, I2{}); break;
            default: patch(p, I3{}); break;
        }
    };

    T acc0 = T(0), acc1 = T(0), acc3 = T(0), accmax = T(0);

#pragma unroll
    for (int q = 0; q <= kDepth; ++q) issue_p(kb - 1 + q);
    cp_wait<kDepth - 1>();
    patch_p(kb - 1);
    patch_p(kb);
    __syncthreads();
    Face<T> Fb, Gc;
    {
        const N4* bp = sm.plane[(kb - 1 + 4) & 3];
        face_forward4<T>(bp[ty * (TX + 1) + tx], bp[ty * (TX + 1) + tx + 1], bp[(ty + 1) * (TX + 1) + tx],
                         bp[(ty + 1) * (TX + 1) + tx + 1], Fb);
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        Gc.p[f] = P{T(0), T(0)};
        Gc.z[f] = T(0);
    }

    // one element layer with compile-time ring slots: top plane k+1 in slot ST, bottom plane k in SB
    auto layer = [&](int k, auto STc) {
        constexpr int ST = decltype(STc)::value;
        constexpr int SB = (ST + 3) & 3;
        constexpr int SI = (ST + 2) & 3;   // plane k+3 is issued into the slot of plane k-1
        constexpr int SN = (ST + 1) & 3;   // plane k+2, patched at the end of this layer
        issue(k + 1 + kDepth, std::integral_constant<int, SI>{});

        const N4* tp = sm.plane[ST];
        Face<T> Ft;
        face_forward4<T>(tp[ty * (TX + 1) + tx], tp[ty * (TX + 1) + tx + 1], tp[(ty + 1) * (TX + 1) + tx],
                         tp[(ty + 1) * (TX + 1) + tx + 1], Ft);
        Face<T> S;
        const bool elem_in = col_in && k >= 0 && k < a.nz;
        if (elem_in) {
            const T Ee = sm.ebuf[ST][ty][tx];
            T uh[24];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const P sum = padd(Ft.p[f], Fb.p[f]), dif = psub(Ft.p[f], Fb.p[f]);
                uh[3 * f + 0] = sum.x;
                uh[3 * f + 1] = sum.y;
                uh[3 * f + 2] = Ft.z[f] + Fb.z[f];
                uh[12 + 3 * f + 0] = dif.x;
                uh[12 + 3 * f + 1] = dif.y;
                uh[12 + 3 * f + 2] = Ft.z[f] - Fb.z[f];
            }
            T v[24];
            haar_apply(kh.v, uh, v);
            if (MODE == OP_RESID) {
                if (a.gt && owner && k + 1 >= kb && k + 1 < ke) {
                    T en = T(0);
#pragma unroll
                    for (int i = 3; i < 24; ++i) en = fma(uh[i], v[i], en);
                    const long long e = (long long)k * eplane + ecol;
                    a.gt[e] = -a.Ed[e] * en;
                }
            }
            const P E2{Ee, Ee};
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const P vs{v[3 * f], v[3 * f + 1]}, vd{v[12 + 3 * f], v[12 + 3 * f + 1]};
                S.p[f] = pfma(E2, psub(vs, vd), Gc.p[f]);
                Gc.p[f] = pmul(E2, padd(vs, vd));
                const T zs = v[3 * f + 2], zd = v[12 + 3 * f + 2];
                S.z[f] = fma(Ee, zs - zd, Gc.z[f]);
                Gc.z[f] = Ee * (zs + zd);
            }
        } else {
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                S.p[f] = Gc.p[f];
                S.z[f] = Gc.z[f];
                Gc.p[f] = P{T(0), T(0)};
                Gc.z[f] = T(0);
            }
        }
        Fb = Ft;

        const bool out_plane = k >= kb;
        P Xp, Yp;
        T Xz, Yz;
        {
            const P sx0 = psub(S.p[0], S.p[2]), sx1 = padd(S.p[0], S.p[2]);
            const P dx0 = psub(S.p[1], S.p[3]), dx1 = padd(S.p[1], S.p[3]);
            const P c00 = psub(sx0, dx0), c10 = padd(sx0, dx0), c01 = psub(sx1, dx1), c11 = padd(sx1, dx1);
            const T zsx0 = S.z[0] - S.z[2], zsx1 = S.z[0] + S.z[2], zdx0 = S.z[1] - S.z[3], zdx1 = S.z[1] + S.z[3];
            const T z00 = zsx0 - zdx0, z10 = zsx0 + zdx0, z01 = zsx1 - zdx1, z11 = zsx1 + zdx1;
            P n01, n00;
            n01.x = __shfl_down_sync(0xffffffffu, c01.x, 1);
            n01.y = __shfl_down_sync(0xffffffffu, c01.y, 1);
            n00.x = __shfl_down_sync(0xffffffffu, c00.x, 1);
            n00.y = __shfl_down_sync(0xffffffffu, c00.y, 1);
            const T m01 = __shfl_down_sync(0xffffffffu, z01, 1);
            const T m00 = __shfl_down_sync(0xffffffffu, z00, 1);
            Xp = padd(c11, n01);
            Xz = z11 + m01;
            Yp = padd(c10, n00);
            Yz = z10 + m00;
        }
        if (out_plane) sm.ybuf[ty][tx] = N4{Yp.x, Yp.y, Yz, T(0)};
        __syncthreads();   // (A)
        if (out_plane && owner) {
            const N4 yb = sm.ybuf[ty + 1][tx];
            const T Kx3[3] = {Xp.x + yb.x, Xp.y + yb.y, Xz + yb.z};
            const long long pofs = 3 * (long long)k * nplane;
            const int oidx = (ty + 1) * (TX + 1) + tx + 1;
            const N4 xs = sm.plane[SB][oidx];
            const T xv3[3] = {xs.x, xs.y, xs.z};
            uint32_t mk = 0;
            if (hm) mk = (sm.mword[SB][oidx] >> (8 * ((own_n + (unsigned)((long long)k * nplane)) & 3u))) & 0xffu;
            T* yo = a.y + pofs + own3;
            const T* xo = a.x + pofs + own3;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                T Kx = Kx3[c], xv = xv3[c];
                if ((mk >> c) & 1) {               // K^ is the identity on fixed DOFs
                    xv = xo[c];
                    Kx = xv;
                }
                if (MODE == OP_APPLY) {
                    yo[c] = Kx;
                } else if (MODE == OP_Q) {
                    yo[c] = Kx;
                    acc0 = fma(xv, Kx, acc0);
                } else if (MODE == OP_BMINUS) {
                    yo[c] = sm.eb[SB][ty][tx][c] - Kx;
                } else if (MODE == OP_SMOOTH) {
                    const T bv = sm.eb[SB][ty][tx][c];
                    const T yv = xv + a.omega * (bv - Kx) * sm.ed[SB][ty][tx][c];
                    yo[c] = yv;
                    acc0 = fma(bv, yv, acc0);
                } else if (MODE == OP_RESID) {
                    const T bv = sm.eb[SB][ty][tx][c];
                    const T rv2 = bv - Kx;
                    yo[c] = rv2;
                    if (a.z) {
                        const T zv = rv2 * sm.ed[SB][ty][tx][c];
                        a.z[pofs + own3 + c] = zv;
                        acc0 = fma(rv2, zv, acc0);
                    }
                    acc1 = fma(rv2, rv2, acc1);
                    accmax = tmax(accmax, tabs(rv2));
                    acc3 = fma(bv, xv, acc3);
                }
            }
        }
        cp_wait<kDepth - 1>();     // plane k+2 (and its layer, operands) landed
        patch(k + 2, std::integral_constant<int, SN>{});
        __syncthreads();   // (B)
    };

    // four layers per trip with every ring slot a compile-time constant (the carried
    // faces change registers without copies); the layers before the first slot-0 top
    // plane and the last ones dispatch on the slot one at a time
    for (int k = kb - 1; k < ke;) {
        if (((k + 1 + 4) & 3) == 0 && k + 4 <= ke) {
            layer(k, I0{});
            layer(k + 1, I1{});
            layer(k + 2, I2{});
            layer(k + 3, I3{});
            k += 4;
            continue;
        }
        switch ((k + 1 + 4) & 3) {
            case 0: layer(k, I0{}); break;
            case 1: layer(k, I1{}); break;
            case 2: layer(k, I2{}); break;
            default: layer(k, I3{}); break;
        }
        ++k;
    }
    cp_wait<0>();
    double* sh_red = sm.red;

    if (MODE == OP_SMOOTH && a.first_step == 2) {
        // last fine-level sweep of a V-cycle: r^T z with r the cycle's right-hand side
        T v[1] = {acc0};
        const int kind[1] = {0};
        double tot[1];
        block_reduce<T, 1>(v, kind, reinterpret_cast<T*>(sh_red));
        if (finish_reduction<T, 1>(v, kind, a.red, a.counter, tot, sh_red, bid, nblocks) && tid == 0) {
            a.sc->rz = tot[0];
            if (!isfinite(tot[0])) set_err(&a.sc->err, TO_ERR_NONFINITE);
        }
    }
    if (MODE == OP_Q) {
        T v[1] = {acc0};
        const int kind[1] = {0};
        double tot[1];
        block_reduce<T, 1>(v, kind, reinterpret_cast<T*>(sh_red));
        if (finish_reduction<T, 1>(v, kind, a.red, a.counter, tot, sh_red, bid, nblocks) && tid == 0) {
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
        T v[4] = {acc0, acc1, accmax, acc3};
        const int kind[4] = {0, 0, 1, 0};
        double tot[4];
        block_reduce<T, 4>(v, kind, reinterpret_cast<T*>(sh_red));
        if (finish_reduction<T, 4>(v, kind, a.red, a.counter, tot, sh_red, bid, nblocks) && tid == 0) {
            DevScalars* sc = a.sc;
            sc->rz = tot[0];
            if (a.first_step) {   // the residual at u_k: tracking error and compliance estimate
                sc->res2 = sqrt(tot[1]);
                sc->res_inf = tot[2];
                sc->J = tot[3];
            }
            if (!isfinite(tot[1]) || !isfinite(tot[0])) set_err(&sc->err, TO_ERR_NONFINITE);
        }
    }
}

template <typename T, int TX, int TY, int MODE>
__global__ void __launch_bounds__(TX * TY, (sizeof(T) == 4 ? (MODE == OP_RESID ? 2 : 3) : 1)) k_operator(const OpArgs<T> a) {
    op_body<T, TX, TY, MODE>(a, a.kh, blockIdx.x, blockIdx.y, blockIdx.z, linear_block(), grid_blocks());
}

// Many problems in one launch: each CTA takes one (problem, tile) pair of a compact
// map built on the host (no CTA of a small problem idles in a grid sized for the
// largest one); the problem's arguments come from a device table, and the element
// matrix constants are common to the batch.
template <typename T, int TX, int TY, int MODE>
__global__ void __launch_bounds__(TX * TY, (sizeof(T) == 4 ? (MODE == OP_RESID ? 2 : 3) : 1))
    k_operator_batch(const OpArgs<T>* __restrict__ tab, const int2* __restrict__ map, const HaarK<T> kh) {
    const int2 m = map[blockIdx.x];
    const OpArgs<T> a = tab[m.x];
    const int gx = (a.nx + 1 + TX - 2) / (TX - 1), gy = (a.ny + 1 + TY - 2) / (TY - 1);
    const int gz = (a.nz + 1 + a.kchunk - 1) / a.kchunk;
    const int t = m.y;
    op_body<T, TX, TY, MODE>(a, kh, t % gx, (t / gx) % gy, t / (gx * gy), (unsigned)t, (unsigned)(gx * gy * gz));
}

// the kernel's in-plane offsets are 32-bit
static bool plane_fits(int nx, int ny) { return 3LL * (nx + 1) * (ny + 1) < (1LL << 31); }

// the table of a batched launch: the problems' arguments, then the (problem, tile) map,
// round-robin over the problems tile by tile; *total = the map's length (the grid)
template <typename T>
static int upload_op_table(const std::vector<OpArgs<T>>& h, void** dev, int* total) {
    const int n = (int)h.size();
    std::vector<int> tiles(n);
    int mt = 0;
    for (int p = 0; p < n; ++p) {
        const OpArgs<T>& a = h[p];
        if (!plane_fits(a.nx, a.ny)) return fail(TO_ERR_ARG, "grid plane too large for the operator kernel");
        const int gx = (a.nx + 1 + 30) / 31, gy = (a.ny + 1 + 6) / 7, gz = (a.nz + 1 + a.kchunk - 1) / a.kchunk;
        if ((long long)gx * gy * gz > kMaxRedBlocks) return fail(TO_ERR_ARG, "batched problem too large for the reduction slots");
        tiles[p] = gx * gy * gz;
        mt = mt > tiles[p] ? mt : tiles[p];
    }
    std::vector<int2> map;
    for (int t = 0; t < mt; ++t)
        for (int p = 0; p < n; ++p)
            if (t < tiles[p]) map.push_back(make_int2(p, t));
    static_assert(sizeof(OpArgs<T>) % alignof(int2) == 0, "map alignment");
    const size_t ab = sizeof(OpArgs<T>) * (size_t)n, mb = sizeof(int2) * map.size();
    if (*dev) cudaFree(*dev);
    *dev = nullptr;
    if (cudaMalloc(dev, ab + mb) != cudaSuccess) return fail(TO_ERR_CUDA, "table allocation");
    if (cudaMemcpy(*dev, h.data(), ab, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(static_cast<char*>(*dev) + ab, map.data(), mb, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(TO_ERR_CUDA, "table upload");
    *total = (int)map.size();
    return TO_OK;
}

int choose_kchunk(long long columns, int planes, long long slots);

template <typename T>
static void fill_haar(const to_problem* P, double scale_h, HaarK<T>& kh) {
    for (int n = 0; n < kHaarNnz; ++n) kh.v[n] = (T)(P->haar[n] * scale_h);
}

template <typename T, int TX, int TY>
static int launch_t(to_problem* P, int level, int mode, const void* x, void* y, const void* b,
                    cudaStream_t s, double omega, int first, const OpOut* out) {
    const Level& L = P->lv[level];
    if (!plane_fits(L.nx, L.ny)) return fail(TO_ERR_ARG, "grid plane too large for the operator kernel");
    OpArgs<T> a{};
    a.nx = L.nx;
    a.ny = L.ny;
    a.nz = L.nz;
    a.x = (const T*)x;
    a.y = (T*)y;
    a.b = (const T*)b;
    a.dinv = (const T*)L.dinv;
    a.E = (const T*)L.E;
    a.mask = L.mask;
    a.tmask = L.tmask;
    fill_haar<T>(P, L.h / P->g.h, a.kh);
    a.omega = (T)omega;
    a.red = P->red;
    a.sc = P->sc;
    a.first_step = first;
    if (mode == OP_RESID) {
        a.counter = P->counters + 0;
        a.z = (P->prm.precond == TO_PRECOND_JACOBI && level == 0) ? (T*)P->z : nullptr;
        a.Ed = (const T*)P->Ed;
        a.gt = (T*)P->gt;
        if (out) {   // caller-supplied outputs (to_residual): z = r / d and g~ / Hs, either optional
            a.z = (T*)out->z;
            a.gt = (T*)out->gt;
        }
    } else if (mode == OP_Q) {
        a.counter = P->counters + 1;
    } else if (mode == OP_SMOOTH) {
        a.counter = P->counters + 6;
    }
    const int gx = (L.nx + 1 + TX - 2) / (TX - 1);
    const int gy = (L.ny + 1 + TY - 2) / (TY - 1);
    int kchunk = P->tile_z > 0 ? P->tile_z : L.kchunk;
    if (kchunk <= 0) kchunk = choose_kchunk((long long)gx * gy, L.nz + 1, (long long)P->op_occ[mode] * P->num_sms);
    if (kchunk > L.nz + 1) kchunk = L.nz + 1;
    a.kchunk = kchunk;
    const int gz = (L.nz + 1 + kchunk - 1) / kchunk;
    if ((long long)gx * gy * gz > kMaxRedBlocks && (mode == OP_RESID || mode == OP_Q || mode == OP_SMOOTH))
        return fail(TO_ERR_ARG, "operator grid exceeds the reduction scratch; raise tile_z");
    dim3 grid(gx, gy, gz), block(TX, TY);
    const size_t smem = sizeof(OpSmem<T, TX, TY, kRing>);
    switch (mode) {
        case OP_APPLY: k_operator<T, TX, TY, OP_APPLY><<<grid, block, smem, s>>>(a); break;
        case OP_RESID: k_operator<T, TX, TY, OP_RESID><<<grid, block, smem, s>>>(a); break;
        case OP_Q: k_operator<T, TX, TY, OP_Q><<<grid, block, smem, s>>>(a); break;
        case OP_SMOOTH: k_operator<T, TX, TY, OP_SMOOTH><<<grid, block, smem, s>>>(a); break;
        case OP_BMINUS: k_operator<T, TX, TY, OP_BMINUS><<<grid, block, smem, s>>>(a); break;
        default: return fail(TO_ERR_ARG, "bad operator mode");
    }
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

// ----------------------------------------------------------------------------- persistent multigrid legs
// The multigrid levels between the fine grid and the one-CTA coarse tail, run as one
// cooperative launch per leg of the V-cycle instead of one launch per step: the down
// leg (the restriction from the fine level, then on every level its pre-smoothing
// sweeps, b - K x and the restriction to the next level) and the up leg (on every level
// the prolongation from the level below and the post-smoothing sweeps, then the
// prolongation to the fine level).  Steps are the same bodies, buffers and order as the
// launch-per-step V-cycle (so the results are bitwise the same); a bounded grid barrier
// separates them.  The fine level's residual (down) and correction target (up) are the
// only pointers that vary between calls: they are kernel arguments.
enum LegKind { LEG_OPER = 0, LEG_RESTRICT = 1, LEG_PROLONG = 2 };

template <typename T>
struct LegStep {
    int kind, mode;                 // LEG_*; OP_SMOOTH / OP_BMINUS for LEG_OPER
    int gx, gy, gz;                 // operator tiles
    OpArgs<T> op;
    int cx, cy, cz;                 // transfers: the coarse grid
    const T* src;                   // restriction: fine residual (nullptr: the launch's fine pointer);
                                    // prolongation: coarse correction
    const uint8_t* mf;
    const uint8_t* mc;
    T* dst;                         // restriction: coarse right-hand side; prolongation: fine target
                                    // (nullptr: the launch's fine pointer)
    const T* dc;                    // restriction: coarse 1 / d
    T* xc;                          // restriction: the coarse first sweep (nullptr: none)
    T omega;
};

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) k_mg_legs(const LegStep<T>* __restrict__ steps, int nsteps, const T* fine_src,
                                                 T* fine_dst, unsigned* bar, int* err) {
    const int tid = threadIdx.x + 32 * threadIdx.y;
    __shared__ OpArgs<T> s_op;   // the current operator step's arguments, read by every thread
    for (int q = 0; q < nsteps; ++q) {
        const LegStep<T>& st = steps[q];
        if (st.kind == LEG_OPER) {
            {   // word by word: no local copy of the step
                const unsigned* src = reinterpret_cast<const unsigned*>(&st.op);
                unsigned* dst = reinterpret_cast<unsigned*>(&s_op);
                for (int w = tid; w < (int)(sizeof(OpArgs<T>) / 4); w += 256) dst[w] = src[w];
            }
            __syncthreads();
            const int nt = st.gx * st.gy * st.gz;
            for (int t = blockIdx.x; t < nt; t += gridDim.x) {
                const int bx = t % st.gx, by = (t / st.gx) % st.gy, bz = t / (st.gx * st.gy);
                if (st.mode == OP_SMOOTH) op_body<T, 32, 8, OP_SMOOTH>(s_op, s_op.kh, bx, by, bz, (unsigned)t, (unsigned)nt);
                else op_body<T, 32, 8, OP_BMINUS>(s_op, s_op.kh, bx, by, bz, (unsigned)t, (unsigned)nt);
                __syncthreads();   // the next tile reuses the shared-memory ring
            }
        } else if (st.kind == LEG_RESTRICT) {
            // node indices in 32 bits (the legs are built only while the fine level has fewer
            // than 2^31 nodes): unsigned divisions instead of 64-bit ones
            const T* tf = st.src ? st.src : fine_src;
            const unsigned nxc = st.cx + 1, nxyc = nxc * (unsigned)(st.cy + 1);
            const unsigned n = nxyc * (unsigned)(st.cz + 1);
            for (unsigned i = blockIdx.x * 256u + tid; i < n; i += gridDim.x * 256u) {
                const unsigned K = i / nxyc, r = i - K * nxyc, J = r / nxc, I = r - J * nxc;
                restrict_node<T, int, true>(st.cx, st.cy, st.cz, (int)I, (int)J, (int)K, tf, st.mf, st.mc, st.dst, st.dc,
                                            st.xc, st.omega);
            }
        } else {
            T* xf = st.dst ? st.dst : fine_dst;
            const unsigned nxf = 2 * st.cx + 1, nxyf = nxf * (unsigned)(2 * st.cy + 1);
            const unsigned n = nxyf * (unsigned)(2 * st.cz + 1);
            for (unsigned i = blockIdx.x * 256u + tid; i < n; i += gridDim.x * 256u) {
                const unsigned z = i / nxyf, r = i - z * nxyf, y = r / nxf, x = r - y * nxf;
                prolong_node<T, int>(st.cx, st.cy, st.cz, (int)x, (int)y, (int)z, st.src, st.mc, st.mf, xf);
            }
        }
        if (q + 1 < nsteps && !grid_barrier(bar, err)) return;
    }
}

// the operator arguments and tile grid of one launch on level `level` (as launch_t)
template <typename T>
static int level_op_args(to_problem* P, int level, int mode, const void* x, void* y, const void* b, double omega,
                         OpArgs<T>& a, int& gx, int& gy, int& gz) {
    constexpr int TX = 32, TY = 8;
    const Level& L = P->lv[level];
    if (!plane_fits(L.nx, L.ny)) return fail(TO_ERR_ARG, "grid plane too large for the operator kernel");
    a = OpArgs<T>{};
    a.nx = L.nx;
    a.ny = L.ny;
    a.nz = L.nz;
    a.x = (const T*)x;
    a.y = (T*)y;
    a.b = (const T*)b;
    a.dinv = (const T*)L.dinv;
    a.E = (const T*)L.E;
    a.mask = L.mask;
    a.tmask = L.tmask;
    fill_haar<T>(P, L.h / P->g.h, a.kh);
    a.omega = (T)omega;
    a.red = P->red;
    a.sc = P->sc;
    a.first_step = 0;
    a.counter = P->counters + 6;
    gx = (L.nx + 1 + TX - 2) / (TX - 1);
    gy = (L.ny + 1 + TY - 2) / (TY - 1);
    int kchunk = P->tile_z > 0 ? P->tile_z : L.kchunk;
    if (kchunk <= 0) kchunk = choose_kchunk((long long)gx * gy, L.nz + 1, (long long)P->op_occ[mode] * P->num_sms);
    if (kchunk > L.nz + 1) kchunk = L.nz + 1;
    a.kchunk = kchunk;
    gz = (L.nz + 1 + kchunk - 1) / kchunk;
    return TO_OK;
}

// the two leg programs of the V-cycle's levels 1 .. tail - 1, in the order and with the
// buffers of the launch-per-step V-cycle (first sweeps fused into the restrictions)
template <typename T>
static int legs_build_t(to_problem* P) {
    const int L = (int)P->lv.size();
    const int tail = P->mg_tail;
    const int nu1 = P->prm.mg_nu_pre, nu2 = P->prm.mg_nu_post;
    const double om = P->prm.mg_omega;
    const bool odd = (nu1 - 1 + nu2) % 2 != 0;   // the first sweep's target: t if odd, else x
    std::vector<LegStep<T>> down, up;
    std::vector<void*> cur(L, nullptr), oth(L, nullptr);
    auto restrict_step = [&](int l, const void* src) {   // level l -> l + 1
        const Level& F = P->lv[l];
        const Level& C = P->lv[l + 1];
        LegStep<T> st{};
        st.kind = LEG_RESTRICT;
        st.cx = C.nx;
        st.cy = C.ny;
        st.cz = C.nz;
        st.src = (const T*)src;
        st.mf = F.mask;
        st.mc = C.mask;
        st.dst = (T*)C.b;
        st.dc = (const T*)C.dinv;
        st.xc = (l + 1 < L - 1) ? (T*)(odd ? C.t : C.x) : nullptr;
        st.omega = (T)om;
        down.push_back(st);
    };
    auto oper_step = [&](std::vector<LegStep<T>>& prog, int l, int mode, void* x, void* y) {
        LegStep<T> st{};
        st.kind = LEG_OPER;
        st.mode = mode;
        int rc = level_op_args<T>(P, l, mode, x, y, P->lv[l].b, om, st.op, st.gx, st.gy, st.gz);
        prog.push_back(st);
        return rc;
    };
    restrict_step(0, nullptr);
    for (int l = 1; l < tail; ++l) {
        const Level& F = P->lv[l];
        cur[l] = odd ? F.t : F.x;
        oth[l] = cur[l] == F.t ? F.x : F.t;
        for (int it = 1; it < nu1; ++it) {
            if (int rc = oper_step(down, l, OP_SMOOTH, cur[l], oth[l])) return rc;
            std::swap(cur[l], oth[l]);
        }
        if (int rc = oper_step(down, l, OP_BMINUS, cur[l], oth[l])) return rc;
        restrict_step(l, oth[l]);
    }
    for (int l = tail - 1; l >= 1; --l) {
        const Level& F = P->lv[l];
        const Level& C = P->lv[l + 1];
        LegStep<T> pr{};
        pr.kind = LEG_PROLONG;
        pr.cx = C.nx;
        pr.cy = C.ny;
        pr.cz = C.nz;
        pr.src = (const T*)C.x;
        pr.mc = C.mask;
        pr.mf = F.mask;
        pr.dst = (T*)cur[l];
        up.push_back(pr);
        for (int it = 0; it < nu2; ++it) {
            if (int rc = oper_step(up, l, OP_SMOOTH, cur[l], oth[l])) return rc;
            std::swap(cur[l], oth[l]);
        }
        if (cur[l] != F.x) return fail(TO_ERR_STATE, "multigrid legs: buffer parity");
    }
    {
        const Level& C = P->lv[1];
        LegStep<T> pr{};
        pr.kind = LEG_PROLONG;
        pr.cx = C.nx;
        pr.cy = C.ny;
        pr.cz = C.nz;
        pr.src = (const T*)C.x;
        pr.mc = C.mask;
        pr.mf = P->lv[0].mask;
        pr.dst = nullptr;
        up.push_back(pr);
    }
    int maxt = 1;
    for (const auto* prog : {&down, &up})
        for (const LegStep<T>& st : *prog)
            if (st.kind == LEG_OPER) maxt = std::max(maxt, st.gx * st.gy * st.gz);
    const size_t bytes = sizeof(LegStep<T>) * (down.size() + up.size());
    void* d = nullptr;
    TO_CUDA(cudaMalloc(&d, bytes));
    TO_CUDA(cudaMemcpy(d, down.data(), sizeof(LegStep<T>) * down.size(), cudaMemcpyHostToDevice));
    TO_CUDA(cudaMemcpy(static_cast<char*>(d) + sizeof(LegStep<T>) * down.size(), up.data(),
                       sizeof(LegStep<T>) * up.size(), cudaMemcpyHostToDevice));
    P->legs_prog = d;
    P->legs_n[0] = (int)down.size();
    P->legs_n[1] = (int)up.size();
    // co-resident CTAs: the operator's residency (it bounds the shared memory) on every SM
    const size_t smem = sizeof(OpSmem<T, 32, 8, kRing>);
    TO_CUDA(cudaFuncSetAttribute(k_mg_legs<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    TO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mg_legs<T>, 256, smem));
    if (occ < 1) return TO_OK;   // no cooperative residency: the launch-per-step V-cycle stays
    P->legs_grid = std::min(maxt, occ * P->num_sms);
    return TO_OK;
}

int mg_legs_build(to_problem* P) {
    P->legs_grid = 0;
    if (P->prm.precond != TO_PRECOND_MG || P->prm.mg_legs == 0 || P->prm.op_kernel != 0 || P->mg_tail < 2) return TO_OK;
    if (P->lv[0].n_node >= (1LL << 31)) return TO_OK;   // the legs index nodes in 32 bits
    return P->prec == TO_FP64 ? legs_build_t<double>(P) : legs_build_t<float>(P);
}

// one leg: 0 down (fine residual `fine` restricted), 1 up (the correction added into `fine`)
int mg_legs_launch(to_problem* P, int leg, void* fine, cudaStream_t s) {
    const size_t stride = P->prec == TO_FP64 ? sizeof(LegStep<double>) : sizeof(LegStep<float>);
    const void* steps = static_cast<const char*>(P->legs_prog) + (leg ? stride * P->legs_n[0] : 0);
    int n = P->legs_n[leg];
    unsigned* bar = P->counters + 20;
    int* err = &P->sc->err;
    const void* fsrc = leg ? nullptr : fine;
    void* fdst = leg ? fine : nullptr;
    void* args[] = {(void*)&steps, (void*)&n, (void*)&fsrc, (void*)&fdst, (void*)&bar, (void*)&err};
    const dim3 block(32, 8);
    if (P->prec == TO_FP64) {
        TO_CUDA(cudaLaunchCooperativeKernel((const void*)k_mg_legs<double>, dim3(P->legs_grid), block, args,
                                            sizeof(OpSmem<double, 32, 8, kRing>), s));
    } else {
        TO_CUDA(cudaLaunchCooperativeKernel((const void*)k_mg_legs<float>, dim3(P->legs_grid), block, args,
                                            sizeof(OpSmem<float, 32, 8, kRing>), s));
    }
    return TO_OK;
}

template <typename T, int TX, int TY>
static int init_t(to_problem* P) {
    const size_t smem = sizeof(OpSmem<T, TX, TY, kRing>);
    const void* fns[5] = {(const void*)k_operator<T, TX, TY, OP_APPLY>, (const void*)k_operator<T, TX, TY, OP_RESID>,
                          (const void*)k_operator<T, TX, TY, OP_Q>, (const void*)k_operator<T, TX, TY, OP_SMOOTH>,
                          (const void*)k_operator<T, TX, TY, OP_BMINUS>};
    for (int m = 0; m < 5; ++m) {
        TO_CUDA(cudaFuncSetAttribute(fns[m], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int occ = 0;
        TO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fns[m], TX * TY, smem));
        P->op_occ[m] = occ > 0 ? occ : 1;
    }
    return TO_OK;
}

// shared-memory opt-in and residency of the operator kernels (on the problem's device, before any capture)
int operator_init(to_problem* P) {
    if (P->prec == TO_FP64) return init_t<double, 32, 8>(P);
    int rc = init_t<float, 32, 8>(P);
    if (!rc) rc = operator_tma_init(P);
    return rc ? rc : operator_tc_init(P);
}

// Tile autotuner of a problem's operator: for every multigrid level (or the fine grid
// alone), time the damped-Jacobi sweep (the most frequent operator launch) for every
// distinct split of the level's node planes into chunks (the cost model's choice
// first), twice, and keep the fastest for all of that level's operator launches.
// Inputs and outputs are the level's scratch vectors: timing only, no state the
// method reads is changed.
int operator_autotune(to_problem* P, cudaStream_t s) {
    cudaEvent_t e0, e1;
    TO_CUDA(cudaEventCreate(&e0));
    TO_CUDA(cudaEventCreate(&e1));
    int rc = TO_OK;
    const int L = (int)P->lv.size();
    for (int l = 0; l < L && !rc; ++l) {
        Level& Lv = P->lv[l];
        if (l > 0 && l == P->mg_tail) break;   // the one-CTA tail takes over from here
        if (l > 0 && l == L - 1) break;        // the dense coarsest solve
        const void* x = l == 0 ? P->u : Lv.x;
        void* y = l == 0 ? P->tmp_v : Lv.t;
        const void* b = l == 0 ? P->r : Lv.b;
        if (!x || !y || !b) continue;
        const int planes = Lv.nz + 1;
        const int gx = (Lv.nx + 1 + 30) / 31, gy = (Lv.ny + 1 + 6) / 7;
        const int model = choose_kchunk((long long)gx * gy, planes, (long long)P->op_occ[OP_SMOOTH] * P->num_sms);
        std::vector<int> cand{model};
        for (int kc = 1; kc <= planes && kc <= 64; ++kc) {
            const int gz = (planes + kc - 1) / kc;
            if (kc > 1 && (planes + kc - 2) / (kc - 1) == gz) continue;   // same split as a shorter chunk
            if (kc != model && (long long)gx * gy * gz <= kMaxRedBlocks) cand.push_back(kc);
        }
        int best = model;
        float best_t = -1.f;
        for (int round = 0; round < 2 && !rc; ++round)
            for (size_t c = 0; c < cand.size() && !rc; ++c) {
                Lv.kchunk = cand[c];
                for (int r = 0; r < 2 && !rc; ++r) rc = launch_operator(P, l, OP_SMOOTH, x, y, b, s, 0.5, 0);
                cudaEventRecord(e0, s);
                for (int r = 0; r < 5 && !rc; ++r) rc = launch_operator(P, l, OP_SMOOTH, x, y, b, s, 0.5, 0);
                cudaEventRecord(e1, s);
                if (rc) break;
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = fail(TO_ERR_CUDA, "autotune timing");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (best_t < 0.f || ms < best_t) {
                    best_t = ms;
                    best = cand[c];
                }
            }
        Lv.kchunk = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

// Node planes per CTA tile for one launch: the CTA count is gx * gy * ceil(planes / kchunk)
// and a CTA walks kchunk + 1 planes (one recomputed halo layer).  With `slots` CTAs
// resident at once the launch takes about ceil(CTAs / slots) rounds of the longest
// walk; pick the chunk that minimises rounds x walk (the fewest CTAs on ties).
int choose_kchunk(long long columns, int planes, long long slots) {
    long long best_cost = -1, best_ctas = 0;
    int best = planes;
    for (int kc = 1; kc <= planes; ++kc) {
        const long long gz = (planes + kc - 1) / kc;
        if (kc > 1 && (planes + kc - 2) / (kc - 1) == gz) continue;   // same split as a shorter chunk
        const long long ctas = columns * gz;
        const long long cost = ((ctas + slots - 1) / slots) * (kc + 1);
        if (best_cost < 0 || cost < best_cost || (cost == best_cost && ctas < best_ctas)) {
            best_cost = cost;
            best_ctas = ctas;
            best = kc;
        }
    }
    return best;
}

// Per CTA tile column of the operator's 32 x 8 tiling: does its node footprint
// (x from 31 bx - 1 to 31 bx + 31, y from 7 by - 1 to 7 by + 7, every z) hold a
// fixed DOF?  Tiles without one skip all mask handling.
int build_tile_mask(Level& L, const uint8_t* mask_host) {
    const int nxn = L.nx + 1, nyn = L.ny + 1, nzn = L.nz + 1;
    std::vector<uint8_t> col((size_t)nxn * nyn, 0);
    for (int k = 0; k < nzn; ++k)
        for (int j = 0; j < nyn; ++j)
            for (int i = 0; i < nxn; ++i)
                if (mask_host[(size_t)i + (size_t)nxn * ((size_t)j + (size_t)nyn * k)]) col[(size_t)i + (size_t)nxn * j] = 1;
    const int gx = (nxn + 29) / 31 + 1, gy = (nyn + 5) / 7 + 1;   // generous: covers (n + 1 + 30) / 31 tiles
    std::vector<uint8_t> t((size_t)gx * gy, 0);
    const int gxk = (L.nx + 1 + 32 - 2) / 31;
    for (int by = 0; by < gy; ++by)
        for (int bx = 0; bx < gxk; ++bx) {
            uint8_t f = 0;
            for (int j = std::max(7 * by - 1, 0); j <= std::min(7 * by + 7, nyn - 1) && !f; ++j)
                for (int i = std::max(31 * bx - 1, 0); i <= std::min(31 * bx + 31, nxn - 1); ++i)
                    if (col[(size_t)i + (size_t)nxn * j]) {
                        f = 1;
                        break;
                    }
            t[(size_t)bx + (size_t)gxk * by] = f;
        }
    void* d = nullptr;
    TO_CUDA(cudaMalloc(&d, t.size()));
    TO_CUDA(cudaMemcpy(d, t.data(), t.size(), cudaMemcpyHostToDevice));
    L.tmask = (uint8_t*)d;
    return build_tile_mask64(L, mask_host);
}

int launch_operator(to_problem* P, int level, int mode, const void* x, void* y, const void* b,
                    cudaStream_t s, double omega, int first, const OpOut* out) {
    if (operator_tma_applicable(P, level, x, y, b)) return launch_operator_tma(P, level, mode, x, y, b, s, omega, first, out);
    if (operator_tc_applicable(P, level)) return launch_operator_tc(P, level, mode, x, y, b, s, omega, first, out);
    if (P->prec == TO_FP64) return launch_t<double, 32, 8>(P, level, mode, x, y, b, s, omega, first, out);
    return launch_t<float, 32, 8>(P, level, mode, x, y, b, s, omega, first, out);
}

}  // namespace to

// ----------------------------------------------------------------------------- batched launches
namespace to {

template <typename T>
static OpArgs<T> batch_args(to_problem* P, int mode, int first, int kchunk) {
    const Level& L = P->lv[0];
    OpArgs<T> a{};
    a.nx = L.nx;
    a.ny = L.ny;
    a.nz = L.nz;
    a.kchunk = L.nz + 1 < kchunk ? L.nz + 1 : kchunk;
    a.E = (const T*)L.E;
    a.mask = L.mask;
    a.tmask = L.tmask;
    a.dinv = (const T*)L.dinv;
    a.red = P->red;
    a.sc = P->sc;
    a.first_step = first;
    fill_haar<T>(P, 1.0, a.kh);
    if (mode == OP_RESID) {
        a.x = (const T*)P->u;
        a.y = (T*)P->r;
        a.b = (const T*)P->f;
        a.z = P->prm.precond == TO_PRECOND_JACOBI ? (T*)P->z : nullptr;   // multigrid: z comes from the V-cycle
        a.Ed = (const T*)P->Ed;
        a.gt = (T*)P->gt;
        a.counter = P->counters + 0;
    } else if (mode == OP_Q) {
        a.x = (const T*)P->z;
        a.y = (T*)P->q;
        a.counter = P->counters + 1;
    } else {   // OP_APPLY into scratch: the tile autotuner's timing runs
        a.x = (const T*)P->u;
        a.y = (T*)P->tmp_v;
    }
    return a;
}

template <typename T>
static int op_table_t(to_problem* const* probs, int n, int mode, int first, void** dev, int* max_tiles, int kchunk) {
    std::vector<OpArgs<T>> h(n);
    for (int i = 0; i < n; ++i) h[i] = batch_args<T>(probs[i], mode, first, kchunk);
    return upload_op_table<T>(h, dev, max_tiles);
}

// device tables of operator arguments for a list of problems (node planes per tile:
// kchunk), and the common element constants
int op_tables_build(to_problem* const* probs, int n, void** resid, void** q_first, void** q, void** kh_host,
                    int* max_tiles, int kchunk) {
    const int prec = probs[0]->prec;
    int mt = 0, rc;
    if (prec == TO_FP64) {
        if ((rc = op_table_t<double>(probs, n, OP_RESID, 1, resid, &mt, kchunk)) ||
            (rc = op_table_t<double>(probs, n, OP_Q, 1, q_first, &mt, kchunk)) || (rc = op_table_t<double>(probs, n, OP_Q, 0, q, &mt, kchunk)))
            return rc;
        if (!*kh_host) {
            HaarK<double>* kh = (HaarK<double>*)malloc(sizeof(HaarK<double>));
            fill_haar<double>(probs[0], 1.0, *kh);
            *kh_host = kh;
        }
    } else {
        if ((rc = op_table_t<float>(probs, n, OP_RESID, 1, resid, &mt, kchunk)) ||
            (rc = op_table_t<float>(probs, n, OP_Q, 1, q_first, &mt, kchunk)) || (rc = op_table_t<float>(probs, n, OP_Q, 0, q, &mt, kchunk)))
            return rc;
        if (!*kh_host) {
            HaarK<float>* kh = (HaarK<float>*)malloc(sizeof(HaarK<float>));
            fill_haar<float>(probs[0], 1.0, *kh);
            *kh_host = kh;
        }
    }
    *max_tiles = mt;
    // shared-memory opt-in of the batched kernels
    const size_t smem = prec == TO_FP64 ? sizeof(OpSmem<double, 32, 8, kRing>) : sizeof(OpSmem<float, 32, 8, kRing>);
    const void* fns[5];
    if (prec == TO_FP64) {
        fns[0] = (const void*)k_operator_batch<double, 32, 8, OP_RESID>;
        fns[1] = (const void*)k_operator_batch<double, 32, 8, OP_Q>;
        fns[2] = (const void*)k_operator_batch<double, 32, 8, OP_APPLY>;
        fns[3] = (const void*)k_operator_batch<double, 32, 8, OP_SMOOTH>;
        fns[4] = (const void*)k_operator_batch<double, 32, 8, OP_BMINUS>;
    } else {
        fns[0] = (const void*)k_operator_batch<float, 32, 8, OP_RESID>;
        fns[1] = (const void*)k_operator_batch<float, 32, 8, OP_Q>;
        fns[2] = (const void*)k_operator_batch<float, 32, 8, OP_APPLY>;
        fns[3] = (const void*)k_operator_batch<float, 32, 8, OP_SMOOTH>;
        fns[4] = (const void*)k_operator_batch<float, 32, 8, OP_BMINUS>;
    }
    for (const void* f : fns) TO_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return TO_OK;
}

int batch_operator_launch(int prec, int mode, const void* tab, const void* kh, int max_tiles, int n, cudaStream_t s);

// One batched multigrid sweep's table: problem i applies `mode` (OP_SMOOTH or OP_BMINUS)
// on its level `level` from x[i] into y[i] with right-hand side b[i]; `first` = 2 on the
// fine level's last sweep (it also reduces b^T y, the r^T z of the lower-level step).
template <typename T>
static int op_table_level_t(to_problem* const* probs, int n, int level, int mode, const void* const* x, void* const* y,
                            const void* const* b, double omega, int first, int kchunk, void** dev, int* max_tiles) {
    std::vector<OpArgs<T>> h(n);
    for (int i = 0; i < n; ++i) {
        to_problem* P = probs[i];
        const Level& L = P->lv[level];
        OpArgs<T>& a = h[i];
        a = OpArgs<T>{};
        a.nx = L.nx;
        a.ny = L.ny;
        a.nz = L.nz;
        a.kchunk = L.nz + 1 < kchunk ? L.nz + 1 : kchunk;
        a.x = (const T*)x[i];
        a.y = (T*)y[i];
        a.b = (const T*)b[i];
        a.dinv = (const T*)L.dinv;
        a.E = (const T*)L.E;
        a.mask = L.mask;
        a.tmask = L.tmask;
        a.omega = (T)omega;
        a.red = P->red;
        a.sc = P->sc;
        a.first_step = first;
        a.counter = mode == OP_SMOOTH ? P->counters + 6 : nullptr;
    }
    return upload_op_table<T>(h, dev, max_tiles);
}

int op_table_level(to_problem* const* probs, int n, int level, int mode, const void* const* x, void* const* y,
                   const void* const* b, double omega, int first, int kchunk, void** dev, int* max_tiles) {
    return probs[0]->prec == TO_FP64
               ? op_table_level_t<double>(probs, n, level, mode, x, y, b, omega, first, kchunk, dev, max_tiles)
               : op_table_level_t<float>(probs, n, level, mode, x, y, b, omega, first, kchunk, dev, max_tiles);
}

// host copy of a level's element constants (K_e scales with the element size: h_level / h_0)
void* level_haar(const to_problem* P, int level) {
    if (P->prec == TO_FP64) {
        HaarK<double>* kh = (HaarK<double>*)malloc(sizeof(HaarK<double>));
        if (kh) fill_haar<double>(P, P->lv[level].h / P->g.h, *kh);
        return kh;
    }
    HaarK<float>* kh = (HaarK<float>*)malloc(sizeof(HaarK<float>));
    if (kh) fill_haar<float>(P, P->lv[level].h / P->g.h, *kh);
    return kh;
}

// Tile autotuner of the batched operator: time the batch's K u into scratch (no scalar
// side effects) for each candidate number of node planes per tile and return the fastest.
int batch_autotune_kchunk(to_problem* const* probs, int n, const void* kh, cudaStream_t s, int* best_out, float* us_out) {
    const int prec = probs[0]->prec;
    static const int cand[] = {2, 4, 8, 16, 32};
    void* tab = nullptr;
    cudaEvent_t e0, e1;
    TO_CUDA(cudaEventCreate(&e0));
    TO_CUDA(cudaEventCreate(&e1));
    int best = 8;
    float best_t = -1.f;
    int rc = TO_OK;
    for (int kc : cand) {
        int mt = 0;
        rc = prec == TO_FP64 ? op_table_t<double>(probs, n, OP_APPLY, 0, &tab, &mt, kc)
                             : op_table_t<float>(probs, n, OP_APPLY, 0, &tab, &mt, kc);
        if (rc) break;
        for (int r = 0; r < 2 && !rc; ++r) rc = batch_operator_launch(prec, OP_APPLY, tab, kh, mt, n, s);
        if (rc) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 5 && !rc; ++r) rc = batch_operator_launch(prec, OP_APPLY, tab, kh, mt, n, s);
        cudaEventRecord(e1, s);
        if (rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = fail(TO_ERR_CUDA, "autotune timing");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best_t < 0.f || ms < best_t) {
            best_t = ms;
            best = kc;
        }
    }
    if (tab) cudaFree(tab);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *best_out = best;
    if (us_out) *us_out = best_t * 1000.f / 5.f;
    return TO_OK;
}

template <typename T>
static void batch_launch_t(int mode, const void* tab, int n, const void* kh, dim3 grid, cudaStream_t s) {
    const size_t smem = sizeof(OpSmem<T, 32, 8, kRing>);
    const HaarK<T>& k = *(const HaarK<T>*)kh;
    const OpArgs<T>* t = (const OpArgs<T>*)tab;
    const int2* m = reinterpret_cast<const int2*>(t + n);
    const dim3 block(32, 8);
    switch (mode) {
        case OP_RESID: k_operator_batch<T, 32, 8, OP_RESID><<<grid, block, smem, s>>>(t, m, k); break;
        case OP_Q: k_operator_batch<T, 32, 8, OP_Q><<<grid, block, smem, s>>>(t, m, k); break;
        case OP_SMOOTH: k_operator_batch<T, 32, 8, OP_SMOOTH><<<grid, block, smem, s>>>(t, m, k); break;
        case OP_BMINUS: k_operator_batch<T, 32, 8, OP_BMINUS><<<grid, block, smem, s>>>(t, m, k); break;
        default: k_operator_batch<T, 32, 8, OP_APPLY><<<grid, block, smem, s>>>(t, m, k); break;
    }
}

// `tiles`: the length of the table's (problem, tile) map
int batch_operator_launch(int prec, int mode, const void* tab, const void* kh, int tiles, int n, cudaStream_t s) {
    const dim3 grid(tiles);
    if (prec == TO_FP64) batch_launch_t<double>(mode, tab, n, kh, grid, s);
    else batch_launch_t<float>(mode, tab, n, kh, grid, s);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

}  // namespace to
