// C entry points (include/to.h): argument checks, device memory owned by the
// problem, and stream-ordered calls into the kernels.
#include <cstdint>
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "device.cuh"

namespace to {
int project_coop_blocks(int prec, int num_sms, int* out);
int launch_rowsum(to_problem* P, cudaStream_t s);
int run_inner(to_problem* P, void* u, int nsteps, int primary, cudaStream_t s, int resid_done);
int launch_filter_prescaled_T(to_problem* P, const void* x, void* y, cudaStream_t s);

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <typename T>
__global__ void k_fill(T* p, long long n, T v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

int dalloc(void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) return fail(TO_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return TO_OK;
}

void dfree(void*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

int fill_scalar(to_problem* P, void* p, long long n, double v, cudaStream_t s) {
    const int nb = (int)std::min<long long>((n + 255) / 256, 1024);
    if (P->prec == TO_FP64)
        k_fill<double><<<nb > 0 ? nb : 1, 256, 0, s>>>((double*)p, n, v);
    else
        k_fill<float><<<nb > 0 ? nb : 1, 256, 0, s>>>((float*)p, n, (float)v);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

}  // namespace
}  // namespace to

using namespace to;

extern "C" void to_default_params(to_params* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = TO_FP32_MIXED;
    o->precond = TO_PRECOND_JACOBI;
    o->inner_mode = TO_INNER_SD;
    o->n_inner = 5;
    o->beta = 0.5;
    o->alpha0 = 0.0;
    o->alpha_scale = 0.2;
    o->m = 0.75;
    o->mean_proj = 0;
    o->mg_levels = 0;
    o->mg_nu_pre = 2;
    o->mg_nu_post = 2;
    o->mg_omega = 0.5;
    o->krylov_dim = 20;
    o->mg_legs = 0;
    o->tile_z = -1;   // the cost model: measured per level, the autotuner's isolated timings lost in the graph
}

static int validate(const to_grid* g, const to_material* m, const to_loads* L, const to_bcs* B, const to_params* p) {
    if (!g || !m || !L || !B || !p) return fail(TO_ERR_ARG, "null argument");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return fail(TO_ERR_ARG, "grid dimensions must be >= 1");
    if (!(g->h > 0.0)) return fail(TO_ERR_ARG, "element edge h must be > 0");
    const double nn = (double)(g->nx + 1) * (g->ny + 1) * (g->nz + 1);
    if (nn * 3 > 4.0e9) return fail(TO_ERR_ARG, "grid too large");
    if (!(m->E0 > m->Emin) || !(m->Emin >= 0.0)) return fail(TO_ERR_ARG, "need E0 > Emin >= 0");
    if (!(m->nu >= 0.0 && m->nu < 0.5)) return fail(TO_ERR_ARG, "need 0 <= nu < 0.5");
    if (!(m->p >= 1.0)) return fail(TO_ERR_ARG, "need p >= 1");
    if (!(m->rho_min >= 0.0 && m->rho_max > m->rho_min)) return fail(TO_ERR_ARG, "need 0 <= rho_min < rho_max");
    if (!(m->volfrac > 0.0)) return fail(TO_ERR_ARG, "need volfrac > 0");
    if (m->volfrac < m->rho_min) return fail(TO_ERR_INFEASIBLE, "volume bound below n_elem * rho_min: X is empty");
    if (L->n < 0 || (L->n > 0 && (!L->dof || !L->val))) return fail(TO_ERR_ARG, "bad load list");
    if (B->n < 0 || (B->n > 0 && !B->dof)) return fail(TO_ERR_ARG, "bad fixture list");
    if (p->precision != TO_FP64 && p->precision != TO_FP32_MIXED) return fail(TO_ERR_ARG, "bad precision");
    if (p->precond < 0 || p->precond > 3) return fail(TO_ERR_ARG, "bad preconditioner");
    if (p->precond == TO_PRECOND_KRYLOV && (p->krylov_dim < 0 || p->krylov_dim > 30))
        return fail(TO_ERR_ARG, "krylov_dim must lie in [0, 30]");
    if (p->adj_stride < -1) return fail(TO_ERR_ARG, "adj_stride must be >= -1");
    if (p->op_kernel < 0 || p->op_kernel > 2) return fail(TO_ERR_ARG, "op_kernel must be 0, 1 or 2");
    if (p->inner_mode < TO_INNER_SD || p->inner_mode > TO_INNER_PCG) return fail(TO_ERR_ARG, "bad inner mode");
    if (p->n_inner < 0) return fail(TO_ERR_ARG, "n_inner must be >= 0");
    if (!(p->m >= 0.0)) return fail(TO_ERR_ARG, "alpha exponent m must be >= 0");
    const long long ndof = 3LL * (long long)nn;
    for (int64_t i = 0; i < L->n; ++i)
        if (L->dof[i] < 0 || L->dof[i] >= ndof || !std::isfinite(L->val[i])) return fail(TO_ERR_ARG, "load DOF out of range or value not finite");
    for (int64_t i = 0; i < B->n; ++i)
        if (B->dof[i] < 0 || B->dof[i] >= ndof) return fail(TO_ERR_ARG, "fixed DOF out of range");
    if (B->n == 0) return fail(TO_ERR_SINGULAR, "no fixed DOF: K is singular");
    return TO_OK;
}

extern "C" void to_destroy(to_problem* P) {
    if (!P) return;
    DeviceGuard dg(P->device);
    void** bufs[] = {&P->rho, &P->rhot, &P->Ed, &P->Hs, &P->gt, &P->grad, &P->tmp_e, &P->stencil_w,
                     &P->u, &P->f, &P->r, &P->z, &P->q, &P->tmp_v, &P->coarse_A, &P->coarse_L, &P->iters, &P->gj_work, &P->gj_tab,
                     &P->legs_prog};
    for (void** b : bufs) dfree(*b);
    void* st = P->stencil;
    dfree(st);
    for (auto& L : P->lv) {
        dfree(L.E);
        dfree(L.dinv);
        void* mk = L.mask;
        dfree(mk);
        void* tm = L.tmask;
        dfree(tm);
        void* tm64 = L.tmask64;
        dfree(tm64);
        dfree(L.tcb);
        dfree(L.x);
        dfree(L.b);
        dfree(L.t);
    }
    if (P->gexec) cudaGraphExecDestroy(P->gexec);
    for (int p = 0; p < 2; ++p)
        for (int f = 0; f < 3; ++f)
            if (P->gexec_pipe[p][f]) cudaGraphExecDestroy(P->gexec_pipe[p][f]);
    if (P->gstream) cudaStreamSynchronize(P->gstream);
    if (P->ev_in) cudaEventDestroy(P->ev_in);
    if (P->ev_out) cudaEventDestroy(P->ev_out);
    if (P->side) cudaStreamSynchronize(P->side);
    if (P->ev_fork) cudaEventDestroy(P->ev_fork);
    if (P->ev_join) cudaEventDestroy(P->ev_join);
    if (P->ev_ljoin) cudaEventDestroy(P->ev_ljoin);
    if (P->side) cudaStreamDestroy(P->side);
    if (P->dside) cudaStreamSynchronize(P->dside);
    if (P->ev_dfork) cudaEventDestroy(P->ev_dfork);
    if (P->ev_djoin) cudaEventDestroy(P->ev_djoin);
    if (P->dside) cudaStreamDestroy(P->dside);
    if (P->gstream) cudaStreamDestroy(P->gstream);
    void* p;
    p = P->ke_dev; dfree(p);
    p = P->kry_q; dfree(p);
    p = P->kry_s; dfree(p);
    p = P->kry_part; dfree(p);
    p = P->ps_buf; dfree(p);
    p = P->sc; dfree(p);
    p = P->red; dfree(p);
    p = P->red_d; dfree(p);
    p = P->alt_rhot; dfree(p);
    p = P->alt_Ed; dfree(p);
    for (void* q : P->alt_E) dfree(q);
    for (void* q : P->alt_dinv) dfree(q);
    p = P->alt_coarse_L; dfree(p);
    p = P->alt_gj_tab; dfree(p);
    p = P->counters; dfree(p);
    p = P->dstats; dfree(p);
    p = P->rho_stage; dfree(p);
    if (P->stats_pinned) cudaFreeHost(P->stats_pinned);
    delete P;
}

extern "C" int to_create(const to_grid* g, const to_material* m, const to_loads* L, const to_bcs* B,
                         const to_params* prm, int device, to_problem** out) {
    if (!out) return fail(TO_ERR_ARG, "out is null");
    *out = nullptr;
    int rc = validate(g, m, L, B, prm);
    if (rc) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(TO_ERR_CUDA, "no such CUDA device");
    DeviceGuard dg(device);
    if (!dg.ok) return fail(TO_ERR_CUDA, "cudaSetDevice failed");

    to_problem* P = new (std::nothrow) to_problem();
    if (!P) return fail(TO_ERR_ARG, "out of host memory");
    P->device = device;
    P->prec = prm->precision;
    P->g = *g;
    P->mat = *m;
    P->prm = *prm;
    P->esz = P->prec == TO_FP64 ? 8 : 4;
    P->n_elem = (int64_t)g->nx * g->ny * g->nz;
    P->n_node = (int64_t)(g->nx + 1) * (g->ny + 1) * (g->nz + 1);
    P->n_dof = 3 * P->n_node;
    P->tile_z = prm->tile_z > 0 ? prm->tile_z : 0;
    auto bail = [&](int code) {
        to_destroy(P);
        return code;
    };

    if ((rc = build_element_matrix(m->nu, P->ke))) return bail(rc);
    if ((rc = build_haar(P->ke, g->h, P->haar))) return bail(rc);
    P->kdiag = g->h * P->ke[0];
    for (int i = 1; i < 24; ++i)
        if (std::fabs(P->ke[i * 24 + i] - P->ke[0]) > 1e-14) return bail(fail(TO_ERR_ARG, "unequal element diagonal"));

    int dev_sms = 0;
    if (cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return bail(fail(TO_ERR_CUDA, "device query failed"));
    P->num_sms = dev_sms;
    if ((rc = project_coop_blocks(P->prec, P->num_sms, &P->coop_blocks))) return bail(rc);
    if ((rc = operator_init(P)) || (rc = mg_cluster_init(P))) return bail(rc);
    if (cudaStreamCreateWithFlags(&P->gstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&P->dside, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&P->ev_dfork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&P->ev_djoin, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(TO_ERR_CUDA, "stream / event creation failed"));

    // filter stencil: offsets with w = rmin - |d| > 0 (identity when rmin <= 0)
    std::vector<int4> st;
    std::vector<double> sw;
    const int R = (int)std::ceil(m->rmin) + 1;
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                const double w = m->rmin - std::sqrt((double)(dx * dx + dy * dy + dz * dz));
                if (w > 0.0) {
                    st.push_back(make_int4(dx, dy, dz, dx + g->nx * (dy + g->ny * dz)));
                    sw.push_back(w);
                }
            }
    if (st.empty()) {
        st.push_back(make_int4(0, 0, 0, 0));
        sw.push_back(1.0);
    }
    if (st.size() > 1024) return bail(fail(TO_ERR_ARG, "filter radius too large (more than 1024 stencil points)"));
    P->n_stencil = (int)st.size();
    P->filter_ext = 0;
    for (const int4& o : st) P->filter_ext = std::max(P->filter_ext, std::max(std::abs(o.x), std::max(std::abs(o.y), std::abs(o.z))));

    // level 0 (the fine grid)
    Level L0{};
    L0.nx = g->nx; L0.ny = g->ny; L0.nz = g->nz;
    L0.n_elem = P->n_elem; L0.n_node = P->n_node; L0.n_dof = P->n_dof;
    L0.h = g->h;
    L0.kdiag = P->kdiag;
    P->lv.push_back(L0);
    Level& F = P->lv[0];

    const size_t es = P->esz;
    const size_t ne = (size_t)P->n_elem, nd = (size_t)P->n_dof;
    if ((rc = dalloc(&P->rho, ne * es)) || (rc = dalloc(&P->rhot, ne * es)) || (rc = dalloc(&F.E, ne * es)) ||
        (rc = dalloc(&P->Ed, ne * es)) || (rc = dalloc(&P->Hs, ne * es)) || (rc = dalloc(&P->gt, ne * es)) ||
        (rc = dalloc(&P->grad, ne * es)) || (rc = dalloc(&P->tmp_e, ne * es)) || (rc = dalloc(&P->u, nd * es)) ||
        (rc = dalloc(&P->f, nd * es)) || (rc = dalloc(&P->r, nd * es)) || (rc = dalloc(&P->z, nd * es)) ||
        (rc = dalloc(&P->q, nd * es)) || (rc = dalloc(&P->tmp_v, nd * es)) || (rc = dalloc(&F.dinv, nd * es)))
        return bail(rc);
    void* mk = nullptr;
    // masks are read as aligned 4-byte words: round the allocation up
    if ((rc = dalloc(&mk, ((size_t)P->n_node + 7) & ~(size_t)3))) return bail(rc);
    F.mask = (uint8_t*)mk;
    void* stp = nullptr;
    if ((rc = dalloc(&stp, st.size() * sizeof(int4))) || (rc = dalloc(&P->stencil_w, sw.size() * es))) return bail(rc);
    P->stencil = (int4*)stp;
    void* p = nullptr;
    if ((rc = dalloc(&p, sizeof(DevScalars)))) return bail(rc);
    P->sc = (DevScalars*)p;
    if ((rc = dalloc(&p, sizeof(double) * (size_t)kMaxRedBlocks * (kRedQ + 2 * 12)))) return bail(rc);
    P->red = (double*)p;
    if ((rc = dalloc(&p, sizeof(double) * (size_t)kMaxRedBlocks * (kRedQ + 2 * 12)))) return bail(rc);
    P->red_d = (double*)p;
    if ((rc = dalloc(&p, sizeof(unsigned) * 64))) return bail(rc);
    P->counters = (unsigned*)p;
    if ((rc = dalloc(&p, sizeof(to_stats) * 256))) return bail(rc);
    P->dstats = (to_stats*)p;
    P->dstats_cap = 256;

    // host-built tables: mask, load vector, stencil
    std::vector<uint8_t> hmask((size_t)P->n_node, 0);
    for (int64_t i = 0; i < B->n; ++i) hmask[(size_t)(B->dof[i] / 3)] |= (uint8_t)(1u << (B->dof[i] % 3));
    std::vector<double> hf(nd, 0.0);
    for (int64_t i = 0; i < L->n; ++i) hf[(size_t)L->dof[i]] += L->val[i];
    for (size_t i = 0; i < nd; ++i)
        if ((hmask[i / 3] >> (i % 3)) & 1) hf[i] = 0.0;

    if ((rc = build_tile_mask(F, hmask.data()))) return bail(rc);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return bail(fail(TO_ERR_CUDA, "stream"));
    auto upload = [&](void* dst, const void* src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
    };
    bool ok = cudaMemsetAsync(F.mask, 0, ((size_t)P->n_node + 7) & ~(size_t)3, s) == cudaSuccess &&
              upload(F.mask, hmask.data(), hmask.size()) && upload(P->stencil, st.data(), st.size() * sizeof(int4));
    std::vector<float> hf32, sw32;
    if (P->prec == TO_FP64) {
        ok = ok && upload(P->f, hf.data(), nd * 8) && upload(P->stencil_w, sw.data(), sw.size() * 8);
    } else {
        hf32.assign(hf.begin(), hf.end());
        sw32.assign(sw.begin(), sw.end());
        ok = ok && upload(P->f, hf32.data(), nd * 4) && upload(P->stencil_w, sw32.data(), sw32.size() * 4);
    }
    DevScalars hsc{};
    hsc.k = 1;
    hsc.alpha0 = prm->alpha0 > 0.0 ? prm->alpha0 : 0.0;
    ok = ok && upload(P->sc, &hsc, sizeof hsc);
    ok = ok && cudaMemsetAsync(P->counters, 0, sizeof(unsigned) * 64, s) == cudaSuccess;
    ok = ok && cudaMemsetAsync(P->u, 0, nd * es, s) == cudaSuccess;
    if (!ok) {
        cudaStreamDestroy(s);
        return bail(fail(TO_ERR_CUDA, "upload failed"));
    }
    if ((rc = fill_scalar(P, P->rho, P->n_elem, m->volfrac > m->rho_max ? m->rho_max : m->volfrac, s)) ||
        (rc = launch_rowsum(P, s))) {
        cudaStreamDestroy(s);
        return bail(rc);
    }
    if (prm->proj_sort && (rc = dalloc(&P->ps_buf, projsort_bytes(P)))) {
        cudaStreamDestroy(s);
        return bail(rc);
    }
    if (prm->precond == TO_PRECOND_KRYLOV && (rc = krylov_build(P))) {
        cudaStreamDestroy(s);
        return bail(rc);
    }
    if (prm->precond == TO_PRECOND_MG && (rc = mg_build(P))) {
        cudaStreamDestroy(s);
        return bail(rc);
    }
    if ((rc = project_cluster_setup(P)) || (rc = operator_tc_build(P))) {
        cudaStreamDestroy(s);
        return bail(rc);
    }
    if ((rc = launch_moduli(P, s)) || (rc = refresh_preconditioner(P, s)) ||
        (prm->tile_z == 0 && (rc = operator_autotune(P, s))) || (rc = mg_legs_build(P))) {
        cudaStreamDestroy(s);
        return bail(rc);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) return bail(fail(TO_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e)));
    *out = P;
    return TO_OK;
}

extern "C" int to_sizes(const to_problem* P, int64_t* n_elem, int64_t* n_dof) {
    if (!P) return fail(TO_ERR_ARG, "null problem");
    if (n_elem) *n_elem = P->n_elem;
    if (n_dof) *n_dof = P->n_dof;
    return TO_OK;
}

#define TO_ENTER(P)                                                   \
    if (!(P)) return fail(TO_ERR_ARG, "null problem");                \
    DeviceGuard dg_((P)->device);                                     \
    if (!dg_.ok) return fail(TO_ERR_CUDA, "cudaSetDevice failed");   \
    cudaStream_t s = (cudaStream_t)stream;

extern "C" int to_set_design(to_problem* P, const void* rho_dev, void* stream) {
    TO_ENTER(P);
    if (!rho_dev) return fail(TO_ERR_ARG, "rho is null");
    TO_CUDA(cudaMemcpyAsync(P->rho, rho_dev, P->n_elem * P->esz, cudaMemcpyDeviceToDevice, s));
    P->fwd_id = 0;   // iterates kept by a truncated forward belong to the old design
    int rc = launch_moduli(P, s);
    if (rc) return rc;
    P->precond_stale = 1;   // refreshed by the next to_inner_solve (to_step refreshes every iteration)
    P->pipe_ready = 0;
    P->design_check = 0;
    return TO_OK;
}

extern "C" int to_apply_K(to_problem* P, const void* u_dev, void* y_dev, void* stream) {
    TO_ENTER(P);
    if (!u_dev || !y_dev) return fail(TO_ERR_ARG, "null vector");
    if (u_dev == y_dev) return fail(TO_ERR_ARG, "u and y must not overlap");
    return launch_operator(P, 0, OP_APPLY, u_dev, y_dev, nullptr, s);
}

extern "C" int to_residual(to_problem* P, const void* u_dev, void* r_dev, void* z_dev, void* gt_dev,
                           double* scalars_out, void* stream) {
    TO_ENTER(P);
    if (!u_dev || !r_dev) return fail(TO_ERR_ARG, "null vector");
    if (u_dev == r_dev || u_dev == z_dev || (z_dev && z_dev == r_dev)) return fail(TO_ERR_ARG, "vectors must not overlap");
    if (P->precond_stale) {   // 1 / diag(K^) of the current design
        if (int rc0 = refresh_preconditioner(P, s)) return rc0;
        P->precond_stale = 0;
    }
    const OpOut out{z_dev, gt_dev};
    int rc = launch_operator(P, 0, OP_RESID, u_dev, r_dev, P->f, s, 0.0, 1, &out);
    if (rc) return rc;
    if (scalars_out) {
        DevScalars h;
        TO_CUDA(cudaMemcpyAsync(&h, P->sc, sizeof h, cudaMemcpyDeviceToHost, s));
        TO_CUDA(cudaStreamSynchronize(s));
        scalars_out[0] = z_dev ? h.rz : 0.0;
        scalars_out[1] = h.res2;
        scalars_out[2] = h.res_inf;
        scalars_out[3] = h.J;
        if (h.err) return fail(h.err, "device-side error in the residual");
    }
    return TO_OK;
}

extern "C" int to_smooth(to_problem* P, const void* x_dev, const void* b_dev, void* y_dev, double omega, void* stream) {
    TO_ENTER(P);
    if (!x_dev || !b_dev || !y_dev) return fail(TO_ERR_ARG, "null vector");
    if (y_dev == x_dev || y_dev == b_dev) return fail(TO_ERR_ARG, "y must not overlap x or b");
    if (!std::isfinite(omega)) return fail(TO_ERR_ARG, "omega must be finite");
    if (P->precond_stale) {
        if (int rc0 = refresh_preconditioner(P, s)) return rc0;
        P->precond_stale = 0;
    }
    return launch_operator(P, 0, OP_SMOOTH, x_dev, y_dev, b_dev, s, omega, 0);
}

extern "C" int to_inner_solve(to_problem* P, void* u_dev, int32_t nsteps, double* res_out, void* stream) {
    TO_ENTER(P);
    if (!u_dev || nsteps < 0) return fail(TO_ERR_ARG, "bad arguments");
    if (P->precond_stale) {
        if (int rc0 = refresh_preconditioner(P, s)) return rc0;
        P->precond_stale = 0;
    }
    void* gt = P->gt;
    P->gt = nullptr;
    int rc = run_inner(P, u_dev, nsteps, 0, s, 0);
    if (!rc && res_out) rc = launch_operator(P, 0, OP_RESID, u_dev, P->r, P->f, s, 0.0, 1);
    P->gt = gt;
    if (rc) return rc;
    if (res_out) {
        DevScalars h;
        TO_CUDA(cudaMemcpyAsync(&h, P->sc, sizeof h, cudaMemcpyDeviceToHost, s));
        TO_CUDA(cudaStreamSynchronize(s));
        *res_out = h.res2;
        if (h.err) return fail(h.err, "device-side error in the lower-level steps");
    }
    return TO_OK;
}

extern "C" int to_sensitivity(to_problem* P, const void* u_dev, void* g_dev, void* stream) {
    TO_ENTER(P);
    if (!u_dev || !g_dev) return fail(TO_ERR_ARG, "null vector");
    int rc = launch_energy(P, u_dev, s);
    if (rc) return rc;
    return launch_filter_prescaled_T(P, P->gt, g_dev, s);
}

extern "C" int to_filter(to_problem* P, const void* x_dev, void* y_dev, int32_t transpose, void* stream) {
    TO_ENTER(P);
    if (!x_dev || !y_dev || x_dev == y_dev) return fail(TO_ERR_ARG, "bad vectors");
    return launch_filter(P, x_dev, y_dev, transpose ? 1 : 0, s);
}

extern "C" int to_project(to_problem* P, const void* w_dev, void* rho_dev, double* lambda_out, void* stream) {
    TO_ENTER(P);
    if (!w_dev || !rho_dev) return fail(TO_ERR_ARG, "null vector");
    int rc = launch_project(P, w_dev, nullptr, nullptr, rho_dev, 0, s);
    if (rc) return rc;
    if (lambda_out) {
        DevScalars h;
        TO_CUDA(cudaMemcpyAsync(&h, P->sc, sizeof h, cudaMemcpyDeviceToHost, s));
        TO_CUDA(cudaStreamSynchronize(s));
        *lambda_out = h.lambda;
        if (h.err) return fail(h.err, "device-side error in the projection");
    }
    return TO_OK;
}

__global__ void k_reset_rec(to::DevScalars* sc) { sc->rec = 0; }

// Capture one outer iteration on the library stream; on any failure the
// iteration is launched kernel by kernel from then on.
static int capture_outer(to_problem* P) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(P->gstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        P->graph_state = -1;
        return TO_OK;
    }
    const int rc = outer_iteration(P, P->gstream);
    const cudaError_t e = cudaStreamEndCapture(P->gstream, &g);
    if (rc != TO_OK || e != cudaSuccess || !g) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        P->graph_state = -1;
        return TO_OK;
    }
    const cudaError_t ei = cudaGraphInstantiate(&P->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        P->gexec = nullptr;
        P->graph_state = -1;
        return TO_OK;
    }
    P->graph_state = 1;
    return TO_OK;
}

// The same for the pipelined iteration of the live set (one graph per set: the kernels'
// pointers differ)
static int capture_pipelined(to_problem* P, int fresh) {
    const int p = P->set_parity;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(P->gstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        P->pipe_state[p][fresh] = -1;
        return TO_OK;
    }
    const int rc = outer_iteration_pipelined(P, P->gstream, fresh);
    const cudaError_t e = cudaStreamEndCapture(P->gstream, &g);
    if (rc != TO_OK || e != cudaSuccess || !g) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        P->pipe_state[p][fresh] = -1;
        return TO_OK;
    }
    const cudaError_t ei = cudaGraphInstantiate(&P->gexec_pipe[p][fresh], g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        P->gexec_pipe[p][fresh] = nullptr;
        P->pipe_state[p][fresh] = -1;
        return TO_OK;
    }
    P->pipe_state[p][fresh] = 1;
    return TO_OK;
}

extern "C" int to_step(to_problem* P, int32_t n_outer, to_stats* stats_out, void* stream) {
    TO_ENTER(P);
    if (n_outer < 0) return fail(TO_ERR_ARG, "n_outer must be >= 0");
    if (n_outer == 0) return TO_OK;
    P->fwd_id = 0;   // the outer iterations change the design
    if (n_outer > P->dstats_cap) {
        TO_CUDA(cudaStreamSynchronize(s));
        TO_CUDA(cudaStreamSynchronize(P->gstream));
        void* p = P->dstats;
        dfree(p);
        int cap = P->dstats_cap;
        while (cap < n_outer) cap *= 2;
        if (int rc = dalloc(&p, sizeof(to_stats) * (size_t)cap)) return rc;
        P->dstats = (to_stats*)p;
        P->dstats_cap = cap;
        if (P->gexec) cudaGraphExecDestroy(P->gexec);   // the captured record kernel holds the old ring
        P->gexec = nullptr;
        if (P->graph_state == 1) P->graph_state = 0;
        for (int p = 0; p < 2; ++p)
            for (int f = 0; f < 3; ++f) {
                if (P->gexec_pipe[p][f]) cudaGraphExecDestroy(P->gexec_pipe[p][f]);
                P->gexec_pipe[p][f] = nullptr;
                if (P->pipe_state[p][f] == 1) P->pipe_state[p][f] = 0;
            }
    }
    // run on the library stream, ordered after the caller's stream and before its next work
    TO_CUDA(cudaEventRecord(P->ev_in, s));
    TO_CUDA(cudaStreamWaitEvent(P->gstream, P->ev_in, 0));
    k_reset_rec<<<1, 1, 0, P->gstream>>>(P->sc);
    TO_CUDA(cudaGetLastError());
    // Pipelined iterations (each builds the next design's preconditioner beside its own
    // lower-level steps) unless the persistent multigrid legs or a batch hold this
    // problem's buffer pointers, or the second set could not be allocated.
    bool pipe = P->prm.mg_legs == 0 && !P->in_batch && P->alt_alloc != 2;
    if (pipe && pipe_alloc(P) != TO_OK) {
        cudaGetLastError();
        pipe = false;
    }
    if (pipe) {
        // the first iteration computes the live set itself unless the last to_step left it;
        // after to_set_state only if the design it brought differs (decided on the device)
        int fresh = P->pipe_ready ? 0 : (P->design_check ? 2 : 1);
        P->pipe_ready = 0;
        P->design_check = 0;
        for (int i = 0; i < n_outer; ++i, fresh = 0) {
            const int p = P->set_parity;
            if (P->prm.no_graph == 0 && P->pipe_state[p][fresh] == 0) {
                int rc = capture_pipelined(P, fresh);
                if (rc) return rc;
            }
            if (P->pipe_state[p][fresh] == 1) {
                TO_CUDA(cudaGraphLaunch(P->gexec_pipe[p][fresh], P->gstream));
            } else {
                int rc = outer_iteration_pipelined(P, P->gstream, fresh);
                if (rc) return rc;
            }
            pipe_swap(P);   // the set built for rho_{k+1} is live from here on
        }
        P->pipe_ready = 1;
    } else {
        if (P->prm.no_graph == 0 && P->graph_state == 0) {
            int rc = capture_outer(P);
            if (rc) return rc;
        }
        for (int i = 0; i < n_outer; ++i) {
            if (P->graph_state == 1) {
                TO_CUDA(cudaGraphLaunch(P->gexec, P->gstream));
            } else {
                int rc = outer_iteration(P, P->gstream);
                if (rc) return rc;
            }
        }
        P->pipe_ready = 0;   // the moduli lag rho by one iteration here
        P->design_check = 0;
    }
    P->precond_stale = 0;   // the last iteration refreshed it for its own moduli (pipelined: for rho)
    TO_CUDA(cudaEventRecord(P->ev_out, P->gstream));
    TO_CUDA(cudaStreamWaitEvent(s, P->ev_out, 0));
    P->last_step_n = n_outer;
    if (stats_out) {
        TO_CUDA(cudaMemcpyAsync(stats_out, P->dstats, sizeof(to_stats) * (size_t)n_outer, cudaMemcpyDeviceToHost, s));
        TO_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < n_outer; ++i)
            if (stats_out[i].status) return fail(stats_out[i].status, "device-side error during the outer iterations");
    }
    return TO_OK;
}

extern "C" int to_get_stats(to_problem* P, int32_t n, to_stats* stats_out, void* stream) {
    TO_ENTER(P);
    if (!stats_out) return fail(TO_ERR_ARG, "stats_out is null");
    if (n < 1 || n > P->last_step_n) return fail(TO_ERR_ARG, "n must lie in [1, n_outer of the last to_step call]");
    TO_CUDA(cudaMemcpyAsync(stats_out, P->dstats, sizeof(to_stats) * (size_t)n, cudaMemcpyDeviceToHost, s));
    return TO_OK;
}

extern "C" int to_get_state(to_problem* P, void* rho_dev, void* u_dev, int64_t* k_out, double* alpha0_out, void* stream) {
    TO_ENTER(P);
    if (rho_dev) TO_CUDA(cudaMemcpyAsync(rho_dev, P->rho, P->n_elem * P->esz, cudaMemcpyDeviceToDevice, s));
    if (u_dev) TO_CUDA(cudaMemcpyAsync(u_dev, P->u, P->n_dof * P->esz, cudaMemcpyDeviceToDevice, s));
    if (k_out || alpha0_out) {
        DevScalars h;
        TO_CUDA(cudaMemcpyAsync(&h, P->sc, sizeof h, cudaMemcpyDeviceToHost, s));
        TO_CUDA(cudaStreamSynchronize(s));
        if (k_out) *k_out = h.k;
        if (alpha0_out) *alpha0_out = h.alpha0;
    }
    return TO_OK;
}

__global__ void k_set_counters(to::DevScalars* sc, long long k, double alpha0, int set_k, int set_a, void* host_out,
                               void* host_rec) {
    if (set_k) sc->k = k;
    if (set_a) sc->alpha0 = alpha0 > 0.0 ? alpha0 : 0.0;
    sc->host_out = host_out;
    sc->host_rec = host_rec;
}

// rho <- rho_in, compared bitwise with the old rho: comparison number seq found a
// difference iff afterwards sc->dchanged == sc->dseq.  Also sets k and alpha0 (set_counters)
// and the host buffers of the next iteration's outputs.
template <typename W>
__global__ void k_take_design(const W* __restrict__ in, W* __restrict__ rho, long long n, to::DevScalars* sc,
                              unsigned seq, int set_counters, long long k, double alpha0, void* host_out,
                              void* host_rec) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (set_counters) {
            sc->k = k;
            sc->alpha0 = alpha0 > 0.0 ? alpha0 : 0.0;
        }
        sc->dseq = seq;
        sc->host_out = host_out;
        sc->host_rec = host_rec;
    }
    bool diff = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const W v = in[i];
        diff |= v != rho[i];
        rho[i] = v;
    }
    if (__any_sync(0xffffffffu, diff) && (threadIdx.x & 31) == 0) sc->dchanged = seq;
}

// The design in from rho_dev (device memory), with k and alpha0 (set_counters), rho~ and
// the moduli.  The live set (moduli, 1 / d, coarsest inverse) was built for the current
// rho when a pipelined to_step left it: then the incoming design is compared with rho on
// the device, and the moduli here and the next to_step's rebuild run only if it differs.
static int take_design(to_problem* P, const void* rho_dev, bool set_counters, long long k, double alpha0,
                       cudaStream_t s, void* host_out = nullptr, void* host_rec = nullptr) {
    const bool check = rho_dev && P->pipe_ready && !P->in_batch &&
                       (P->prm.precond != TO_PRECOND_MG || mg_refresh_gatable(P));
    if (check) {
        const long long n = P->n_elem;
        long long nb = (n + 255) / 256;
        if (nb > 4LL * P->num_sms) nb = 4LL * P->num_sms;
        if (nb < 1) nb = 1;
        const unsigned seq = ++P->dseq_host;
        // compared as bit patterns (a NaN equals itself, -0 differs from +0)
        if (P->prec == TO_FP64)
            k_take_design<unsigned long long><<<(unsigned)nb, 256, 0, s>>>(
                (const unsigned long long*)rho_dev, (unsigned long long*)P->rho, n, P->sc, seq, set_counters ? 1 : 0, k,
                alpha0, host_out, host_rec);
        else
            k_take_design<unsigned><<<(unsigned)nb, 256, 0, s>>>((const unsigned*)rho_dev, (unsigned*)P->rho, n, P->sc,
                                                                 seq, set_counters ? 1 : 0, k, alpha0, host_out, host_rec);
        TO_CUDA(cudaGetLastError());
    } else {
        if (rho_dev) TO_CUDA(cudaMemcpyAsync(P->rho, rho_dev, P->n_elem * P->esz, cudaMemcpyDefault, s));
        const int sc_ = set_counters ? 1 : 0;
        k_set_counters<<<1, 1, 0, s>>>(P->sc, k, alpha0, sc_, sc_, host_out, host_rec);
        TO_CUDA(cudaGetLastError());
    }
    int rc = launch_moduli(P, s, check ? &P->sc->dchanged : nullptr);
    if (rc) return rc;
    P->fwd_id = 0;
    P->precond_stale = 1;   // refreshed by the next to_inner_solve (to_step refreshes every iteration)
    P->pipe_ready = 0;
    P->design_check = check ? 1 : 0;
    return TO_OK;
}

extern "C" int to_set_state(to_problem* P, const void* rho_dev, const void* u_dev, int64_t k, double alpha0, void* stream) {
    TO_ENTER(P);
    if (k < 1) return fail(TO_ERR_ARG, "k must be >= 1");
    if (u_dev) TO_CUDA(cudaMemcpyAsync(P->u, u_dev, P->n_dof * P->esz, cudaMemcpyDeviceToDevice, s));
    return take_design(P, rho_dev, true, (long long)k, alpha0, s);
}

// the device alias of page-locked host memory aligned to `align` bytes for the kernels
// that read or write it in place, or nullptr (pageable or misaligned memory: copies instead)
static void* host_alias(const void* p, size_t align) {
    if ((uintptr_t)p % align != 0) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer || (uintptr_t)at.devicePointer % align != 0) return nullptr;
    return at.devicePointer;
}

extern "C" int to_step_host(to_problem* P, const void* rho_in, void* rho_out, to_stats* stats_out, void* stream) {
    TO_ENTER(P);
    if (!rho_in) return fail(TO_ERR_ARG, "rho_in is null");
    const size_t bytes = P->n_elem * P->esz;
    if (!stats_out && !P->stats_pinned) {
        void* h = nullptr;
        TO_CUDA(cudaMallocHost(&h, sizeof(to_stats)));
        P->stats_pinned = (to_stats*)h;
    }
    to_stats* rec = stats_out ? stats_out : P->stats_pinned;
    // Page-locked buffers are used in place through their device aliases: the comparing
    // copy reads the design over the host link, the iteration writes the new design from
    // its design branch (beside the lower-level steps) and its record with the record.
    // Pageable ones are copied before and after.
    const void* in = host_alias(rho_in, P->esz);
    if (!in) {
        if (!P->rho_stage)
            if (int rc = dalloc(&P->rho_stage, bytes)) return rc;
        TO_CUDA(cudaMemcpyAsync(P->rho_stage, rho_in, bytes, cudaMemcpyHostToDevice, s));
        in = P->rho_stage;
    }
    void* out = rho_out ? host_alias(rho_out, P->esz) : nullptr;
    void* rec_dev = host_alias(rec, alignof(to_stats));
    int rc = take_design(P, in, false, 0, 0.0, s, out, rec_dev);
    if (!rc) rc = to_step(P, 1, nullptr, stream);
    if (rc) {
        // nothing may write into the caller's buffers later
        k_set_counters<<<1, 1, 0, s>>>(P->sc, 0, 0.0, 0, 0, nullptr, nullptr);
        cudaStreamSynchronize(s);
        return rc;
    }
    if (rho_out && !out) TO_CUDA(cudaMemcpyAsync(rho_out, P->rho, bytes, cudaMemcpyDeviceToHost, s));
    if (!rec_dev) TO_CUDA(cudaMemcpyAsync(rec, P->dstats, sizeof(to_stats), cudaMemcpyDeviceToHost, s));
    TO_CUDA(cudaStreamSynchronize(s));
    if (rec->status) return fail(rec->status, "device-side error in the outer iteration");
    return TO_OK;
}

namespace to {
int barrier_selftest(to_problem* P, int absent, long long spin_limit, cudaStream_t s);
}

extern "C" int to_barrier_selftest(to_problem* P, int32_t absent_block, int64_t spin_limit, void* stream) {
    TO_ENTER(P);
    if (spin_limit < 1 || spin_limit > (int64_t)kBarrierSpins) return fail(TO_ERR_ARG, "spin_limit out of range");
    if (absent_block < -1) return fail(TO_ERR_ARG, "absent_block must be >= -1");
    return barrier_selftest(P, absent_block, spin_limit, s);
}

__global__ void k_clear_err(to::DevScalars* sc) { sc->err = 0; }

extern "C" int to_check(to_problem* P, void* stream) {
    TO_ENTER(P);
    DevScalars h;
    TO_CUDA(cudaMemcpyAsync(&h, P->sc, sizeof h, cudaMemcpyDeviceToHost, s));
    TO_CUDA(cudaStreamSynchronize(s));
    if (h.err) {
        // a device-side wait gave up: clear the flag and the barrier / reduction words
        k_clear_err<<<1, 1, 0, s>>>(P->sc);
        TO_CUDA(cudaMemsetAsync(P->counters, 0, sizeof(unsigned) * 64, s));
        TO_CUDA(cudaStreamSynchronize(s));
        return fail(h.err, "device-side error flag was set");
    }
    return TO_OK;
}
