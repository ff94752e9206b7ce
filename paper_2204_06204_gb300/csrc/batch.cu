// Many independent design problems advanced together: one kernel launch per
// phase of the outer iteration (Algorithms 1 / 3) covers every problem, and
// the whole batched iteration is captured once as a CUDA graph.
//
// Each problem keeps its own buffers, scalars, reduction slots and stats ring
// (it is an ordinary to_problem); the batched kernels read a device table of
// per-problem arguments indexed by blockIdx.y (blockIdx.x for the projection's
// clusters).  Phases, per outer iteration:
//   design   rho -> rho~ -> E, E'/Hs            k_filter_batch (moduli)
//   diag     Jacobi diagonal                     k_b_diag
//   (multigrid: coarse moduli and diagonals, dense coarsest operators and their
//    inverses, one launch per step and level; see the batched multigrid in mg.cu)
//   resid    r = f - K u, z = r/d, sensitivity   k_operator_batch<OP_RESID>
//   (multigrid: z = V-cycle(r), r^T z in its last sweep)
//   n_inner x (Q apply, update[, V-cycle])       k_operator_batch<OP_Q>, k_b_update
//   filterT  g = C^T g~, ||g||_inf, alpha_k      k_filter_batch (transpose, statistics)
//   project  one thread-block cluster per problem (distributed shared memory
//            for the pass totals: no grid-wide barrier between problems)
//   record   per-problem stats                    k_b_record
// Requirements: every problem uses steepest descent with the same n_inner and
// the same preconditioner (Jacobi, or multigrid with the same smoothing
// parameters), the same precision, device, element size and material moduli
// (the element matrix constants are common to the launch).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "projection.cuh"

namespace cg = cooperative_groups;

namespace to {
template <typename T>
SimpT<T> simp_params(const to_material& m);

int batch_operator_launch(int prec, int mode, const void* tab, const void* kh, int max_tiles, int n, cudaStream_t s);
int filter_table_build(to_problem* const* probs, int n, int mode, void** dev, int* max_tiles, size_t* smem);
int filter_batch_launch(int prec, int mode, const void* tab, int max_tiles, int n, size_t smem, cudaStream_t s);
int batch_autotune_kchunk(to_problem* const* probs, int n, const void* kh, cudaStream_t s, int* best_out, float* us_out);
int op_tables_build(to_problem* const* probs, int n, void** resid, void** q_first, void** q, void** kh_host,
                    int* max_tiles, int kchunk);

template <typename T>
struct BProb {
    int nx, ny, nz;
    long long n_elem, n_dof;
    const T* rho;
    T* E;
    T* grad;
    const uint8_t* mask;
    T* dinv;   // 1 / diag(K^)
    double kdiag;
    T* u;
    T* r;
    T* z;
    const T* q;
    T* wbuf;
    double* red;
    unsigned* counters;
    DevScalars* sc;
    to_stats* dstats;
    int dstats_cap;
    double vbar, lo, hi;
    int mean_proj;
};

template <typename T>
__global__ void __launch_bounds__(256) k_b_diag(const BProb<T>* __restrict__ tab) {
    const BProb<T>& P = tab[blockIdx.y];
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const long long nn = P.n_dof / 3;
    for (long long n = blockIdx.x * 256LL + threadIdx.x; n < nn; n += (long long)gridDim.x * 256) {
        const int i = (int)(n % (nx + 1)), j = (int)((n / (nx + 1)) % (ny + 1)), k = (int)(n / ((long long)(nx + 1) * (ny + 1)));
        T s = T(0);
        for (int dk = -1; dk <= 0; ++dk)
            for (int dj = -1; dj <= 0; ++dj)
                for (int di = -1; di <= 0; ++di) {
                    const int ei = i + di, ej = j + dj, ek = k + dk;
                    if (ei < 0 || ei >= nx || ej < 0 || ej >= ny || ek < 0 || ek >= nz) continue;
                    s += P.E[ei + (long long)nx * (ej + (long long)ny * ek)];
                }
        const uint8_t mk = P.mask[n];
        const T v = T(1) / ((T)P.kdiag * s);
        for (int c = 0; c < 3; ++c) P.dinv[3 * n + c] = ((mk >> c) & 1) ? T(1) : v;
    }
}

// u += beta z, r -= beta q and (Jacobi) z = r / d with r^T z, per problem
template <typename T, bool JACOBI>
__global__ void __launch_bounds__(256) k_b_update(const BProb<T>* __restrict__ tab) {
    __shared__ double sh[32 * kRedQ];
    const BProb<T>& P = tab[blockIdx.y];
    __shared__ T s_beta;
    if (threadIdx.x == 0) s_beta = (T)P.sc->beta;   // one conversion per block
    __syncthreads();
    const T beta = s_beta;
    T acc = T(0);
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < P.n_dof; i += (long long)gridDim.x * 256) {
        P.u[i] += beta * P.z[i];
        const T ri = P.r[i] - beta * P.q[i];
        P.r[i] = ri;
        if (JACOBI) {
            const T zn = ri * P.dinv[i];
            P.z[i] = zn;
            acc += ri * zn;
        }
    }
    if (!JACOBI) return;
    T v[1] = {acc};
    const int kind[1] = {0};
    double tot[1];
    block_reduce<T, 1>(v, kind, reinterpret_cast<T*>(sh));
    if (finish_reduction<T, 1>(v, kind, P.red, P.counters + 4, tot, sh, blockIdx.x, gridDim.x) && threadIdx.x == 0)
        P.sc->rz = tot[0];
}

// ----------------------------------------------------------------------------- projection, one cluster per problem
constexpr int kClusterCTAs = 8;

// Cluster size (CTAs per problem) and CTA size are launch parameters: the
// batched path launches 8 CTAs of 256 threads per problem, a single problem
// 16 CTAs of 1024 threads.  Each CTA takes a contiguous chunk of its problem.
template <typename T, bool CACHE>
__global__ void __launch_bounds__(1024) k_b_project(const BProb<T>* __restrict__ tab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ ProjPart slots[2];
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank(), csize = cl.num_blocks();
    const BProb<T>& P = tab[blockIdx.x / csize];
    const long long n = P.n_elem;
    const long long chunk = (n + csize - 1) / csize;
    ProjIO io;
    io.n = n;
    io.b0 = (long long)rank * chunk;
    io.b1 = min(io.b0 + chunk, n);
    io.vbar = P.vbar;
    io.lo = P.lo;
    io.hi = P.hi;
    io.fused = 1;
    io.mean_proj = P.mean_proj;
    io.writer = rank == 0;
    io.wdirect = 0;
    ClusterComm comm{slots};
    T* rho = const_cast<T*>(P.rho);
    projection_body<T, CACHE>(comm, io, nullptr, P.rho, P.grad, reinterpret_cast<T*>(smem_raw), P.wbuf, rho, P.sc);
    cl.sync();   // no CTA leaves while another may still read its slots
}

template <typename T>
int launch_cluster_project(const BProb<T>* tab, int n_problems, int csize, int threads, bool cache, size_t smem,
                           cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_problems * csize));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cache) TO_CUDA(cudaLaunchKernelEx(&cfg, k_b_project<T, true>, tab));
    else TO_CUDA(cudaLaunchKernelEx(&cfg, k_b_project<T, false>, tab));
    return TO_OK;
}

// shared-memory and non-portable cluster-size opt-in of the cluster projection
template <typename T>
int cluster_project_attrs(size_t smem) {
    TO_CUDA(cudaFuncSetAttribute(k_b_project<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TO_CUDA(cudaFuncSetAttribute(k_b_project<T, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    TO_CUDA(cudaFuncSetAttribute(k_b_project<T, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    return TO_OK;
}

template <typename T>
__global__ void k_b_record(const BProb<T>* __restrict__ tab, int n, int reset) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    DevScalars* sc = tab[p].sc;
    if (reset) {
        sc->rec = 0;
        return;
    }
    to_stats s;
    s.k = sc->k;
    s.J = sc->J;
    s.res_inf = sc->res_inf;
    s.res2 = sc->res2;
    s.drho_inf = sc->drho_inf;
    s.volume = sc->volume;
    s.lambda = sc->lambda;
    s.alpha = sc->alpha;
    s.gmax = sc->gmax;
    s.beta_first = sc->beta_first;
    s.beta_last = sc->beta;
    s.proj_iters = sc->proj_iters;
    s.status = sc->err;
    const int slot = sc->rec;
    if (slot >= 0 && slot < tab[p].dstats_cap) tab[p].dstats[slot] = s;
    sc->rec = slot + 1;
    sc->k += 1;
    sc->beta_first = 0.0;
    sc->beta = 0.0;
}

}  // namespace to

// ----------------------------------------------------------------------------- host side
struct to_batch {
    std::vector<to_problem*> probs;
    int n = 0, prec = TO_FP32_MIXED, n_inner = 0, device = 0;
    void* btab = nullptr;                 // BProb<T>[n]
    void* tab_resid = nullptr;            // OpArgs<T>[n]
    void* tab_q_first = nullptr;
    void* tab_q = nullptr;
    void* kh = nullptr;                   // host copy of HaarK<T>
    int max_tiles = 0, grid_x = 0;
    int kchunk = 8;                       // node planes per operator tile, picked by the autotuner
    float tune_us = 0.f;                  // the batch's K u at that choice
    size_t proj_smem = 0;
    bool proj_cache = true;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_state = 0;
    to::BatchMG* mg = nullptr;            // batched multigrid tables (multigrid batches)
    void* ftab[2] = {nullptr, nullptr};   // batched filter tables: design, gradient
    int ftiles[2] = {0, 0};
    size_t fsmem[2] = {0, 0};
    // Pipelined iterations (as to_step's): the tables over the members' second design sets;
    // swapped with the live ones above (and every member's sets) after each iteration
    struct Alt {
        void* btab = nullptr;
        void* tab_resid = nullptr;
        void* tab_q_first = nullptr;
        void* tab_q = nullptr;
        void* ftab0 = nullptr;
        to::BatchMG* mg = nullptr;
    } alt;
    int pipe = 0;                         // the second sets and their tables exist
    int parity = 0;
    cudaStream_t dside = nullptr;         // the design branch
    cudaEvent_t ev_dfork = nullptr, ev_djoin = nullptr;
    cudaGraphExec_t gexec_pipe[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [parity][fresh]
    int pipe_state[2][2] = {{0, 0}, {0, 0}};
};

using namespace to;

namespace {

template <typename T>
int build_tables_t(to_batch* B) {
    std::vector<BProb<T>> h(B->n);
    long long max_elem = 0, max_dof = 0;
    for (int i = 0; i < B->n; ++i) {
        to_problem* P = B->probs[i];
        BProb<T>& b = h[i];
        b.nx = P->g.nx;
        b.ny = P->g.ny;
        b.nz = P->g.nz;
        b.n_elem = P->n_elem;
        b.n_dof = P->n_dof;
        b.rho = (const T*)P->rho;
        b.E = (T*)P->lv[0].E;
        b.grad = (T*)P->grad;
        b.mask = P->lv[0].mask;
        b.dinv = (T*)P->lv[0].dinv;
        b.kdiag = P->kdiag;
        b.u = (T*)P->u;
        b.r = (T*)P->r;
        b.z = (T*)P->z;
        b.q = (const T*)P->q;
        b.wbuf = (T*)P->tmp_e;
        b.red = P->red;
        b.counters = P->counters;
        b.sc = P->sc;
        b.dstats = P->dstats;
        b.dstats_cap = P->dstats_cap;
        b.vbar = P->mat.volfrac * (double)P->n_elem;
        b.lo = P->mat.rho_min;
        b.hi = P->mat.rho_max;
        b.mean_proj = P->prm.mean_proj;
        max_elem = std::max<long long>(max_elem, (long long)P->n_elem);
        max_dof = std::max<long long>(max_dof, (long long)P->n_dof);
    }
    if (!B->btab && cudaMalloc(&B->btab, sizeof(BProb<T>) * (size_t)B->n) != cudaSuccess)
        return fail(TO_ERR_CUDA, "batch table allocation");
    if (cudaMemcpy(B->btab, h.data(), sizeof(BProb<T>) * (size_t)B->n, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(TO_ERR_CUDA, "batch table upload");
    // grid-stride width for the elementwise phases: enough blocks for the largest problem
    B->grid_x = (int)std::min<long long>((max_dof + 255) / 256, 64);
    const long long chunk = (max_elem + kClusterCTAs - 1) / kClusterCTAs;
    B->proj_smem = (size_t)chunk * sizeof(T);
    B->proj_cache = B->proj_smem <= 96 * 1024;
    if (!B->proj_cache) B->proj_smem = 0;
    if (int rc = cluster_project_attrs<T>(160 * 1024)) return rc;
    return TO_OK;
}

template <typename T>
int iteration_t(to_batch* B, cudaStream_t s) {
    const BProb<T>* tab = (const BProb<T>*)B->btab;
    const dim3 g2(B->grid_x, B->n);
    int rc;
    if ((rc = filter_batch_launch(B->prec, 0, B->ftab[0], B->ftiles[0], B->n, B->fsmem[0], s))) return rc;
    k_b_diag<T><<<g2, 256, 0, s>>>(tab);
    TO_CUDA(cudaGetLastError());
    if (B->mg && (rc = batch_mg_refresh(B->mg, s))) return rc;
    if ((rc = batch_operator_launch(B->prec, OP_RESID, B->tab_resid, B->kh, B->max_tiles, B->n, s))) return rc;
    if (B->mg && (rc = batch_mg_vcycle(B->mg, s))) return rc;
    for (int it = 0; it < B->n_inner; ++it) {
        rc = batch_operator_launch(B->prec, OP_Q, it == 0 ? B->tab_q_first : B->tab_q, B->kh, B->max_tiles, B->n, s);
        if (rc) return rc;
        if (B->mg) k_b_update<T, false><<<g2, 256, 0, s>>>(tab);
        else k_b_update<T, true><<<g2, 256, 0, s>>>(tab);
        TO_CUDA(cudaGetLastError());
        if (B->mg && it + 1 < B->n_inner && (rc = batch_mg_vcycle(B->mg, s))) return rc;
    }
    if (B->mg && (rc = batch_mg_join(B->mg, s))) return rc;   // the refresh branch, if no tail joined it
    if ((rc = filter_batch_launch(B->prec, 1, B->ftab[1], B->ftiles[1], B->n, B->fsmem[1], s))) return rc;
    if ((rc = launch_cluster_project<T>(tab, B->n, kClusterCTAs, 256, B->proj_cache, B->proj_smem, s))) return rc;
    k_b_record<T><<<(B->n + 63) / 64, 64, 0, s>>>(tab, B->n, 0);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

// The same iteration with the next designs' moduli, diagonals and (multigrid) coarse
// refresh built on the design branch into the members' second sets (B->alt tables)
// while the lower-level steps run on the live sets; `fresh`: the live sets are
// computed first.  The kernels see the same inputs as in iteration_t.
template <typename T>
int iteration_pipelined_t(to_batch* B, cudaStream_t s, bool fresh) {
    const BProb<T>* tab = (const BProb<T>*)B->btab;
    const BProb<T>* tabn = (const BProb<T>*)B->alt.btab;
    const dim3 g2(B->grid_x, B->n);
    int rc;
    if (fresh) {
        if ((rc = filter_batch_launch(B->prec, 0, B->ftab[0], B->ftiles[0], B->n, B->fsmem[0], s))) return rc;
        k_b_diag<T><<<g2, 256, 0, s>>>(tab);
        TO_CUDA(cudaGetLastError());
        if (B->mg && (rc = batch_mg_refresh(B->mg, s))) return rc;
    }
    if ((rc = batch_operator_launch(B->prec, OP_RESID, B->tab_resid, B->kh, B->max_tiles, B->n, s))) return rc;
    cudaStream_t d = B->dside;
    TO_CUDA(cudaEventRecord(B->ev_dfork, s));
    TO_CUDA(cudaStreamWaitEvent(d, B->ev_dfork, 0));
    if ((rc = filter_batch_launch(B->prec, 1, B->ftab[1], B->ftiles[1], B->n, B->fsmem[1], d))) return rc;
    if ((rc = launch_cluster_project<T>(tab, B->n, kClusterCTAs, 256, B->proj_cache, B->proj_smem, d))) return rc;
    // the live inverses (fresh: still on the multigrid branch) share the assembled
    // operators and the inversion scratch with the next ones
    if (fresh && B->mg && (rc = batch_mg_wait(B->mg, d))) return rc;
    if ((rc = filter_batch_launch(B->prec, 0, B->alt.ftab0, B->ftiles[0], B->n, B->fsmem[0], d))) return rc;
    k_b_diag<T><<<g2, 256, 0, d>>>(tabn);
    TO_CUDA(cudaGetLastError());
    if (B->alt.mg && (rc = batch_mg_refresh_inline(B->alt.mg, d))) return rc;
    TO_CUDA(cudaEventRecord(B->ev_djoin, d));
    if (B->mg && (rc = batch_mg_vcycle(B->mg, s))) return rc;
    for (int it = 0; it < B->n_inner; ++it) {
        rc = batch_operator_launch(B->prec, OP_Q, it == 0 ? B->tab_q_first : B->tab_q, B->kh, B->max_tiles, B->n, s);
        if (rc) return rc;
        if (B->mg) k_b_update<T, false><<<g2, 256, 0, s>>>(tab);
        else k_b_update<T, true><<<g2, 256, 0, s>>>(tab);
        TO_CUDA(cudaGetLastError());
        if (B->mg && it + 1 < B->n_inner && (rc = batch_mg_vcycle(B->mg, s))) return rc;
    }
    if (B->mg && (rc = batch_mg_join(B->mg, s))) return rc;
    TO_CUDA(cudaStreamWaitEvent(s, B->ev_djoin, 0));
    k_b_record<T><<<(B->n + 63) / 64, 64, 0, s>>>(tab, B->n, 0);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

// the live tables and every member's live set become the other ones
void batch_swap(to_batch* B) {
    std::swap(B->btab, B->alt.btab);
    std::swap(B->tab_resid, B->alt.tab_resid);
    std::swap(B->tab_q_first, B->alt.tab_q_first);
    std::swap(B->tab_q, B->alt.tab_q);
    std::swap(B->ftab[0], B->alt.ftab0);
    std::swap(B->mg, B->alt.mg);
    for (to_problem* P : B->probs) pipe_swap(P);
    B->parity ^= 1;
}

// the members' second sets and the tables over them (built with the sets swapped in)
int build_alt(to_batch* B) {
    for (to_problem* P : B->probs)
        if (P->alt_alloc == 2 || pipe_alloc(P) != TO_OK) {
            cudaGetLastError();
            return TO_OK;   // no pipelining for this batch
        }
    if (cudaStreamCreateWithFlags(&B->dside, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_dfork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_djoin, cudaEventDisableTiming) != cudaSuccess)
        return fail(TO_ERR_CUDA, "batch stream / event creation failed");
    const int n = B->n;
    for (to_problem* P : B->probs) pipe_swap(P);
    // build the second tables into the live fields, then exchange the two
    std::swap(B->btab, B->alt.btab);
    std::swap(B->tab_resid, B->alt.tab_resid);
    std::swap(B->tab_q_first, B->alt.tab_q_first);
    std::swap(B->tab_q, B->alt.tab_q);
    std::swap(B->ftab[0], B->alt.ftab0);
    std::swap(B->mg, B->alt.mg);
    void* kh = nullptr;
    int mt = 0, ft = 0;
    size_t fs = 0;
    int rc = B->prec == TO_FP64 ? build_tables_t<double>(B) : build_tables_t<float>(B);
    if (!rc) rc = op_tables_build(B->probs.data(), n, &B->tab_resid, &B->tab_q_first, &B->tab_q, &kh, &mt, B->kchunk);
    free(kh);
    if (!rc && B->alt.mg) rc = batch_mg_build(B->probs.data(), n, B->kchunk, &B->mg);
    if (!rc) rc = filter_table_build(B->probs.data(), n, 0, &B->ftab[0], &ft, &fs);
    std::swap(B->btab, B->alt.btab);
    std::swap(B->tab_resid, B->alt.tab_resid);
    std::swap(B->tab_q_first, B->alt.tab_q_first);
    std::swap(B->tab_q, B->alt.tab_q);
    std::swap(B->ftab[0], B->alt.ftab0);
    std::swap(B->mg, B->alt.mg);
    for (to_problem* P : B->probs) pipe_swap(P);
    if (rc) return rc;
    B->pipe = 1;
    return TO_OK;
}

void destroy_batch(to_batch* B) {
    if (!B) return;
    if (B->stream) cudaStreamSynchronize(B->stream);
    if (B->dside) cudaStreamSynchronize(B->dside);
    if (B->gexec) cudaGraphExecDestroy(B->gexec);
    for (int p = 0; p < 2; ++p)
        for (int f = 0; f < 2; ++f)
            if (B->gexec_pipe[p][f]) cudaGraphExecDestroy(B->gexec_pipe[p][f]);
    if (B->ev_dfork) cudaEventDestroy(B->ev_dfork);
    if (B->ev_djoin) cudaEventDestroy(B->ev_djoin);
    if (B->dside) cudaStreamDestroy(B->dside);
    {
        void* ps[] = {B->alt.btab, B->alt.tab_resid, B->alt.tab_q_first, B->alt.tab_q, B->alt.ftab0};
        for (void* p : ps)
            if (p) cudaFree(p);
        batch_mg_free(B->alt.mg);
    }
    if (B->ev_in) cudaEventDestroy(B->ev_in);
    if (B->ev_out) cudaEventDestroy(B->ev_out);
    if (B->stream) cudaStreamDestroy(B->stream);
    void* ps[] = {B->btab, B->tab_resid, B->tab_q_first, B->tab_q, B->ftab[0], B->ftab[1]};
    for (void* p : ps)
        if (p) cudaFree(p);
    free(B->kh);
    batch_mg_free(B->mg);
    delete B;
}

}  // namespace


extern "C" int to_batch_create(to_problem* const* problems, int32_t n, to_batch** out) {
    if (!out) return fail(TO_ERR_ARG, "out is null");
    *out = nullptr;
    if (!problems || n < 1) return fail(TO_ERR_ARG, "need at least one problem");
    const to_problem* P0 = problems[0];
    if (!P0) return fail(TO_ERR_ARG, "null problem");
    for (int i = 0; i < n; ++i) {
        const to_problem* P = problems[i];
        if (!P) return fail(TO_ERR_ARG, "null problem");
        const bool pre_ok = P->prm.precond == P0->prm.precond &&
                            (P0->prm.precond == TO_PRECOND_JACOBI ||
                             (P0->prm.precond == TO_PRECOND_MG && P->prm.mg_nu_pre == P0->prm.mg_nu_pre &&
                              P->prm.mg_nu_post == P0->prm.mg_nu_post && P->prm.mg_omega == P0->prm.mg_omega));
        if (P->prec != P0->prec || P->device != P0->device || !pre_ok || P->prm.inner_mode != TO_INNER_SD ||
            P->prm.n_inner != P0->prm.n_inner || P->g.h != P0->g.h || P->mat.E0 != P0->mat.E0 ||
            P->mat.Emin != P0->mat.Emin || P->mat.p != P0->mat.p || P->mat.nu != P0->mat.nu)
            return fail(TO_ERR_ARG,
                        "batched problems must share precision, device, element size, material moduli and n_inner, "
                        "and use steepest descent with the same preconditioner (Jacobi, or multigrid with the same "
                        "smoothing parameters)");
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(P0->device) != cudaSuccess) return fail(TO_ERR_CUDA, "cudaSetDevice failed");
    to_batch* B = new to_batch();
    B->probs.assign(problems, problems + n);
    for (to_problem* P : B->probs) P->in_batch += 1;   // the batch's tables hold their buffer pointers
    B->n = n;
    B->prec = P0->prec;
    B->n_inner = P0->prm.n_inner;
    B->device = P0->device;
    int rc = P0->prec == TO_FP64 ? build_tables_t<double>(B) : build_tables_t<float>(B);
    if (!rc && (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming) != cudaSuccess))
        rc = fail(TO_ERR_CUDA, "batch stream / event creation failed");
    // tile shapes: time the batched operator for each candidate depth, keep the fastest
    if (!rc) rc = op_tables_build(B->probs.data(), n, &B->tab_resid, &B->tab_q_first, &B->tab_q, &B->kh, &B->max_tiles, 8);
    if (!rc && P0->tile_z > 0) B->kchunk = P0->tile_z;   // a fixed tile depth: no autotuning
    else if (!rc) rc = batch_autotune_kchunk(B->probs.data(), n, B->kh, B->stream, &B->kchunk, &B->tune_us);
    if (!rc) rc = op_tables_build(B->probs.data(), n, &B->tab_resid, &B->tab_q_first, &B->tab_q, &B->kh, &B->max_tiles, B->kchunk);
    if (!rc && P0->prm.precond == TO_PRECOND_MG) rc = batch_mg_build(B->probs.data(), n, B->kchunk, &B->mg);
    for (int m = 0; m < 2 && !rc; ++m) rc = filter_table_build(B->probs.data(), n, m, &B->ftab[m], &B->ftiles[m], &B->fsmem[m]);
    if (!rc) rc = build_alt(B);
    if (prev >= 0) cudaSetDevice(prev);
    if (rc) {
        destroy_batch(B);
        return rc;
    }
    *out = B;
    return TO_OK;
}

extern "C" int to_batch_tile(const to_batch* B, int32_t* kchunk_out, double* us_out) {
    if (!B) return fail(TO_ERR_ARG, "null batch");
    if (kchunk_out) *kchunk_out = B->kchunk;
    if (us_out) *us_out = (double)B->tune_us;
    return TO_OK;
}

extern "C" void to_batch_destroy(to_batch* B) {
    if (!B) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(B->device);
    destroy_batch(B);
    if (prev >= 0) cudaSetDevice(prev);
}

extern "C" int to_batch_step(to_batch* B, int32_t n_outer, to_stats* stats_out, void* stream) {
    if (!B) return fail(TO_ERR_ARG, "null batch");
    if (n_outer < 0) return fail(TO_ERR_ARG, "n_outer must be >= 0");
    if (n_outer == 0) return TO_OK;
    for (to_problem* P : B->probs) P->fwd_id = 0;   // the outer iterations change every design
    for (to_problem* P : B->probs)
        if (n_outer > P->dstats_cap)
            return fail(TO_ERR_ARG, "n_outer exceeds a problem's stats ring (run to_step once with that many iterations "
                                    "to grow it, or use fewer outer iterations per call)");
    for (to_problem* P : B->probs) P->last_step_n = n_outer;   // each member's ring holds this call's records
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(B->device) != cudaSuccess) return fail(TO_ERR_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = TO_OK;
    auto body = [&]() -> int {
        TO_CUDA(cudaEventRecord(B->ev_in, s));
        TO_CUDA(cudaStreamWaitEvent(B->stream, B->ev_in, 0));
        if (B->prec == TO_FP64)
            k_b_record<double><<<(B->n + 63) / 64, 64, 0, B->stream>>>((const BProb<double>*)B->btab, B->n, 1);
        else
            k_b_record<float><<<(B->n + 63) / 64, 64, 0, B->stream>>>((const BProb<float>*)B->btab, B->n, 1);
        TO_CUDA(cudaGetLastError());
        if (B->pipe) {
            // the first iteration computes the live sets unless the last batched step left them
            bool fresh = false;
            for (to_problem* P : B->probs) fresh = fresh || !P->pipe_ready;
            for (to_problem* P : B->probs) P->pipe_ready = P->design_check = 0;
            for (int i = 0; i < n_outer; ++i, fresh = false) {
                const int p = B->parity, f = fresh ? 1 : 0;
                if (B->pipe_state[p][f] == 0) {
                    cudaGraph_t g = nullptr;
                    B->pipe_state[p][f] = -1;
                    if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                        const int r2 = B->prec == TO_FP64 ? iteration_pipelined_t<double>(B, B->stream, fresh)
                                                          : iteration_pipelined_t<float>(B, B->stream, fresh);
                        if (cudaStreamEndCapture(B->stream, &g) == cudaSuccess && g && r2 == TO_OK &&
                            cudaGraphInstantiate(&B->gexec_pipe[p][f], g, 0) == cudaSuccess)
                            B->pipe_state[p][f] = 1;
                        if (g) cudaGraphDestroy(g);
                    }
                    cudaGetLastError();
                }
                if (B->pipe_state[p][f] == 1) {
                    TO_CUDA(cudaGraphLaunch(B->gexec_pipe[p][f], B->stream));
                } else {
                    const int r2 = B->prec == TO_FP64 ? iteration_pipelined_t<double>(B, B->stream, fresh)
                                                      : iteration_pipelined_t<float>(B, B->stream, fresh);
                    if (r2) return r2;
                }
                batch_swap(B);   // the sets built for the next designs are live from here on
            }
            for (to_problem* P : B->probs) P->pipe_ready = 1;
        } else if (B->graph_state == 0) {
            cudaGraph_t g = nullptr;
            B->graph_state = -1;
            if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const int r2 = B->prec == TO_FP64 ? iteration_t<double>(B, B->stream) : iteration_t<float>(B, B->stream);
                if (cudaStreamEndCapture(B->stream, &g) == cudaSuccess && g && r2 == TO_OK &&
                    cudaGraphInstantiate(&B->gexec, g, 0) == cudaSuccess)
                    B->graph_state = 1;
                if (g) cudaGraphDestroy(g);
            }
            cudaGetLastError();
        }
        for (int i = 0; i < n_outer && !B->pipe; ++i) {
            if (B->graph_state == 1) {
                TO_CUDA(cudaGraphLaunch(B->gexec, B->stream));
            } else {
                const int r2 = B->prec == TO_FP64 ? iteration_t<double>(B, B->stream) : iteration_t<float>(B, B->stream);
                if (r2) return r2;
            }
        }
        if (!B->pipe)
            for (to_problem* P : B->probs) P->pipe_ready = P->design_check = 0;   // the moduli lag rho by one iteration here
        TO_CUDA(cudaEventRecord(B->ev_out, B->stream));
        TO_CUDA(cudaStreamWaitEvent(s, B->ev_out, 0));
        if (stats_out) {
            for (int p = 0; p < B->n; ++p)
                TO_CUDA(cudaMemcpyAsync(stats_out + (size_t)p * n_outer, B->probs[p]->dstats,
                                        sizeof(to_stats) * (size_t)n_outer, cudaMemcpyDeviceToHost, s));
            TO_CUDA(cudaStreamSynchronize(s));
            for (int p = 0; p < B->n; ++p)
                for (int i = 0; i < n_outer; ++i)
                    if (stats_out[(size_t)p * n_outer + i].status)
                        return fail(stats_out[(size_t)p * n_outer + i].status, "device-side error in a batched problem");
        }
        return TO_OK;
    };
    rc = body();
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}
