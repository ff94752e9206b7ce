// Lower-level steps and the outer iteration.
//
// Lower level (Algorithm 1 / 3, line 1, widened to n_inner steps warm-started
// from the previous u): steepest descent on P_f(u) = 1/2 u^T K u - f^T u along
// z = M^-1 r with the exact line search beta = r^T z / z^T K z, or the literal
// constant-beta step u <- u + beta M^-1 (f - K u).
//
// Outer iteration k (Algorithms 1 / 3):
//   rho~ = C(rho_k), E, E'                        launch_moduli
//   M for this design (diagonal / V-cycle)        launch_diag | mg_refresh
//   r = f - K u_k, g~ = -E' u^T k_e u (at u_k), J  fused operator epilogue
//   n_inner lower-level steps                     operator + update kernels
//   g = C^T g~, ||g||_inf, 1^T g                  launch_sens_filter_T
//   rho_{k+1} = Proj_X(rho_k - alpha_k g)        launch_project (fused)
//   stats record, k += 1                          launch_record
// Every scalar stays on the device; nothing synchronises with the host.
#include "device.cuh"

namespace to {

int project_coop_blocks(int prec, int num_sms, int* out);

static int grid_1d(long long n, int threads, int num_sms) {
    long long b = (n + threads - 1) / threads;
    if (b > 4LL * num_sms) b = 4LL * num_sms;
    return (int)(b < 1 ? 1 : b);
}

// u += beta z; r -= beta q; (Jacobi) z = r / d and r^T z (dinv = 1 / d)
template <typename T, bool JACOBI>
__global__ void __launch_bounds__(256) k_update_sd(long long n, T* __restrict__ u, T* __restrict__ r, T* __restrict__ z,
                                                   const T* __restrict__ q, const T* __restrict__ dinv, double* red,
                                                   unsigned* counter, DevScalars* sc) {
    __shared__ double sh[32 * kRedQ];
    __shared__ T s_beta;
    if (threadIdx.x == 0) s_beta = (T)sc->beta;   // one conversion per block
    __syncthreads();
    const T beta = s_beta;
    T acc = T(0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T zi = z[i];
        u[i] += beta * zi;
        const T ri = r[i] - beta * q[i];
        r[i] = ri;
        if (JACOBI) {
            const T zn = ri * dinv[i];
            z[i] = zn;
            acc += ri * zn;
        }
    }
    if (JACOBI) {
        T v[1] = {acc};
        const int kind[1] = {0};
        double tot[1];
        block_reduce<T, 1>(v, kind, reinterpret_cast<T*>(sh));
        if (finish_reduction<T, 1>(v, kind, red, counter, tot, sh, linear_block(), grid_blocks()) && threadIdx.x == 0) sc->rz = tot[0];
    }
}

// Conjugate gradients: u += alpha p, r -= alpha q (alpha = r^T z / p^T q from the q = K p
// pass); keeps the previous r^T z, and with the Jacobi M also z = r / d and the new r^T z
template <typename T, bool JACOBI>
__global__ void __launch_bounds__(256) k_cg_update(long long n, T* __restrict__ u, T* __restrict__ r, T* __restrict__ z,
                                                   const T* __restrict__ p, const T* __restrict__ q, const T* __restrict__ dinv,
                                                   double* red, unsigned* counter, DevScalars* sc) {
    __shared__ double sh[32 * kRedQ];
    __shared__ T s_alpha;
    if (threadIdx.x == 0) {
        s_alpha = (T)sc->beta;
        if (blockIdx.x == 0) sc->rz_old = sc->rz;   // read before the new r^T z is written (by the last block,
                                                    // or by the preconditioner that follows)
    }
    __syncthreads();
    const T alpha = s_alpha;
    T acc = T(0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        u[i] += alpha * p[i];
        const T ri = r[i] - alpha * q[i];
        r[i] = ri;
        if (JACOBI) {
            const T zn = ri * dinv[i];
            z[i] = zn;
            acc += ri * zn;
        }
    }
    if (JACOBI) {
        T v[1] = {acc};
        const int kind[1] = {0};
        double tot[1];
        block_reduce<T, 1>(v, kind, reinterpret_cast<T*>(sh));
        if (finish_reduction<T, 1>(v, kind, red, counter, tot, sh, linear_block(), grid_blocks()) && threadIdx.x == 0) sc->rz = tot[0];
    }
}

// p = z + (r^T z / previous r^T z) p
template <typename T>
__global__ void __launch_bounds__(256) k_cg_dir(long long n, const T* __restrict__ z, T* __restrict__ p, const DevScalars* sc) {
    __shared__ T s_b;
    if (threadIdx.x == 0) s_b = sc->rz_old != 0.0 ? (T)(sc->rz / sc->rz_old) : T(0);
    __syncthreads();
    const T b = s_b;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = z[i] + b * p[i];
}

// r^T z (after a V-cycle)
template <typename T>
__global__ void __launch_bounds__(256) k_dot_rz(long long n, const T* __restrict__ r, const T* __restrict__ z, double* red,
                                                unsigned* counter, DevScalars* sc) {
    __shared__ double sh[32 * kRedQ];
    T acc = T(0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += r[i] * z[i];
    T v[1] = {acc};
    const int kind[1] = {0};
    double tot[1];
    block_reduce<T, 1>(v, kind, reinterpret_cast<T*>(sh));
    if (finish_reduction<T, 1>(v, kind, red, counter, tot, sh, linear_block(), grid_blocks()) && threadIdx.x == 0) sc->rz = tot[0];
}

// u += beta z  (Richardson)
template <typename T>
__global__ void k_axpy(long long n, T* __restrict__ u, const T* __restrict__ z, T beta) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        u[i] += beta * z[i];
}

__global__ void k_record(DevScalars* sc, to_stats* st, int cap) {
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
    if (slot >= 0 && slot < cap) st[slot] = s;
    if (sc->host_rec) *(to_stats*)sc->host_rec = s;
    sc->host_rec = nullptr;
    sc->host_out = nullptr;   // the design's copy ran on the design branch, joined before this
    sc->rec = slot + 1;
    sc->k += 1;
    sc->beta_first = 0.0;
    sc->beta = 0.0;
}

__global__ void k_set_beta(DevScalars* sc, double beta) {
    sc->beta = beta;
    if (sc->beta_first == 0.0) sc->beta_first = beta;
}

// the new design into the host buffer that to_step_host left in sc->host_out (a device
// alias of page-locked memory), n words; nothing when none is set
__global__ void k_host_out(const DevScalars* __restrict__ sc, const unsigned* __restrict__ rho, long long n) {
    unsigned* dst = (unsigned*)sc->host_out;
    if (!dst) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = rho[i];
}

int launch_host_out(to_problem* P, cudaStream_t s) {
    const long long nw = (long long)(P->n_elem * P->esz / 4);
    k_host_out<<<grid_1d(nw, 256, P->num_sms), 256, 0, s>>>(P->sc, (const unsigned*)P->rho, nw);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

int launch_record(to_problem* P, cudaStream_t s) {
    k_record<<<1, 1, 0, s>>>(P->sc, P->dstats, P->dstats_cap);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

template <typename T>
static int update_t(to_problem* P, void* u, cudaStream_t s) {
    const int nb = grid_1d(P->n_dof, 256, P->num_sms);
    if (P->prm.precond == TO_PRECOND_JACOBI)
        k_update_sd<T, true><<<nb, 256, 0, s>>>(P->n_dof, (T*)u, (T*)P->r, (T*)P->z, (const T*)P->q,
                                                (const T*)P->lv[0].dinv, P->red, P->counters + 4, P->sc);
    else
        k_update_sd<T, false><<<nb, 256, 0, s>>>(P->n_dof, (T*)u, (T*)P->r, (T*)P->z, (const T*)P->q,
                                                 (const T*)P->lv[0].dinv, P->red, P->counters + 4, P->sc);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

// z = M^-1 r for the non-Jacobi preconditioners, followed by r^T z
template <typename T>
static int precond_t(to_problem* P, cudaStream_t s) {
    const int nb = grid_1d(P->n_dof, 256, P->num_sms);
    if (P->prm.precond == TO_PRECOND_MG) {
        int rc = mg_vcycle(P, P->r, P->z, s);
        if (rc) return rc;
        if (P->prm.mg_nu_post > 0 && P->lv.size() > 1) return TO_OK;   // r^T z fused into the last sweep
    } else if (P->prm.precond == TO_PRECOND_KRYLOV) {
        int rc = krylov_apply(P, P->r, P->z, s);
        if (rc) return rc;
    } else if (P->prm.precond == TO_PRECOND_NONE) {
        TO_CUDA(cudaMemcpyAsync(P->z, P->r, P->n_dof * sizeof(T), cudaMemcpyDeviceToDevice, s));
    } else {
        return TO_OK;  // Jacobi z is produced inside the fused kernels
    }
    k_dot_rz<T><<<nb, 256, 0, s>>>(P->n_dof, (const T*)P->r, (const T*)P->z, P->red, P->counters + 5, P->sc);
    TO_CUDA(cudaGetLastError());
    return TO_OK;
}

int launch_precond(to_problem* P, const void*, void*, cudaStream_t s) {
    return P->prec == TO_FP64 ? precond_t<double>(P, s) : precond_t<float>(P, s);
}

// out = in / d (the Jacobi M^-1 as a separate pass; dinv = 1 / d)
template <typename T>
__global__ void __launch_bounds__(256) k_mul_dinv(long long n, const T* __restrict__ in, const T* __restrict__ dinv,
                                                  T* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = in[i] * dinv[i];
}

// out = M^-1 in for any preconditioner (in and out distinct)
template <typename T>
static int apply_M_t(to_problem* P, const void* in, void* out, cudaStream_t s) {
    const int nb = grid_1d(P->n_dof, 256, P->num_sms);
    switch (P->prm.precond) {
        case TO_PRECOND_MG: return mg_vcycle(P, in, out, s);
        case TO_PRECOND_KRYLOV: return krylov_apply(P, in, out, s);
        case TO_PRECOND_NONE:
            TO_CUDA(cudaMemcpyAsync(out, in, P->n_dof * sizeof(T), cudaMemcpyDeviceToDevice, s));
            return TO_OK;
        default:
            k_mul_dinv<T><<<nb, 256, 0, s>>>(P->n_dof, (const T*)in, (const T*)P->lv[0].dinv, (T*)out);
            TO_CUDA(cudaGetLastError());
            return TO_OK;
    }
}

// Residual at u (with the fused sensitivity when `primary`; already launched by the
// caller when `resid_done`), then nsteps steps.
int run_inner(to_problem* P, void* u, int nsteps, int primary, cudaStream_t s, int resid_done) {
    int rc;
    void* gt_save = P->gt;
    if (!resid_done) {
        if (!primary) P->gt = nullptr;
        rc = launch_operator(P, 0, OP_RESID, u, P->r, P->f, s, 0.0, 1);
        P->gt = gt_save;
        if (rc) return rc;
    }
    if (P->prm.inner_mode == TO_INNER_PCG) {
        // preconditioned conjugate gradients from u: p = z, then per iteration q = K p with
        // alpha = r^T z / p^T q, the update, z = M^-1 r, p = z + beta p
        const int nb = grid_1d(P->n_dof, 256, P->num_sms);
        const bool jac = P->prm.precond == TO_PRECOND_JACOBI;
        if ((rc = launch_precond(P, P->r, P->z, s))) return rc;
        TO_CUDA(cudaMemcpyAsync(P->tmp_v, P->z, P->n_dof * P->esz, cudaMemcpyDeviceToDevice, s));
        for (int it = 0; it < nsteps; ++it) {
            if ((rc = launch_operator(P, 0, OP_Q, P->tmp_v, P->q, nullptr, s, 0.0, it == 0))) return rc;
            if (P->prec == TO_FP64) {
                if (jac) k_cg_update<double, true><<<nb, 256, 0, s>>>(P->n_dof, (double*)u, (double*)P->r, (double*)P->z, (const double*)P->tmp_v, (const double*)P->q, (const double*)P->lv[0].dinv, P->red, P->counters + 4, P->sc);
                else k_cg_update<double, false><<<nb, 256, 0, s>>>(P->n_dof, (double*)u, (double*)P->r, (double*)P->z, (const double*)P->tmp_v, (const double*)P->q, (const double*)P->lv[0].dinv, P->red, P->counters + 4, P->sc);
            } else {
                if (jac) k_cg_update<float, true><<<nb, 256, 0, s>>>(P->n_dof, (float*)u, (float*)P->r, (float*)P->z, (const float*)P->tmp_v, (const float*)P->q, (const float*)P->lv[0].dinv, P->red, P->counters + 4, P->sc);
                else k_cg_update<float, false><<<nb, 256, 0, s>>>(P->n_dof, (float*)u, (float*)P->r, (float*)P->z, (const float*)P->tmp_v, (const float*)P->q, (const float*)P->lv[0].dinv, P->red, P->counters + 4, P->sc);
            }
            TO_CUDA(cudaGetLastError());
            if (it + 1 == nsteps) break;
            if (!jac && (rc = launch_precond(P, P->r, P->z, s))) return rc;
            if (P->prec == TO_FP64) k_cg_dir<double><<<nb, 256, 0, s>>>(P->n_dof, (const double*)P->z, (double*)P->tmp_v, P->sc);
            else k_cg_dir<float><<<nb, 256, 0, s>>>(P->n_dof, (const float*)P->z, (float*)P->tmp_v, P->sc);
            TO_CUDA(cudaGetLastError());
        }
    } else if (P->prm.inner_mode == TO_INNER_PFBTO) {
        // Algorithm 2: u <- u - beta K M^-1 M^-1 (K u - f) = u + beta K M^-1 M^-1 r
        const int nb = grid_1d(P->n_dof, 256, P->num_sms);
        for (int it = 0; it < nsteps; ++it) {
            if (it > 0) {
                P->gt = nullptr;
                rc = launch_operator(P, 0, OP_RESID, u, P->r, P->f, s, 0.0, 0);
                P->gt = gt_save;
                if (rc) return rc;
            }
            if ((rc = P->prec == TO_FP64 ? apply_M_t<double>(P, P->r, P->z, s) : apply_M_t<float>(P, P->r, P->z, s)) ||
                (rc = P->prec == TO_FP64 ? apply_M_t<double>(P, P->z, P->tmp_v, s) : apply_M_t<float>(P, P->z, P->tmp_v, s)) ||
                (rc = launch_operator(P, 0, OP_APPLY, P->tmp_v, P->q, nullptr, s, 0.0, 0)))
                return rc;
            if (P->prec == TO_FP64)
                k_axpy<double><<<nb, 256, 0, s>>>(P->n_dof, (double*)u, (const double*)P->q, P->prm.beta);
            else
                k_axpy<float><<<nb, 256, 0, s>>>(P->n_dof, (float*)u, (const float*)P->q, (float)P->prm.beta);
            TO_CUDA(cudaGetLastError());
        }
    } else if (P->prm.inner_mode == TO_INNER_SD) {
        if ((rc = launch_precond(P, P->r, P->z, s))) return rc;
        for (int it = 0; it < nsteps; ++it) {
            if ((rc = launch_operator(P, 0, OP_Q, P->z, P->q, nullptr, s, 0.0, it == 0))) return rc;
            if ((rc = P->prec == TO_FP64 ? update_t<double>(P, u, s) : update_t<float>(P, u, s))) return rc;
            if (it + 1 < nsteps && (rc = launch_precond(P, P->r, P->z, s))) return rc;
        }
    } else {
        const int nb = grid_1d(P->n_dof, 256, P->num_sms);
        k_set_beta<<<1, 1, 0, s>>>(P->sc, P->prm.beta);
        for (int it = 0; it < nsteps; ++it) {
            if (it > 0) {
                P->gt = nullptr;
                rc = launch_operator(P, 0, OP_RESID, u, P->r, P->f, s, 0.0, 0);
                P->gt = gt_save;
                if (rc) return rc;
            }
            if ((rc = launch_precond(P, P->r, P->z, s))) return rc;
            if (P->prec == TO_FP64)
                k_axpy<double><<<nb, 256, 0, s>>>(P->n_dof, (double*)u, (const double*)P->z, P->prm.beta);
            else
                k_axpy<float><<<nb, 256, 0, s>>>(P->n_dof, (float*)u, (const float*)P->z, (float)P->prm.beta);
            TO_CUDA(cudaGetLastError());
        }
    }
    return TO_OK;
}

int refresh_preconditioner(to_problem* P, cudaStream_t s, bool join, bool inline_inv) {
    int rc = launch_diag(P, 0, s);
    if (rc) return rc;
    if (P->prm.precond == TO_PRECOND_MG) return mg_refresh(P, s, join, inline_inv);
    return TO_OK;
}

int outer_iteration(to_problem* P, cudaStream_t s) {
    int rc;
    if ((rc = launch_moduli(P, s))) return rc;
    // the coarsest inverse overlaps the residual and the fine-level smoothing: its
    // branch is joined by the first coarse solve, and in any case before the iteration ends
    if ((rc = refresh_preconditioner(P, s, false))) return rc;
    // the residual at u_k with the sensitivity at u_k fused
    if ((rc = launch_operator(P, 0, OP_RESID, P->u, P->r, P->f, s, 0.0, 1))) return rc;
    // The design update (filter transpose, gradient step, projection) reads rho_k and the
    // sensitivity at u_k only, and the lower-level steps read K(rho_k) only: the update
    // runs on a branch beside the steps (its reductions have their own scratch and
    // counters; the two write disjoint device scalars) and is joined before the record.
    TO_CUDA(cudaEventRecord(P->ev_dfork, s));
    TO_CUDA(cudaStreamWaitEvent(P->dside, P->ev_dfork, 0));
    if ((rc = launch_sens_filter_T(P, P->dside))) return rc;
    if ((rc = launch_project(P, nullptr, P->rho, P->grad, P->rho, 1, P->dside))) return rc;
    if ((rc = launch_host_out(P, P->dside))) return rc;
    TO_CUDA(cudaEventRecord(P->ev_djoin, P->dside));
    if ((rc = run_inner(P, P->u, P->prm.n_inner, 1, s, 1))) return rc;
    if (P->prm.precond == TO_PRECOND_MG) TO_CUDA(cudaStreamWaitEvent(s, P->ev_join, 0));
    P->coarse_wait = 0;
    TO_CUDA(cudaStreamWaitEvent(s, P->ev_djoin, 0));
    return launch_record(P, s);
}

// ----------------------------------------------------------------------------- gated refresh
// After to_set_state the live set is rebuilt only if the design it brought differs from
// the one the set was built for: sc->dchanged == sc->dseq, written on the device by
// to_set_state's copy (which has also recomputed rho~ and the moduli where the design
// differs).  Every rebuild kernel reads that pair and returns at once unless they are
// equal, so an unchanged design costs one near-empty launch each; level 0's 1 / d is the
// only one on the main stream, the coarse
// levels (moduli, 1 / d, the coarsest operator) and the coarsest inverse run on the
// multigrid branch beside the residual.  The V-cycle's first restriction to level 1 waits
// for the levels (ev_ljoin), the coarse solves for the inverse (ev_join).  (Conditional
// graph nodes measured slower: each costs several microseconds even when its body does
// not run, and the graph around them slowed down too.)
static int gated_refresh(to_problem* P, cudaStream_t s) {
    const unsigned* changed = &P->sc->dchanged;
    if (P->prm.precond != TO_PRECOND_MG) return launch_diag(P, 0, s, changed);
    TO_CUDA(cudaEventRecord(P->ev_fork, s));
    TO_CUDA(cudaStreamWaitEvent(P->side, P->ev_fork, 0));
    int rc = launch_diag(P, 0, s, changed);
    if (!rc) rc = mg_refresh_levels(P, P->side, changed);
    if (rc) return rc;
    TO_CUDA(cudaEventRecord(P->ev_ljoin, P->side));
    if ((rc = mg_refresh_inverse(P, P->side, changed))) return rc;
    TO_CUDA(cudaEventRecord(P->ev_join, P->side));
    P->levels_wait = 1;   // the V-cycle's first restriction joins the levels
    P->coarse_wait = 1;   // the coarse solves join the inverse
    return TO_OK;
}

// The same iteration with the next design's preconditioner built beside it.  The live
// set (moduli, diagonals, coarsest inverse) belongs to rho_k on entry (fresh = 0), or is
// computed first as in outer_iteration, its inverse on the multigrid branch (fresh = 1),
// or where to_set_state found rho_k changed (fresh = 2, gated_refresh).  After the
// residual at u_k the design branch forms rho_{k+1} (filter transpose, step,
// projection), then its moduli, diagonals, coarse moduli and coarsest inverse, all
// into the other set, while the lower-level steps run on the live set; the caller
// swaps the sets afterwards.  Every kernel sees the same inputs as in
// outer_iteration, so the iterates are the same.
int outer_iteration_pipelined(to_problem* P, cudaStream_t s, int fresh) {
    int rc;
    const bool mg = P->prm.precond == TO_PRECOND_MG;
    if (fresh == 2) {
        if ((rc = gated_refresh(P, s))) return rc;
    } else if (fresh && ((rc = launch_moduli(P, s)) || (rc = refresh_preconditioner(P, s, false, false)))) {
        return rc;
    }
    if ((rc = launch_operator(P, 0, OP_RESID, P->u, P->r, P->f, s, 0.0, 1))) return rc;
    TO_CUDA(cudaEventRecord(P->ev_dfork, s));
    TO_CUDA(cudaStreamWaitEvent(P->dside, P->ev_dfork, 0));
    if ((rc = launch_sens_filter_T(P, P->dside))) return rc;
    if ((rc = launch_project(P, nullptr, P->rho, P->grad, P->rho, 1, P->dside))) return rc;
    if ((rc = launch_host_out(P, P->dside))) return rc;   // (to_step_host: the design out, beside the steps)
    // the live inverse (fresh: still on the multigrid branch) shares the assembled
    // operator and the inversion scratch with the next one
    if (fresh && mg) TO_CUDA(cudaStreamWaitEvent(P->dside, P->ev_join, 0));
    pipe_swap(P);   // enqueue the next design's refresh into the other set
    rc = launch_moduli(P, P->dside);
    if (!rc) rc = refresh_preconditioner(P, P->dside, false, true);
    pipe_swap(P);
    if (rc) return rc;
    TO_CUDA(cudaEventRecord(P->ev_djoin, P->dside));
    P->coarse_wait = fresh ? 1 : 0;   // else the live inverse was completed before this iteration
    rc = run_inner(P, P->u, P->prm.n_inner, 1, s, 1);
    P->coarse_wait = 0;               // joined below (fresh: through the design branch)
    P->levels_wait = 0;
    if (rc) return rc;
    TO_CUDA(cudaStreamWaitEvent(s, P->ev_djoin, 0));
    return launch_record(P, s);
}

}  // namespace to
