// Internal definitions of the GB300 first-order bilevel topology optimiser.
// Public ABI: include/to.h.  Nothing here is exported.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <string>
#include <vector>

#include "../../include/to.h"

namespace to {

// ----------------------------------------------------------------------------- errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
#define TO_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return ::to::fail(TO_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// ----------------------------------------------------------------------------- device scalars
// Device-resident scalars of the outer loop; read by kernels, never copied to
// the host except through to_stats / to_get_state / to_check.
// State of the projection's multiplier search (device.cuh: proj_search_step)
struct ProjSearch {
    double lam, lo_b, hi_b;
    double pU, pL, pF;   // sets that produced lam (when have_prev)
    bool have_prev, done;
};

struct DevScalars {
    double rz, zq, beta, beta_first;   // lower-level step sizes (Algorithm 1 / 3, line 1)
    double rz_old;                     // conjugate gradients: r^T z of the previous iteration
    double J, res_inf, res2;           // f^T u_k, residual norms at u_k
    double gmax, gsum;                 // ||g||_inf and 1^T g of dJ/drho
    double alpha0, alpha;              // high-level step size alpha_k = alpha0 k^-m
    double lambda, drho_inf, volume;   // projection results
    long long k;                       // 1-based outer iteration counter
    int err;                           // first device-side error (TO_ERR_*), 0 if none
    int proj_iters;
    int n_inner_done;
    int rec;                           // next stats slot written by the record kernel
    ProjSearch ps;                     // the projection's search, carried between its kernels
    int proj_active;                   // the volume bound is active at this projection (lambda > 0)
    // to_set_state's comparison of the incoming design with the live set's: call number dseq
    // found a difference iff dchanged == dseq (gates: a kernel given &dchanged returns at once
    // when gate[0] != gate[1])
    unsigned dchanged, dseq;
    // to_step_host: device aliases of page-locked host buffers that the next iteration
    // writes its new design into (after the projection) and its record into (with the
    // record); cleared by the record kernel (nullptr: none)
    void* host_out;
    void* host_rec;
};
static_assert(offsetof(DevScalars, dseq) == offsetof(DevScalars, dchanged) + sizeof(unsigned),
              "a gate reads dchanged and dseq as one pair");

// Reduction scratch: one slot of up to kRedQ doubles per block, plus a
// completion counter; the last block to finish sums the slots in block order
// (deterministic) and writes the totals.
constexpr int kRedQ = 4;
constexpr int kMaxRedBlocks = 8192;

// ----------------------------------------------------------------------------- operator constants
// The unit-modulus hex8 element matrix in the sum/difference (Haar) basis of
// its 2x2x2 nodes has 45 non-zeros in fixed positions; kHaarRow/kHaarCol list
// them (coefficient DOF = 3 * (4 zeta + 2 eta + xi) + component, zeta / eta / xi
// = 0 for a sum and 1 for a difference along z / y / x).
constexpr int kHaarNnz = 45;
extern const int kHaarRow[kHaarNnz];
extern const int kHaarCol[kHaarNnz];

template <typename T>
struct HaarK {
    T v[kHaarNnz];  // values for element edge h (K_e scales with h in 3-D)
};

// 24x24 unit-modulus, unit-size hex8 stiffness (row-major), built by exact
// integration of the Lame bilinear form; its Haar-basis non-zeros; validation.
int build_element_matrix(double nu, double ke[24 * 24]);
int build_haar(const double ke[24 * 24], double h, double out[kHaarNnz]);

// ----------------------------------------------------------------------------- problem
struct Level {
    int nx, ny, nz;
    int64_t n_elem, n_node, n_dof;
    double h;
    void* E = nullptr;        // element moduli (T)
    void* dinv = nullptr;     // 1 / diag(K^) (T): the Jacobi scaling, applied by multiplication
    uint8_t* mask = nullptr;  // per node: bit c set = DOF c fixed
    uint8_t* tmask = nullptr; // per operator tile column: any fixed node in its footprint
    uint8_t* tmask64 = nullptr; // the same for the 64 x kTmaTileY tiles of the TMA operator
    void* tcb = nullptr;      // element matrix of edge h as split BF16 pieces (tensor-core operator)
    void* x = nullptr;        // V-cycle vectors (T)
    void* b = nullptr;
    void* t = nullptr;
    double kdiag = 0.0;       // k_e[ll] (all equal on a cube)
    int kchunk = 0;           // node planes per operator tile picked by the autotuner (0: cost model)
};

struct to_problem_impl;

}  // namespace to

struct to_problem {
    int device = 0;
    int prec = TO_FP32_MIXED;
    to_grid g{};
    to_material mat{};
    to_params prm{};
    int64_t n_elem = 0, n_node = 0, n_dof = 0;
    size_t esz = 4;                // bytes per vector entry
    double ke[24 * 24];            // unit element matrix (host, double)
    double haar[to::kHaarNnz];     // Haar non-zeros for edge h
    double kdiag = 0.0;            // k_e[ll] for edge h

    // design and filter
    void* rho = nullptr;
    void* rhot = nullptr;
    void* Ed = nullptr;            // dE/drho~
    void* Hs = nullptr;            // filter row sums
    void* gt = nullptr;            // dJ/drho~
    void* grad = nullptr;          // dJ/drho
    void* tmp_e = nullptr;         // element scratch
    int n_stencil = 0;
    int filter_ext = 0;            // largest |dx|, |dy|, |dz| of the stencil
    int4* stencil = nullptr;       // (dx, dy, dz, -) offsets
    void* stencil_w = nullptr;     // weights (T)

    // solver vectors (n_dof each)
    void* u = nullptr;
    void* f = nullptr;
    void* r = nullptr;
    void* z = nullptr;
    void* q = nullptr;
    void* tmp_v = nullptr;

    // multigrid hierarchy (level 0 aliases E, d, mask of the fine grid)
    std::vector<to::Level> lv;
    void* coarse_A = nullptr;      // dense coarsest operator (T), n_c x n_c
    void* coarse_L = nullptr;      // scaled inverse (T), n_c x n_c, then the n_c scale factors
    int n_coarse = 0;
    void* gj_work = nullptr;       // blocked coarsest inversion (n_coarse > 160): work matrix, block column, pivot
    void* gj_tab = nullptr;        // its one-entry argument table
    int mg_tail = 0;               // first level of the one-CTA coarse tail (0: none)
    void* legs_prog = nullptr;     // the V-cycle's persistent legs over levels 1 .. tail - 1 (device steps)
    int legs_n[2] = {0, 0};        // steps of the down and up legs
    int legs_grid = 0;             // co-resident CTAs of their cooperative launches (0: not used)
    int precond_stale = 0;         // the design changed outside to_step: refresh before the next lower-level solve

    // Krylov preconditioner (Eq. LSP): basis of D + 2 columns (leading dimension kry_ld),
    // device coefficients, per-block partials of its streaming passes
    void* kry_q = nullptr;
    void* kry_s = nullptr;
    double* kry_part = nullptr;
    long long kry_ld = 0;
    int kry_blocks = 0;
    double* ke_dev = nullptr;      // 24x24 unit element matrix (device, double)

    // device scalars, reductions, stats
    to::DevScalars* sc = nullptr;
    double* red = nullptr;         // kMaxRedBlocks * kRedQ doubles
    double* red_d = nullptr;       // the same for the design update (filter^T statistics, projection),
                                   // which runs beside the lower-level steps
    // completion counters / barrier words (64): [0] residual, [1] z^T q, [2] filter^T statistics,
    // [4] update, [5] r^T z, [6] smoother r^T z, [7] f^T u, [8..9] grid barrier,
    // [10..11] projection first / final pass, [12] Krylov passes
    unsigned* counters = nullptr;
    to_stats* dstats = nullptr;    // device stats ring
    int dstats_cap = 0;
    void* rho_stage = nullptr;     // to_step_host: the design copied in from the host
    to_stats* stats_pinned = nullptr;   // to_step_host without stats_out: the record read back
    int last_step_n = 0;           // outer iterations of the last to_step call (its records: slots 0 .. n - 1)

    // truncated-solve iterates u_0 .. u_T kept for the reverse sweep
    void* iters = nullptr;
    int iters_cap = 0;
    int iters_T = -1;
    double iters_beta = 0.0;
    int iters_stride = 1;          // every iters_stride-th iterate kept (1: all)
    int64_t fwd_id = 0;            // id of the kept iterates; 0: none, or the design changed since
    int64_t fwd_count = 0;

    // can one 16-CTA cluster run the projection's search passes
    int cluster16 = 0;
    // scratch of the sort-based multiplier (proj_sort)
    void* ps_buf = nullptr;

    // captured outer iteration (replayed by to_step) on a library-owned stream
    cudaStream_t gstream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_state = 0;           // 0: not captured yet, 1: ready, -1: capture unavailable
    cudaStream_t side = nullptr;   // branch for the coarsest inverse (overlaps the fine-level work)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaStream_t dside = nullptr;  // branch for the design update (overlaps the lower-level steps)
    cudaEvent_t ev_dfork = nullptr, ev_djoin = nullptr;
    // Pipelined outer iterations: the next iteration's design-dependent data (rho~, E', every
    // level's moduli and 1 / d, the coarsest inverse with its inversion table) are built on
    // the design branch into a second set of buffers, swapped with the live set after the
    // iteration; set_parity says which physical set is live (one captured graph per set).
    void* alt_rhot = nullptr;
    void* alt_Ed = nullptr;
    std::vector<void*> alt_E, alt_dinv;
    void* alt_coarse_L = nullptr;
    void* alt_gj_tab = nullptr;
    int alt_alloc = 0;
    int set_parity = 0;
    // [set][variant]: 0 the live set is current, 1 it is rebuilt first, 2 it is rebuilt by
    // kernels that do nothing unless dchanged says to_set_state brought a different design
    cudaGraphExec_t gexec_pipe[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    int pipe_state[2][3] = {{0, 0, 0}, {0, 0, 0}};   // as graph_state, per set and variant
    int pipe_ready = 0;            // the live set belongs to the current rho (a pipelined to_step left it)
    int design_check = 0;          // to_set_state compared its design with the live set's (variant 2 may run)
    unsigned dseq_host = 0;        // number of those comparisons
    int levels_wait = 0;           // variant 2: the coarse levels are rebuilt on the branch; the first
    cudaEvent_t ev_ljoin = nullptr;   // restriction to level 1 waits for ev_ljoin
    int in_batch = 0;              // a batch's tables hold this problem's buffers: no swapping
    int coarse_wait = 0;           // a forked coarsest inverse may still run: coarse solves wait for ev_join

    // launch configuration of the operator kernel; resident CTAs per SM of each mode
    int tile_x = 32, tile_y = 8, tile_z = 8;
    int op_occ[5] = {0, 0, 0, 0, 0};
    int tma_occ[5] = {0, 0, 0, 0, 0};  // the FP32 TMA operator: resident CTAs per SM of each mode
    int tma_ready = 0;                 // its shared-memory opt-ins are set
    int mgc_ok = 0;                    // the 16-CTA cluster of the level above the coarse tail can be resident
    int tc_occ[5] = {0, 0, 0, 0, 0};   // the tensor-core FP32 operator: resident CTAs per SM of each mode
    int tc_ready = 0;                  // its shared-memory opt-ins are set and tensor memory suffices
    int num_sms = 0;
    int coop_blocks = 0;           // co-resident blocks for the projection kernel
};

namespace to {

// kernels/launchers (templated on the vector type T = float | double)
template <typename T> struct Launch;

int launch_filter(to_problem* P, const void* x, void* y, int transpose, cudaStream_t s);
// rho -> rho~, E, E'; with gate (&sc->dchanged), only where the design changed (read on the device)
int launch_moduli(to_problem* P, cudaStream_t s, const unsigned* gate = nullptr);
int launch_diag(to_problem* P, int level, cudaStream_t s, const unsigned* gate = nullptr);   // gate: as launch_moduli

enum OpMode { OP_APPLY = 0, OP_RESID = 1, OP_Q = 2, OP_SMOOTH = 3, OP_BMINUS = 4 };
// OP_RESID outputs named by the caller instead of the problem's buffers (nullptr skips one)
struct OpOut {
    void* z;    // r / d
    void* gt;   // -E'_e u_e^T k_e u_e / Hs_e
};
// y = K^ x (+ mode epilogue) on multigrid level `level` (0 = fine grid).
int launch_operator(to_problem* P, int level, int mode, const void* x, void* y,
                    const void* b, cudaStream_t s, double omega = 0.0, int first = 0,
                    const OpOut* out = nullptr);

int launch_project(to_problem* P, const void* w, const void* rho_in, const void* g,
                   void* rho_out, int fused, cudaStream_t s);
int launch_update_sd(to_problem* P, cudaStream_t s);
int launch_precond(to_problem* P, const void* r, void* z, cudaStream_t s);
int launch_sens_filter_T(to_problem* P, cudaStream_t s);
int launch_energy(to_problem* P, const void* u, cudaStream_t s);
int launch_record(to_problem* P, cudaStream_t s);
int launch_host_out(to_problem* P, cudaStream_t s);   // rho into sc->host_out, if set
int operator_init(to_problem* P);
int build_tile_mask(Level& L, const uint8_t* mask_host);
// the FP32 operator with TMA staging (optma.cu): node rows per tile, set-up, applicability
constexpr int kTmaTileY = 8;
int operator_tma_init(to_problem* P);
bool operator_tma_applicable(const to_problem* P, int level, const void* x, const void* y, const void* b);
int launch_operator_tma(to_problem* P, int level, int mode, const void* x, void* y, const void* b, cudaStream_t s,
                        double omega, int first, const OpOut* out);
int build_tile_mask64(Level& L, const uint8_t* mask_host);
// the FP32 operator with the element contraction on the tensor cores (optc.cu)
int operator_tc_init(to_problem* P);
int operator_tc_build(to_problem* P);
bool operator_tc_applicable(const to_problem* P, int level);
int launch_operator_tc(to_problem* P, int level, int mode, const void* x, void* y, const void* b, cudaStream_t s,
                       double omega, int first, const OpOut* out);
int project_cluster_setup(to_problem* P);
int krylov_build(to_problem* P);
int operator_autotune(to_problem* P, cudaStream_t s);
int projsort_lambda(to_problem* P, const void* w, cudaStream_t s);
size_t projsort_bytes(const to_problem* P);
int krylov_apply(to_problem* P, const void* b, void* x, cudaStream_t s);
int launch_richardson(to_problem* P, cudaStream_t s);

// multigrid
int mg_build(to_problem* P);
// coarse moduli, diagonals, the coarsest inverse (on a forked branch of s; join: s waits for it
// at once, else the first coarse solve on s does)
int mg_refresh(to_problem* P, cudaStream_t s, bool join = true, bool inline_inv = false);
// coarse moduli, 1 / d and the coarsest operator; its inverse (gate: as launch_moduli)
int mg_refresh_levels(to_problem* P, cudaStream_t s, const unsigned* gate = nullptr);
int mg_refresh_inverse(to_problem* P, cudaStream_t s, const unsigned* gate = nullptr);
bool mg_refresh_gatable(const to_problem* P);   // the inverse takes a gate (one-CTA register form)
// the diagonal and (multigrid) the refresh above; inline_inv: the coarsest inverse on s itself
int refresh_preconditioner(to_problem* P, cudaStream_t s, bool join = true, bool inline_inv = false);
// the second set of design-dependent buffers (allocated once) and the swap of the two sets
int pipe_alloc(to_problem* P);
void pipe_swap(to_problem* P);
int mg_vcycle(to_problem* P, const void* r, void* z, cudaStream_t s);
int mg_legs_build(to_problem* P);
// the level just above the coarse tail in one 16-CTA cluster (mgcl.cu)
int mg_cluster_init(to_problem* P);
bool mg_cluster_applicable(const to_problem* P, int l);
int mg_cluster_down(const to_problem* P, int l, void* x_first, void* x_iter, void* cfirst, cudaStream_t s);
int mg_cluster_up(const to_problem* P, int l, void* x_iter, void* x_out, cudaStream_t s);
int mg_legs_launch(to_problem* P, int leg, void* fine, cudaStream_t s);

int outer_iteration(to_problem* P, cudaStream_t s);
// one outer iteration that also builds the next design's set; the live set must match rho,
// or `fresh`: the iteration first computes the live set itself
int outer_iteration_pipelined(to_problem* P, cudaStream_t s, int fresh);   // fresh: variant 0, 1 or 2
int inner_steps(to_problem* P, int nsteps, int from_resid, cudaStream_t s);

// batched multigrid (mg.cu): the V-cycle and the per-iteration refresh of many problems
struct BatchMG;
int batch_mg_build(to_problem* const* probs, int n, int kchunk, BatchMG** out);
int batch_mg_refresh(const BatchMG* M, cudaStream_t s);
int batch_mg_vcycle(const BatchMG* M, cudaStream_t s);
int batch_mg_join(const BatchMG* M, cudaStream_t s);
int batch_mg_refresh_inline(const BatchMG* M, cudaStream_t s);
int batch_mg_wait(const BatchMG* M, cudaStream_t s);
int batch_mg_launches(const BatchMG* M, int* refresh, int* vcycle);
void batch_mg_free(BatchMG* M);

}  // namespace to
