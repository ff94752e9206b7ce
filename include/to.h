/*
 * to.h -- C ABI of the GB300 first-order bilevel topology optimiser.
 *
 * Method: arXiv 2204.06204, "First-Order Bilevel Topology Optimization for
 * Fast Mechanical Design".  One outer iteration (Algorithms 1 and 3) refines
 * the lower-level solution of K(v) u = f by a few (preconditioned) descent
 * steps instead of an exact solve, takes the approximate sensitivity
 * -1/2 u^T dK/dv u at the current u (Sec. III, exact-gradient formula, used
 * with the approximate u), chains it through the material filter
 * (Remark 3.1) and projects the gradient step onto
 * X = {lo <= v <= hi, 1^T v <= vbar} (Sec. IV-B, Eq. piecewiseLinearEQ,
 * Algorithm 4).  Here the design v is written rho, the discretisation is
 * hex8 on an nx x ny x nz voxel grid, the stiffness parameterisation is the
 * power law of Sec. III in its modified form E_e = Emin + rho~_e^p (E0-Emin),
 * and the compliance reported is J = f^T u (= 2 l of Eq. (opt)).
 *
 * Conventions (all entry points)
 *   node  n = i + (nx+1) * (j + (ny+1) * k)        0 <= i <= nx, ...
 *   DOF   d = 3 n + c, c = 0 (x), 1 (y), 2 (z)     n_dof  = 3 (nx+1)(ny+1)(nz+1)
 *   element e = i + nx * (j + ny * k)             n_elem = nx ny nz
 *   Fixed DOFs are eliminated: K^ = m K m + (I - m), m the free-DOF indicator,
 *   so K^ is the identity on fixed rows and columns.
 *
 * Precision is fixed per problem by to_params.precision:
 *   TO_FP64        every vector, scalar and product in double  -> pointers are double*
 *   TO_FP32_MIXED  vectors, products and element work in float; global dot
 *                  products, norms, step sizes and the volume multiplier in
 *                  double                                     -> pointers are float*
 *
 * Memory and streams
 *   Pointers named *_dev are device pointers on the problem's device, borrowed
 *   for the call only (never freed, never kept).  Pointers named *_host or
 *   plain scalar out-pointers are host memory.  The library owns its internal
 *   buffers (design, filtered design, moduli, solver vectors, multigrid
 *   levels, reduction scratch) and frees them in to_destroy.  `stream` is a
 *   cudaStream_t (NULL = legacy default stream); every call is stream-ordered
 *   on it.  A call that returns a host value synchronises that stream.
 *
 * Errors
 *   Every int-returning call returns TO_OK (0) or a TO_ERR_* code and never
 *   throws or aborts.  to_last_error() returns a per-thread message for the
 *   last failure.  Device-side checks (non-finite step sizes, a grid barrier
 *   that waits too long) set a device flag that is reported by the next call
 *   that synchronises (to_step with stats, to_check, the *_out variants).
 */
#ifndef TO_H
#define TO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    TO_OK = 0,
    TO_ERR_ARG = 1,          /* invalid argument (null pointer, size, enum value)   */
    TO_ERR_CUDA = 2,         /* a CUDA runtime call failed                          */
    TO_ERR_NONFINITE = 3,    /* NaN / Inf met in a step size or reduction            */
    TO_ERR_INFEASIBLE = 4,   /* vbar < n_elem * lo: X is empty                       */
    TO_ERR_TIMEOUT = 5,      /* a device-side wait hit its iteration limit           */
    TO_ERR_SINGULAR = 6,     /* no fixed DOF (K singular) or a failed coarse factor  */
    TO_ERR_STATE = 7         /* call not valid in the current state                  */
};

enum { TO_FP64 = 0, TO_FP32_MIXED = 1 };
enum { TO_PRECOND_JACOBI = 0, TO_PRECOND_MG = 1, TO_PRECOND_NONE = 2, TO_PRECOND_KRYLOV = 3 };
enum { TO_INNER_SD = 0, TO_INNER_RICHARDSON = 1, TO_INNER_PFBTO = 2, TO_INNER_PCG = 3 };

typedef struct to_problem to_problem;      /* opaque */
typedef struct to_batch to_batch;          /* opaque: many problems advanced together */

/* Voxel grid: element counts and edge length h (> 0). */
typedef struct {
    int32_t nx, ny, nz;
    double h;
} to_grid;

/* Material and design bounds (Sec. III power law; X of Eq. (opt)).
 * E0 > Emin >= 0, 0 <= nu < 0.5, p >= 1, 0 < volfrac, rmin >= 0 (filter
 * radius in voxels; < 1 means no filtering), 0 <= rho_min < rho_max.
 * vbar = volfrac * n_elem. */
typedef struct {
    double E0, Emin, nu, p;
    double volfrac, rmin, rho_min, rho_max;
} to_material;

/* Load vector f: n entries (global DOF, value), host arrays read during
 * to_create only.  Repeated DOFs add; loads on fixed DOFs are dropped. */
typedef struct {
    int64_t n;
    const int64_t* dof;
    const double* val;
} to_loads;

/* Fixed DOFs (u = 0), host array read during to_create only. */
typedef struct {
    int64_t n;
    const int64_t* dof;
} to_bcs;

/* Solver parameters.
 *   precision   TO_FP64 | TO_FP32_MIXED
 *   precond     M of the lower-level step: Jacobi diagonal, multigrid V-cycle, none,
 *               or the Krylov preconditioner of Eq. (LSP) (Sec. IV-C): M^-1 b is the
 *               vector of span{b, K b, ..., K^D b} whose K-image is closest to b;
 *               with inner_mode TO_INNER_RICHARDSON and beta = 1 this is
 *               Algorithm CPFBTO
 *   inner_mode  TO_INNER_SD: steepest descent with the exact line search
 *               beta = r^T z / z^T K z; TO_INNER_RICHARDSON: constant beta
 *               (the literal step of Algorithms 1 / 3); TO_INNER_PFBTO: the step of
 *               Algorithm 2, u <- u - beta K M^-1 M^-1 (K u - f) (two applications
 *               of M and one of K per step); TO_INNER_PCG: n_inner iterations of
 *               preconditioned conjugate gradients from u (the near-exact solve of
 *               the nested method, PGD, Sec. V)
 *   n_inner     lower-level steps per outer iteration (>= 0)
 *   beta        step of TO_INNER_RICHARDSON and TO_INNER_PFBTO
 *   alpha0      > 0: alpha_k = alpha0 k^-m.  <= 0: alpha0 = alpha_scale / ||g||_inf
 *               fixed at the first iteration with g != 0
 *   m           exponent of the alpha schedule (Sec. V uses 3/4)
 *   mean_proj   1: g <- g - mean(g) before the step (Sec. IV-B)
 *   mg_levels   0 = automatic; mg_nu_pre / mg_nu_post smoothing sweeps;
 *               mg_omega damped-Jacobi weight
 *   tile_x, tile_y, tile_z   node planes per operator tile (tile_z): > 0 fixed; 0: picked
 *               per multigrid level by an autotuner at to_create (the sweep is timed for
 *               every distinct split of the level's planes into chunks of up to 64 and
 *               the cost model's choice); < 0 (the default): the cost
 *               model alone (waves of resident CTAs x planes walked).  In a batch
 *               (to_batch_create) the first problem's tile_z > 0 fixes the batched
 *               launches' planes per tile; otherwise the batch autotunes it.  tile_x /
 *               tile_y are reserved (the tile is 32 x 8 threads)
 *   no_graph    0: to_step replays one captured CUDA graph per outer iteration;
 *               1: to_step launches the kernels one by one
 *   krylov_dim  D of Eq. (LSP), 0 <= D <= 30 (the paper uses 20); it costs D + 1
 *               operator applications and (D + 2) vectors of n_dof per application
 *   proj_sort   0: the projection's multiplier by the safeguarded Newton search;
 *               1: by the paper's parallel form of Algorithm 4 (a radix sort of the
 *               2E breakpoints and scans, Sec. IV-D); the same rho
 *   adj_stride  iterates of to_compliance_truncated kept for its reverse sweep:
 *               0 or 1: all of u_0 .. u_T ((T + 1) n_dof entries);  s > 1: every s-th
 *               (u_0, u_s, u_2s, ...) plus one segment of s + 1, the reverse sweep
 *               recomputing each segment from its kept iterate (one more forward
 *               pass; (ceil(T / s) + s + 1) n_dof entries);  -1: s = ceil(sqrt(T)).
 *               The gradient is bitwise the same in every mode.
 *   op_kernel   0 (default): the operator K^ x runs the general kernel (cp.async
 *               staging, 31 x 7 node tiles, one element column per thread);
 *               1: FP32 problems run the TMA-staged kernel (64 x 8 node tiles, element
 *               pairs in packed FP32x2, persistent CTAs) wherever its vectors are
 *               16-byte aligned, its copy coordinates fit 32 bits and the grid spans
 *               its copy boxes, else the general kernel;  2: FP32 problems run the
 *               tensor-core kernel (the element contraction as tcgen05.mma on split-BF16
 *               operands with FP32 accumulation in tensor memory, 31 x 7 node tiles;
 *               about 2^-17 per product term instead of FP32's 2^-24: within the 1e-5
 *               operator tolerance, not within the multigrid trajectory's) where the GPU
 *               holds its shared and tensor memory, else the general kernel.  FP64
 *               problems and batches always use the general kernel.  All give the same
 *               K^ x up to rounding
 *   mg_legs     0 (default): the multigrid levels between the fine grid and the one-CTA
 *               coarse tail run one launch per step; 1: as two cooperative launches per
 *               V-cycle (the down leg's smoothing, residuals and restrictions, the up leg's
 *               prolongations and smoothing), separated inside by bounded grid barriers
 *               (general operator kernel only).  The same steps, buffers and order: bitwise
 *               the same results
 *   mg_cluster  0 (default): every multigrid level above the one-CTA coarse tail runs one
 *               launch per step;  1: FP32 problems run the level just above the tail in
 *               one 16-CTA thread-block cluster (two launches per V-cycle around the tail,
 *               the level's vectors in shared memory, sweeps separated by cluster barriers)
 *               where that level has at most 16 element layers and 512 elements per layer
 *               and the GPU can hold the cluster.  The same V-cycle up to the order of sums;
 *               measured at the speed of the launched steps on the 128x64x64 cantilever */
typedef struct {
    int32_t precision, precond, inner_mode, n_inner;
    double beta, alpha0, alpha_scale, m;
    int32_t mean_proj, mg_levels, mg_nu_pre, mg_nu_post;
    double mg_omega;
    int32_t tile_x, tile_y, tile_z, no_graph;
    int32_t krylov_dim, proj_sort;
    int32_t adj_stride, op_kernel;
    int32_t mg_legs, mg_cluster;
} to_params;

/* Per-outer-iteration record (host copy). */
typedef struct {
    int64_t k;          /* outer iteration index, 1-based                           */
    double J;           /* f^T u_k (compliance estimate at the iterate entering k)  */
    double res_inf;     /* ||K(rho~_k) u_k - f||_inf  (tracking error, Sec. V)      */
    double res2;        /* ||K(rho~_k) u_k - f||_2                                   */
    double drho_inf;    /* ||rho_{k+1} - rho_k||_inf (Sec. V termination quantity)   */
    double volume;      /* 1^T rho_{k+1}                                             */
    double lambda;      /* volume multiplier of the projection (0 if inactive)       */
    double alpha;       /* alpha_k                                                   */
    double gmax;        /* ||dJ/drho||_inf                                            */
    double beta_first;  /* first and last lower-level step sizes of this iteration   */
    double beta_last;
    int32_t proj_iters; /* passes of the multiplier search                           */
    int32_t status;     /* TO_OK or the first device-side error of this iteration    */
} to_stats;

/* Fill *out with defaults: FP32-mixed, Jacobi, steepest descent, 5 inner
 * steps, beta 0.5, alpha0 automatic with scale 0.2, m = 0.75, no mean
 * projection, automatic multigrid with 2 + 2 sweeps and omega 0.5. */
void to_default_params(to_params* out);

/* Create a problem on CUDA device `device` (the caller's current device is
 * restored).  Copies loads and fixtures, builds the element matrix, the filter
 * weights and (for TO_PRECOND_MG) the multigrid hierarchy, sets
 * rho = volfrac everywhere, u = 0, k = 1.  Errors: TO_ERR_ARG, TO_ERR_CUDA,
 * TO_ERR_INFEASIBLE, TO_ERR_SINGULAR (no fixed DOF).  *out is NULL on error. */
int to_create(const to_grid* grid, const to_material* mat, const to_loads* loads,
              const to_bcs* bcs, const to_params* params, int device, to_problem** out);

/* Free everything the problem owns.  NULL is ignored. */
void to_destroy(to_problem* P);

/* Sizes of the problem's vectors. */
int to_sizes(const to_problem* P, int64_t* n_elem, int64_t* n_dof);

/* Set the design rho (n_elem entries) and recompute rho~ = C(rho), E and dE/drho~
 * (Sec. III power law through the filter of Remark 3.1).  The operator of
 * to_apply_K, to_inner_solve and to_sensitivity uses this design; the next
 * to_inner_solve first refreshes the preconditioner for it (to_step refreshes
 * it every outer iteration). */
int to_set_design(to_problem* P, const void* rho_dev, void* stream);

/* y = K^(rho~) u, the matrix-free hex8 operator of Sec. III (K = sum_e E_e K_e with
 * fixtures eliminated).  u, y: n_dof entries, node-major xyz-interleaved;
 * u and y must not overlap. */
int to_apply_K(to_problem* P, const void* u_dev, void* y_dev, void* stream);

/* The residual at u and what the first step of an outer iteration takes from it
 * (Algorithms 1 / 3: line 2 evaluates the sensitivity at u_k; line 1's descent
 * step starts from r = f - K u_k), all in one pass of the operator:
 *   r_dev   (n_dof, required)  r = f - K^(rho~) u
 *   z_dev   (n_dof, may be NULL) z = r / diag(K^), the Jacobi-preconditioned residual
 *           ("damped Jacobi", Sec. IV-A)
 *   gt_dev  (n_elem, may be NULL) -E'_e u_e^T k_e u_e / Hs_e: the element sensitivity
 *           with respect to rho~ (Sec. III, exact-gradient formula at u, J = f^T u)
 *           divided by the filter row sum Hs_e = sum_i max(0, rmin - |c_e - c_i|), the
 *           form the filter transpose consumes (to_sensitivity returns the chained
 *           dJ/drho)
 *   scalars_out (host, 4 doubles, may be NULL; synchronises) r^T z (0 without z),
 *           ||r||_2, ||r||_inf, f^T u, reduced in double.
 * u must not overlap r or z.  The Jacobi diagonal of the current design is
 * refreshed first if the design changed since the last lower-level solve. */
int to_residual(to_problem* P, const void* u_dev, void* r_dev, void* z_dev, void* gt_dev,
                double* scalars_out, void* stream);

/* One damped-Jacobi sweep y = x + omega diag(K^)^-1 (b - K^ x) on the fine grid: the
 * smoother of the multigrid preconditioner M (the paper names multigrid as prior
 * art for M, Sec. IV-A; "damped Jacobi" is its Jacobi step).  x, b, y: n_dof
 * entries; y must not overlap x or b. */
int to_smooth(to_problem* P, const void* x_dev, const void* b_dev, void* y_dev, double omega, void* stream);

/* nsteps lower-level steps on K^(rho~) u = f from the given u (in place), with the
 * problem's preconditioner and inner_mode (Algorithm 1 / 3, line 1).  If res_out
 * is not NULL it receives ||f - K^ u||_2 after the steps (synchronises). */
int to_inner_solve(to_problem* P, void* u_dev, int32_t nsteps, double* res_out, void* stream);

/* g = dJ/drho at the displacement u for the current design: the element term
 * -E'_e u_e^T k_e u_e (Sec. III, exact-gradient formula applied to u; J = f^T u)
 * chained through the filter transpose.  u: n_dof, g: n_elem entries. */
int to_sensitivity(to_problem* P, const void* u_dev, void* g_dev, void* stream);

/* Density filter of Remark 3.1 as a linear cone of radius rmin:
 * transpose = 0: y_e = sum_i H_ei x_i / Hs_e;  transpose = 1: y_i = sum_e H_ei x_e / Hs_e.
 * x, y: n_elem entries, must not overlap. */
int to_filter(to_problem* P, const void* x_dev, void* y_dev, int32_t transpose, void* stream);

/* rho = Proj_X(w): clamp(w - lambda, rho_min, rho_max) with lambda = 0 if the clamp meets
 * the volume bound, else the root of Eq. (piecewiseLinearEQ) (Sec. IV-B), found
 * by a safeguarded Newton search over the breakpoints in double precision.
 * w, rho: n_elem entries (may alias).  lambda_out (host, may be NULL) synchronises. */
int to_project(to_problem* P, const void* w_dev, void* rho_dev, double* lambda_out, void* stream);

/* Run n_outer outer iterations (Algorithms 1 / 3 with the problem's M) on the
 * problem's own state (rho_k, u_k, k).  If stats_out is not NULL it receives
 * n_outer records and the call synchronises; the return value then also
 * reports device-side errors.  Without stats_out nothing is copied back.
 * Each iteration builds the next design's moduli and preconditioner beside its
 * own lower-level steps (in a second buffer set, allocated on the first call:
 * one more copy of rho~, E', every level's moduli and 1 / d and the coarsest
 * inverse); the iterates are those of the sequential order, bit for bit.  On
 * return the operator of to_apply_K, to_inner_solve and to_sensitivity is that of
 * the returned design rho_{k+n}.  With mg_legs = 1, or while the problem belongs
 * to a batch, the iterations run in the sequential order and the moduli on return
 * are those of rho_{k+n-1}. */
int to_step(to_problem* P, int32_t n_outer, to_stats* stats_out, void* stream);

/* The records of the first n outer iterations of the last to_step call, or of the
 * last to_batch_step call of a batch the problem belongs to, whichever came last
 * (1 <= n <= its n_outer), copied into stats_out (host memory for n records) asynchronously on
 * `stream`, ordered after that call when the stream is the same: for a caller that
 * reads a step's results without the synchronisation to_step does for stats_out (to_step
 * with stats_out = NULL, then this, then one synchronisation of its own).  The copy is
 * asynchronous when stats_out is page-locked.  Device-side errors appear in each
 * record's status once the stream has completed; this call reports none itself.
 * TO_ERR_ARG for a null stats_out or n outside that range.  Not in the paper: an
 * interface convenience. */
int to_get_stats(to_problem* P, int32_t n, to_stats* stats_out, void* stream);

/* Read / write the outer state: rho (n_elem), u (n_dof), the 1-based iteration
 * counter k and alpha0 (<= 0 means not yet fixed).  Any pointer may be NULL to
 * skip that part.  to_set_state recomputes rho~ and the moduli.  After a to_step
 * (outside a batch), to_set_state compares the rho it is given with the problem's
 * rho bit for bit on the device; where they are equal the moduli and the next
 * to_step's rebuild of the preconditioner are skipped on the device (no
 * synchronisation), so a host loop that feeds back the design to_get_state returned
 * pays no rebuild.  The results are the same either way. */
int to_get_state(to_problem* P, void* rho_dev, void* u_dev, int64_t* k_out, double* alpha0_out, void* stream);
int to_set_state(to_problem* P, const void* rho_dev, const void* u_dev, int64_t k, double alpha0, void* stream);

/* One outer iteration (Algorithms 1 / 3) fed from host memory, for a loop that keeps
 * the design on the host: rho_in (n_elem entries, host, page-locked for an
 * asynchronous copy) is copied in and becomes rho as to_set_state would make it (k,
 * alpha0 and u are kept; an unchanged design skips its rebuild), one to_step
 * iteration runs, the new design is copied to rho_out (host, n_elem entries; may be
 * NULL) and the iteration's record to stats_out (host, one record; may be NULL), and
 * `stream` is synchronised once.  Page-locked rho_in / rho_out / stats_out are read
 * and written by kernels through their device aliases (no separate copy; the new
 * design is written as soon as the iteration's projection has formed it); pageable
 * ones are copied.  Returns the record's status: TO_OK or the first
 * device-side error of the iteration.  The first call allocates a device buffer of
 * n_elem entries (and, without stats_out, one page-locked record), kept until
 * to_destroy.  TO_ERR_ARG for a null rho_in.  Not in the paper: an interface for
 * serving loops. */
int to_step_host(to_problem* P, const void* rho_in, void* rho_out, to_stats* stats_out, void* stream);

/* Batches of independent design problems (each advanced exactly as to_step
 * advances it: Algorithms 1 / 3 with its own lambda, beta, alpha and state).
 * to_batch_create groups existing problems (not copied, not owned: destroy the
 * batch before its problems).  They must share precision, device, element
 * size h, E0 / Emin / p / nu and n_inner, and use TO_INNER_SD with the same
 * preconditioner: TO_PRECOND_JACOBI, or TO_PRECOND_MG with the same nu_pre,
 * nu_post and omega, every grid halving at least twice (each problem's coarse
 * levels below 1024 elements run as one CTA, all problems' in one launch;
 * TO_ERR_ARG otherwise); grids, loads, fixtures, volume fractions, filter
 * radii and multigrid depths may differ.  to_batch_step runs n_outer outer
 * iterations of every problem with one kernel launch per phase (per multigrid
 * step and level) for the whole batch (captured once as a CUDA graph); stats_out (may be NULL) receives n problems x n_outer records,
 * problem-major, and then the call synchronises.  n_outer must not exceed any
 * problem's stats ring (256 after to_create; a longer to_step grows it). */
int to_batch_create(to_problem* const* problems, int32_t n, to_batch** out);
void to_batch_destroy(to_batch* batch);
int to_batch_step(to_batch* batch, int32_t n_outer, to_stats* stats_out, void* stream);

/* The batched operator's tile shape chosen by the autotuner at to_batch_create:
 * to_batch_create times the batch's K u (into scratch, no state change) for tiles
 * of 2, 4, 8, 16 and 32 node planes and keeps the fastest.  kchunk_out receives
 * the planes per tile, us_out the measured microseconds of one batched K u at that
 * choice; either pointer may be NULL.  No counterpart in the paper. */
int to_batch_tile(const to_batch* batch, int32_t* kchunk_out, double* us_out);

/* Differentiable compliance through a truncated lower-level solve.
 * J(rho) = f^T u_T where u_0 = 0 and u_{j+1} = u_j + beta D^-1 (f - K^(rho~) u_j),
 * D = diag K^ (the literal constant-beta step of Algorithms 1 / 3 with the Jacobi M),
 * j < T_steps.  Sets the problem's design to rho (as to_set_design), keeps the
 * iterates that to_params.adj_stride asks for (all of u_0 .. u_T by default; the
 * problem grows its iterate buffer when a call needs more) and, if J_out is not
 * NULL, returns J (synchronises).  Requires precond = TO_PRECOND_JACOBI
 * (TO_ERR_STATE otherwise).  As T grows the gradient tends to the exact
 * sensitivity of Sec. III. */
int to_compliance_truncated(to_problem* P, const void* rho_dev, int32_t T_steps, double beta,
                            double* J_out, void* stream);

/* g = scale * dJ/drho for the last to_compliance_truncated call: a reverse sweep
 * over the kept iterates (adjoint lambda_T = f, lambda_j = lambda_{j+1} - K^ s_j,
 * s_j = beta D^-1 lambda_{j+1}) with the element terms
 * -E'_e [ s_e^T k_e u_j,e + sum_{d in e} k_dd s_d z_j,d ] (z_j = D^-1 r_j, the
 * dependence of D on rho included), chained through the filter transpose;
 * iterates not kept are recomputed segment by segment.  g: n_elem entries.
 * TO_ERR_STATE if no forward call preceded, or if the design changed since it
 * (to_set_design, to_set_state, to_step, a batch step). */
int to_compliance_truncated_grad(to_problem* P, double scale, void* g_dev, void* stream);

/* Identifier of the iterates the last to_compliance_truncated call kept: > 0 and
 * different for every forward call; 0 when none are kept or the design changed
 * since (then to_compliance_truncated_grad returns TO_ERR_STATE).  A caller that
 * interleaves several forward calls on one problem compares it with the value
 * read after its own forward to know whether its iterates are still there. */
int to_compliance_truncated_id(const to_problem* P, int64_t* id_out);

/* Allocation-free projection.  The paper has no counterpart: this entry point
 * exists for callers that may not allocate device memory, for instance code
 * running inside a host framework that owns every device byte through its own
 * pool, or a long-running service that must not call cudaMalloc / cudaFree
 * (cudaFree synchronises the whole device) once it is serving.  It computes
 * what to_project computes for a problem with n_elem = n, vbar, rho_min = lo and
 * rho_max = hi, without a to_problem and without allocating: its scratch (block
 * partials, barrier words, result scalars) is one static device array of about
 * 200 KB that every GPU loading this library holds until the process exits.
 *   w_dev, rho_dev  n entries on the current device (double for TO_FP64, float for
 *                   TO_FP32_MIXED); they may alias.
 *   n               1 <= n <= 2,097,152; larger n returns TO_ERR_ARG (also when the
 *                   device cannot keep every per-block chunk in shared memory).
 *   lambda_out      host, may be NULL; when set the call synchronises `stream`.
 * Device-side errors (a non-finite w, a grid barrier that gave up) are kept in the
 * array until a call with lambda_out != NULL reads them: that call returns the
 * error, whether this call or an earlier one made without lambda_out raised it,
 * and clears it.  A caller that never passes lambda_out never sees them.
 * The first call on a device looks up the array's device address and the
 * kernel's co-residency limit for that device (with it current); make that first
 * call before any stream capture.  Every call shares the one array and resets the
 * parts that must start at zero, so calls that overlap on the GPU (different
 * streams or threads) race: serialise them. */
int to_project_noalloc(const void* w_dev, void* rho_dev, int64_t n, int32_t precision, double vbar,
                       double lo, double hi, double* lambda_out, void* stream);

/* Failure-detection self-test of the grid barrier that the projection's
 * cooperative kernel uses between its passes (no counterpart in the paper).  It
 * launches up to 8 co-resident blocks that meet at that barrier with an
 * iteration limit of spin_limit polls (1 <= spin_limit <= 2^24; 2^24 is the
 * limit the library itself uses, about a second).  absent_block = -1: every
 * block arrives and the call returns TO_OK.  absent_block = b >= 0: block b skips
 * the barrier, the others wait for it until the limit runs out and then return,
 * and the call returns TO_ERR_TIMEOUT.  Either way the call synchronises, clears
 * the barrier words and the problem's device error flag, and leaves the context
 * usable: no kernel waits without a bound. */
int to_barrier_selftest(to_problem* P, int32_t absent_block, int64_t spin_limit, void* stream);

/* Synchronise the stream and report (and clear) the device error flag. */
int to_check(to_problem* P, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* to_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TO_H */
