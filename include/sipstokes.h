/*
 * sipstokes.h -- C ABI of a GB300 (sm_103a) library for the symmetric interior
 * penalty discontinuous Galerkin (SIP-DG) discretisation of heterogeneous
 * 2D Stokes flow and its block / hp-multigrid preconditioned Krylov solver,
 * after Charrier, May & Schnepp, arXiv 1607.03777.
 *
 * Discretisation (paper Sec. 3-4): a regular nx x ny Cartesian grid of
 * [0,lx] x [0,ly]; velocity in discontinuous Q_k^2, pressure in
 * discontinuous Q_{k-1}, 1 <= k <= 6; element-wise constant viscosity eta_K
 * (assumption ASh1).  Basis: tensor products of orthonormal Legendre
 * polynomials l_i = sqrt((2i+1)/2) P_i on the reference square (Sec. 5).
 *
 * Vector layouts (all FP64 unless the name ends in _f32):
 *   velocity  u[e][c][j][i]  e = ey*nx + ex, c = component (x, y),
 *                            i = x-degree (fastest), j = y-degree, 0..k
 *                            -> n_u = nx*ny*2*(k+1)^2 entries
 *   pressure  p[e][j][i]     0 <= i, j < k  -> n_p = nx*ny*k^2 entries
 *   Q_1 (p-coarse) vectors   u1[e][c][j][i], i, j in {0, 1} -> 8 per element
 *   continuous bilinear      v[(vy*(nx+1)+vx)][c] -> 2 (nx+1)(ny+1) entries
 *
 * Conventions:
 *   - Vector arguments are caller-owned DEVICE pointers on the problem's
 *     device, 8-byte (FP64) / 4-byte (FP32) aligned, and must not overlap
 *     unless stated.  Host arrays are named *_host.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous with respect to the host unless they return a host value.
 *   - Every call returns a sip_status; on failure a message is available from
 *     sip_last_error() on the owning context.  No C++ exception crosses the ABI.
 *   - Handles are opaque, created and destroyed by the library.
 */
#ifndef SIPSTOKES_H
#define SIPSTOKES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SIP_OK = 0,
    SIP_ERR_INVALID_ARG = 1,   /* bad size, k, eta <= 0, non-finite input ... */
    SIP_ERR_OOM = 2,           /* device allocation failed / over budget      */
    SIP_ERR_CUDA = 3,          /* a CUDA runtime call failed                  */
    SIP_ERR_NOT_CONVERGED = 4, /* iteration cap reached before the tolerance  */
    SIP_ERR_BREAKDOWN = 5,     /* Krylov breakdown or non-finite iterate      */
    SIP_ERR_TIMEOUT = 6,       /* a served request passed its deadline        */
    SIP_ERR_REJECTED = 7,      /* server admission refused the request        */
    SIP_ERR_NOT_READY = 8,     /* result not available yet                    */
    SIP_ERR_CANCELLED = 9      /* a served request was cancelled              */
} sip_status;

/* Boundary condition of one side of the rectangle (Sec. 2, eqs.
 * neumann_bc / navier_dirichlet_bc).  SIP_BC_DIRICHLET (u = 0, imposed by
 * the symmetric Nitsche analogue of the Navier terms) is an extension that
 * the paper does not use. */
typedef enum { SIP_BC_NAVIER = 0, SIP_BC_NEUMANN = 1, SIP_BC_DIRICHLET = 2 } sip_bc;

/* Precision of the viscous preconditioner.  The outer FGMRES, its residual,
 * B, B^T and the S* scaling are always FP64.
 *   SIP_PREC_FP64            everything FP64;
 *   SIP_PREC_MIXED           V-cycle (smoother, transfers, coarse solve) FP32,
 *                            inner PCG iterate and operator FP64;
 *   SIP_PREC_MIXED_F32_INNER V-cycle and inner PCG both FP32. */
typedef enum {
    SIP_PREC_FP64 = 0,
    SIP_PREC_MIXED = 1,
    SIP_PREC_MIXED_F32_INNER = 2
} sip_precision;

typedef struct sip_ctx sip_ctx;
typedef struct sip_problem sip_problem;

typedef struct {
    int nx, ny;             /* elements per direction, >= 1                     */
    double lx, ly;          /* domain size, > 0                                 */
    int k;                  /* velocity degree 1..6 (pressure k-1)              */
    int bc[4];              /* sip_bc of the left, right, bottom, top side      */
    const double* eta_host; /* nx*ny element viscosities, > 0, copied           */
    double penalty_scale;   /* multiplies sigma_e; 1.0 = the paper's choice     */
    /* hp-multigrid (Sec. 6): coarse space Q^2_1 then n_hlevels coarsenings of
     * the continuous bilinear problem; 0 = A_p(Q^2_1) (LU of A_1). */
    int n_hlevels;
    int cheb_steps_p;       /* Chebyshev / block-Jacobi steps per side, paper 2 */
    int cheb_steps_h;       /* Chebyshev / point-Jacobi steps on h-levels, 3    */
    int eig_iters;          /* GMRES steps of the eigen estimate, paper 10      */
    double cheb_lo, cheb_hi;/* bound factors, paper 0.1 and 1.1                 */
    uint64_t seed;          /* SplitMix64 stream of the eigen-estimate vector   */
    sip_precision precision;
    /* p-coarse space (Sec. 6.1): SIP_COARSE_Q1 (element-wise bilinear, then the
     * continuous bilinear h-hierarchy, Sec. 6.1.2) or SIP_COARSE_Q0 (element-
     * wise constants, A_0 = P^T A P, coarsened as a grid of the element
     * centres, Sec. 6.1.1: needs nx - 1 and ny - 1 divisible by 2^n_hlevels,
     * i.e. odd element counts; n_hlevels = 0 solves A_0 directly, at most
     * 8192 elements). */
    int coarse;
    /* Mixed forms only (no counterpart in the paper, which is FP64): the FP32
     * operator of the V-cycle is evaluated in FP64 arithmetic (on the same
     * FP32 data) on the mesh tiles of 32 x 2 elements whose tile or
     * one-element halo holds an element with eta >= mixed_fp64_ratio x
     * min(eta); elsewhere in FP32.  In FP32 arithmetic the nearly rigid
     * motion of an inclusion much stiffer than the medium cancels to
     * rounding noise of size eps_32 eta_K |u|, which swamps the residual of
     * the soft medium: at contrast 1e6 the FP32 V-cycle stops reducing the
     * residual altogether.  Default 1e3; 0 = FP32 arithmetic everywhere.
     * At k = 6, which has no staged kernel, the whole FP32 operator takes
     * FP64 arithmetic as soon as one tile is marked. */
    double mixed_fp64_ratio;
} sip_problem_desc;

/* values of sip_problem_desc.coarse */
enum { SIP_COARSE_Q1 = 0, SIP_COARSE_Q0 = 1 };

/* Fill a descriptor with the paper's defaults (Sec. 6-7): Navier on every
 * side, penalty_scale 1, n_hlevels 0, 2 p-level and 3 h-level smoothing
 * steps, 10 eigen-estimate iterations, bounds 0.1 / 1.1, seed 0, FP64,
 * Q^2_1 coarse space; mixed_fp64_ratio 1e3. */
void sip_problem_desc_default(sip_problem_desc* desc);

/* ---- context ------------------------------------------------------------ */
/* Create a context bound to CUDA device `device`. */
sip_status sip_ctx_create(int device, sip_ctx** out);
void sip_ctx_destroy(sip_ctx* ctx);
/* Message of the last failing call made through ctx (or one of its
 * problems); valid until the next call on ctx.  Never NULL. */
const char* sip_last_error(const sip_ctx* ctx);

/* ---- problem ------------------------------------------------------------ */
/* Create a problem: copies eta, derives the element-wise penalties and
 * allocates the device state.  The multigrid set-up runs on first use (or
 * through sip_problem_setup).  Errors: INVALID_ARG (nx, ny < 1, k outside
 * 1..6, non-positive or non-finite eta / lengths, a mesh that cannot be
 * coarsened n_hlevels times), OOM, CUDA. */
sip_status sip_problem_create(sip_ctx* ctx, const sip_problem_desc* desc, sip_problem** out);
void sip_problem_destroy(sip_problem* prob);
/* Replace the element viscosities (host or device array of nx*ny, finite and
 * positive) and mark the multigrid set-up stale: the next call that needs it
 * rebuilds it in the buffers already held (no new device allocation). */
sip_status sip_problem_update_eta(sip_problem* prob, const double* eta, void* stream);
/* Number of velocity and pressure dofs and the device bytes held. */
sip_status sip_problem_sizes(const sip_problem* prob, int64_t* n_u, int64_t* n_p,
                             int64_t* device_bytes);
/* Kernel schedule in force (no counterpart in the paper).  The first set-up
 * of a problem of a new (degree, precision, mesh) times the candidate kernels
 * on the device and keeps the fastest; later problems of the same shape reuse
 * the choice.  apply[0] / apply[1]: SIP apply kernel of the FP64 / FP32
 * operator: 1 component-split thread pair per element, 2 one thread per
 * element, 3 shared-memory tile, 4 / 5 component-split thread pair on
 * element blocks staged through shared memory with 2 / 4 tile rows, 6 (FP32
 * operator only) one thread per element and one warp per tile row on
 * element blocks staged with asynchronous 16-byte copies.  An FP32 operator
 * with split-precision tiles (see mixed_fp64_ratio) reports 4: its marked
 * tiles run the staged kernel with FP64 arithmetic, the others kernel 6;
 * fused[0] / fused[1]: 1 if a p-level smoother step is one launch (apply,
 * block-Jacobi and Chebyshev update together), 0 if it is the apply and
 * block-Jacobi launches.  Either array may be NULL; the values are those of
 * the last set-up (defaults before). */
sip_status sip_problem_schedule(const sip_problem* prob, int apply[2], int fused[2]);
/* Pin the kernel schedule of this problem (no counterpart in the paper):
 * apply[t] in 0..6 with the codes of sip_problem_schedule (0 = autotuned;
 * 1, 2, 4, 5, 6 need k <= 5; 6 only for apply[1]), fused[t] in -1..1 (-1 = autotuned; 1 takes effect
 * only for k <= 3).  Either array may be NULL (unchanged).  The operator
 * entry points use a pinned apply kernel at once; the multigrid set-up is
 * marked stale, so the next call that needs it rebuilds it (in the buffers
 * already held) with the pinned kernels.  Errors: INVALID_ARG. */
sip_status sip_problem_set_schedule(sip_problem* prob, const int apply[2], const int fused[2]);

/* ---- operators (paper Sec. 4) ------------------------------------------- */
/* y_u = A x_u: the SIP viscous operator, eq. stiffness_form -- volume term
 * 2 eta eps(u):eps(v), interior-face consistency, symmetry and penalty
 * terms, Navier-face terms -- applied matrix-free (closed-form 1D modal
 * factors, no assembled matrix).  sigma_e = penalty_scale * 4 eta_e
 * (k+1)^2 |e|/|K| x {1 interior, 2 boundary} (Lemma 4.4 with tau = 0,
 * Lemma 4.1, eq. eta_face).  x_u and y_u must not overlap. */
sip_status sip_apply_A(sip_problem* prob, const double* x_u, double* y_u, void* stream);
/* The same operator in FP32 arithmetic (inputs and outputs FP32). */
sip_status sip_apply_A_f32(sip_problem* prob, const float* x_u, float* y_u, void* stream);
/* y_u = B p: (B p)_v = b_h(v, p), eq. divergence_form.  x_p: n_p, y_u: n_u. */
sip_status sip_apply_B(sip_problem* prob, const double* x_p, double* y_u, void* stream);
/* y_p = B^T u: (B^T u)_q = b_h(u, q).  x_u: n_u, y_p: n_p. */
sip_status sip_apply_Bt(sip_problem* prob, const double* x_u, double* y_p, void* stream);

/* ---- hp-multigrid pieces (paper Sec. 6) ------------------------------------
 * The multigrid set-up runs once per problem, on the device, on first use or
 * here: element-block Jacobi inverses (FP64 factorisation), eigenvalue
 * estimates, Galerkin coarse operators and the coarsest-level inverse.
 * The entry points below act on FP64 vectors with the FP64 hierarchy
 * (built on demand also for SIP_PREC_MIXED problems). */
sip_status sip_problem_setup(sip_problem* prob, void* stream);
/* Largest eigenvalue estimate lambda* of the smoother's preconditioned
 * operator: level -1 = p-level M^{-1}A (element-block Jacobi), level l >= 0 =
 * continuous level l (point-Jacobi D^{-1}A_l); from eig_iters GMRES (Arnoldi)
 * steps started from the SplitMix64 vector of stream seed (p-level) or
 * seed + 1 + l (h-level l); the Chebyshev interval is [cheb_lo, cheb_hi] x
 * lambda* (Sec. 6).  Synchronous. */
sip_status sip_lambda_max(sip_problem* prob, int level, double* out);
/* z_u = M^{-1} r_u, M = the diagonal element blocks of A (Sec. 6, eq. smoother). */
sip_status sip_block_jacobi(sip_problem* prob, const double* r_u, double* z_u, void* stream);
/* r1 = R r_u = P^T r_u: keep the hierarchical modes i, j <= 1 (Sec. 6). */
sip_status sip_p_restrict(sip_problem* prob, const double* r_u, double* r1, void* stream);
/* y_u += P e1: inject Q_1 modes into Q_k (zero fill of the rest). */
sip_status sip_p_prolong_add(sip_problem* prob, const double* e1, double* y_u, void* stream);
/* y1 = A_1 x1, A_1 = P^T A P: the SIP operator on the Q_1 modes with the
 * penalty of degree k (Sec. 6 Galerkin coarse operator). */
sip_status sip_apply_A1(sip_problem* prob, const double* x1, double* y1, void* stream);
/* u1 = P_cd v: continuous bilinear vertex values -> element modal Q_1
 * coefficients (Sec. 6.1.2); v has 2 (nx+1)(ny+1) entries. */
sip_status sip_cd_prolong(sip_problem* prob, const double* v, double* u1, void* stream);
/* v = R_dc u1 = P_cd^T u1. */
sip_status sip_dc_restrict(sip_problem* prob, const double* u1, double* v, void* stream);
/* Number of vertex-grid levels (n_hlevels + 1 for A_hp(Q^2_1) and for the
 * Q^2_0 coarse space, 0 for A_p(Q^2_1)) and the vertex grid of level l
 * (l = 0 finest: the mesh vertices for Q^2_1, the element centres for
 * Q^2_0). */
sip_status sip_hlevel_dims(sip_problem* prob, int level, int* n_levels, int* nvx, int* nvy);
/* Copy the Galerkin 9-point 2x2-block stencil of level l into S (device,
 * nvx*nvy*36 doubles, S[v][t][c][c'], t = (dy+1)*3 + (dx+1)): level 0 is
 * A_1c = P_cd^T A_1 P_cd (Q^2_1) or A_0 = P_0^T A P_0 (Q^2_0), level l+1 is
 * P_h^T A_l P_h (bilinear P_h). */
sip_status sip_hlevel_stencil(sip_problem* prob, int level, double* S, void* stream);
/* y = A_l x on continuous level l (vectors of 2 nvx nvy). */
sip_status sip_hlevel_apply(sip_problem* prob, int level, const double* x, double* y, void* stream);
/* x = A_c^{-1} b on the coarsest level (LU / Cholesky set-up, dense inverse):
 * A_1 (Q^2_1) or A_0 (Q^2_0) itself for n_hlevels = 0, else the coarsest
 * vertex-grid level. */
sip_status sip_coarse_solve(sip_problem* prob, const double* b, double* x, void* stream);
/* z_u = one V-cycle of Algorithm 1 (y0 = 0) applied to r_u: Chebyshev /
 * element-block Jacobi pre-smoothing, restriction to Q_1 (or Q_0), coarse
 * correction (LU of A_1, or P_cd + continuous h-cycle + R_dc; with Q^2_0 the
 * h-cycle of A_0 on the element centres, or its LU), prolongation,
 * post-smoothing. */
sip_status sip_vcycle(sip_problem* prob, const double* r_u, double* z_u, void* stream);
/* The same V-cycle computed entirely in FP32 (the mixed-precision form). */
sip_status sip_vcycle_f32(sip_problem* prob, const float* r_u, float* z_u, void* stream);
/* y_u ~ A^{-1} t_u by PCG preconditioned with the V-cycle, from y = 0 until
 * ||A y - t|| < rtol ||t|| (Sec. 6) or max_it iterations; *its receives the
 * count.  Synchronous. */
sip_status sip_inner_solve(sip_problem* prob, const double* t_u, double* y_u, double rtol,
                           int max_it, int* its, void* stream);

/* ---- Stokes solve (paper Sec. 5-7) ---------------------------------------- */
typedef struct {
    double rtol;        /* stop when ||b - K x||_2 <= rtol ||b||_2 (true residual)  */
    int max_outer;      /* FGMRES iteration cap (all restarts)                      */
    int restart;        /* FGMRES restart length                                    */
    double inner_rtol;  /* inner PCG relative tolerance (paper 1e-3)                */
    int max_inner;      /* inner iteration cap                                      */
    int inner_loop;     /* 0: each inner PCG solve is one CUDA graph launch whose   *
                         *    loop runs on the device (default); 1: host-driven     *
                         *    loop, one read-back per iteration.  Same arithmetic:  *
                         *    both give bit-identical iterates.                     */
    int inner_krylov;   /* 0: automatic (PCG for SIP_PREC_FP64, flexible CG for the *
                         *    mixed forms, whose FP32 V-cycle is not exactly the    *
                         *    same linear operator at every application);          *
                         *    1: PCG; 2: flexible CG, FCG(1) (device loop only);    *
                         *    3: GCR, restarted after inner_restart directions, the *
                         *    method of the six-inclusion runs (Sec. 7.3): flexible,*
                         *    minimises and tests ||t - A y||_2 (inner_norm does   *
                         *    not apply); device loop only, not with               *
                         *    SIP_PREC_MIXED_F32_INNER                              */
    int inner_norm;     /* inner stopping test of the CG variants, relative to the  *
                         *    first value: 0 (default): the residual               *
                         *    ||t - A y||_2 (Sec. 7.1), whose outer iteration      *
                         *    counts stay flat in the viscosity contrast; 1: the   *
                         *    preconditioned residual ||V(t - A y)||_2 (PETSc's    *
                         *    CG default): fewer V-cycles on a single jump, but    *
                         *    the outer count grows with the contrast on the six   *
                         *    inclusions of Sec. 7.3 (device loop only)            */
    int inner_restart;  /* GCR restart length, 1..64 (default 30); GCR stores      *
                         *    2 x inner_restart FP64 vectors of n_u on the device  */
    int outer_krylov;   /* 0: FGMRES (default); 1: GCR, restarted after `restart`  *
                         *    directions, the outer method of the six-inclusion    *
                         *    runs (Sec. 7.3); both minimise the residual, both     *
                         *    stop on the residual recomputed from x, and both     *
                         *    stop early (NOT_CONVERGED) when two consecutive      *
                         *    restarts on which the recurrence met rtol fail to    *
                         *    halve that residual (the FP64 attainable accuracy)   */
    int refine;         /* 0 (default): off.  n > 0: iterative refinement, at most *
                         *    n correction solves: x and r = b - K x are carried   *
                         *    in double-double (sip_residual_dd), each correction  *
                         *    K d = r is an ordinary solve in the problem's        *
                         *    precision asking for the reduction still missing.    *
                         *    Stops when ||r|| <= rtol ||b|| (evaluated in         *
                         *    double-double) or when a step fails to halve ||r||. *
                         *    Reaches residuals below FP64's attainable accuracy   *
                         *    for high viscosity contrasts, in place of the        *
                         *    paper's quadruple precision (Sec. 7.4).  sip_solve   *
                         *    returns the iterate rounded to FP64, whose residual  *
                         *    can lie above rtol at such contrasts; sip_solve_dd   *
                         *    returns the double-double iterate itself.            */
    double time_limit_ms;  /* 0 (default): none.  > 0: wall-clock limit of the  *
                            *    solve (sip_solve, sip_solve_batch: from the    *
                            *    call; served requests: from submission).  It   *
                            *    is checked between outer iterations: a solve   *
                            *    past it stops with SIP_ERR_TIMEOUT and keeps   *
                            *    its last iterate; a queued request past it is  *
                            *    reported with SIP_ERR_TIMEOUT unsolved.  No    *
                            *    counterpart in the paper.                      */
} sip_solve_opts;

typedef struct {
    int status;            /* sip_status of the solve                           */
    int outer_its;         /* FGMRES iterations                                 */
    int inner_total;       /* inner PCG iterations, summed                      */
    int inner_max;
    double inner_avg;
    double rel_residual;   /* ||b - K x||_2 / ||b||_2 recomputed in FP64        *
                            * (in double-double with refine > 0)               */
    double setup_ms;       /* multigrid set-up time of this call (0 if reused)  */
    double solve_ms;
    double lambda_max_p;
    int64_t kernel_launches;
    int refine_steps;      /* correction solves of iterative refinement (0: off) */
} sip_solve_report;

/* rtol 1e-8, max_outer 500, restart 100, inner_rtol 1e-3, max_inner 200,
 * inner_loop 0, inner_krylov 0, inner_norm 0, inner_restart 30,
 * outer_krylov 0, refine 0, time_limit_ms 0. */
void sip_solve_opts_default(sip_solve_opts* opts);
/* Solve [A B; B^T 0][u; p] = [f; g] (eq. discretestokes) by right-
 * preconditioned FGMRES (or GCR, opts->outer_krylov) with the upper
 * block-triangular preconditioner (eq. discretestokespc) whose Schur block is
 * the saddle matrix's own Schur complement -B^T A^{-1} B approximated by -S*,
 * S* the pressure mass scaled by 1/eta_K (diagonal, Sec. 5): y_p = -S*^{-1}
 * x_p, y_u ~ A^{-1}(x_u - B y_p) by the inner Krylov solve (PCG, FCG or
 * GCR) with the hp-multigrid V-cycle.  Orthogonalisation: classical
 * Gram-Schmidt twice.
 * Without a Neumann side the constant pressure is projected out of every
 * pressure vector and p is returned with zero mean (Sec. 5).  g_p may be NULL
 * (g = 0, eq. rhs_f).  Outer state, residuals and S* are FP64; the
 * preconditioner runs in the problem's precision.  Returns the status also
 * in report->status (NOT_CONVERGED / BREAKDOWN keep the last iterate in u, p).
 * Synchronous. */
sip_status sip_solve(sip_problem* prob, const double* f_u, const double* g_p, double* u,
                     double* p, const sip_solve_opts* opts, sip_solve_report* report,
                     void* stream);

/* r = b - K x for b = [f_u; g_p] (g_p may be NULL: 0) and x = [x_u; x_p] in
 * double-double arithmetic (about 106 significant bits): the operator of
 * sip_apply_A / sip_apply_B / sip_apply_Bt (eq. discretestokes, the same
 * FP64 coefficients) evaluated exactly enough that the residual of an FP64
 * iterate is not lost in rounding at high viscosity contrast (the precision
 * question of Sec. 7.4).  x_u, x_p, r_u, r_p are device arrays of
 * interleaved (hi, lo) double pairs, value = hi + lo: 2 n_u and 2 n_p
 * doubles, caller-owned, not overlapping.  Stream-ordered. */
sip_status sip_residual_dd(sip_problem* prob, const double* f_u, const double* g_p,
                           const double* x_u, const double* x_p, double* r_u, double* r_p,
                           void* stream);

/* The refined solve of sip_solve (opts->refine > 0, required) returning its
 * double-double iterate (Sec. 7.4 solves high-contrast problems in quadruple
 * precision; the iterate of the refinement carries about 106 bits): u_dd, p_dd
 * are 2 n_u / 2 n_p doubles of interleaved (hi, lo) pairs, value = hi + lo,
 * caller-owned device buffers, the layout sip_residual_dd reads.  The
 * relative residual the report gives (and that rtol bounds) is that of this
 * iterate; rounded to FP64 (what sip_solve returns) it can lie above rtol
 * when ||K|| eps_64 ||x|| > rtol ||b|| (viscosity contrasts of 1e6 and more).
 * Without a Neumann face the pressure is fixed only up to a constant (the
 * FP64 outputs of sip_solve have zero mean).  Errors as sip_solve, and
 * INVALID_ARG without refinement. */
sip_status sip_solve_dd(sip_problem* prob, const double* f_u, const double* g_p, double* u_dd,
                        double* p_dd, const sip_solve_opts* opts, sip_solve_report* report,
                        void* stream);

/* ---- batches and serving ----------------------------------------------------
 * Not in the paper (it solves one problem at a time on one CPU core): many
 * independent Stokes problems of different mesh sizes, degrees and viscosity
 * fields solved concurrently on one GPU.  Every solve in flight owns a
 * stream, its device-resident multigrid and Krylov state and its captured
 * V-cycle graph; solves in flight together overlap on the device.  Device
 * memory of in-flight work is stream-ordered (no device-wide
 * synchronisation between requests). */
typedef struct sip_server sip_server;

/* Solve problems[i] with right-hand side f_u[i] into u[i], p[i] (device
 * pointers), n_streams solves in flight at a time (<= 0: 8), each on its own
 * host thread and stream; each result equals the same solve alone, bit for
 * bit.  reports may be NULL or hold n entries.  Returns SIP_OK when every
 * solve converged, else the status of a failing one (each report holds its
 * own).  Synchronous. */
sip_status sip_solve_batch(sip_ctx* ctx, int n, sip_problem* const* problems,
                           const double* const* f_u, double* const* u, double* const* p,
                           const sip_solve_opts* opts, sip_solve_report* reports, int n_streams);
/* The same solves with the inner solves of up to `group` problems at a time
 * (<= 0: 32) batched into one CUDA graph: each problem's outer FGMRES runs on
 * its own host thread and stream, and where it needs an inner solve it
 * waits until every problem of its group still solving needs one; the last
 * to arrive launches one inner loop for all of them, in which every stage
 * (each step of the V-cycle, Algorithm 1, and of the Krylov iteration) is
 * one launch over a work list of (problem, tile) items per polynomial
 * degree, and the loop runs on the device until every problem has met its
 * stopping test.  The problems thus advance through their outer iterations
 * in lockstep, and the number of launches per stage does not grow with the
 * group.  Results equal the same solves alone to rounding (the dot products
 * are blocked differently), not bit for bit.  Needs one precision
 * (SIP_PREC_FP64 or SIP_PREC_MIXED) for all problems, the default inner
 * method and stopping test on the device loop, the Q^2_1 coarse space with
 * 1..11 h-coarsenings, k <= 5 and one smoothing schedule with 2..8 h-level
 * steps; else SIP_ERR_INVALID_ARG.  A round lasts as long as its slowest
 * inner solve: grouping pays where launches, not the device, limit a solve
 * (on a GB300, 48 meshes of 32^2 elements solve 1.45x faster grouped than
 * on 32 concurrent streams; meshes of 64^2 break even; 128^2 are faster
 * through sip_solve_batch).  Synchronous. */
sip_status sip_solve_batch_grouped(sip_ctx* ctx, int n, sip_problem* const* problems,
                                   const double* const* f_u, double* const* u, double* const* p,
                                   const sip_solve_opts* opts, sip_solve_report* reports,
                                   int group);
/* Device bytes a problem of this description holds after a solve with the
 * given FGMRES restart length (the server's admission estimate). */
int64_t sip_problem_footprint(const sip_problem_desc* desc, int restart);
/* A request server on ctx's device: at most max_slots solves in flight and
 * at most budget_bytes of estimated device footprint admitted at once.
 * Requests are admitted in arrival order as slots and memory free up; while
 * the oldest queued request does not fit the free budget, later requests
 * that fit may run ahead of it, at most 4 x max_slots of them, after which
 * it waits alone for memory (bounded backfilling, no starvation). */
sip_status sip_server_create(sip_ctx* ctx, int64_t budget_bytes, int max_slots, sip_server** out);
/* Queue one request: the problem desc (eta_host copied), the element
 * densities rho_host (copied; body force (0, -g rho_K)), host outputs u_host
 * (n_u) and p_host (n_p) that must stay valid until the request is reported
 * done, options (NULL = defaults; opts->time_limit_ms is a deadline counted
 * from this call).  Non-blocking.  Non-finite or non-positive eta,
 * non-finite rho or g: SIP_ERR_INVALID_ARG (nothing queued).  A request whose
 * footprint exceeds the whole budget is refused (SIP_ERR_REJECTED, also
 * reported by poll). */
sip_status sip_server_submit(sip_server* server, const sip_problem_desc* desc,
                             const double* rho_host, double g, double* u_host, double* p_host,
                             const sip_solve_opts* opts, uint64_t request_id);
/* Move up to cap finished requests into ids / reports (report.solve_ms =
 * submit-to-result latency in ms); *n_done receives the count. */
sip_status sip_server_poll(sip_server* server, uint64_t* ids, sip_solve_report* reports, int cap,
                           int* n_done);
/* Cancel request `request_id`: a queued request is dropped and reported
 * by poll with SIP_ERR_CANCELLED; a running one stops at its next outer
 * iteration and is reported with SIP_ERR_CANCELLED (its outputs hold the
 * last iterate).  Returns SIP_OK, or SIP_ERR_INVALID_ARG when no queued or
 * running request has this id (finished requests cannot be cancelled). */
sip_status sip_server_cancel(sip_server* server, uint64_t request_id);
/* Block until every queued and running request has finished. */
sip_status sip_server_drain(sip_server* server);
sip_status sip_server_stats(sip_server* server, int* queued, int* running,
                            int64_t* bytes_in_use);
/* Stop the workers (queued requests are dropped, running ones finish). */
void sip_server_destroy(sip_server* server);

/* ---- set-up helpers (paper Sec. 7.3) -------------------------------------- */
/* Element-wise material of inclusions (Sec. 7.3): eta_K = max of eta over
 * the open element, rho_K = min of rho, where eta(x) = max(eta_bg, eta_i over
 * the closed inclusions containing x); an element takes an inclusion's
 * density only when it lies inside that single inclusion.
 * shapes_host: n_shapes records of 7 doubles (kind, a, b, c, d, eta_i, rho_i):
 *   kind 0 = disc, centre (a, b), radius c (d unused);
 *   kind 1 = box [a, b] x [c, d];
 * with eta_i >= eta_bg and rho_i >= rho_bg.  eta_out, rho_out: device arrays
 * of nx*ny.  Synchronises `stream` before returning. */
sip_status sip_rasterise_inclusions(sip_ctx* ctx, int nx, int ny, double lx, double ly,
                                    const double* shapes_host, int n_shapes, double eta_bg,
                                    double rho_bg, double* eta_out, double* rho_out,
                                    void* stream);
/* Allocation-free variant of sip_rasterise_inclusions (the paper has no
 * counterpart: this is a service to callers that must not allocate device
 * memory -- e.g. code running inside a framework that owns all device memory
 * through its own pool and budget, or a latency-bound loop where cudaMalloc /
 * cudaFree would synchronise the whole device).  Same arguments, same results.
 * The inclusion records are staged in a fixed device array compiled into the
 * library (SIP_NOALLOC_MAX_SHAPES records, 224 KiB on every GPU that loads
 * the library, held until the process exits) instead of a fresh allocation;
 * n_shapes > SIP_NOALLOC_MAX_SHAPES is rejected with SIP_ERR_INVALID_ARG.
 * The first call on a device looks up the array's device address, so make
 * that first call before any stream capture.  All calls share the one
 * array: calls whose copies and kernels may overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller.  The
 * records are copied with cudaMemcpyAsync on `stream`; the call does not
 * synchronise the stream (a pinned shapes_host must stay valid until the
 * stream has passed the copy). */
#define SIP_NOALLOC_MAX_SHAPES 4096
sip_status sip_rasterise_inclusions_noalloc(sip_ctx* ctx, int nx, int ny, double lx, double ly,
                                            const double* shapes_host, int n_shapes,
                                            double eta_bg, double rho_bg, double* eta_out,
                                            double* rho_out, void* stream);
/* f_u = the load vector of the body force f = (0, -g rho_K) (eq. rhs_f,
 * Sec. 7.3); rho: device array of nx*ny. */
sip_status sip_rhs_body_force(sip_problem* prob, const double* rho, double g, double* f_u,
                              void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SIPSTOKES_H */
