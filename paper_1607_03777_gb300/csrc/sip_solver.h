// Solver-side declarations: kernel launchers of the smoother, transfer and
// Krylov translation units, and the multigrid / Krylov drivers.
#pragma once

#include <memory>

#include "sip_internal.h"

namespace sip {

// ---- smoother.cu
void launch_classify(int nx, int ny, const double* eta, int* emap, int* uniq_list, int* n_uniq,
                     cudaStream_t s);
template <typename T>
void launch_build_blocks(int N, const OpGeom& g, const int* spec, int count, const double* eta,
                         T* out, cudaStream_t s);
// uniq_hi (may be null): unique blocks applied in FP64 from uniq_inv64
template <typename T>
void launch_bj_apply(int N, int ne, const T* r, T* out, T* x, const int* emap, const T* cls_inv,
                     const int* cls_sym, const T* uniq_inv, const T* eta, T c1, T c2, bool x_zero,
                     cudaStream_t s, const unsigned char* uniq_hi = nullptr,
                     const double* uniq_inv64 = nullptr);
// Block-Jacobi apply arguments of one element set (one member of a batch).
template <typename T>
struct BJBatchArgs {
    int ne;
    const T* r;
    T* out;
    T* x;
    const int* emap;
    const T* cls_inv;
    const int* cls_sym;
    const T* uniq_inv;
    const T* eta_inv;
    const unsigned char* uniq_hi;
    const double* uniq_inv64;   // FP64 inverses of the unique blocks (flagged ones read)
    T c1, c2;
    int x_zero;
};
// elements per CTA of the block-Jacobi kernels
int bj_group(int N);
// CTA b: member items[b].x (args[items[b].x]), element group items[b].y
template <typename T>
void launch_bj_apply_batch(int N, const BJBatchArgs<T>* args, const int2* items, int n_items,
                           const int* active, cudaStream_t s);
void launch_mark_uniq_hi(int nx, int ny, const int* list, const int* n_uniq_dev, int n_uniq,
                         const double* eta, double ratio, unsigned char* flag, cudaStream_t s);

// ---- transfer.cu
// M = 2: Q^2_1 modes (8 per element), M = 1: Q^2_0 (2 per element)
template <typename T>
void launch_p_restrict(size_t ne, int N, const T* r, T* r1, cudaStream_t s, int M = 2);
template <typename T>
void launch_p_prolong_add(size_t ne, int N, const T* e1, T* y, cudaStream_t s, int M = 2);
template <typename T> void launch_pcd(int nx, int ny, const T* v, T* out, cudaStream_t s);
template <typename T> void launch_rdc(int nx, int ny, const T* r, T* out, cudaStream_t s);
template <typename T>
void launch_stencil_apply(int nvx, int nvy, const T* S, const T* x, T* y, T alpha, const T* z,
                          T beta, cudaStream_t s);
template <typename T> void launch_stencil_dinv(size_t nv, const T* S, T* dinv, cudaStream_t s);
template <typename T>
void launch_jacobi_cheb(size_t n, const T* r, const T* dinv, T* d, T* x, T c1, T c2, bool x_zero,
                        cudaStream_t s);
template <typename T> void launch_ph_add(int nxc, int nyc, const T* xc, T* yf, cudaStream_t s);
template <typename T>
void launch_hcheb_first(size_t n, const T* b, const T* dinv, T* r, T* d, T* x, T c2,
                        cudaStream_t s);
template <typename T>
void launch_hcheb_start(int nvx, int nvy, const T* S, const T* dinv, const T* b, const T* x, T* r,
                        T* d, T c2, cudaStream_t s);
template <typename T>
void launch_hcheb_step(int nvx, int nvy, const T* S, const T* dinv, T* r, const T* d_old,
                       T* d_new, T* x, T c1, T c2, bool pend, cudaStream_t s);
template <typename T> void launch_rh(int nxc, int nyc, const T* rf, T* rc, cudaStream_t s);
template <typename T>
void launch_probe_vertices(int nvx, int nvy, int col, int cp, T* x, cudaStream_t s);
template <typename T> void launch_extract_stencil(int nvx, int nvy, const T* Y, T* S, cudaStream_t s);
template <typename T> void launch_probe_elements(int nx, int ny, int col, int l, T* x, cudaStream_t s);
template <typename T> void launch_dense_symv(int n, const T* M, const T* x, T* y, cudaStream_t s);
void launch_band_chol_inverse(int n, int bw, const double* L, double* X, cudaStream_t s);
template <typename T> void launch_convert(size_t n, const double* a, T* b, cudaStream_t s);

// ---- krylov.cu
size_t reduction_workspace_doubles(int max_vectors);
template <typename T>
void launch_mdot(int m, size_t n, const T* V, size_t ldv, const T* w, double* out, double* ws,
                 cudaStream_t s);
template <typename T>
void launch_dot(size_t n, const T* x, const T* y, double* out, double* ws, cudaStream_t s);
template <typename T>
void launch_maxpy(int m, size_t n, const T* V, size_t ldv, const double* h, double sign, T* w,
                  cudaStream_t s);
template <typename T>
void launch_pcg_update(size_t n, const T* d, const T* q, T* y, T* r, const double* num,
                       const double* den, cudaStream_t s);
template <typename T>
void launch_pcg_dir(size_t n, const T* z, T* d, const double* num, const double* den,
                    cudaStream_t s);
template <typename T> void launch_axpby(size_t n, T a, const T* x, T b, T* y, cudaStream_t s);
template <typename T> void launch_scale_inv_sqrt(size_t n, const double* s2, T* v, cudaStream_t s);
template <typename T> void launch_vmul(size_t n, const T* x, const T* sc, T* y, cudaStream_t s);
template <typename Ti, typename To> void launch_cast(size_t n, const Ti* a, To* b, cudaStream_t s);
void launch_zero_mean_pressure(size_t ne, int mp, double* p, double* ws, cudaStream_t s);
void launch_splitmix_uniform(size_t n, uint64_t seed, double* out, cudaStream_t s);
// true when every entry is finite and positive (synchronises s)
bool eta_valid(size_t n, const double* eta, cudaStream_t s);

// ---- host helpers (solver.cu)
double hessenberg_max_real_eig(const std::vector<double>& H, int m);  // H: m x m row-major
// Cholesky of a symmetric band matrix (lower band storage A[i][bw-1-(i-j)]),
// in place; returns false if a pivot is not positive.
bool band_cholesky(std::vector<double>& A, int n, int bw);

// Small pinned host scratch for scalar read-backs.
struct HostScalars {
    double* p = nullptr;
    HostScalars();
    ~HostScalars();
};

template <typename T>
struct HLevel {
    int nx = 0, ny = 0;       // elements of this level's grid
    int nvx = 0, nvy = 0;     // vertices
    size_t n = 0;             // dofs = 2 nvx nvy
    DeviceBuffer S, dinv, b, x, r, d, d2;
    double lmax = 0.0;
};

template <typename T>
struct Multigrid {
    sip_problem* P = nullptr;
    int N = 0, nb = 0;
    size_t ne = 0, n_u = 0;
    // element-block Jacobi
    DeviceBuffer emap, uniq_list, n_uniq_d, cls_inv, uniq_inv, eta_T;
    DeviceBuffer cls_sym;   // reflection-symmetry type of each class block (sip_parity.cuh)
    int n_uniq = 0;
    double lmax_p = 0.0;
    // p-level work
    DeviceBuffer pb, pr, pd, pd2, r1, e1, vin, vout;
    // continuous hierarchy (h[0] = finest continuous level)
    std::vector<HLevel<T>> h;
    // coarsest direct solve (dense inverse)
    DeviceBuffer cinv;
    int nc = 0;
    // reductions
    DeviceBuffer ws, sc;
    HostScalars hs;
    DeviceBuffer cg_r, cg_d, cg_q;   // inner PCG vectors (outside the graph)
    // FP32 operator only: split-precision tiles (flags per tile, their list)
    DeviceBuffer hi_flag, hi_list, hi_scr;
    int n_hi = 0;
    // unique blocks whose face neighbour is much stiffer: applied in FP64 from
    // FP64 inverses (FP32 operator only)
    DeviceBuffer uniq_hi, uniq_inv64;
    const unsigned char* bj_hi() const { return n_hi > 0 ? uniq_hi.as<unsigned char>() : nullptr; }
    const double* bj_inv64() const { return n_hi > 0 ? uniq_inv64.as<double>() : nullptr; }
    // set-up scratch, kept so that a repeated set-up allocates nothing
    DeviceBuffer scr_V, scr_tmp, scr_b, scr_spec, scr_L, scr_X, scr_Y, scr_xv, scr_t1, scr_t2;
    std::vector<DeviceBuffer> scr_S64;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t graph_stream = nullptr;
    int64_t graph_kernels = 0;
    int setup_gen = 0;   // incremented by every set-up (graphs holding its kernels go stale)
    bool ready = false;

    ~Multigrid();
    void setup(cudaStream_t s);
    // z = V(r): one V-cycle of Algorithm 1 with y0 = 0 (r, z of length n_u)
    void vcycle(const T* r, T* z, cudaStream_t s);
    void vcycle_direct(cudaStream_t s);   // vin -> vout, kernels only
    void vcycle_on(const T* b, T* y, cudaStream_t s);   // b -> y, kernels only
    // z = V(r) for FP64 vectors: r rounded to T, the cycle in T, z widened
    void vcycle_widen(const double* r, double* z, cudaStream_t s);
    void bj(const T* r, T* z, cudaStream_t s);
    void coarse_solve(const T* b1, T* e1, cudaStream_t s);
    void hlevel_apply(int l, const T* x, T* y, cudaStream_t s);
    // choose fused or split p-level smoother steps by timing (tune.cu)
    void tune_smoother(cudaStream_t s);
    int inner_pcg(const T* t, T* y, double rtol, int maxit, cudaStream_t s, double* final_rel);
    int64_t bytes() const;

   private:
    // fused p-level smoother steps: available for N <= 4, chosen by the
    // schedule, and not overridden by SIP_APPLY_KERNEL=elem1 / tile
    bool use_fused() const;
    void smooth_p(const T* b, T* y, bool zero, cudaStream_t s);
    void hcycle(int l, cudaStream_t s);
    void smooth_h(int l, bool zero, cudaStream_t s);
    double estimate_p(cudaStream_t s);
    double estimate_h(int l, cudaStream_t s);
    void build_blocks(cudaStream_t s);
    void mark_split_tiles(cudaStream_t s);
    // r1 = R (b - A y) in one launch where a kernel for it exists
    bool residual_restrict(const T* y, const T* b, T* r1, cudaStream_t s);
    void build_coarse_from_band(const std::vector<double>& band, int n, int bw, cudaStream_t s);
};

// Graph-resident inner PCG (inner_graph.cu).
struct InnerLoop;
struct InnerLoopDeleter {
    void operator()(InnerLoop* p) const;
};

// FGMRES storage of one problem (FP64): Krylov basis V, flexible basis Z.
struct Workspace {
    int restart = 0;
    size_t n = 0;
    DeviceBuffer V, Z, w, x, r, b, tu, yu64, sinv, ws, sc, hbuf;
    DeviceBuffer cg_r, cg_d, cg_q, cg_z, sc_in;   // FP64 inner PCG of the mixed form
    DeviceBuffer gcr_z, gcr_q;                    // inner GCR directions [m][n_u] each
    DeviceBuffer t32, y32;                        // FP32 inner PCG (SIP_PREC_MIXED_F32_INNER)
    HostScalars hs, hs_in;
    std::unique_ptr<InnerLoop, InnerLoopDeleter> loop;
    bool sinv_ready = false;
    int64_t bytes() const;
};

// Pick the apply kernel of each precision the problem runs in by timing
// (tune.cu); cached per degree, precision and mesh.
void tune_apply(sip_problem* P, cudaStream_t s);

int inner_pcg_mixed(sip_problem* P, Workspace& W, const double* t, double* y, double rtol,
                    int maxit, cudaStream_t s);
// Batched inner solves (batch.cu): a group of problems whose solves run on
// host threads registered with one collector share one batched inner loop.
struct BatchCollector;
BatchCollector*& batch_collector();   // the calling thread's group (null: none)
// the inner solve through the group's rendezvous when the calling thread
// belongs to a group (*used = true), else nothing (*used = false)
int batched_inner(sip_problem* P, const double* t, double* y, cudaStream_t s, bool* used);
BatchCollector* make_collector(const std::vector<sip_problem*>& probs, bool mixed, double rtol,
                               int maxit);
void free_collector(BatchCollector* c);
void collector_leave(BatchCollector* c, sip_problem* P);
int64_t collector_rounds(const BatchCollector* c);

// The same inner solve (FP64 iterate; V-cycle in FP32 when mixed, else FP64)
// as one graph launch with a device-side loop; returns the iteration count.
// flexible: FCG(1) directions instead of PCG's; pnorm: stop on the
// preconditioned residual ||V r|| instead of ||r||; gcr_restart > 0: GCR
// restarted after that many directions (<= 64) instead of CG, stopping on
// ||r|| (flexible and pnorm are then ignored).
int inner_pcg_graph(sip_problem* P, Workspace& W, bool mixed, bool flexible, bool pnorm,
                    const double* t, double* y, double rtol, int maxit, cudaStream_t s,
                    int gcr_restart = 0);

sip_status run_solve(sip_problem* P, const double* f_u, const double* g_p, double* u,
                     double* p, const sip_solve_opts& o, sip_solve_report* rep,
                     cudaStream_t s);

// r = b - K x with b = [f; g] (g may be null: 0) and x, r in double-double
// (interleaved hi, lo pairs): velocity and pressure parts separately.
void residual_dd(sip_problem* P, const double* f_u, const double* g_p, const double* x_u,
                 const double* x_p, double* r_u, double* r_p, cudaStream_t s);

// Iterative refinement (o.refine > 0): FP64 / mixed solves of K d = r for
// the residual r = b - K x evaluated in double-double, x accumulated in
// double-double, until the residual meets o.rtol or stops halving.
// u, p (FP64, the iterate rounded) may be null; u_dd, p_dd (may be null)
// receive the double-double iterate as interleaved (hi, lo) pairs.
sip_status run_solve_refined(sip_problem* P, const double* f_u, const double* g_p, double* u,
                             double* p, const sip_solve_opts& o, sip_solve_report* rep,
                             cudaStream_t s, double* u_dd = nullptr, double* p_dd = nullptr);

// Throws Error(SIP_ERR_INVALID_ARG) unless the options are valid for a
// problem of this precision (every solve entry point checks them).
void require_valid_opts(const sip_solve_opts& o, int precision);
// Message of a solve's failing status.
const char* status_message(sip_status st);
// Device bytes of one problem solved with these options (admission).
int64_t estimate_problem_bytes(const sip_problem_desc& d, const sip_solve_opts& o);

// run_solve_refined when o.refine > 0, else run_solve (every entry point)
inline sip_status solve_dispatch(sip_problem* P, const double* f_u, const double* g_p, double* u,
                                 double* p, const sip_solve_opts& o, sip_solve_report* rep,
                                 cudaStream_t s) {
    return o.refine > 0 ? run_solve_refined(P, f_u, g_p, u, p, o, rep, s)
                        : run_solve(P, f_u, g_p, u, p, o, rep, s);
}

}  // namespace sip

struct sip_problem {
    sip_ctx* ctx = nullptr;
    sip_problem_desc desc{};
    int k = 0, n = 0, nb = 0, mp = 0;
    int64_t ne = 0, n_u = 0, n_p = 0;
    sip::OpGeom geom{};      // the SIP operator of degree k
    sip::OpGeom geom1{};     // the Galerkin Q_1 operator (fine-k penalty)
    std::vector<double> eta_host;
    sip::DeviceBuffer eta_d, eta_f, eta_inv_d, eta_inv_f;
    // refresh the FP32 copy and the FP64 / FP32 reciprocals of eta_d
    void derive_eta(cudaStream_t s);
    std::unique_ptr<sip::Multigrid<double>> mg64;
    std::unique_ptr<sip::Multigrid<float>> mg32;
    std::unique_ptr<sip::Workspace> ws;
    // iterative refinement: eta, x, K x, B x_p in double-double; residual and
    // correction in FP64; norm scratch and its pinned read-back (created on
    // first use, kept: freeing pinned memory would synchronise the device)
    sip::DeviceBuffer eta_dd, rf_x, rf_y, rf_t, rf_r, rf_d, rf_scr;
    std::unique_ptr<sip::HostScalars> rf_hs;
    double setup_ms = 0.0;
    // kernel schedule pinned by sip_problem_set_schedule ([0] FP64, [1] FP32):
    // apply 0 = autotuned, else sip_problem_schedule's code; fused -1 = autotuned
    int pin_apply[2] = {0, 0};
    int pin_fused[2] = {-1, -1};
    int64_t device_bytes() const;
    void ensure_setup(cudaStream_t s);
};
