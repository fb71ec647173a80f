// hp-multigrid set-up and cycle (Sec. 6, Algorithm 1), the inner PCG on the
// viscous block and the outer right-preconditioned FGMRES with the upper
// block-triangular preconditioner (Sec. 5).  Host code orchestrates device
// kernels; the V-cycle is captured once into a CUDA graph.
#include <algorithm>
#include <chrono>
#include <complex>
#include <cstdlib>
#include <cstring>

#include "dd.cuh"
#include "sip_solver.h"

namespace sip {

int64_t& launch_counter() {
    static thread_local int64_t n = 0;
    return n;
}

cudaStream_t& alloc_stream() {
    static thread_local cudaStream_t s = nullptr;
    return s;
}

bool& release_on_legacy() {
    static thread_local bool on = false;
    return on;
}

StopCtl& stop_ctl() {
    static thread_local StopCtl c;
    return c;
}

double steady_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

sip_status stop_requested() {
    const StopCtl& c = stop_ctl();
    if (c.cancel && *c.cancel) return SIP_ERR_CANCELLED;
    if (c.deadline_ms > 0.0 && steady_ms() > c.deadline_ms) return SIP_ERR_TIMEOUT;
    return SIP_OK;
}

bool& pdl_enabled() {
    static thread_local bool on = [] {
        const char* v = std::getenv("SIP_PDL");
        return !(v && std::string(v) == "0");
    }();
    return on;
}

namespace {

__global__ void k_splitmix(size_t n, uint64_t seed, double* out) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= n) return;
    // SplitMix64 (Steele, Lea & Flood 2014) as a counter-based hash
    uint64_t z = seed + (uint64_t(g) + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    out[g] = double(z >> 11) * 0x1.0p-52 - 1.0;
}

template <typename T>
const T* eta_of(sip_problem* P);
template <>
const double* eta_of<double>(sip_problem* P) { return P->eta_d.as<double>(); }
template <>
const float* eta_of<float>(sip_problem* P) { return P->eta_f.as<float>(); }
template <typename T>
const T* eta_inv_of(sip_problem* P);
template <>
const double* eta_inv_of<double>(sip_problem* P) { return P->eta_inv_d.as<double>(); }
template <>
const float* eta_inv_of<float>(sip_problem* P) { return P->eta_inv_f.as<float>(); }

// Chebyshev recurrence for SPD operators on [lo, hi] (Saad, Iterative
// Methods for Sparse Linear Systems, Sec. 12.3): coefficients of step s
// (s = 0 first update): d_s = c1 d_{s-1} + c2 M^{-1} r_s.
struct Cheb {
    double theta, delta, sigma;
    explicit Cheb(double lo, double hi)
        : theta(0.5 * (hi + lo)), delta(0.5 * (hi - lo)), sigma(theta / delta) {}
};

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

inline double read_scalar(const double* dev, double* host, cudaStream_t s) {
    SIP_CUDA(cudaMemcpyAsync(host, dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    SIP_CUDA(cudaStreamSynchronize(s));
    return *host;
}

}  // namespace

void launch_splitmix_uniform(size_t n, uint64_t seed, double* out, cudaStream_t s) {
    launch_k(k_splitmix, unsigned((n + 255) / 256), 256, 0, s, n, seed, out);
    SIP_CHECK_LAUNCH();
}

namespace {
__global__ void k_check_positive(size_t n, const double* v, int* bad) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g < n && !(isfinite(v[g]) && v[g] > 0.0)) atomicOr(bad, 1);
}
}  // namespace

bool eta_valid(size_t n, const double* eta, cudaStream_t s) {
    DeviceBuffer flag;
    flag.alloc(sizeof(int));
    SIP_CUDA(cudaMemsetAsync(flag.ptr, 0, sizeof(int), s));
    launch_k(k_check_positive, unsigned((n + 255) / 256), 256, 0, s, n, eta, flag.as<int>());
    SIP_CHECK_LAUNCH();
    int bad = 0;
    SIP_CUDA(cudaMemcpyAsync(&bad, flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    SIP_CUDA(cudaStreamSynchronize(s));
    return bad == 0;
}

// Pinned blocks for scalar read-backs come from a per-thread free list:
// pinned allocation synchronises the device, so it happens once per block
// and thread, never in a steady-state solve.
namespace {
struct PinnedPool {
    std::vector<double*> free_blocks;
    ~PinnedPool() {
        for (double* p : free_blocks) cudaFreeHost(p);
    }
};
PinnedPool& pinned_pool() {
    static thread_local PinnedPool pool;
    return pool;
}
}  // namespace

HostScalars::HostScalars() {
    auto& pool = pinned_pool();
    if (!pool.free_blocks.empty()) {
        p = pool.free_blocks.back();
        pool.free_blocks.pop_back();
        return;
    }
    if (cudaMallocHost(&p, 256 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        throw Error(SIP_ERR_OOM, "pinned host allocation failed");
    }
}
HostScalars::~HostScalars() {
    if (p) pinned_pool().free_blocks.push_back(p);
}

// ---------------------------------------------------------------- host math
// Eigenvalues of a small real upper Hessenberg matrix by the shifted QR
// algorithm in complex arithmetic (Wilkinson shifts, Givens rotations,
// deflation); returns the largest real part.
double hessenberg_max_real_eig(const std::vector<double>& Hin, int m) {
    using C = std::complex<double>;
    std::vector<C> A(size_t(m) * m);
    for (int i = 0; i < m * m; ++i) A[i] = Hin[i];
    auto at = [&](int i, int j) -> C& { return A[size_t(i) * m + j]; };
    std::vector<C> eig;
    int n = m;
    int guard = 0;
    while (n > 0) {
        if (n == 1) {
            eig.push_back(at(0, 0));
            break;
        }
        // deflation test on the last subdiagonal
        const double sub = std::abs(at(n - 1, n - 2));
        const double dia = std::abs(at(n - 1, n - 1)) + std::abs(at(n - 2, n - 2));
        if (sub <= 1e-15 * (dia > 0 ? dia : 1.0) || guard > 1000) {
            eig.push_back(at(n - 1, n - 1));
            --n;
            guard = 0;
            continue;
        }
        ++guard;
        // Wilkinson shift from the trailing 2x2 block
        const C a = at(n - 2, n - 2), b = at(n - 2, n - 1), c = at(n - 1, n - 2), d = at(n - 1, n - 1);
        const C tr = a + d, det = a * d - b * c;
        const C disc = std::sqrt(tr * tr - 4.0 * det);
        const C l1 = 0.5 * (tr + disc), l2 = 0.5 * (tr - disc);
        const C mu = std::abs(l1 - d) < std::abs(l2 - d) ? l1 : l2;
        for (int i = 0; i < n; ++i) at(i, i) -= mu;
        // QR by Givens rotations G_k acting on rows k, k+1; then RQ
        std::vector<C> cs(n - 1), sn(n - 1);
        for (int k = 0; k < n - 1; ++k) {
            const C x = at(k, k), y = at(k + 1, k);
            const double r = std::sqrt(std::norm(x) + std::norm(y));
            C cc = 1.0, ss = 0.0;
            if (r > 0) {
                cc = x / r;
                ss = y / r;
            }
            cs[k] = cc;
            sn[k] = ss;
            for (int j = k; j < n; ++j) {
                const C t1 = at(k, j), t2 = at(k + 1, j);
                at(k, j) = std::conj(cc) * t1 + std::conj(ss) * t2;
                at(k + 1, j) = -ss * t1 + cc * t2;
            }
        }
        for (int k = 0; k < n - 1; ++k) {
            const C cc = cs[k], ss = sn[k];
            for (int i = 0; i <= std::min(k + 1, n - 1); ++i) {
                const C t1 = at(i, k), t2 = at(i, k + 1);
                at(i, k) = t1 * cc + t2 * ss;
                at(i, k + 1) = -t1 * std::conj(ss) + t2 * std::conj(cc);
            }
        }
        for (int i = 0; i < n; ++i) at(i, i) += mu;
    }
    double best = -1e300;
    for (const C& e : eig) best = std::max(best, e.real());
    return best;
}

bool band_cholesky(std::vector<double>& A, int n, int bw) {
    auto L = [&](int i, int j) -> double& { return A[size_t(i) * bw + (bw - 1 - (i - j))]; };
    for (int j = 0; j < n; ++j) {
        const int k0 = std::max(0, j - bw + 1);
        double d = L(j, j);
        for (int k = k0; k < j; ++k) d -= L(j, k) * L(j, k);
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        L(j, j) = d;
        const int i1 = std::min(n - 1, j + bw - 1);
        for (int i = j + 1; i <= i1; ++i) {
            const int kk0 = std::max(k0, i - bw + 1);
            double s = L(i, j);
            for (int k = kk0; k < j; ++k) s -= L(i, k) * L(j, k);
            L(i, j) = s / d;
        }
    }
    return true;
}

// ---------------------------------------------------------------- multigrid
template <typename T>
Multigrid<T>::~Multigrid() {
    if (graph) cudaGraphExecDestroy(graph);
    if (graph_stream) cudaStreamDestroy(graph_stream);
}

template <typename T>
int64_t Multigrid<T>::bytes() const {
    int64_t b = int64_t(uniq_hi.bytes + uniq_inv64.bytes + hi_flag.bytes + hi_list.bytes +
                        emap.bytes + uniq_list.bytes + n_uniq_d.bytes + cls_inv.bytes +
                        uniq_inv.bytes + cls_sym.bytes + pb.bytes + pr.bytes + pd.bytes + pd2.bytes + r1.bytes + e1.bytes +
                        vin.bytes + vout.bytes + cinv.bytes + ws.bytes + sc.bytes + cg_r.bytes +
                        cg_d.bytes + cg_q.bytes);
    for (const auto& l : h)
        b += int64_t(l.S.bytes + l.dinv.bytes + l.b.bytes + l.x.bytes + l.r.bytes + l.d.bytes +
                     l.d2.bytes);
    return b;
}

template <typename T>
void Multigrid<T>::build_blocks(cudaStream_t s) {
    emap.alloc(ne * sizeof(int));
    uniq_list.alloc(ne * sizeof(int));
    n_uniq_d.alloc(sizeof(int));
    SIP_CUDA(cudaMemsetAsync(n_uniq_d.ptr, 0, sizeof(int), s));
    launch_classify(P->geom.nx, P->geom.ny, P->eta_d.as<double>(), emap.as<int>(),
                    uniq_list.as<int>(), n_uniq_d.as<int>(), s);
    int nu = 0;
    SIP_CUDA(cudaMemcpyAsync(&nu, n_uniq_d.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    SIP_CUDA(cudaStreamSynchronize(s));
    n_uniq = nu;
    std::vector<int> spec(16);
    for (int m = 0; m < 16; ++m) spec[m] = -(m + 1);
    DeviceBuffer& dspec = scr_spec;
    dspec.alloc(16 * sizeof(int));
    SIP_CUDA(cudaMemcpyAsync(dspec.ptr, spec.data(), 16 * sizeof(int), cudaMemcpyHostToDevice, s));
    cls_inv.alloc(size_t(16) * nb * nb * sizeof(T));
    launch_build_blocks<T>(N, P->geom, dspec.as<int>(), 16, P->eta_d.as<double>(), cls_inv.template as<T>(), s);
    uniq_inv.alloc(size_t(std::max(n_uniq, 1)) * nb * nb * sizeof(T));
    launch_build_blocks<T>(N, P->geom, uniq_list.as<int>(), n_uniq, P->eta_d.as<double>(),
                           uniq_inv.template as<T>(), s);
    // Reflection symmetry of each class block: x-faces of one kind (both
    // interior, or both boundary with the same condition) make the block
    // commute with x -> -x, likewise in y; confirmed on the computed inverse
    // (couplings between modes of different parity must vanish), else dense.
    const int NBl = nb;
    std::vector<T> ch(size_t(16) * NBl * NBl);
    SIP_CUDA(cudaMemcpyAsync(ch.data(), cls_inv.ptr, ch.size() * sizeof(T), cudaMemcpyDeviceToHost, s));
    SIP_CUDA(cudaStreamSynchronize(s));   // dspec is released on return
    std::vector<int> par(NBl), sym(16, 0);
    for (int q = 0; q < NBl; ++q) {
        const int c = q / (N * N), j = (q / N) % N, i = q % N;
        par[q] = ((i + (c == 0)) & 1) | (((j + (c == 1)) & 1) << 1);
    }
    const int* bc = P->geom.bc;
    for (int m = 0; m < 16; ++m) {
        const bool bl = m & 1, br = m & 2, bb = m & 4, bt = m & 8;
        const bool sx = bl == br && (!bl || bc[0] == bc[1]);
        const bool sy = bb == bt && (!bb || bc[2] == bc[3]);
        int t = (sx ? 1 : 0) | (sy ? 2 : 0);
        if (t) {
            const T* M = ch.data() + size_t(m) * NBl * NBl;
            double mx = 0.0, off = 0.0;
            for (int a = 0; a < NBl; ++a)
                for (int b2 = 0; b2 < NBl; ++b2) {
                    const double v = std::abs(double(M[size_t(a) * NBl + b2]));
                    mx = std::max(mx, v);
                    if ((par[a] & t) != (par[b2] & t)) off = std::max(off, v);
                }
            if (!(off <= 1e-10 * mx)) t = 0;
        }
        sym[m] = t;
    }
    cls_sym.alloc(16 * sizeof(int));
    SIP_CUDA(cudaMemcpyAsync(cls_sym.ptr, sym.data(), 16 * sizeof(int), cudaMemcpyHostToDevice, s));
    SIP_CUDA(cudaStreamSynchronize(s));   // sym is released on return
}

template <typename T>
void Multigrid<T>::bj(const T* r, T* z, cudaStream_t s) {
    launch_bj_apply<T>(N, int(ne), r, z, nullptr, emap.as<int>(), cls_inv.template as<T>(),
                       cls_sym.as<int>(), uniq_inv.template as<T>(),
                       eta_inv_of<T>(P), T(0), T(1), true, s, bj_hi(), bj_inv64());
}

// Arnoldi (GMRES) estimate of the largest eigenvalue of the preconditioned
// operator (Sec. 6): m steps from the normalised start vector V[0];
// classical Gram-Schmidt applied twice; largest real part of the Hessenberg
// eigenvalues.  Every step stays on the device (the projections and norms
// land in device memory, the normalisation divides by a device scalar); the
// Hessenberg matrix is read back once at the end, where the first
// (near-)breakdown truncates it exactly as a step-by-step loop would stop.
// `op(v, w)` writes w = M^{-1} A v.
namespace {
template <typename T, class Op>
double arnoldi_lmax(size_t n, int m, T* Vp, DeviceBuffer& hbuf, double* ws, HostScalars& hs,
                    Op op, cudaStream_t s) {
    // device layout: pass-1 projections [m][m+1], pass-2 projections [m][m+1],
    // squared norms [m + 1] (slot m: the start vector)
    const size_t np = size_t(m) * (m + 1);
    hbuf.alloc((2 * np + m + 1) * sizeof(double));
    double* H1 = hbuf.as<double>();
    double* H2 = H1 + np;
    double* Hn = H2 + np;
    launch_dot<T>(n, Vp, Vp, Hn + m, ws, s);
    launch_scale_inv_sqrt<T>(n, Hn + m, Vp, s);
    for (int j = 0; j < m; ++j) {
        T* w = Vp + size_t(j + 1) * n;
        op(Vp + size_t(j) * n, w);
        launch_mdot<T>(j + 1, n, Vp, n, w, H1 + size_t(j) * (m + 1), ws, s);
        launch_maxpy<T>(j + 1, n, Vp, n, H1 + size_t(j) * (m + 1), -1.0, w, s);
        launch_mdot<T>(j + 1, n, Vp, n, w, H2 + size_t(j) * (m + 1), ws, s);
        launch_maxpy<T>(j + 1, n, Vp, n, H2 + size_t(j) * (m + 1), -1.0, w, s);
        launch_dot<T>(n, w, w, Hn + j, ws, s);
        if (j + 1 < m) launch_scale_inv_sqrt<T>(n, Hn + j, w, s);
    }
    std::vector<double> hh(2 * np + m + 1);
    SIP_CUDA(cudaMemcpyAsync(hh.data(), H1, hh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    SIP_CUDA(cudaStreamSynchronize(s));
    (void)hs;
    std::vector<double> H(size_t(m + 1) * m, 0.0);
    int size = m;
    for (int j = 0; j < m; ++j) {
        for (int i = 0; i <= j; ++i)
            H[size_t(i) * m + j] = hh[size_t(j) * (m + 1) + i] + hh[np + size_t(j) * (m + 1) + i];
        const double hn = std::sqrt(hh[2 * np + j]);
        if (j + 1 < m) H[size_t(j + 1) * m + j] = hn;
        if (!(hn > 1e-14 * std::abs(H[size_t(j) * m + j]))) {
            size = j + 1;
            break;
        }
    }
    std::vector<double> Hs(size_t(size) * size);
    for (int i = 0; i < size; ++i)
        for (int j = 0; j < size; ++j) Hs[size_t(i) * size + j] = H[size_t(i) * m + j];
    return hessenberg_max_real_eig(Hs, size);
}
}  // namespace

template <typename T>
double Multigrid<T>::estimate_p(cudaStream_t s) {
    const int m = std::max(1, std::min<int>(P->desc.eig_iters, int(n_u)));
    DeviceBuffer &V = scr_V, &tmp = scr_tmp, &b64 = scr_b;
    V.alloc(size_t(m + 1) * n_u * sizeof(T));
    tmp.alloc(n_u * sizeof(T));
    b64.alloc(n_u * sizeof(double));
    T* Vp = V.template as<T>();
    launch_splitmix_uniform(n_u, P->desc.seed, b64.as<double>(), s);
    launch_cast<double, T>(n_u, b64.as<double>(), tmp.template as<T>(), s);
    bj(tmp.template as<T>(), Vp, s);
    return arnoldi_lmax<T>(n_u, m, Vp, scr_t2, ws.as<double>(), hs,
                           [&](const T* v, T* w) {
                               launch_apply_sip<T>(N, P->geom, v, tmp.template as<T>(), eta_of<T>(P),
                                                   T(1), nullptr, T(0), s);
                               bj(tmp.template as<T>(), w, s);
                           },
                           s);
}

template <typename T>
double Multigrid<T>::estimate_h(int l, cudaStream_t s) {
    HLevel<T>& L = h[l];
    const size_t n = L.n;
    const int m = std::max(1, std::min<int>(P->desc.eig_iters, int(n)));
    DeviceBuffer &V = scr_V, &tmp = scr_tmp, &b64 = scr_b;
    V.alloc(size_t(m + 1) * n * sizeof(T));
    tmp.alloc(n * sizeof(T));
    b64.alloc(n * sizeof(double));
    T* Vp = V.template as<T>();
    launch_splitmix_uniform(n, P->desc.seed + 1 + uint64_t(l), b64.as<double>(), s);
    launch_cast<double, T>(n, b64.as<double>(), tmp.template as<T>(), s);
    launch_vmul<T>(n, tmp.template as<T>(), L.dinv.template as<T>(), Vp, s);
    return arnoldi_lmax<T>(n, m, Vp, scr_t2, ws.as<double>(), hs,
                           [&](const T* v, T* w) {
                               launch_stencil_apply<T>(L.nvx, L.nvy, L.S.template as<T>(), v,
                                                       tmp.template as<T>(), T(1), nullptr, T(0), s);
                               launch_vmul<T>(n, tmp.template as<T>(), L.dinv.template as<T>(), w, s);
                           },
                           s);
}

template <typename T>
void Multigrid<T>::build_coarse_from_band(const std::vector<double>& band_in, int n, int bw,
                                          cudaStream_t s) {
    std::vector<double> band = band_in;
    if (!band_cholesky(band, n, bw))
        throw Error(SIP_ERR_BREAKDOWN, "coarsest operator is not positive definite");
    DeviceBuffer &Ld = scr_L, &X = scr_X;
    Ld.alloc(band.size() * sizeof(double));
    X.alloc(size_t(n) * n * sizeof(double));
    SIP_CUDA(cudaMemcpyAsync(Ld.ptr, band.data(), band.size() * sizeof(double),
                             cudaMemcpyHostToDevice, s));
    launch_band_chol_inverse(n, bw, Ld.as<double>(), X.as<double>(), s);
    cinv.alloc(size_t(n) * n * sizeof(T));
    launch_convert<T>(size_t(n) * n, X.as<double>(), cinv.template as<T>(), s);
    nc = n;
    SIP_CUDA(cudaStreamSynchronize(s));
}

// Mixed form: the FP32 operator evaluates the tiles near elements with
// eta >= ratio x min(eta) in FP64 arithmetic (apply_stage.cu; for k = 6,
// which has no staged kernel, the whole operator: apply.cu); the FP64
// operator has no such tiles.
template <typename T>
void Multigrid<T>::mark_split_tiles(cudaStream_t s) {
    n_hi = 0;
    const double ratio = P->desc.mixed_fp64_ratio;
    if (sizeof(T) == 4 && ratio > 0.0) {
        const int nt = split_tile_count(P->desc.nx, P->desc.ny);
        hi_flag.alloc(size_t(nt));
        hi_list.alloc(size_t(nt) * sizeof(int));
        hi_scr.alloc(32);
        n_hi = mark_hi_tiles(P->desc.nx, P->desc.ny, P->eta_d.as<double>(), ratio,
                             hi_flag.as<unsigned char>(), hi_list.as<int>(), hi_scr.as<int>(), s);
        if (n_hi > 0) {
            split_fork_prepare();   // the side stream, before any graph capture
            // FP32 sums of an element block whose face neighbour is much
            // stiffer cancel the block's small components the same way
            uniq_hi.alloc(size_t(std::max(n_uniq, 1)));
            launch_mark_uniq_hi(P->desc.nx, P->desc.ny, uniq_list.as<int>(), n_uniq_d.as<int>(),
                                n_uniq, P->eta_d.as<double>(), std::max(1.0, 0.1 * ratio),
                                uniq_hi.as<unsigned char>(), s);
            // their inverses are also kept in FP64 (an ill-conditioned inverse
            // rounded to FP32 is wrong along its stiff directions)
            uniq_inv64.alloc(size_t(std::max(n_uniq, 1)) * nb * nb * sizeof(double));
            launch_build_blocks<double>(N, P->geom, uniq_list.as<int>(), n_uniq,
                                        P->eta_d.as<double>(), uniq_inv64.as<double>(), s);
        }
    }
    if (sizeof(T) == 4) {
        P->geom.n_hi = n_hi;
        P->geom.hi_flag = n_hi > 0 ? hi_flag.as<unsigned char>() : nullptr;
        P->geom.hi_tiles = n_hi > 0 ? hi_list.as<int>() : nullptr;
    }
}

template <typename T>
bool Multigrid<T>::residual_restrict(const T* y, const T* b, T* r1, cudaStream_t s) {
    const bool split = sizeof(T) == 4 && P->geom.n_hi > 0;
    if (split || apply_variant<T>(P->geom) == APPLY_STAGE)
        return launch_apply_sip_stage<T>(N, P->geom, y, nullptr, eta_of<T>(P), T(-1), b, T(1), r1,
                                         s);
    return use_fused() && launch_residual_restrict_elem<T>(N, P->geom, y, b, eta_of<T>(P), r1, s);
}

template <typename T>
void Multigrid<T>::setup(cudaStream_t s) {
    const sip_problem_desc& d = P->desc;
    N = P->n;
    nb = P->nb;
    ne = size_t(P->ne);
    n_u = size_t(P->n_u);
    const int nx = d.nx, ny = d.ny;
    ws.alloc(reduction_workspace_doubles(128) * sizeof(double));
    sc.alloc(256 * sizeof(double));
    pb.alloc(n_u * sizeof(T));
    pr.alloc(n_u * sizeof(T));
    pd.alloc(n_u * sizeof(T));
    if (cheb_elem_available(N)) pd2.alloc(n_u * sizeof(T));
    vin.alloc(n_u * sizeof(T));
    vout.alloc(n_u * sizeof(T));
    r1.alloc(ne * 8 * sizeof(T));
    e1.alloc(ne * 8 * sizeof(T));
    cg_r.alloc(n_u * sizeof(T));
    cg_d.alloc(n_u * sizeof(T));
    cg_q.alloc(n_u * sizeof(T));
    build_blocks(s);
    mark_split_tiles(s);
    lmax_p = estimate_p(s);
    tune_smoother(s);

    const OpGeom& g1 = P->geom1;
    const bool q0 = d.coarse == SIP_COARSE_Q0;
    if (d.n_hlevels == 0 && !q0) {
        // A_p(Q^2_1): the coarse problem A_1 = P^T A P itself, by probing with
        // 9 element colours x 8 local dofs, then a band Cholesky.
        const int n1 = int(ne * 8);
        if (n1 > 65536)
            throw Error(SIP_ERR_INVALID_ARG,
                        "A_p(Q^2_1) coarse direct solve limited to 8192 elements; use n_hlevels > 0");
        const int bw = 8 * nx + 8;
        std::vector<double> band(size_t(n1) * bw, 0.0);
        DeviceBuffer &x = scr_t1, &y = scr_t2;
        x.alloc(size_t(n1) * sizeof(double));
        y.alloc(size_t(n1) * sizeof(double));
        std::vector<double> yh(n1);
        for (int col = 0; col < 9; ++col)
            for (int l = 0; l < 8; ++l) {
                launch_probe_elements<double>(nx, ny, col, l, x.as<double>(), s);
                launch_apply_sip<double>(2, g1, x.as<double>(), y.as<double>(), P->eta_d.as<double>(),
                                         1.0, nullptr, 0.0, s);
                SIP_CUDA(cudaMemcpyAsync(yh.data(), y.ptr, n1 * sizeof(double), cudaMemcpyDeviceToHost, s));
                SIP_CUDA(cudaStreamSynchronize(s));
                for (int ey = col / 3; ey < ny; ey += 3)
                    for (int ex = col % 3; ex < nx; ex += 3) {
                        const int e = ey * nx + ex;
                        const int cdof = 8 * e + l;
                        const int nbr[5] = {e, ex > 0 ? e - 1 : -1, ex < nx - 1 ? e + 1 : -1,
                                            ey > 0 ? e - nx : -1, ey < ny - 1 ? e + nx : -1};
                        for (int q = 0; q < 5; ++q) {
                            if (nbr[q] < 0) continue;
                            for (int rl = 0; rl < 8; ++rl) {
                                const int rdof = 8 * nbr[q] + rl;
                                if (rdof >= cdof && rdof - cdof < bw)
                                    band[size_t(rdof) * bw + (bw - 1 - (rdof - cdof))] = yh[rdof];
                            }
                        }
                    }
            }
        build_coarse_from_band(band, n1, bw, s);
    } else {
        // vertex-grid levels: level 0 = A_1c = P_cd^T A_1 P_cd on the mesh
        // vertices (Q^2_1), or A_0 = P_0^T A P_0 on the element centres
        // (Q^2_0, an (nx-1) x (ny-1) grid of intervals); then Galerkin
        // P_h^T A_l P_h; stencils formed in FP64 by probing with 9 vertex
        // colours x 2 components.  With Q^2_0 and no coarsening, level 0 is
        // the coarsest and is solved directly (A_p(Q^2_0)).
        const int L = d.n_hlevels;
        h.resize(L + 1);
        std::vector<DeviceBuffer>& S64 = scr_S64;
        S64.resize(L + 1);
        const int gx = q0 ? nx - 1 : nx, gy = q0 ? ny - 1 : ny;
        for (int l = 0; l <= L; ++l) {
            h[l].nx = gx >> l;
            h[l].ny = gy >> l;
            h[l].nvx = h[l].nx + 1;
            h[l].nvy = h[l].ny + 1;
            h[l].n = size_t(2) * h[l].nvx * h[l].nvy;
        }
        for (int l = 0; l <= L; ++l) {
            HLevel<T>& Lv = h[l];
            const size_t nv = size_t(Lv.nvx) * Lv.nvy;
            DeviceBuffer &Y = scr_Y, &xv = scr_xv;
            Y.alloc(size_t(18) * Lv.n * sizeof(double));
            xv.alloc(Lv.n * sizeof(double));
            DeviceBuffer &t1 = scr_t1, &t2 = scr_t2;
            if (l == 0) {
                t1.alloc((q0 ? n_u : ne * 8) * sizeof(double));
                t2.alloc((q0 ? n_u : ne * 8) * sizeof(double));
            } else {
                t1.alloc(h[l - 1].n * sizeof(double));
                t2.alloc(h[l - 1].n * sizeof(double));
            }
            for (int col = 0; col < 9; ++col)
                for (int cp = 0; cp < 2; ++cp) {
                    double* y = Y.as<double>() + size_t(col * 2 + cp) * Lv.n;
                    launch_probe_vertices<double>(Lv.nvx, Lv.nvy, col, cp, xv.as<double>(), s);
                    if (l == 0 && q0) {
                        SIP_CUDA(cudaMemsetAsync(t1.ptr, 0, n_u * sizeof(double), s));
                        launch_p_prolong_add<double>(ne, N, xv.as<double>(), t1.as<double>(), s, 1);
                        launch_apply_sip<double>(N, P->geom, t1.as<double>(), t2.as<double>(),
                                                 P->eta_d.as<double>(), 1.0, nullptr, 0.0, s);
                        launch_p_restrict<double>(ne, N, t2.as<double>(), y, s, 1);
                    } else if (l == 0) {
                        launch_pcd<double>(nx, ny, xv.as<double>(), t1.as<double>(), s);
                        launch_apply_sip<double>(2, g1, t1.as<double>(), t2.as<double>(),
                                                 P->eta_d.as<double>(), 1.0, nullptr, 0.0, s);
                        launch_rdc<double>(nx, ny, t2.as<double>(), y, s);
                    } else {
                        const HLevel<T>& F = h[l - 1];
                        SIP_CUDA(cudaMemsetAsync(t1.ptr, 0, F.n * sizeof(double), s));
                        launch_ph_add<double>(Lv.nx, Lv.ny, xv.as<double>(), t1.as<double>(), s);
                        launch_stencil_apply<double>(F.nvx, F.nvy, S64[l - 1].as<double>(),
                                                     t1.as<double>(), t2.as<double>(), 1.0, nullptr,
                                                     0.0, s);
                        launch_rh<double>(Lv.nx, Lv.ny, t2.as<double>(), y, s);
                    }
                }
            S64[l].alloc(nv * 36 * sizeof(double));
            launch_extract_stencil<double>(Lv.nvx, Lv.nvy, Y.as<double>(), S64[l].as<double>(), s);
            Lv.S.alloc(nv * 36 * sizeof(T));
            launch_convert<T>(nv * 36, S64[l].as<double>(), Lv.S.template as<T>(), s);
            Lv.dinv.alloc(Lv.n * sizeof(T));
            launch_stencil_dinv<T>(nv, Lv.S.template as<T>(), Lv.dinv.template as<T>(), s);
            for (DeviceBuffer* b : {&Lv.b, &Lv.x, &Lv.r, &Lv.d, &Lv.d2}) b->alloc(Lv.n * sizeof(T));
            SIP_CUDA(cudaStreamSynchronize(s));
        }
        for (int l = 0; l < L; ++l) h[l].lmax = estimate_h(l, s);
        // coarsest level: band Cholesky of the stencil matrix, dof 2 v + c
        HLevel<T>& C = h[L];
        const int n = int(C.n);
        const int bw = 2 * C.nvx + 4;
        std::vector<double> Sh(size_t(C.nvx) * C.nvy * 36);
        SIP_CUDA(cudaMemcpyAsync(Sh.data(), S64[L].ptr, Sh.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, s));
        SIP_CUDA(cudaStreamSynchronize(s));
        std::vector<double> band(size_t(n) * bw, 0.0);
        for (int vy = 0; vy < C.nvy; ++vy)
            for (int vx = 0; vx < C.nvx; ++vx) {
                const int v = vy * C.nvx + vx;
                for (int t = 0; t < 9; ++t) {
                    const int wx = vx + t % 3 - 1, wy = vy + t / 3 - 1;
                    if (wx < 0 || wx >= C.nvx || wy < 0 || wy >= C.nvy) continue;
                    const int w = wy * C.nvx + wx;
                    for (int c = 0; c < 2; ++c)
                        for (int cp = 0; cp < 2; ++cp) {
                            const int i = 2 * v + c, j = 2 * w + cp;
                            if (i >= j && i - j < bw)
                                band[size_t(i) * bw + (bw - 1 - (i - j))] =
                                    Sh[size_t(v) * 36 + t * 4 + c * 2 + cp];
                        }
                }
            }
        build_coarse_from_band(band, n, bw, s);
    }

    ++setup_gen;
    // capture the V-cycle (vin -> vout) once
    if (graph) {
        SIP_CUDA(cudaGraphExecDestroy(graph));
        graph = nullptr;
    }
    if (!graph_stream) SIP_CUDA(cudaStreamCreateWithFlags(&graph_stream, cudaStreamNonBlocking));
    SIP_CUDA(cudaStreamSynchronize(s));
    const int64_t before = launch_counter();
    SIP_CUDA(cudaStreamBeginCapture(graph_stream, cudaStreamCaptureModeThreadLocal));
    try {
        vcycle_direct(graph_stream);
    } catch (...) {
        cudaGraph_t gtmp;
        cudaStreamEndCapture(graph_stream, &gtmp);
        if (gtmp) cudaGraphDestroy(gtmp);
        throw;
    }
    cudaGraph_t gr;
    SIP_CUDA(cudaStreamEndCapture(graph_stream, &gr));
    graph_kernels = launch_counter() - before;
    launch_counter() = before;
    SIP_CUDA(cudaGraphInstantiate(&graph, gr, 0));
    cudaGraphDestroy(gr);
    ready = true;
}

template <typename T>
bool Multigrid<T>::use_fused() const {
    static const bool env_off = [] {
        const char* v = std::getenv("SIP_APPLY_KERNEL");
        return v && (std::string(v) == "elem1" || std::string(v) == "tile");
    }();
    // SIP_FUSED_SMOOTHER=0 / 1 pins the choice (profiling runs, where timings
    // taken under the profiler would mislead the autotuner)
    static const int forced = [] {
        const char* v = std::getenv("SIP_FUSED_SMOOTHER");
        return v ? (std::string(v) == "1" ? 1 : 0) : -1;
    }();
    if (env_off || !pd2.ptr || !cheb_elem_available(N)) return false;
    // the fused step evaluates the operator in T everywhere
    if (sizeof(T) == 4 && P->geom.n_hi > 0) return false;
    if (forced >= 0) return forced == 1;
    return P->geom.fused[sizeof(T) == 4 ? 1 : 0] != 0;
}

template <typename T>
void Multigrid<T>::smooth_p(const T* b, T* y, bool zero, cudaStream_t s) {
    const Cheb ch(P->desc.cheb_lo * lmax_p, P->desc.cheb_hi * lmax_p);
    T* r = pr.template as<T>();
    T* dd = pd.template as<T>();
    const T* eta = eta_of<T>(P);
    const T* einv0 = eta_inv_of<T>(P);
    const int steps = P->desc.cheb_steps_p;
    // fused path (N <= 4): each step after the first is one launch
    //   r = z - A d, d' = c1 d + c2 M^{-1} r, y += d'   (directions ping-pong);
    // from a non-zero y the first step only forms r = b - A y and d, and
    // its y update is deferred into the next launch (x = y cannot be
    // written while neighbours read it).
    if (steps >= 2 && use_fused()) {
        T* dA = dd;
        T* dB = pd2.template as<T>();
        bool pend = false;
        const int* em = emap.as<int>();
        const T* ci = cls_inv.template as<T>();
        const T* ui = uniq_inv.template as<T>();
        const int* cs = cls_sym.as<int>();
        if (zero) {
            // d = c2 M^{-1} b, y = d; the next step's residual is b - A d
            launch_bj_apply<T>(N, int(ne), b, dA, y, em, ci, cs, ui, einv0, T(0), T(1.0 / ch.theta),
                               true, s, bj_hi(), bj_inv64());
        } else {
            launch_cheb_elem<T>(N, P->geom, y, b, r, eta, em, ci, cs, ui, einv0, nullptr, dA, nullptr,
                                T(0), T(1.0 / ch.theta), false, s);
            pend = true;
        }
        const T* zsrc = zero ? b : r;
        double rho = 1.0 / ch.sigma;
        for (int st = 1; st < steps; ++st) {
            const double rn = 1.0 / (2.0 * ch.sigma - rho);
            launch_cheb_elem<T>(N, P->geom, dA, zsrc, r, eta, em, ci, cs, ui, einv0, dA, dB, y,
                                T(rn * rho), T(2.0 * rn / ch.delta), pend, s);
            pend = false;
            std::swap(dA, dB);
            zsrc = r;
            rho = rn;
        }
        return;
    }
    if (zero)
        launch_axpby<T>(n_u, T(1), b, T(0), r, s);
    else
        launch_apply_sip<T>(N, P->geom, y, r, eta, T(-1), b, T(1), s);   // r = b - A y
    double rho = 1.0 / ch.sigma;
    const T* einv = eta_inv_of<T>(P);
    launch_bj_apply<T>(N, int(ne), r, dd, y, emap.as<int>(), cls_inv.template as<T>(),
                       cls_sym.as<int>(), uniq_inv.template as<T>(), einv,
                       T(0), T(1.0 / ch.theta), zero, s, bj_hi(), bj_inv64());
    for (int st = 1; st < P->desc.cheb_steps_p; ++st) {
        launch_apply_sip<T>(N, P->geom, dd, r, eta, T(-1), r, T(1), s);  // r -= A d
        const double rn = 1.0 / (2.0 * ch.sigma - rho);
        launch_bj_apply<T>(N, int(ne), r, dd, y, emap.as<int>(), cls_inv.template as<T>(),
                           cls_sym.as<int>(), uniq_inv.template as<T>(),
                           einv, T(rn * rho), T(2.0 * rn / ch.delta), false, s, bj_hi(),
                           bj_inv64());
        rho = rn;
    }
}

template <typename T>
void Multigrid<T>::smooth_h(int l, bool zero, cudaStream_t s) {
    HLevel<T>& L = h[l];
    const Cheb ch(P->desc.cheb_lo * L.lmax, P->desc.cheb_hi * L.lmax);
    T* r = L.r.template as<T>();
    T* dA = L.d.template as<T>();    // Chebyshev directions, ping-pong
    T* dB = L.d2.template as<T>();
    T* x = L.x.template as<T>();
    const T* b = L.b.template as<T>();
    const T* S = L.S.template as<T>();
    const T* dinv = L.dinv.template as<T>();
    const int steps = P->desc.cheb_steps_h;
    bool pend = false;
    if (zero) {
        launch_hcheb_first<T>(L.n, b, dinv, r, dA, x, T(1.0 / ch.theta), s);
    } else if (steps >= 2) {
        // r = b - A x, d = c2 D^{-1} r; x += d deferred to the next step
        launch_hcheb_start<T>(L.nvx, L.nvy, S, dinv, b, x, r, dA, T(1.0 / ch.theta), s);
        pend = true;
    } else {
        launch_stencil_apply<T>(L.nvx, L.nvy, S, x, r, T(-1), b, T(1), s);   // r = b - A x
        launch_jacobi_cheb<T>(L.n, r, dinv, dA, x, T(0), T(1.0 / ch.theta), false, s);
    }
    double rho = 1.0 / ch.sigma;
    for (int st = 1; st < steps; ++st) {
        const double rn = 1.0 / (2.0 * ch.sigma - rho);
        launch_hcheb_step<T>(L.nvx, L.nvy, S, dinv, r, dA, dB, x, T(rn * rho),
                             T(2.0 * rn / ch.delta), pend, s);
        pend = false;
        std::swap(dA, dB);
        rho = rn;
    }
}

template <typename T>
void Multigrid<T>::hcycle(int l, cudaStream_t s) {
    const int L = int(h.size()) - 1;
    HLevel<T>& Lv = h[l];
    if (l == L) {
        launch_dense_symv<T>(nc, cinv.template as<T>(), Lv.b.template as<T>(), Lv.x.template as<T>(), s);
        return;
    }
    smooth_h(l, true, s);
    launch_stencil_apply<T>(Lv.nvx, Lv.nvy, Lv.S.template as<T>(), Lv.x.template as<T>(), Lv.r.template as<T>(), T(-1),
                            Lv.b.template as<T>(), T(1), s);
    HLevel<T>& C = h[l + 1];
    launch_rh<T>(C.nx, C.ny, Lv.r.template as<T>(), C.b.template as<T>(), s);
    hcycle(l + 1, s);
    launch_ph_add<T>(C.nx, C.ny, C.x.template as<T>(), Lv.x.template as<T>(), s);
    smooth_h(l, false, s);
}

template <typename T>
void Multigrid<T>::coarse_solve(const T* b1, T* x1, cudaStream_t s) {
    if (P->desc.coarse == SIP_COARSE_Q0) {   // b1, x1: 2 constants per element
        SIP_CUDA(cudaMemcpyAsync(h[0].b.ptr, b1, h[0].n * sizeof(T), cudaMemcpyDeviceToDevice, s));
        hcycle(0, s);
        SIP_CUDA(cudaMemcpyAsync(x1, h[0].x.ptr, h[0].n * sizeof(T), cudaMemcpyDeviceToDevice, s));
        return;
    }
    if (h.empty()) {
        launch_dense_symv<T>(nc, cinv.template as<T>(), b1, x1, s);
        return;
    }
    const int nx = P->desc.nx, ny = P->desc.ny;
    launch_rdc<T>(nx, ny, b1, h[0].b.template as<T>(), s);
    hcycle(0, s);
    launch_pcd<T>(nx, ny, h[0].x.template as<T>(), x1, s);
}

template <typename T>
void Multigrid<T>::vcycle_direct(cudaStream_t s) {
    vcycle_on(vin.template as<T>(), vout.template as<T>(), s);
}

template <typename T>
void Multigrid<T>::vcycle_on(const T* b, T* y, cudaStream_t s) {
    smooth_p(b, y, true, s);
    if (P->desc.coarse == SIP_COARSE_Q0) {
        // coarse correction on the element-wise constants: the residual's
        // (0,0) modes are the finest vertex-grid level's right-hand side
        launch_apply_sip<T>(N, P->geom, y, pr.template as<T>(), eta_of<T>(P), T(-1), b, T(1), s);
        launch_p_restrict<T>(ne, N, pr.template as<T>(), h[0].b.template as<T>(), s, 1);
        hcycle(0, s);
        launch_p_prolong_add<T>(ne, N, h[0].x.template as<T>(), y, s, 1);
        smooth_p(b, y, false, s);
        return;
    }
    // r1 = R (b - A y)
    if (!residual_restrict(y, b, r1.template as<T>(), s)) {
        launch_apply_sip<T>(N, P->geom, y, pr.template as<T>(), eta_of<T>(P), T(-1), b, T(1), s);
        launch_p_restrict<T>(ne, N, pr.template as<T>(), r1.template as<T>(), s);
    }
    coarse_solve(r1.template as<T>(), e1.template as<T>(), s);
    launch_p_prolong_add<T>(ne, N, e1.template as<T>(), y, s);
    smooth_p(b, y, false, s);
}

template <typename T>
void Multigrid<T>::vcycle(const T* r, T* z, cudaStream_t s) {
    if (r != vin.template as<T>())
        SIP_CUDA(cudaMemcpyAsync(vin.ptr, r, n_u * sizeof(T), cudaMemcpyDeviceToDevice, s));
    SIP_CUDA(cudaGraphLaunch(graph, s));
    launch_counter() += graph_kernels;
    if (z != vout.template as<T>())
        SIP_CUDA(cudaMemcpyAsync(z, vout.ptr, n_u * sizeof(T), cudaMemcpyDeviceToDevice, s));
}

template <typename T>
void Multigrid<T>::hlevel_apply(int l, const T* x, T* y, cudaStream_t s) {
    launch_stencil_apply<T>(h[l].nvx, h[l].nvy, h[l].S.template as<T>(), x, y, T(1), nullptr, T(0), s);
}

// PCG on A y = t from y = 0, preconditioned by the V-cycle; stops when
// ||t - A y|| < rtol ||t||.  Scalars alpha, beta stay on the device; one
// host read-back (the residual norm) per iteration.
template <typename T>
int Multigrid<T>::inner_pcg(const T* t, T* y, double rtol, int maxit, cudaStream_t s,
                            double* final_rel) {
    T* r = cg_r.template as<T>();
    T* dd = cg_d.template as<T>();
    T* q = cg_q.template as<T>();
    T* z = vout.template as<T>();
    double* scd = sc.as<double>();   // [0] rz, [1] dq, [2] rr, [3] rz_new
    double* wsd = ws.as<double>();
    const T* eta = eta_of<T>(P);
    SIP_CUDA(cudaMemsetAsync(y, 0, n_u * sizeof(T), s));
    launch_dot<T>(n_u, t, t, scd + 2, wsd, s);
    const double nt = std::sqrt(read_scalar(scd + 2, hs.p, s));
    if (final_rel) *final_rel = 0.0;
    if (nt == 0.0) return 0;
    if (!std::isfinite(nt)) throw Error(SIP_ERR_BREAKDOWN, "non-finite inner right-hand side");
    launch_axpby<T>(n_u, T(1), t, T(0), r, s);
    vcycle(r, z, s);
    launch_dot<T>(n_u, r, z, scd + 0, wsd, s);
    launch_axpby<T>(n_u, T(1), z, T(0), dd, s);
    int it = 0;
    for (it = 1; it <= maxit; ++it) {
        launch_apply_sip<T>(N, P->geom, dd, q, eta, T(1), nullptr, T(0), s);
        launch_dot<T>(n_u, dd, q, scd + 1, wsd, s);
        launch_pcg_update<T>(n_u, dd, q, y, r, scd + 0, scd + 1, s);
        launch_dot<T>(n_u, r, r, scd + 2, wsd, s);
        const double rr = std::sqrt(read_scalar(scd + 2, hs.p, s));
        if (!std::isfinite(rr)) throw Error(SIP_ERR_BREAKDOWN, "non-finite inner residual");
        if (final_rel) *final_rel = rr / nt;
        if (rr < rtol * nt) break;
        if (it == maxit) break;
        vcycle(r, z, s);
        launch_dot<T>(n_u, r, z, scd + 3, wsd, s);
        launch_pcg_dir<T>(n_u, z, dd, scd + 3, scd + 0, s);
        SIP_CUDA(cudaMemcpyAsync(scd + 0, scd + 3, sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    return std::min(it, maxit);
}

template <typename T>
void Multigrid<T>::vcycle_widen(const double* r, double* z, cudaStream_t s) {
    launch_cast<double, T>(n_u, r, vin.template as<T>(), s);
    SIP_CUDA(cudaGraphLaunch(graph, s));
    launch_counter() += graph_kernels;
    launch_cast<T, double>(n_u, vout.template as<T>(), z, s);
}

template struct Multigrid<double>;
template struct Multigrid<float>;

// Inner PCG of the mixed form: FP64 iterate, residual, operator and dot
// products; the V-cycle (smoother, transfers, coarse solve) in FP32, the
// residual rounded to FP32 on the way in and the correction widened on the
// way out.  Same stopping test as the FP64 form.
int inner_pcg_mixed(sip_problem* P, Workspace& W, const double* t, double* y, double rtol,
                    int maxit, cudaStream_t s) {
    Multigrid<float>& mg = *P->mg32;
    const size_t n_u = size_t(P->n_u);
    double* r = W.cg_r.as<double>();
    double* dd = W.cg_d.as<double>();
    double* q = W.cg_q.as<double>();
    double* z = W.cg_z.as<double>();
    double* scd = W.sc_in.as<double>();   // [0] rz, [1] dq, [2] rr, [3] rz_new
    double* wsd = W.ws.as<double>();
    double* hp = W.hs_in.p;
    const double* eta = P->eta_d.as<double>();
    SIP_CUDA(cudaMemsetAsync(y, 0, n_u * sizeof(double), s));
    launch_dot<double>(n_u, t, t, scd + 2, wsd, s);
    const double nt = std::sqrt(read_scalar(scd + 2, hp, s));
    if (nt == 0.0) return 0;
    if (!std::isfinite(nt)) throw Error(SIP_ERR_BREAKDOWN, "non-finite inner right-hand side");
    launch_axpby<double>(n_u, 1.0, t, 0.0, r, s);
    mg.vcycle_widen(r, z, s);
    launch_dot<double>(n_u, r, z, scd + 0, wsd, s);
    launch_axpby<double>(n_u, 1.0, z, 0.0, dd, s);
    int it = 0;
    for (it = 1; it <= maxit; ++it) {
        launch_apply_sip<double>(P->n, P->geom, dd, q, eta, 1.0, nullptr, 0.0, s);
        launch_dot<double>(n_u, dd, q, scd + 1, wsd, s);
        launch_pcg_update<double>(n_u, dd, q, y, r, scd + 0, scd + 1, s);
        launch_dot<double>(n_u, r, r, scd + 2, wsd, s);
        const double rr = std::sqrt(read_scalar(scd + 2, hp, s));
        if (!std::isfinite(rr)) throw Error(SIP_ERR_BREAKDOWN, "non-finite inner residual");
        if (rr < rtol * nt || it == maxit) break;
        mg.vcycle_widen(r, z, s);
        launch_dot<double>(n_u, r, z, scd + 3, wsd, s);
        launch_pcg_dir<double>(n_u, z, dd, scd + 3, scd + 0, s);
        SIP_CUDA(cudaMemcpyAsync(scd + 0, scd + 3, sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    return std::min(it, maxit);
}

// ---------------------------------------------------------------- FGMRES
int64_t Workspace::bytes() const {
    return int64_t(V.bytes + Z.bytes + w.bytes + x.bytes + r.bytes + b.bytes + tu.bytes +
                   yu64.bytes + sinv.bytes + ws.bytes + sc.bytes + hbuf.bytes + cg_r.bytes +
                   cg_d.bytes + cg_q.bytes + cg_z.bytes + sc_in.bytes + gcr_z.bytes +
                   gcr_q.bytes);
}

namespace {

__global__ void k_sinv(size_t ne, int mp, double area_quarter, const double* eta, double* out) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g < ne * mp) out[g] = -eta[g / mp] / area_quarter;
}

}  // namespace

sip_status run_solve(sip_problem* P, const double* f_u, const double* g_p, double* u_out,
                     double* p_out, const sip_solve_opts& o, sip_solve_report* rep,
                     cudaStream_t s) {
    const double t_start = now_ms();
    const int64_t launches0 = launch_counter();
    const double setup0 = P->setup_ms;
    P->ensure_setup(s);
    const double setup_ms = P->setup_ms - setup0;
    const bool f32_inner = P->desc.precision == SIP_PREC_MIXED_F32_INNER;
    const bool mixed = P->desc.precision == SIP_PREC_MIXED || f32_inner;
    const size_t n_u = size_t(P->n_u), n_p = size_t(P->n_p), n = n_u + n_p;
    const bool singular = P->desc.bc[0] != SIP_BC_NEUMANN && P->desc.bc[1] != SIP_BC_NEUMANN &&
                          P->desc.bc[2] != SIP_BC_NEUMANN && P->desc.bc[3] != SIP_BC_NEUMANN;
    const int restart = std::max(1, std::min(o.restart, o.max_outer));
    if (!P->ws || P->ws->restart < restart) {
        auto w = std::make_unique<Workspace>();
        w->restart = restart;
        w->n = n;
        w->V.alloc(size_t(restart + 1) * n * sizeof(double));
        w->Z.alloc(size_t(restart) * n * sizeof(double));
        for (DeviceBuffer* b : {&w->w, &w->x, &w->r, &w->b}) b->alloc(n * sizeof(double));
        w->tu.alloc(n_u * sizeof(double));
        w->yu64.alloc(n_u * sizeof(double));
        w->sinv.alloc(n_p * sizeof(double));
        w->ws.alloc(reduction_workspace_doubles(restart + 2) * sizeof(double));
        w->sc.alloc(size_t(restart + 8) * sizeof(double));
        w->hbuf.alloc(size_t(restart + 8) * sizeof(double));
        P->ws = std::move(w);
    }
    Workspace& W = *P->ws;
    if (!W.sinv_ready) {
        // Schur block of the preconditioner: the saddle matrix's own Schur
        // complement -B^T A^{-1} B, approximated by -S*, S* = the pressure mass
        // (h_x h_y / 4 on the orthonormal basis) scaled by 1/eta_K; stored
        // here as the diagonal of its inverse, -eta_K / (h_x h_y / 4)
        launch_k(k_sinv, unsigned((n_p + 255) / 256), 256, 0, s, 
            size_t(P->ne), P->mp, 0.25 * P->geom.hx * P->geom.hy, P->eta_d.as<double>(),
            W.sinv.as<double>());
        SIP_CHECK_LAUNCH();
        W.sinv_ready = true;
    }
    if (f32_inner) {
        W.t32.alloc(n_u * sizeof(float));
        W.y32.alloc(n_u * sizeof(float));
    } else if (mixed) {
        for (DeviceBuffer* b : {&W.cg_r, &W.cg_d, &W.cg_q, &W.cg_z}) b->alloc(n_u * sizeof(double));
        W.sc_in.alloc(8 * sizeof(double));
    }
    double* V = W.V.as<double>();
    double* Z = W.Z.as<double>();
    double* wv = W.w.as<double>();
    double* x = W.x.as<double>();
    double* b = W.b.as<double>();
    double* r = W.r.as<double>();
    double* sc = W.sc.as<double>();
    double* wsd = W.ws.as<double>();
    double* hp = W.hs.p;
    const double* eta = P->eta_d.as<double>();

    // b = [f; g]
    SIP_CUDA(cudaMemcpyAsync(b, f_u, n_u * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (g_p)
        SIP_CUDA(cudaMemcpyAsync(b + n_u, g_p, n_p * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else
        SIP_CUDA(cudaMemsetAsync(b + n_u, 0, n_p * sizeof(double), s));
    SIP_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));

    auto project = [&](double* v) {
        if (singular) launch_zero_mean_pressure(size_t(P->ne), P->mp, v + n_u, wsd, s);
    };
    // y = K v  (w_u = A v_u + B v_p, w_p = B^T v_u)
    auto applyK = [&](const double* v, double* y) {
        launch_apply_B<double>(P->k, P->geom, v + n_u, W.tu.as<double>(), s);
        launch_apply_sip<double>(P->n, P->geom, v, y, eta, 1.0, W.tu.as<double>(), 1.0, s);
        launch_apply_Bt<double>(P->k, P->geom, v, y + n_u, s);
    };
    int inner_total = 0, inner_max = 0, inner_calls = 0;
    // the inner PCG runs as one graph launch with a device-side loop unless
    // the options ask for the host-driven loop (same arithmetic)
    const bool host_loop = o.inner_loop == 1;
    // flexible CG where the V-cycle is FP32 (automatic choice), else PCG;
    // inner_krylov 3: GCR restarted after inner_restart directions
    const bool flexible = o.inner_krylov == 2 || (o.inner_krylov == 0 && mixed && !host_loop);
    const int gcr_restart = o.inner_krylov == 3 ? o.inner_restart : 0;
    // z = P^{-1} v
    auto precond = [&](const double* v, double* z) {
        launch_vmul<double>(n_p, v + n_u, W.sinv.as<double>(), z + n_u, s);   // y_p = -S*^{-1} v_p
        project(z);
        launch_apply_B<double>(P->k, P->geom, z + n_u, W.tu.as<double>(), s);
        launch_axpby<double>(n_u, 1.0, v, -1.0, W.tu.as<double>(), s);        // t = v_u - B y_p
        int its;
        if (f32_inner) {
            launch_cast<double, float>(n_u, W.tu.as<double>(), W.t32.as<float>(), s);
            its = P->mg32->inner_pcg(W.t32.as<float>(), W.y32.as<float>(), o.inner_rtol,
                                     o.max_inner, s, nullptr);
            launch_cast<float, double>(n_u, W.y32.as<float>(), z, s);
        } else if (host_loop) {
            its = mixed ? inner_pcg_mixed(P, W, W.tu.as<double>(), z, o.inner_rtol, o.max_inner, s)
                        : P->mg64->inner_pcg(W.tu.as<double>(), z, o.inner_rtol, o.max_inner, s,
                                             nullptr);
        } else {
            bool batched = false;
            its = batched_inner(P, W.tu.as<double>(), z, s, &batched);
            if (!batched)
                its = inner_pcg_graph(P, W, mixed, flexible, o.inner_norm == 1, W.tu.as<double>(),
                                      z, o.inner_rtol, o.max_inner, s, gcr_restart);
        }
        inner_total += its;
        inner_max = std::max(inner_max, its);
        ++inner_calls;
    };
    auto norm = [&](const double* v) {
        launch_dot<double>(n, v, v, sc, wsd, s);
        return std::sqrt(read_scalar(sc, hp, s));
    };

    launch_axpby<double>(n, 1.0, b, 0.0, r, s);
    project(r);
    const double beta0 = norm(b);
    sip_status st = SIP_ERR_NOT_CONVERGED;
    int total = 0;
    double rel = 0.0;
    if (beta0 == 0.0) {
        st = SIP_OK;
    } else if (!std::isfinite(beta0)) {
        throw Error(SIP_ERR_INVALID_ARG, "non-finite right-hand side");
    }
    std::vector<double> H(size_t(restart + 1) * restart), cs(restart), sn(restart), gv(restart + 1);
    bool recur_conv = false;   // the last cycle ended on the recurrence's residual
    double rn_false = 0.0;     // residual after the previous such cycle
    auto stagnated = [&](double rn) {
        if (!recur_conv) return false;
        if (rn_false > 0.0 && rn > 0.5 * rn_false) return true;
        rn_false = rn;
        return false;
    };
    if (o.outer_krylov == 1 && st == SIP_ERR_NOT_CONVERGED) {
        // GCR (Eisenstat, Elman & Schultz 1983), the outer method of the
        // six-inclusion runs (Sec. 7.3): z_j = P^{-1} r, q_j = K z_j, both
        // orthogonalised against the stored pairs (classical Gram-Schmidt
        // twice, coefficients on the device) and scaled to ||q_j|| = 1;
        // x += <r, q_j> z_j, r -= <r, q_j> q_j.  The pairs live in V (q) and
        // Z (z) and are dropped after `restart` of them; whenever the
        // recurrence's residual meets the tolerance, the residual is
        // recomputed from x and GCR continues from it if it does not.
        double* sq = sc + restart + 1;     // ||q_j||^2
        double* sa = sc + restart + 2;     // <r, q_j>
        double* sone = sc + restart + 3;   // 1.0
        double* sq0 = sc + restart + 4;    // ||K z_j||^2 before the projections
        static const double one = 1.0;
        SIP_CUDA(cudaMemcpyAsync(sone, &one, sizeof(double), cudaMemcpyHostToDevice, s));
        bool broke = false;
        sip_status stop_st = SIP_OK;
        for (;;) {
            applyK(x, r);
            launch_axpby<double>(n, 1.0, b, -1.0, r, s);
            project(r);
            const double rn = norm(r);
            rel = rn / beta0;
            if (!std::isfinite(rn)) {
                st = SIP_ERR_BREAKDOWN;
                break;
            }
            if (rn <= o.rtol * beta0) {
                st = SIP_OK;
                break;
            }
            if (broke) {
                st = SIP_ERR_BREAKDOWN;
                break;
            }
            if (stop_st != SIP_OK) {
                st = stop_st;
                break;
            }
            if (total >= o.max_outer || stagnated(rn)) break;
            int j = 0;
            recur_conv = false;
            while (total < o.max_outer) {
                if (j == restart) j = 0;
                double* zj = Z + size_t(j) * n;
                double* qj = V + size_t(j) * n;
                precond(r, zj);
                applyK(zj, qj);
                project(qj);
                launch_dot<double>(n, qj, qj, sq0, wsd, s);
                if (j > 0) {
                    for (int pass = 0; pass < 2; ++pass) {
                        launch_mdot<double>(j, n, V, n, qj, sc, wsd, s);
                        launch_maxpy<double>(j, n, V, n, sc, -1.0, qj, s);
                        launch_maxpy<double>(j, n, Z, n, sc, -1.0, zj, s);
                    }
                }
                launch_dot<double>(n, qj, qj, sq, wsd, s);
                // a direction with K z_j in the span of the stored q_i (or
                // K z_j = 0) cannot be normalised: stop with the iterate so far
                SIP_CUDA(cudaMemcpyAsync(hp, sq, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
                SIP_CUDA(cudaStreamSynchronize(s));
                const double qq = hp[0], qq0 = hp[sq0 - sq];
                if (!(qq > 1e-28 * qq0) || !std::isfinite(qq)) {
                    broke = true;
                    break;
                }
                launch_scale_inv_sqrt<double>(n, sq, qj, s);
                launch_scale_inv_sqrt<double>(n, sq, zj, s);
                launch_dot<double>(n, r, qj, sa, wsd, s);
                launch_pcg_update<double>(n, zj, qj, x, r, sa, sone, s);
                ++total;
                ++j;
                const double rr = norm(r);
                if (!std::isfinite(rr)) {
                    broke = true;
                    break;
                }
                if (rr <= o.rtol * beta0) {
                    recur_conv = true;
                    break;
                }
                stop_st = stop_requested();
                if (stop_st != SIP_OK) break;
            }
        }
    }
    while (o.outer_krylov == 0 && st == SIP_ERR_NOT_CONVERGED && total < o.max_outer) {
        const double beta = norm(r);
        if (!std::isfinite(beta)) {
            st = SIP_ERR_BREAKDOWN;
            break;
        }
        launch_axpby<double>(n, 1.0 / beta, r, 0.0, V, s);
        std::fill(H.begin(), H.end(), 0.0);
        std::fill(gv.begin(), gv.end(), 0.0);
        gv[0] = beta;
        int j = 0, jdone = 0;
        bool broke = false;
        sip_status stop_st = SIP_OK;
        recur_conv = false;
        for (j = 0; j < restart && total < o.max_outer; ++j) {
            double* vj = V + size_t(j) * n;
            double* zj = Z + size_t(j) * n;
            precond(vj, zj);
            applyK(zj, wv);
            project(wv);
            for (int pass = 0; pass < 2; ++pass) {
                launch_mdot<double>(j + 1, n, V, n, wv, sc, wsd, s);
                launch_maxpy<double>(j + 1, n, V, n, sc, -1.0, wv, s);
                SIP_CUDA(cudaMemcpyAsync(hp, sc, (j + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
                SIP_CUDA(cudaStreamSynchronize(s));
                for (int i = 0; i <= j; ++i) H[size_t(i) * restart + j] += hp[i];
            }
            const double hn = norm(wv);
            if (!std::isfinite(hn)) {
                broke = true;
                break;
            }
            H[size_t(j + 1) * restart + j] = hn;
            if (hn > 0.0) launch_axpby<double>(n, 1.0 / hn, wv, 0.0, V + size_t(j + 1) * n, s);
            for (int i = 0; i < j; ++i) {
                const double t1 = H[size_t(i) * restart + j], t2 = H[size_t(i + 1) * restart + j];
                H[size_t(i) * restart + j] = cs[i] * t1 + sn[i] * t2;
                H[size_t(i + 1) * restart + j] = -sn[i] * t1 + cs[i] * t2;
            }
            const double a = H[size_t(j) * restart + j], c = H[size_t(j + 1) * restart + j];
            const double den = std::hypot(a, c);
            if (den == 0.0) {
                broke = true;
                break;
            }
            cs[j] = a / den;
            sn[j] = c / den;
            H[size_t(j) * restart + j] = den;
            H[size_t(j + 1) * restart + j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            ++total;
            jdone = j + 1;
            if (std::abs(gv[j + 1]) <= o.rtol * beta0 || hn <= 1e-300) {
                recur_conv = true;
                break;
            }
            stop_st = stop_requested();
            if (stop_st != SIP_OK) break;
        }
        if (jdone > 0) {
            std::vector<double> yk(jdone);
            for (int i = jdone - 1; i >= 0; --i) {
                double t = gv[i];
                for (int k2 = i + 1; k2 < jdone; ++k2) t -= H[size_t(i) * restart + k2] * yk[k2];
                yk[i] = t / H[size_t(i) * restart + i];
            }
            SIP_CUDA(cudaMemcpyAsync(W.hbuf.ptr, yk.data(), jdone * sizeof(double),
                                     cudaMemcpyHostToDevice, s));
            launch_maxpy<double>(jdone, n, Z, n, W.hbuf.as<double>(), 1.0, x, s);
        }
        // true residual r = b - K x
        applyK(x, r);
        launch_axpby<double>(n, 1.0, b, -1.0, r, s);
        project(r);
        const double rn = norm(r);
        rel = rn / beta0;
        if (!std::isfinite(rn)) {
            st = SIP_ERR_BREAKDOWN;
            break;
        }
        if (rn <= o.rtol * beta0) {
            st = SIP_OK;
            break;
        }
        if (broke) {
            st = SIP_ERR_BREAKDOWN;
            break;
        }
        if (stop_st != SIP_OK) {
            st = stop_st;
            break;
        }
        // the recurrence may report convergence while the true residual does
        // not: restart; a second such cycle that does not halve the residual
        // means FP64 has reached its attainable accuracy for this system
        if (stagnated(rn)) break;
    }
    if (singular) launch_zero_mean_pressure(size_t(P->ne), P->mp, x + n_u, wsd, s);
    SIP_CUDA(cudaMemcpyAsync(u_out, x, n_u * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SIP_CUDA(cudaMemcpyAsync(p_out, x + n_u, n_p * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SIP_CUDA(cudaStreamSynchronize(s));
    if (rep) {
        rep->status = st;
        rep->outer_its = total;
        rep->inner_total = inner_total;
        rep->inner_max = inner_max;
        rep->inner_avg = inner_calls ? double(inner_total) / inner_calls : 0.0;
        rep->rel_residual = beta0 == 0.0 ? 0.0 : rel;
        rep->setup_ms = setup_ms;
        rep->solve_ms = now_ms() - t_start - setup_ms;
        rep->lambda_max_p = mixed ? P->mg32->lmax_p : P->mg64->lmax_p;
        rep->kernel_launches = launch_counter() - launches0;
        rep->refine_steps = 0;
    }
    return st;
}

namespace {

__global__ void k_to_dd(size_t n, const double* __restrict__ a, dd* b) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g < n) b[g] = dd(a[g]);
}

// r = [f; g] - y over n entries (the first n_u from f, the rest from g or 0)
__global__ void k_dd_b_minus(size_t n_u, size_t n, const double* __restrict__ f,
                             const double* __restrict__ gp, const dd* __restrict__ y, dd* r) {
    grid_dep_wait();
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double b = i < n_u ? f[i] : (gp ? gp[i - n_u] : 0.0);
    r[i] = dd(b) - y[i];
}

// x += d (double-double accumulation of an FP64 correction)
__global__ void k_dd_add(size_t n, const double* __restrict__ d, dd* x) {
    grid_dep_wait();
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) x[i] = x[i] + dd(d[i]);
}

// v = hi + lo rounded to FP64 (the leading part of a normalised pair)
__global__ void k_dd_round(size_t n, const dd* __restrict__ x, double* v) {
    grid_dep_wait();
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) v[i] = x[i].hi + x[i].lo;
}

inline unsigned blocks_of(size_t n) { return unsigned((n + 255) / 256); }

// r = b - K x with x, r contiguous [u; p] double-double vectors
void residual_dd_contig(sip_problem* P, const double* f_u, const double* g_p, const dd* x, dd* r,
                        cudaStream_t s) {
    const size_t n_u = size_t(P->n_u), n_p = size_t(P->n_p), n = n_u + n_p;
    const size_t ne = size_t(P->ne);
    P->eta_dd.alloc(ne * sizeof(dd));
    P->rf_y.alloc(n * sizeof(dd));
    P->rf_t.alloc(n_u * sizeof(dd));
    dd* eta = P->eta_dd.as<dd>();
    dd* y = P->rf_y.as<dd>();
    dd* t = P->rf_t.as<dd>();
    launch_k(k_to_dd, blocks_of(ne), 256, 0, s, ne, P->eta_d.as<double>(), eta);
    SIP_CHECK_LAUNCH();
    launch_apply_B<dd>(P->k, P->geom, x + n_u, t, s);                       // t = B x_p
    launch_apply_sip_dd(P->n, P->geom, x, y, eta, t, s);                    // y_u = A x_u + t
    launch_apply_Bt<dd>(P->k, P->geom, x, y + n_u, s);                      // y_p = B^T x_u
    launch_k(k_dd_b_minus, blocks_of(n), 256, 0, s, n_u, n, f_u, g_p, static_cast<const dd*>(y),
             r);
    SIP_CHECK_LAUNCH();
}

}  // namespace

void residual_dd(sip_problem* P, const double* f_u, const double* g_p, const double* x_u,
                 const double* x_p, double* r_u, double* r_p, cudaStream_t s) {
    const size_t n_u = size_t(P->n_u), n_p = size_t(P->n_p), n = n_u + n_p;
    P->rf_x.alloc(n * sizeof(dd));
    P->rf_r.alloc(n * sizeof(dd));
    dd* x = P->rf_x.as<dd>();
    dd* r = P->rf_r.as<dd>();
    SIP_CUDA(cudaMemcpyAsync(x, x_u, n_u * sizeof(dd), cudaMemcpyDeviceToDevice, s));
    SIP_CUDA(cudaMemcpyAsync(x + n_u, x_p, n_p * sizeof(dd), cudaMemcpyDeviceToDevice, s));
    residual_dd_contig(P, f_u, g_p, x, r, s);
    SIP_CUDA(cudaMemcpyAsync(r_u, r, n_u * sizeof(dd), cudaMemcpyDeviceToDevice, s));
    SIP_CUDA(cudaMemcpyAsync(r_p, r + n_u, n_p * sizeof(dd), cudaMemcpyDeviceToDevice, s));
}

sip_status run_solve_refined(sip_problem* P, const double* f_u, const double* g_p, double* u_out,
                             double* p_out, const sip_solve_opts& o, sip_solve_report* rep,
                             cudaStream_t s, double* u_dd, double* p_dd) {
    const double t_start = now_ms();
    const int64_t launches0 = launch_counter();
    const size_t n_u = size_t(P->n_u), n_p = size_t(P->n_p), n = n_u + n_p;
    P->rf_x.alloc(n * sizeof(dd));
    P->rf_r.alloc(n * sizeof(dd));
    P->rf_d.alloc(2 * n * sizeof(double));   // FP64 residual [n] and correction [n]
    dd* x = P->rf_x.as<dd>();
    dd* r = P->rf_r.as<dd>();
    double* r64 = P->rf_d.as<double>();
    double* d64 = r64 + n;
    SIP_CUDA(cudaMemsetAsync(x, 0, n * sizeof(dd), s));
    SIP_CUDA(cudaMemcpyAsync(r64, f_u, n_u * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (g_p)
        SIP_CUDA(cudaMemcpyAsync(r64 + n_u, g_p, n_p * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else
        SIP_CUDA(cudaMemsetAsync(r64 + n_u, 0, n_p * sizeof(double), s));
    // norms through a small device scratch (the reduction kernels of the solve)
    P->rf_scr.alloc((8 + reduction_workspace_doubles(2)) * sizeof(double));
    if (!P->rf_hs) P->rf_hs = std::make_unique<HostScalars>();
    double* scr = P->rf_scr.as<double>();
    double* part = scr + 8;
    double* hsp = P->rf_hs->p;
    auto norm = [&](const double* v) {
        launch_dot<double>(n, v, v, scr, part, s);
        return std::sqrt(read_scalar(scr, hsp, s));
    };
    const double nb = norm(r64);
    sip_solve_opts o1 = o;
    o1.refine = 0;
    sip_status st = SIP_ERR_NOT_CONVERGED;
    int outer = 0, inner_total = 0, inner_max = 0, steps = 0;
    double inner_calls = 0.0, setup_ms = 0.0, rel = nb == 0.0 ? 0.0 : 1.0, nr = nb;
    if (nb == 0.0) st = SIP_OK;
    if (!std::isfinite(nb)) throw Error(SIP_ERR_INVALID_ARG, "non-finite right-hand side");
    while (st == SIP_ERR_NOT_CONVERGED && steps < o.refine && outer < o.max_outer) {
        // the correction solve asks for what is left of the reduction
        o1.rtol = std::min(0.5, o.rtol * nb / nr);
        o1.max_outer = o.max_outer - outer;
        sip_solve_report r1{};
        const sip_status s1 = run_solve(P, r64, r64 + n_u, d64, d64 + n_u, o1, &r1, s);
        ++steps;
        outer += r1.outer_its;
        inner_total += r1.inner_total;
        inner_max = std::max(inner_max, r1.inner_max);
        if (r1.inner_avg > 0.0) inner_calls += double(r1.inner_total) / r1.inner_avg;
        setup_ms += r1.setup_ms;
        if (s1 == SIP_ERR_BREAKDOWN && !std::isfinite(norm(d64))) {
            st = SIP_ERR_BREAKDOWN;
            break;
        }
        launch_k(k_dd_add, blocks_of(n), 256, 0, s, n, static_cast<const double*>(d64), x);
        SIP_CHECK_LAUNCH();
        residual_dd_contig(P, f_u, g_p, x, r, s);
        launch_k(k_dd_round, blocks_of(n), 256, 0, s, n, static_cast<const dd*>(r), r64);
        SIP_CHECK_LAUNCH();
        const double nr_new = norm(r64);
        if (!std::isfinite(nr_new)) {
            st = SIP_ERR_BREAKDOWN;
            break;
        }
        rel = nr_new / nb;
        if (nr_new <= o.rtol * nb) {
            st = SIP_OK;
            break;
        }
        if (nr_new > 0.5 * nr) break;   // the correction no longer halves the residual
        nr = nr_new;
    }
    launch_k(k_dd_round, blocks_of(n), 256, 0, s, n, static_cast<const dd*>(x), d64);
    SIP_CHECK_LAUNCH();
    const bool singular = P->desc.bc[0] != SIP_BC_NEUMANN && P->desc.bc[1] != SIP_BC_NEUMANN &&
                          P->desc.bc[2] != SIP_BC_NEUMANN && P->desc.bc[3] != SIP_BC_NEUMANN;
    if (singular) launch_zero_mean_pressure(size_t(P->ne), P->mp, d64 + n_u, part, s);
    if (u_out)
        SIP_CUDA(cudaMemcpyAsync(u_out, d64, n_u * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (p_out)
        SIP_CUDA(cudaMemcpyAsync(p_out, d64 + n_u, n_p * sizeof(double), cudaMemcpyDeviceToDevice,
                                 s));
    // the double-double iterate itself: its residual is the one tested above
    static_assert(sizeof(dd) == 2 * sizeof(double), "(hi, lo) pairs");
    if (u_dd) SIP_CUDA(cudaMemcpyAsync(u_dd, x, n_u * sizeof(dd), cudaMemcpyDeviceToDevice, s));
    if (p_dd)
        SIP_CUDA(cudaMemcpyAsync(p_dd, x + n_u, n_p * sizeof(dd), cudaMemcpyDeviceToDevice, s));
    SIP_CUDA(cudaStreamSynchronize(s));
    if (rep) {
        rep->status = st;
        rep->outer_its = outer;
        rep->inner_total = inner_total;
        rep->inner_max = inner_max;
        rep->inner_avg = inner_calls > 0.0 ? double(inner_total) / inner_calls : 0.0;
        rep->rel_residual = rel;
        rep->setup_ms = setup_ms;
        rep->solve_ms = now_ms() - t_start - setup_ms;
        rep->lambda_max_p = P->mg32 ? P->mg32->lmax_p : (P->mg64 ? P->mg64->lmax_p : 0.0);
        rep->kernel_launches = launch_counter() - launches0;
        rep->refine_steps = steps;
    }
    return st;
}

}  // namespace sip

int64_t sip_problem::device_bytes() const {
    int64_t b = int64_t(eta_d.bytes + eta_f.bytes + eta_inv_d.bytes + eta_inv_f.bytes);
    if (mg64) b += mg64->bytes();
    if (mg32) b += mg32->bytes();
    if (ws) b += ws->bytes();
    b += int64_t(eta_dd.bytes + rf_x.bytes + rf_y.bytes + rf_t.bytes + rf_r.bytes + rf_d.bytes +
                 rf_scr.bytes);
    return b;
}

namespace {
__global__ void k_derive_eta(size_t n, const double* eta, float* ef, double* inv, float* invf) {
    sip::grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const double e = eta[g];
    ef[g] = float(e);
    inv[g] = 1.0 / e;
    invf[g] = float(1.0 / e);
}
}  // namespace

void sip_problem::derive_eta(cudaStream_t s) {
    const size_t n = size_t(ne);
    eta_f.alloc(n * sizeof(float));
    eta_inv_d.alloc(n * sizeof(double));
    eta_inv_f.alloc(n * sizeof(float));
    sip::launch_k(k_derive_eta, unsigned((n + 255) / 256), 256, 0, s, n, eta_d.as<double>(),
                  eta_f.as<float>(), eta_inv_d.as<double>(), eta_inv_f.as<float>());
    SIP_CHECK_LAUNCH();
}

void sip_problem::ensure_setup(cudaStream_t s) {
    const double t0 = sip::now_ms();
    bool did = false;
    const bool fresh = (mg32 == nullptr || !mg32->ready) && (mg64 == nullptr || !mg64->ready);
    if (fresh) sip::tune_apply(this, s);
    if (desc.precision == SIP_PREC_MIXED || desc.precision == SIP_PREC_MIXED_F32_INNER) {
        if (!mg32) {
            mg32 = std::make_unique<sip::Multigrid<float>>();
            mg32->P = this;
        }
        if (!mg32->ready) {
            mg32->setup(s);
            did = true;
        }
    } else {
        if (!mg64) {
            mg64 = std::make_unique<sip::Multigrid<double>>();
            mg64->P = this;
        }
        if (!mg64->ready) {
            mg64->setup(s);
            did = true;
        }
    }
    if (did) setup_ms += sip::now_ms() - t0;
}
