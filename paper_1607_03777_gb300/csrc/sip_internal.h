// Internal declarations shared by the CUDA translation units of the
// SIP-DG Stokes library.  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "../../include/sipstokes.h"

namespace sip {

// ---------------------------------------------------------------- errors
struct Error : std::runtime_error {
    sip_status status;
    Error(sip_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define SIP_CUDA(call)                                                              \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            throw ::sip::Error(SIP_ERR_CUDA, std::string(#call) + ": " +            \
                                                 cudaGetErrorString(e_));           \
    } while (0)

// Host-side count of kernel launches issued by the library (each launcher
// ends with SIP_CHECK_LAUNCH); graph replays add their captured kernel count.
int64_t& launch_counter();

// Programmatic dependent launch.  Kernels are launched with programmatic
// stream serialisation (when enabled), so the next kernel of a chain is
// scheduled while the previous one drains; every kernel starts with
// grid_dep_wait(), which returns once the preceding grid has completed and
// its memory is visible, so the stream order of the data is unchanged and
// only launch latency overlaps.  SIP_PDL=0 launches plainly; the flag is
// also cleared while capturing graph bodies of conditional nodes.
__device__ __forceinline__ void grid_dep_wait() {
#if defined(__CUDA_ARCH__)
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

bool& pdl_enabled();

struct PdlOffScope {
    bool prev;
    PdlOffScope() : prev(pdl_enabled()) { pdl_enabled() = false; }
    ~PdlOffScope() { pdl_enabled() = prev; }
};

template <typename... KArgs, typename... Args>
void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    if (e != cudaSuccess) throw Error(SIP_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
}

#define SIP_CHECK_LAUNCH()                  \
    do {                                    \
        ++::sip::launch_counter();          \
        SIP_CUDA(cudaGetLastError());       \
    } while (0)

// Stop request of the solve running on this host thread, checked between
// outer Krylov iterations: a deadline on the steady clock (ms; 0 = none) and
// a cancel flag (may be null).  A solve that meets it returns
// SIP_ERR_TIMEOUT or SIP_ERR_CANCELLED with its last iterate.
struct StopCtl {
    double deadline_ms = 0.0;
    const volatile bool* cancel = nullptr;
};
StopCtl& stop_ctl();   // per host thread
double steady_ms();
// SIP_OK, or the status of a met stop request
sip_status stop_requested();
struct StopScope {
    StopCtl prev;
    StopScope(double deadline_ms, const volatile bool* cancel) : prev(stop_ctl()) {
        stop_ctl().deadline_ms = deadline_ms;
        stop_ctl().cancel = cancel;
    }
    ~StopScope() { stop_ctl() = prev; }
};

inline void require(bool ok, const std::string& msg) {
    if (!ok) throw Error(SIP_ERR_INVALID_ARG, msg);
}

// ------------------------------------------------------------ 1D tables
// Orthonormal Legendre l_i = sqrt((2i+1)/2) P_i on [-1, 1] (Sec. 5 basis).
// Closed forms of the classical Legendre facts used:
//   P_i(1) = 1, P_i(-1) = (-1)^i, P_i'(1) = i(i+1)/2, P_i'(-1) = (-1)^(i+1) i(i+1)/2
//   P_q' = sum_{p<q, q-p odd} (2p+1) P_p       => int P_p P_q' = 2 for those p
//   int P_a' P_b' = m(m+1), m = min(a,b), when a+b is even (0 otherwise)
// G[a][b] = int l_a' l_b',  D[p][q] = int l_p l_q'.
template <int N, typename T>
struct Tab1D {
    T lp[N], lm[N];   // l_i(+1), l_i(-1)
    T dp[N], dm[N];   // l_i'(+1), l_i'(-1)
    T G[N * N];
    T D[N * N];
};

template <int N, typename T>
Tab1D<N, T> make_tab() {
    Tab1D<N, T> t;
    for (int i = 0; i < N; ++i) {
        double c = std::sqrt((2.0 * i + 1.0) / 2.0);
        double sgn = (i % 2 == 0) ? 1.0 : -1.0;
        t.lp[i] = T(c);
        t.lm[i] = T(sgn * c);
        t.dp[i] = T(c * i * (i + 1) / 2.0);
        t.dm[i] = T(-sgn * c * i * (i + 1) / 2.0);
    }
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            double ca = std::sqrt((2.0 * a + 1.0) / 2.0), cb = std::sqrt((2.0 * b + 1.0) / 2.0);
            int m = a < b ? a : b;
            double g = ((a + b) % 2 == 0 && m >= 1) ? double(m) * (m + 1) : 0.0;
            t.G[a * N + b] = T(ca * cb * g);
            double d = (b > a && (b - a) % 2 == 1) ? 2.0 : 0.0;
            t.D[a * N + b] = T(ca * cb * d);
        }
    return t;
}

// ------------------------------------------------------------ operator
// Geometry and penalty of one SIP operator on the grid.  pen_x / pen_y are
// sigma_e / eta_e for an interior face with x- / y-normal:
// penalty_scale * n_f (1+tau) (k_pen+1)^2 |e|/|K| with n_f = 4, tau = 0 and
// |e|/|K| = 1/h_normal; boundary faces double it (eq. sipg_penalty).
// Kernel schedule of one operator, per precision ([0] FP64, [1] FP32):
// which apply kernel runs and whether the p-level smoother step is fused.
// APPLY_WARP exists for the FP32 operator only (one thread per element, one
// warp per tile row, cp.async staging).
enum ApplyVariant { APPLY_AUTO = 0, APPLY_ELEM2 = 1, APPLY_ELEM1 = 2, APPLY_TILE = 3, APPLY_STAGE = 4,
                    APPLY_WARP = 6 };

struct OpGeom {
    int nx, ny;
    double hx, hy;
    int bc[4];
    double pen_x, pen_y;
    int variant[2];   // ApplyVariant (APPLY_AUTO: component-split for N <= 6, else tile)
    int fused[2];     // p-level smoother step fused into one launch (1) or not (0)
    int stage_rows[2];   // tile rows of the staged apply (2 or 4), per precision
    // split-precision FP32 operator (mixed form at high viscosity contrast):
    // tiles evaluated in FP64 arithmetic on FP32 data; n_hi = 0: none
    const unsigned char* hi_flag;
    const int* hi_tiles;
    int n_hi;
};

inline OpGeom make_geom(int nx, int ny, double lx, double ly, const int bc[4], int k_pen,
                        double penalty_scale) {
    OpGeom g;
    g.nx = nx;
    g.ny = ny;
    g.hx = lx / nx;
    g.hy = ly / ny;
    for (int i = 0; i < 4; ++i) g.bc[i] = bc[i];
    double c = penalty_scale * 4.0 * double(k_pen + 1) * double(k_pen + 1);
    g.variant[0] = g.variant[1] = APPLY_AUTO;
    g.fused[0] = g.fused[1] = 1;
    g.stage_rows[0] = g.stage_rows[1] = 2;
    g.hi_flag = nullptr;
    g.hi_tiles = nullptr;
    g.n_hi = 0;
    g.pen_x = c / g.hx;
    g.pen_y = c / g.hy;
    return g;
}

// y = alpha * (A x) + beta * z (z may be null).  N = polynomial degree + 1
// of the space the operator acts on (N = 2 for the Galerkin A_1).
template <typename T>
void launch_apply_sip(int N, const OpGeom& g, const T* x, T* y, const T* eta, T alpha,
                      const T* z, T beta, cudaStream_t s);
// Thread-per-element variants for N <= 6 (split: two threads per element,
// one per velocity component); returns false for other N.
template <typename T>
bool launch_apply_sip_elem(int N, const OpGeom& g, const T* x, T* y, const T* eta, T alpha,
                           const T* z, T beta, bool split, cudaStream_t s);
// Staged-tile kernels (N <= 6; returns false otherwise): y = alpha A x +
// beta z, or with r1 non-null the Q^2_1 modes of that result into r1 (y
// unused).  For T = float with g.n_hi > 0 the flagged tiles are evaluated in
// FP64 arithmetic (split precision); x must not overlap y.
template <typename T>
bool launch_apply_sip_stage(int N, const OpGeom& g, const T* x, T* y, const T* eta, T alpha,
                            const T* z, T beta, T* r1, cudaStream_t s);
// Warp-row FP32 apply (N <= 6, 16-byte aligned vectors; returns false
// otherwise): y = alpha A x + beta z, z may equal y.  skip (split-precision
// tile flags, 32 x 2 tiles): rows of flagged tiles are left to the FP64
// launch; without it an operator with split-precision tiles is refused.
bool launch_apply_sip_warp(int N, const OpGeom& g, const float* x, float* y, const float* eta,
                           float alpha, const float* z, float beta, const unsigned char* skip,
                           cudaStream_t s);
// Number of split-precision tiles of an nx x ny mesh, and their flags: tile
// t is flagged (and listed) when an element of the tile or of its halo has
// eta >= ratio x min(eta).  scratch: 32 device bytes.  Returns the count
// (synchronises s).
int split_tile_count(int nx, int ny);
// creates this host thread's side stream of the split-precision apply (its
// first use would otherwise fall inside a graph capture)
void split_fork_prepare();
int mark_hi_tiles(int nx, int ny, const double* eta, double ratio, unsigned char* flag, int* list,
                  int* scratch, cudaStream_t s);
// The apply variant in force for precision T: SIP_APPLY_KERNEL (elem2, elem1,
// tile) overrides the operator's schedule.
template <typename T>
int apply_variant(const OpGeom& g);
// Fused p-level smoother step (N <= 4; returns false otherwise, nothing launched):
//   r = z - A x;  d_new = c1 d_old + c2 M^{-1} r;  yv += (pend ? d_old : 0) + d_new
// with M^{-1} the element-block Jacobi inverses (class by emap < 0, scaled by
// eta_inv, else unique).  z may alias r; x must not alias r, d_new or yv.
bool cheb_elem_available(int N);
// r1 = R (b - A y): the residual restricted to the Q^2_1 modes in one launch
// (N <= 4; returns false otherwise, nothing launched).
template <typename T>
bool launch_residual_restrict_elem(int N, const OpGeom& g, const T* y, const T* b, const T* eta,
                                   T* r1, cudaStream_t s);
template <typename T>
bool launch_cheb_elem(int N, const OpGeom& g, const T* x, const T* z, T* r, const T* eta,
                      const int* emap, const T* cls_inv, const int* cls_sym, const T* uniq_inv,
                      const T* eta_inv, const T* d_old, T* d_new, T* yv, T c1, T c2, bool pend,
                      cudaStream_t s);
struct dd;
// y = A x + z in double-double (the tile kernel with T = dd)
void launch_apply_sip_dd(int N, const OpGeom& g, const dd* x, dd* y, const dd* eta, const dd* z,
                         cudaStream_t s);
template <typename T>
void launch_apply_B(int k, const OpGeom& g, const T* p, T* y, cudaStream_t s);
template <typename T>
void launch_apply_Bt(int k, const OpGeom& g, const T* u, T* y, cudaStream_t s);
void launch_rhs_body_force(int k, const OpGeom& g, const double* rho, double grav, double* f,
                           cudaStream_t s);
void launch_rasterise(int nx, int ny, double lx, double ly, const double* shapes, int ns,
                      double eta_bg, double rho_bg, double* eta, double* rho, cudaStream_t s);

// ---------------------------------------------------------- device memory
// Stream on which this host thread's library allocations are ordered
// (stream-ordered allocator, cudaMallocAsync / cudaFreeAsync: no device-wide
// synchronisation, so independent solves on other streams keep running).
// Defaults to the legacy default stream.
cudaStream_t& alloc_stream();

struct AllocStreamScope {
    cudaStream_t prev;
    explicit AllocStreamScope(cudaStream_t s) : prev(alloc_stream()) { alloc_stream() = s; }
    ~AllocStreamScope() { alloc_stream() = prev; }
};

// While set (this thread), buffers are returned on the legacy default stream
// instead of the stream they were allocated on.  Used where the device has
// just been synchronised (problem destruction): the allocation stream may be
// gone by then (a caller's stream, a finished batch worker's stream).
bool& release_on_legacy();

struct ReleaseOnLegacyScope {
    bool prev;
    ReleaseOnLegacyScope() : prev(release_on_legacy()) { release_on_legacy() = true; }
    ~ReleaseOnLegacyScope() { release_on_legacy() = prev; }
};

struct DeviceBuffer {
    void* ptr = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;   // stream the allocation is ordered on
    DeviceBuffer() = default;
    DeviceBuffer(const DeviceBuffer&) = delete;
    DeviceBuffer& operator=(const DeviceBuffer&) = delete;
    DeviceBuffer(DeviceBuffer&& o) noexcept : ptr(o.ptr), bytes(o.bytes), st(o.st) {
        o.ptr = nullptr;
        o.bytes = 0;
    }
    DeviceBuffer& operator=(DeviceBuffer&& o) noexcept {
        if (this != &o) {
            release();
            ptr = o.ptr;
            bytes = o.bytes;
            st = o.st;
            o.ptr = nullptr;
            o.bytes = 0;
        }
        return *this;
    }
    ~DeviceBuffer() { release(); }
    void release() {
        if (ptr) cudaFreeAsync(ptr, release_on_legacy() ? cudaStreamLegacy : st);
        ptr = nullptr;
        bytes = 0;
    }
    // Ensure at least b bytes; an existing buffer that is large enough is
    // kept (re-running a set-up on the same problem allocates nothing).
    void alloc(size_t b) {
        if (ptr && bytes >= b) return;
        release();
        if (b == 0) return;
        st = alloc_stream();
        cudaError_t e = cudaMallocAsync(&ptr, b, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ptr = nullptr;
            throw Error(SIP_ERR_OOM, "device allocation of " + std::to_string(b) + " bytes failed");
        }
        bytes = b;
    }
    template <typename T>
    T* as() const {
        return static_cast<T*>(ptr);
    }
};

}  // namespace sip

struct sip_ctx {
    int device = 0;
    std::string err;
};
