// Inter-level transfers and h-level operators of the hp-multigrid (Sec. 6):
//  - p-restriction / prolongation between Q_k and the hierarchical Q_1 modes
//    (injection and its transpose);
//  - P_cd / R_dc = P_cd^T between continuous bilinears at the vertices and
//    element-wise modal Q_1 coefficients (nodal -> modal);
//  - vertex-centred bilinear P_h / R_h = P_h^T between vertex grids;
//  - the 9-point, 2x2-block stencil operators of the continuous levels, their
//    point-Jacobi / Chebyshev update, and the probing that forms the Galerkin
//    stencils;
//  - a dense symmetric matrix-vector product for the coarsest-level inverse.
#include "sip_internal.h"
#include "sip_level.cuh"

namespace sip {

namespace {

// p-transfers to the coarse space of the M x M lowest modes per component
// (M = 2: Q^2_1, M = 1: Q^2_0), coarse layout [e][c][j][i] with i, j < M.
template <typename T>
__global__ void k_p_restrict(size_t ne, int N, int M, const T* __restrict__ r,
                             T* __restrict__ r1) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int per = 2 * M * M;
    if (g >= ne * per) return;
    const size_t e = g / per;
    const int l = int(g % per), c = l / (M * M), j = (l / M) % M, i = l % M;
    r1[g] = r[e * 2 * N * N + c * N * N + j * N + i];
}

template <typename T>
__global__ void k_p_prolong_add(size_t ne, int N, int M, const T* __restrict__ e1,
                                T* __restrict__ y) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int per = 2 * M * M;
    if (g >= ne * per) return;
    const size_t e = g / per;
    const int l = int(g % per), c = l / (M * M), j = (l / M) % M, i = l % M;
    y[e * 2 * N * N + c * N * N + j * N + i] += e1[g];
}

template <typename T>
__global__ void k_pcd(int nx, int ny, const T* __restrict__ v, T* __restrict__ out) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const size_t ne = size_t(nx) * ny;
    if (g >= ne * 8) return;
    const size_t e = g / 8;
    const int l = int(g % 8), c = l / 4, j = (l / 2) % 2, i = l % 2;
    const int ex = int(e % nx), ey = int(e / nx);
    double acc = 0.0;
    for (int q = 0; q < 2; ++q)
        for (int p = 0; p < 2; ++p)
            acc += hatw(i, p) * hatw(j, q) * double(v[2 * (size_t(ey + q) * (nx + 1) + ex + p) + c]);
    out[g] = T(acc);
}

template <typename T>
__global__ void k_rdc(int nx, int ny, const T* __restrict__ r, T* __restrict__ out) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const size_t nv = size_t(nx + 1) * (ny + 1);
    if (g >= nv * 2) return;
    const int c = int(g % 2);
    const size_t v = g / 2;
    const int vx = int(v % (nx + 1)), vy = int(v / (nx + 1));
    double acc = 0.0;
    for (int q = 0; q < 2; ++q) {          // vertex is corner q (in y) of element row vy - q
        const int ey = vy - q;
        if (ey < 0 || ey >= ny) continue;
        for (int p = 0; p < 2; ++p) {
            const int ex = vx - p;
            if (ex < 0 || ex >= nx) continue;
            const T* re = r + (size_t(ey) * nx + ex) * 8 + c * 4;
            for (int j = 0; j < 2; ++j)
                for (int i = 0; i < 2; ++i) acc += hatw(i, p) * hatw(j, q) * double(re[j * 2 + i]);
        }
    }
    out[g] = T(acc);
}

template <typename T>
bool pair_aligned(const T* p) {
    return (reinterpret_cast<uintptr_t>(p) % (2 * sizeof(T))) == 0;
}

// y = alpha * S x + beta * z for the 9-point 2x2-block stencil on an
// (nvx x nvy) vertex grid; S[v][t][c][c'], t = (dy+1)*3 + (dx+1).
template <typename T, bool VEC>
__global__ void k_stencil_apply(int nvx, int nvy, const T* __restrict__ S, const T* __restrict__ x,
                                T* __restrict__ y, T alpha, const T* __restrict__ z, T beta) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const size_t nv = size_t(nvx) * nvy;
    if (g >= nv * 2) return;
    const int c = int(g % 2);
    const size_t v = g / 2;
    const int vx = int(v % nvx), vy = int(v / nvx);
    const T acc = stencil_row<T, VEC>(nvx, nvy, vx, vy, c, S + v * 36, x);
    T out = alpha * acc;
    if (z) out += beta * z[g];
    y[g] = out;
}

template <typename T>
__global__ void k_stencil_dinv(size_t nv, const T* __restrict__ S, T* __restrict__ dinv) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= nv * 2) return;
    const int c = int(g % 2);
    dinv[g] = T(1) / S[(g / 2) * 36 + 4 * 4 + c * 2 + c];
}

// d = c1 d + c2 D^{-1} r;  x = (x_zero ? 0 : x) + d
template <typename T>
__global__ void k_jacobi_cheb(size_t n, const T* __restrict__ r, const T* __restrict__ dinv, T* d,
                              T* x, T c1, T c2, int x_zero) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= n) return;
    T v = c2 * dinv[g] * r[g];
    if (c1 != T(0)) v += c1 * d[g];
    d[g] = v;
    if (x) x[g] = x_zero ? v : x[g] + v;
}

// First Chebyshev step from a zero iterate: r = b, d = c2 D^{-1} b, x = d.
template <typename T>
__global__ void k_hcheb_first(size_t n, const T* __restrict__ b, const T* __restrict__ dinv,
                              T* __restrict__ r, T* __restrict__ d, T* __restrict__ x, T c2) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const T bv = b[g];
    const T v = c2 * dinv[g] * bv;
    r[g] = bv;
    d[g] = v;
    x[g] = v;
}

// First Chebyshev step from a non-zero iterate, without its x update (x
// is read by neighbours here): r = b - S x, d = c2 D^{-1} r.  The next
// step adds d to x together with its own direction.
template <typename T, bool VEC>
__global__ void k_hcheb_start(int nvx, int nvy, const T* __restrict__ S, const T* __restrict__ dinv,
                              const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ r,
                              T* __restrict__ d, T c2) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const size_t nv = size_t(nvx) * nvy;
    if (g >= nv * 2) return;
    const int c = int(g % 2);
    const size_t v = g / 2;
    const int vx = int(v % nvx), vy = int(v / nvx);
    const T acc = stencil_row<T, VEC>(nvx, nvy, vx, vy, c, S + v * 36, x);
    const T rn = b[g] - acc;
    r[g] = rn;
    d[g] = c2 * dinv[g] * rn;
}

// One fused Chebyshev / point-Jacobi step on a continuous level:
// r -= S d_old;  d_new = c1 d_old + c2 D^{-1} r;  x += d_new (+ d_old when
// pend: the start step's deferred update).  d_old is only read (neighbours
// too), d_new only written: no races.
template <typename T, bool VEC>
__global__ void k_hcheb_step(int nvx, int nvy, const T* __restrict__ S, const T* __restrict__ dinv,
                             T* __restrict__ r, const T* __restrict__ d_old, T* __restrict__ d_new,
                             T* __restrict__ x, T c1, T c2, int pend) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const size_t nv = size_t(nvx) * nvy;
    if (g >= nv * 2) return;
    const int c = int(g % 2);
    const size_t v = g / 2;
    const int vx = int(v % nvx), vy = int(v / nvx);
    const T acc = stencil_row<T, VEC>(nvx, nvy, vx, vy, c, S + v * 36, d_old);
    const T rn = r[g] - acc;
    r[g] = rn;
    const T dn = c1 * d_old[g] + c2 * dinv[g] * rn;
    d_new[g] = dn;
    x[g] += pend ? d_old[g] + dn : dn;
}

// fine (2 nxc + 1)^2 <- coarse (nxc + 1)^2 vertex grid, bilinear (add to y)
template <typename T>
__global__ void k_ph_add(int nxc, int nyc, const T* __restrict__ xc, T* __restrict__ yf) {
    grid_dep_wait();
    const int nfx = 2 * nxc + 1, nfy = 2 * nyc + 1;
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= size_t(nfx) * nfy * 2) return;
    const int c = int(g % 2);
    const size_t v = g / 2;
    const int fx = int(v % nfx), fy = int(v / nfx);
    T acc = T(0);
    const int ix0 = fx / 2, ix1 = (fx + 1) / 2, iy0 = fy / 2, iy1 = (fy + 1) / 2;
    const T wx = (fx % 2) ? T(0.5) : T(1), wy = (fy % 2) ? T(0.5) : T(1);
    if (fx % 2 == 0 && fy % 2 == 0) {
        acc = xc[2 * (size_t(iy0) * (nxc + 1) + ix0) + c];
    } else if (fy % 2 == 0) {
        acc = wx * (xc[2 * (size_t(iy0) * (nxc + 1) + ix0) + c] + xc[2 * (size_t(iy0) * (nxc + 1) + ix1) + c]);
    } else if (fx % 2 == 0) {
        acc = wy * (xc[2 * (size_t(iy0) * (nxc + 1) + ix0) + c] + xc[2 * (size_t(iy1) * (nxc + 1) + ix0) + c]);
    } else {
        acc = wx * wy * (xc[2 * (size_t(iy0) * (nxc + 1) + ix0) + c] + xc[2 * (size_t(iy0) * (nxc + 1) + ix1) + c] +
                         xc[2 * (size_t(iy1) * (nxc + 1) + ix0) + c] + xc[2 * (size_t(iy1) * (nxc + 1) + ix1) + c]);
    }
    yf[g] += acc;
}

// R_h = P_h^T: coarse vertex gathers fine vertices 2I-1 .. 2I+1 with weights 1/2, 1, 1/2
template <typename T>
__global__ void k_rh(int nxc, int nyc, const T* __restrict__ rf, T* __restrict__ rc) {
    grid_dep_wait();
    const int nfx = 2 * nxc + 1, nfy = 2 * nyc + 1;
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= size_t(nxc + 1) * (nyc + 1) * 2) return;
    const int c = int(g % 2);
    const size_t v = g / 2;
    const int I = int(v % (nxc + 1)), J = int(v / (nxc + 1));
    T acc = T(0);
    for (int dy = -1; dy <= 1; ++dy) {
        const int fy = 2 * J + dy;
        if (fy < 0 || fy >= nfy) continue;
        const T wy = dy == 0 ? T(1) : T(0.5);
        for (int dx = -1; dx <= 1; ++dx) {
            const int fx = 2 * I + dx;
            if (fx < 0 || fx >= nfx) continue;
            const T wx = dx == 0 ? T(1) : T(0.5);
            acc += wx * wy * rf[2 * (size_t(fy) * nfx + fx) + c];
        }
    }
    rc[g] = acc;
}

// probe vector: 1 on vertices of colour (vx % 3, vy % 3) == (col % 3, col / 3), component cp
template <typename T>
__global__ void k_probe_vertices(int nvx, int nvy, int col, int cp, T* x) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= size_t(nvx) * nvy * 2) return;
    const int c = int(g % 2);
    const size_t v = g / 2;
    const int vx = int(v % nvx), vy = int(v / nvx);
    x[g] = (c == cp && vx % 3 == col % 3 && vy % 3 == col / 3) ? T(1) : T(0);
}

// S[v][t][c][cp] from the 18 probe results Y[col*2 + cp][v][c]
template <typename T>
__global__ void k_extract_stencil(int nvx, int nvy, const T* __restrict__ Y, T* __restrict__ S) {
    grid_dep_wait();
    const size_t nv = size_t(nvx) * nvy;
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= nv * 36) return;
    const size_t v = g / 36;
    const int rem = int(g % 36), t = rem / 4, c = (rem / 2) % 2, cp = rem % 2;
    const int vx = int(v % nvx), vy = int(v / nvx);
    const int wx = vx + (t % 3) - 1, wy = vy + (t / 3) - 1;
    T val = T(0);
    if (wx >= 0 && wx < nvx && wy >= 0 && wy < nvy) {
        const int col = (wy % 3) * 3 + (wx % 3);
        val = Y[(size_t(col) * 2 + cp) * nv * 2 + 2 * v + c];
    }
    S[g] = val;
}

// probe vector on the Q_1 DG space: unit on local dof l of every element of
// colour (ex % 3, ey % 3) == (col % 3, col / 3)
template <typename T>
__global__ void k_probe_elements(int nx, int ny, int col, int l, T* x) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= size_t(nx) * ny * 8) return;
    const size_t e = g / 8;
    const int ex = int(e % nx), ey = int(e / nx);
    x[g] = (int(g % 8) == l && ex % 3 == col % 3 && ey % 3 == col / 3) ? T(1) : T(0);
}

// y = M x for a dense symmetric n x n matrix (row-major); one warp per row
template <typename T>
__global__ void k_dense_symv(int n, const T* __restrict__ M, const T* __restrict__ x, T* __restrict__ y) {
    grid_dep_wait();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
    if (warp >= n) return;
    const T* row = M + size_t(warp) * n;
    T acc = T(0);
    for (int j = lane; j < n; j += 32) acc += row[j] * x[j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) y[warp] = acc;
}

// Dense inverse from a banded Cholesky factor L (lower, band width bw,
// stored L[i][bw-1-(i-j)] for i-bw < j <= i): thread = column of the inverse.
__global__ void k_band_chol_inverse(int n, int bw, const double* __restrict__ L, double* X) {
    grid_dep_wait();
    // column col of the inverse is kept as X[i][col] (X is symmetric), so the
    // 32 columns of a warp are contiguous and every access is coalesced; the
    // forward solve starts at row col (the entries above it are zero)
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= n) return;
    for (int i = 0; i < col; ++i) X[size_t(i) * n + col] = 0.0;
    for (int i = col; i < n; ++i) {    // L y = e_col
        double s = (i == col) ? 1.0 : 0.0;
        const int j0 = i - bw + 1 > col ? i - bw + 1 : col;
        for (int j = j0; j < i; ++j) s -= L[size_t(i) * bw + (bw - 1 - (i - j))] * X[size_t(j) * n + col];
        X[size_t(i) * n + col] = s / L[size_t(i) * bw + (bw - 1)];
    }
    for (int i = n - 1; i >= 0; --i) { // L^T x = y
        double s = X[size_t(i) * n + col];
        const int j1 = i + bw - 1 < n - 1 ? i + bw - 1 : n - 1;
        for (int j = i + 1; j <= j1; ++j) s -= L[size_t(j) * bw + (bw - 1 - (j - i))] * X[size_t(j) * n + col];
        X[size_t(i) * n + col] = s / L[size_t(i) * bw + (bw - 1)];
    }
}

template <typename T>
__global__ void k_convert(size_t n, const double* __restrict__ a, T* __restrict__ b) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g < n) b[g] = T(a[g]);
}

inline unsigned nblk(size_t n, int t = 256) { return unsigned((n + t - 1) / t); }

}  // namespace

template <typename T>
void launch_p_restrict(size_t ne, int N, const T* r, T* r1, cudaStream_t s, int M) {
    launch_k(k_p_restrict<T>, nblk(ne * 2 * M * M), 256, 0, s, ne, N, M, r, r1);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_p_prolong_add(size_t ne, int N, const T* e1, T* y, cudaStream_t s, int M) {
    launch_k(k_p_prolong_add<T>, nblk(ne * 2 * M * M), 256, 0, s, ne, N, M, e1, y);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_pcd(int nx, int ny, const T* v, T* out, cudaStream_t s) {
    launch_k(k_pcd<T>, nblk(size_t(nx) * ny * 8), 256, 0, s, nx, ny, v, out);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_rdc(int nx, int ny, const T* r, T* out, cudaStream_t s) {
    launch_k(k_rdc<T>, nblk(size_t(nx + 1) * (ny + 1) * 2), 256, 0, s, nx, ny, r, out);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_stencil_apply(int nvx, int nvy, const T* S, const T* x, T* y, T alpha, const T* z,
                          T beta, cudaStream_t s) {
    const unsigned nb = nblk(size_t(nvx) * nvy * 2);
    if (pair_aligned(S) && pair_aligned(x))
        launch_k(k_stencil_apply<T, true>, nb, 256, 0, s, nvx, nvy, S, x, y, alpha, z, beta);
    else
        launch_k(k_stencil_apply<T, false>, nb, 256, 0, s, nvx, nvy, S, x, y, alpha, z, beta);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_stencil_dinv(size_t nv, const T* S, T* dinv, cudaStream_t s) {
    launch_k(k_stencil_dinv<T>, nblk(nv * 2), 256, 0, s, nv, S, dinv);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_jacobi_cheb(size_t n, const T* r, const T* dinv, T* d, T* x, T c1, T c2, bool x_zero,
                        cudaStream_t s) {
    launch_k(k_jacobi_cheb<T>, nblk(n), 256, 0, s, n, r, dinv, d, x, c1, c2, x_zero ? 1 : 0);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_hcheb_first(size_t n, const T* b, const T* dinv, T* r, T* d, T* x, T c2,
                        cudaStream_t s) {
    launch_k(k_hcheb_first<T>, nblk(n), 256, 0, s, n, b, dinv, r, d, x, c2);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_hcheb_start(int nvx, int nvy, const T* S, const T* dinv, const T* b, const T* x, T* r,
                        T* d, T c2, cudaStream_t s) {
    const unsigned nb = nblk(size_t(nvx) * nvy * 2);
    if (pair_aligned(S) && pair_aligned(x))
        launch_k(k_hcheb_start<T, true>, nb, 256, 0, s, nvx, nvy, S, dinv, b, x, r, d, c2);
    else
        launch_k(k_hcheb_start<T, false>, nb, 256, 0, s, nvx, nvy, S, dinv, b, x, r, d, c2);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_hcheb_step(int nvx, int nvy, const T* S, const T* dinv, T* r, const T* d_old,
                       T* d_new, T* x, T c1, T c2, bool pend, cudaStream_t s) {
    const unsigned nb = nblk(size_t(nvx) * nvy * 2);
    if (pair_aligned(S) && pair_aligned(d_old))
        launch_k(k_hcheb_step<T, true>, nb, 256, 0, s, nvx, nvy, S, dinv, r, d_old, d_new, x, c1, c2,
                                                 pend ? 1 : 0);
    else
        launch_k(k_hcheb_step<T, false>, nb, 256, 0, s, nvx, nvy, S, dinv, r, d_old, d_new, x, c1, c2,
                                                  pend ? 1 : 0);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_ph_add(int nxc, int nyc, const T* xc, T* yf, cudaStream_t s) {
    launch_k(k_ph_add<T>, nblk(size_t(2 * nxc + 1) * (2 * nyc + 1) * 2), 256, 0, s, nxc, nyc, xc, yf);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_rh(int nxc, int nyc, const T* rf, T* rc, cudaStream_t s) {
    launch_k(k_rh<T>, nblk(size_t(nxc + 1) * (nyc + 1) * 2), 256, 0, s, nxc, nyc, rf, rc);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_probe_vertices(int nvx, int nvy, int col, int cp, T* x, cudaStream_t s) {
    launch_k(k_probe_vertices<T>, nblk(size_t(nvx) * nvy * 2), 256, 0, s, nvx, nvy, col, cp, x);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_extract_stencil(int nvx, int nvy, const T* Y, T* S, cudaStream_t s) {
    launch_k(k_extract_stencil<T>, nblk(size_t(nvx) * nvy * 36), 256, 0, s, nvx, nvy, Y, S);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_probe_elements(int nx, int ny, int col, int l, T* x, cudaStream_t s) {
    launch_k(k_probe_elements<T>, nblk(size_t(nx) * ny * 8), 256, 0, s, nx, ny, col, l, x);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_dense_symv(int n, const T* M, const T* x, T* y, cudaStream_t s) {
    launch_k(k_dense_symv<T>, nblk(size_t(n) * 32, 128), 128, 0, s, n, M, x, y);
    SIP_CHECK_LAUNCH();
}
void launch_band_chol_inverse(int n, int bw, const double* L, double* X, cudaStream_t s) {
    launch_k(k_band_chol_inverse, nblk(n, 32), 32, 0, s, n, bw, L, X);
    SIP_CHECK_LAUNCH();
}
template <typename T>
void launch_convert(size_t n, const double* a, T* b, cudaStream_t s) {
    launch_k(k_convert<T>, nblk(n), 256, 0, s, n, a, b);
    SIP_CHECK_LAUNCH();
}

#define SIP_INST(T)                                                                              \
    template void launch_p_restrict<T>(size_t, int, const T*, T*, cudaStream_t, int);           \
    template void launch_p_prolong_add<T>(size_t, int, const T*, T*, cudaStream_t, int);        \
    template void launch_pcd<T>(int, int, const T*, T*, cudaStream_t);                          \
    template void launch_rdc<T>(int, int, const T*, T*, cudaStream_t);                          \
    template void launch_stencil_apply<T>(int, int, const T*, const T*, T*, T, const T*, T,     \
                                          cudaStream_t);                                         \
    template void launch_stencil_dinv<T>(size_t, const T*, T*, cudaStream_t);                   \
    template void launch_jacobi_cheb<T>(size_t, const T*, const T*, T*, T*, T, T, bool,         \
                                        cudaStream_t);                                           \
    template void launch_ph_add<T>(int, int, const T*, T*, cudaStream_t);                       \
    template void launch_hcheb_first<T>(size_t, const T*, const T*, T*, T*, T*, T, cudaStream_t); \
    template void launch_hcheb_step<T>(int, int, const T*, const T*, T*, const T*, T*, T*, T, T,  \
                                       bool, cudaStream_t);                                      \
    template void launch_hcheb_start<T>(int, int, const T*, const T*, const T*, const T*, T*, T*, \
                                        T, cudaStream_t);                                        \
    template void launch_rh<T>(int, int, const T*, T*, cudaStream_t);                           \
    template void launch_probe_vertices<T>(int, int, int, int, T*, cudaStream_t);               \
    template void launch_extract_stencil<T>(int, int, const T*, T*, cudaStream_t);              \
    template void launch_probe_elements<T>(int, int, int, int, T*, cudaStream_t);               \
    template void launch_dense_symv<T>(int, const T*, const T*, T*, cudaStream_t);              \
    template void launch_convert<T>(size_t, const double*, T*, cudaStream_t);
SIP_INST(double)
SIP_INST(float)
#undef SIP_INST

}  // namespace sip
