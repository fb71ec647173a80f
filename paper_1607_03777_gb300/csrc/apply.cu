// Matrix-free SIP-DG operators on sm_103a: the viscous operator A
// (eq. stiffness_form), B and B^T (eq. divergence_form), the body-force load
// vector (eq. rhs_f) and the element-wise material rasterisation (Sec. 7.3).
//
// On an affine Cartesian cell every term of the weak form is a sum of
// Kronecker products of 1D reference integrals of the orthonormal Legendre
// basis (G = int l' l', D = int l l', traces l(+-1), l'(+-1)), so the operator
// is applied exactly without quadrature.  Face terms reduce to 1D vectors
// along the face: for the face of K with outward normal s e_d the test mode
// (q along d, m along the face) receives l_q(s) P[m] + l_q'(s) Q[m], where P
// and Q combine the traces of K and its neighbour.
#include <cstdlib>
#include <mutex>

#include "dd.cuh"
#include "sip_face.cuh"
#include "sip_internal.h"

namespace sip {

namespace {

template <int N>
struct TileCfg {
    // elements of one mesh row handled by one CTA
    static constexpr int EX = (N <= 3) ? 32 : (N <= 5 ? 16 : 8);
};

// TS: storage precision of x, y, z and eta; T: arithmetic precision (the
// values are converted to T on their way into shared memory and rounded to
// TS once, at the output).
template <int N, typename TS, typename T>
struct ApplyArgs {
    const TS* x;
    TS* y;
    const TS* eta;
    const TS* z;
    T alpha, beta;
    int nx, ny;
    T hx, hy;
    T two_over_hx, two_over_hy;
    T c2hy_hx, chx_hy, c2hx_hy, chy_hx;   // 2hy/hx, hx/hy, 2hx/hy, hy/hx
    FaceGeo<T> fgx, fgy;                  // faces with x- and y-normal
    int bc[4];
    T pen_x, pen_y;
    Tab1D<N, T> tab;
};

template <int N, typename T>
constexpr size_t apply_smem_elems() {
    constexpr int NN = N * N, NB = 2 * NN, EX = TileCfg<N>::EX, EXH = EX + 2;
    return size_t(3) * EXH * NB      // su
           + 3 * EXH                 // seta
           + 2 * (EX + 1) * 4 * N    // tv, td
           + 2 * EX * 8 * N          // hv, hd
           + 2 * EX * NN             // wx, wy
           + EX * 4 * 2 * 2 * N;     // pq
}

// y = alpha * (A x) + beta * z.  One CTA = EX consecutive elements of one mesh
// row.  Stage 0 stages the x blocks of rows ey-1, ey, ey+1 (one element of
// halo left and right) in shared memory; stage 1 computes face traces and
// the volume cross-term intermediates; stage 2 the face vectors P, Q; stage 3
// writes each output mode once (no atomics; every face is evaluated from
// both sides).
template <int N, typename TS, typename T>
__global__ void __launch_bounds__(256) k_apply_sip(const ApplyArgs<N, TS, T> a) {
    grid_dep_wait();
    constexpr int NN = N * N, NB = 2 * NN, EX = TileCfg<N>::EX, EXH = EX + 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* su = reinterpret_cast<T*>(smem_raw);
    T* seta = su + 3 * EXH * NB;
    T* tv = seta + 3 * EXH;
    T* td = tv + (EX + 1) * 4 * N;
    T* hv = td + (EX + 1) * 4 * N;
    T* hd = hv + EX * 8 * N;
    T* wx = hd + EX * 8 * N;
    T* wy = wx + EX * NN;
    T* pq = wy + EX * NN;

    const int nx = a.nx, ny = a.ny;
    const int ex0 = blockIdx.x * EX, ey = blockIdx.y;
    const int tid = threadIdx.x, nt = blockDim.x;

    // ---- stage 0: load rows ey-1, ey, ey+1, columns ex0-1 .. ex0+EX
    {
        const int exa = ex0 - 1 < 0 ? 0 : ex0 - 1;
        const int exb = ex0 + EX > nx - 1 ? nx - 1 : ex0 + EX;
        const int ncol = exb - exa + 1;
        for (int r = 0; r < 3; ++r) {
            const int eyr = ey + r - 1;
            if (eyr < 0 || eyr >= ny) continue;
            const TS* src = a.x + (size_t(eyr) * nx + exa) * NB;
            T* dst = su + (size_t(r) * EXH + (exa - (ex0 - 1))) * NB;
            const int cnt = ncol * NB;
            for (int q = tid; q < cnt; q += nt) dst[q] = T(src[q]);
            for (int q = tid; q < ncol; q += nt)
                seta[r * EXH + (exa - (ex0 - 1)) + q] = T(a.eta[size_t(eyr) * nx + exa + q]);
        }
    }
    __syncthreads();

    // ---- stage 1a: traces on the EX+1 vertical faces (both sides)
    for (int q = tid; q < (EX + 1) * 4 * N; q += nt) {
        const int j = q % N, c = (q / N) % 2, side = (q / (2 * N)) % 2, f = q / (4 * N);
        const int m = f + side;
        const int ex = ex0 - 1 + m;
        if (ex < 0 || ex >= nx) continue;
        const T* u = su + (EXH + m) * NB + c * NN + j * N;
        const T* lt = side == 0 ? a.tab.lp : a.tab.lm;  // left element sees xi = +1
        const T* dt = side == 0 ? a.tab.dp : a.tab.dm;
        T v = T(0), d = T(0);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            v += u[i] * lt[i];
            d += u[i] * dt[i];
        }
        tv[q] = v;
        td[q] = d * a.two_over_hx;
    }
    // ---- stage 1b: traces on the bottom / top faces of each tile element
    for (int q = tid; q < EX * 8 * N; q += nt) {
        const int i = q % N, c = (q / N) % 2, side = (q / (2 * N)) % 2, face = (q / (4 * N)) % 2,
                  t = q / (8 * N);
        if (ex0 + t >= nx) continue;
        const int r = side == 0 ? 1 : (face == 0 ? 0 : 2);
        const int eyr = ey + r - 1;
        if (eyr < 0 || eyr >= ny) continue;
        const bool plus = side == 0 ? (face == 1) : (face == 0);
        const T* u = su + (r * EXH + t + 1) * NB + c * NN + i;
        const T* lt = plus ? a.tab.lp : a.tab.lm;
        const T* dt = plus ? a.tab.dp : a.tab.dm;
        T v = T(0), d = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            v += u[j * N] * lt[j];
            d += u[j * N] * dt[j];
        }
        hv[q] = v;
        hd[q] = d * a.two_over_hy;
    }
    // ---- stage 1c: volume cross-term intermediates
    //   wx[t][j][a] = sum_i D[a][i] uy[j][i],  wy[t][b][i] = sum_j D[b][j] ux[j][i]
    for (int q = tid; q < EX * 2 * NN; q += nt) {
        const int lo = q % NN, which = (q / NN) % 2, t = q / (2 * NN);
        const T* u = su + (EXH + t + 1) * NB;
        T acc = T(0);
        if (which == 0) {
            const int av = lo % N, j = lo / N;
#pragma unroll
            for (int i = 0; i < N; ++i) acc += a.tab.D[av * N + i] * u[NN + j * N + i];
            wx[t * NN + lo] = acc;
        } else {
            const int i = lo % N, b = lo / N;
#pragma unroll
            for (int j = 0; j < N; ++j) acc += a.tab.D[b * N + j] * u[j * N + i];
            wy[t * NN + lo] = acc;
        }
    }
    __syncthreads();

    // ---- stage 2: face vectors P, Q for faces L, R, B, T of each element
    for (int q = tid; q < EX * 4 * 2 * N; q += nt) {
        const int m = q % N, c = (q / N) % 2, F = (q / (2 * N)) % 4, t = q / (8 * N);
        const int ex = ex0 + t;
        if (ex >= nx) continue;
        const T etaK = seta[EXH + t + 1];
        const T *vo, *dv, *vn, *dn;
        T etaN = T(0), s, pen;
        const FaceGeo<T>* fg;
        int nc, kind, nbr_ok;
        if (F < 2) {  // vertical faces: d = x
            const int f = t + F;                  // face index; L: f = t, R: f = t + 1
            const int own_side = F == 0 ? 1 : 0;  // element is right (L) / left (R) of face
            vo = tv + ((f * 2 + own_side) * 2) * N;
            dv = td + ((f * 2 + own_side) * 2) * N;
            vn = tv + ((f * 2 + 1 - own_side) * 2) * N;
            dn = td + ((f * 2 + 1 - own_side) * 2) * N;
            s = F == 0 ? T(-1) : T(1);
            nbr_ok = F == 0 ? (ex > 0) : (ex < nx - 1);
            kind = nbr_ok ? 0 : 1 + a.bc[F];
            if (nbr_ok) etaN = seta[EXH + t + (F == 0 ? 0 : 2)];
            fg = &a.fgx;
            nc = 0;
            pen = a.pen_x;
        } else {  // horizontal faces: d = y
            const int face = F - 2;
            vo = hv + (((t * 2 + face) * 2 + 0) * 2) * N;
            dv = hd + (((t * 2 + face) * 2 + 0) * 2) * N;
            vn = hv + (((t * 2 + face) * 2 + 1) * 2) * N;
            dn = hd + (((t * 2 + face) * 2 + 1) * 2) * N;
            s = face == 0 ? T(-1) : T(1);
            nbr_ok = face == 0 ? (ey > 0) : (ey < ny - 1);
            kind = nbr_ok ? 0 : 1 + a.bc[F];
            if (nbr_ok) etaN = seta[(face == 0 ? 0 : 2) * EXH + t + 1];
            fg = &a.fgy;
            nc = 1;
            pen = a.pen_y;
        }
        const T eta_e = kind == 0 ? (etaK > etaN ? etaK : etaN) : etaK;
        const T sigma = pen * eta_e * (kind == 0 ? T(1) : T(2));
        T P, Q;
        face_pq<N, T>(kind, c, m, nc, s, *fg, etaK, etaN, sigma, vo, dv, vn, dn, a.tab.D, P, Q);
        pq[((t * 4 + F) * 2 + 0) * 2 * N + c * N + m] = P;
        pq[((t * 4 + F) * 2 + 1) * 2 * N + c * N + m] = Q;
    }
    __syncthreads();

    // ---- stage 3: outputs y_c[b][a]
    for (int q = tid; q < EX * NB; q += nt) {
        const int av = q % N, b = (q / N) % N, c = (q / NN) % 2, t = q / NB;
        const int ex = ex0 + t;
        if (ex >= nx) continue;
        const T* u = su + (EXH + t + 1) * NB;
        const T etaK = seta[EXH + t + 1];
        const T* G = a.tab.G;
        const T* D = a.tab.D;
        T v1 = T(0), v2 = T(0), v3 = T(0);
        if (c == 0) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                v1 += G[av * N + i] * u[b * N + i];
                v2 += G[b * N + i] * u[i * N + av];
                v3 += D[i * N + b] * wx[t * NN + i * N + av];
            }
            v1 *= a.c2hy_hx;
            v2 *= a.chx_hy;
        } else {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                v1 += G[b * N + i] * u[NN + i * N + av];
                v2 += G[av * N + i] * u[NN + b * N + i];
                v3 += D[i * N + av] * wy[t * NN + b * N + i];
            }
            v1 *= a.c2hx_hy;
            v2 *= a.chy_hx;
        }
        T acc = etaK * (v1 + v2 + v3);
        const T* pL = pq + ((t * 4 + 0) * 2) * 2 * N + c * N;
        const T* pR = pq + ((t * 4 + 1) * 2) * 2 * N + c * N;
        const T* pB = pq + ((t * 4 + 2) * 2) * 2 * N + c * N;
        const T* pT = pq + ((t * 4 + 3) * 2) * 2 * N + c * N;
        acc += a.tab.lm[av] * pL[b] + a.tab.dm[av] * pL[2 * N + b];
        acc += a.tab.lp[av] * pR[b] + a.tab.dp[av] * pR[2 * N + b];
        acc += a.tab.lm[b] * pB[av] + a.tab.dm[b] * pB[2 * N + av];
        acc += a.tab.lp[b] * pT[av] + a.tab.dp[b] * pT[2 * N + av];
        const size_t o = (size_t(ey) * nx + ex) * NB + (q - t * NB);
        T out = a.alpha * acc;
        if (a.z) out += a.beta * T(a.z[o]);
        a.y[o] = TS(out);
    }
}

template <int N, typename TS, typename T>
void apply_sip_n(const OpGeom& g, const TS* x, TS* y, const TS* eta, T alpha, const TS* z, T beta,
                 cudaStream_t s) {
    ApplyArgs<N, TS, T> a;
    a.x = x;
    a.y = y;
    a.eta = eta;
    a.z = z;
    a.alpha = alpha;
    a.beta = beta;
    a.nx = g.nx;
    a.ny = g.ny;
    a.hx = T(g.hx);
    a.hy = T(g.hy);
    a.two_over_hx = T(2.0 / g.hx);
    a.two_over_hy = T(2.0 / g.hy);
    a.c2hy_hx = T(2.0 * g.hy / g.hx);
    a.chx_hy = T(g.hx / g.hy);
    a.c2hx_hy = T(2.0 * g.hx / g.hy);
    a.chy_hx = T(g.hy / g.hx);
    a.fgx = make_face_geo<T>(g.hx, g.hy);
    a.fgy = make_face_geo<T>(g.hy, g.hx);
    for (int i = 0; i < 4; ++i) a.bc[i] = g.bc[i];
    a.pen_x = T(g.pen_x);
    a.pen_y = T(g.pen_y);
    a.tab = make_tab<N, T>();
    constexpr int EX = TileCfg<N>::EX;
    const size_t smem = apply_smem_elems<N, T>() * sizeof(T);
    static const bool attr_set = [smem] {   // once per process, thread-safe
        SIP_CUDA(cudaFuncSetAttribute(k_apply_sip<N, TS, T>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        return true;
    }();
    (void)attr_set;
    dim3 grid((g.nx + EX - 1) / EX, g.ny);
    launch_k(k_apply_sip<N, TS, T>, grid, 256, smem, s, a);
    SIP_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ B, B^T
template <int N, typename T>
struct BArgs {
    const T* in;
    T* out;
    int nx, ny;
    T hx, hy;
    int bc[4];
    Tab1D<N, T> tab;
};

// B p: one thread per velocity output (e, c, jq, iq); N = k + 1, pressure
// degree k - 1 (indices < K = N - 1).
template <int N, typename T>
__global__ void k_apply_B(const BArgs<N, T> a) {
    grid_dep_wait();
    constexpr int NN = N * N, NB = 2 * NN, K = N - 1, MP = K * K;
    const size_t gid = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const size_t ne = size_t(a.nx) * a.ny;
    if (gid >= ne * NB) return;
    const int loc = int(gid % NB);
    const size_t e = gid / NB;
    const int ex = int(e % a.nx), ey = int(e / a.nx);
    const int iq = loc % N, jq = (loc / N) % N, c = loc / NN;
    const T* p = a.in + e * MP;
    const T* D = a.tab.D;
    T acc = T(0);
    // volume: -int div(v) p
    if (c == 0 && jq < K) {
        T s = T(0);
        for (int ia = 0; ia < K; ++ia) s += D[ia * N + iq] * p[jq * K + ia];
        acc -= T(0.5) * a.hy * s;
    }
    if (c == 1 && iq < K) {
        T s = T(0);
        for (int jb = 0; jb < K; ++jb) s += D[jb * N + jq] * p[jb * K + iq];
        acc -= T(0.5) * a.hx * s;
    }
    // faces: only the normal component of v sees int {q} [[v.n]]
    for (int F = 0; F < 4; ++F) {
        const int d = F < 2 ? 0 : 1;
        if (c != d) continue;
        const T s = (F % 2 == 0) ? T(-1) : T(1);
        const int qn = d == 0 ? iq : jq;   // test mode along the normal
        const int m = d == 0 ? jq : iq;    // test mode along the face
        if (m >= K) continue;
        int nex = ex, ney = ey;
        if (F == 0) nex--; else if (F == 1) nex++; else if (F == 2) ney--; else ney++;
        const bool interior = nex >= 0 && nex < a.nx && ney >= 0 && ney < a.ny;
        if (!interior && a.bc[F] == SIP_BC_NEUMANN) continue;
        const T* lo = s > 0 ? a.tab.lp : a.tab.lm;
        const T* ln = s > 0 ? a.tab.lm : a.tab.lp;
        T pv = T(0);
        for (int qq = 0; qq < K; ++qq) pv += (d == 0 ? p[m * K + qq] : p[qq * K + m]) * lo[qq];
        const T ht = d == 0 ? a.hy : a.hx;
        if (interior) {
            const T* pn = a.in + (size_t(ney) * a.nx + nex) * MP;
            T pw = T(0);
            for (int qq = 0; qq < K; ++qq) pw += (d == 0 ? pn[m * K + qq] : pn[qq * K + m]) * ln[qq];
            acc += T(0.5) * s * T(0.5) * ht * lo[qn] * (pv + pw);
        } else {
            acc += s * T(0.5) * ht * lo[qn] * pv;
        }
    }
    a.out[gid] = acc;
}

// B^T u: one thread per pressure output (e, jb, ia).
template <int N, typename T>
__global__ void k_apply_Bt(const BArgs<N, T> a) {
    grid_dep_wait();
    constexpr int NN = N * N, NB = 2 * NN, K = N - 1, MP = K * K;
    const size_t gid = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const size_t ne = size_t(a.nx) * a.ny;
    if (gid >= ne * MP) return;
    const int loc = int(gid % MP);
    const size_t e = gid / MP;
    const int ex = int(e % a.nx), ey = int(e / a.nx);
    const int ia = loc % K, jb = loc / K;
    const T* u = a.in + e * NB;
    const T* D = a.tab.D;
    T sx = T(0), sy = T(0);
    for (int i = 0; i < N; ++i) {
        sx += D[ia * N + i] * u[jb * N + i];
        sy += D[jb * N + i] * u[NN + i * N + ia];
    }
    T acc = -T(0.5) * a.hy * sx - T(0.5) * a.hx * sy;
    for (int F = 0; F < 4; ++F) {
        const int d = F < 2 ? 0 : 1;
        const T s = (F % 2 == 0) ? T(-1) : T(1);
        const int qp = d == 0 ? ia : jb;   // pressure mode along the normal
        const int m = d == 0 ? jb : ia;    // along the face
        int nex = ex, ney = ey;
        if (F == 0) nex--; else if (F == 1) nex++; else if (F == 2) ney--; else ney++;
        const bool interior = nex >= 0 && nex < a.nx && ney >= 0 && ney < a.ny;
        if (!interior && a.bc[F] == SIP_BC_NEUMANN) continue;
        const T* lo = s > 0 ? a.tab.lp : a.tab.lm;
        const T* ln = s > 0 ? a.tab.lm : a.tab.lp;
        const T* ud = u + d * NN;
        T v = T(0);
        for (int qq = 0; qq < N; ++qq) v += (d == 0 ? ud[m * N + qq] : ud[qq * N + m]) * lo[qq];
        const T ht = d == 0 ? a.hy : a.hx;
        if (interior) {
            const T* un = a.in + (size_t(ney) * a.nx + nex) * NB + d * NN;
            T w = T(0);
            for (int qq = 0; qq < N; ++qq) w += (d == 0 ? un[m * N + qq] : un[qq * N + m]) * ln[qq];
            acc += T(0.5) * s * T(0.5) * ht * lo[qp] * (v - w);
        } else {
            acc += s * T(0.5) * ht * lo[qp] * v;
        }
    }
    a.out[gid] = acc;
}

template <int N, typename T>
BArgs<N, T> make_bargs(const OpGeom& g, const T* in, T* out) {
    BArgs<N, T> a;
    a.in = in;
    a.out = out;
    a.nx = g.nx;
    a.ny = g.ny;
    a.hx = T(g.hx);
    a.hy = T(g.hy);
    for (int i = 0; i < 4; ++i) a.bc[i] = g.bc[i];
    a.tab = make_tab<N, T>();
    return a;
}

__global__ void k_rhs_body(const double* rho, double grav, double area_half, int nb, size_t ne,
                           double* f) {
    grid_dep_wait();
    const size_t gid = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (gid >= ne * nb) return;
    const size_t e = gid / nb;
    const int loc = int(gid % nb);
    // only the (0,0) mode of the y component: int phi_00 = |K| / 2
    f[gid] = (loc == nb / 2) ? -grav * rho[e] * area_half : 0.0;
}

__global__ void k_rasterise(int nx, int ny, double hx, double hy, const double* shp, int ns,
                            double eta_bg, double rho_bg, double* eta, double* rho) {
    grid_dep_wait();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nx * ny) return;
    const int ex = e % nx, ey = e / nx;
    const double x0 = ex * hx, x1 = x0 + hx, y0 = ey * hy, y1 = y0 + hy;
    double et = eta_bg, rh = rho_bg;
    for (int i = 0; i < ns; ++i) {
        const double* s = shp + 7 * i;
        bool meets, inside;
        if (s[0] == 0.0) {  // disc (cx, cy, r)
            const double cx = s[1], cy = s[2], r = s[3];
            // distance from the centre to the closed cell; the open cell
            // meets the closed disc iff it is below r
            const double dx = fmax(fmax(x0 - cx, cx - x1), 0.0);
            const double dy = fmax(fmax(y0 - cy, cy - y1), 0.0);
            meets = dx * dx + dy * dy < r * r;
            // the cell lies in the disc iff its farthest corner does
            const double fx = fmax(fabs(x0 - cx), fabs(x1 - cx));
            const double fy = fmax(fabs(y0 - cy), fabs(y1 - cy));
            inside = fx * fx + fy * fy <= r * r;
        } else {  // closed box [a, b] x [c, d]
            meets = x0 < s[2] && x1 > s[1] && y0 < s[4] && y1 > s[3];
            inside = x0 >= s[1] && x1 <= s[2] && y0 >= s[3] && y1 <= s[4];
        }
        if (meets) et = fmax(et, s[5]);
        if (inside) rh = fmax(rh, s[6]);
    }
    eta[e] = et;
    rho[e] = rh;
}

}  // namespace

template <typename T>
int apply_variant(const OpGeom& g) {
    static const int forced = [] {
        const char* v = std::getenv("SIP_APPLY_KERNEL");
        if (!v) return int(APPLY_AUTO);
        const std::string e(v);
        return e == "elem2" ? int(APPLY_ELEM2)
                            : (e == "elem1" ? int(APPLY_ELEM1)
                            : (e == "tile" ? int(APPLY_TILE)
                            : (e == "stage" ? int(APPLY_STAGE)
                            : (e == "warp" ? int(APPLY_WARP) : int(APPLY_AUTO)))));
    }();
    return forced != APPLY_AUTO ? forced : g.variant[sizeof(T) == 4 ? 1 : 0];
}
template int apply_variant<double>(const OpGeom&);
template int apply_variant<float>(const OpGeom&);

template <typename T>
void launch_apply_sip(int N, const OpGeom& g, const T* x, T* y, const T* eta, T alpha,
                      const T* z, T beta, cudaStream_t s) {
    // low degrees: thread-per-element kernels with compile-time tables,
    // unless the schedule picks the shared-memory tile kernel
    const int v = apply_variant<T>(g);
    // the split-precision FP32 operator: the staged kernel's two launches
    // (k <= 5), else the tile kernel with FP64 arithmetic throughout
    const bool split = sizeof(T) == 4 && g.n_hi > 0;
    if constexpr (sizeof(T) == 4) {
        if (v == APPLY_WARP && !split &&
            launch_apply_sip_warp(N, g, reinterpret_cast<const float*>(x), reinterpret_cast<float*>(y),
                                  reinterpret_cast<const float*>(eta), float(alpha),
                                  reinterpret_cast<const float*>(z), float(beta), nullptr, s))
            return;
    }
    if ((v == APPLY_STAGE || split) &&
        launch_apply_sip_stage<T>(N, g, x, y, eta, alpha, z, beta, nullptr, s))
        return;
    if constexpr (sizeof(T) == 4) {
        if (split) {
            // no staged kernel at this degree (k = 6): FP64 arithmetic on the
            // FP32 data of the whole mesh rather than FP32 arithmetic on the
            // marked tiles, whose cancellation it cannot afford
            const double a64 = double(alpha), b64 = double(beta);
            switch (N) {
                case 2: apply_sip_n<2, float, double>(g, x, y, eta, a64, z, b64, s); return;
                case 3: apply_sip_n<3, float, double>(g, x, y, eta, a64, z, b64, s); return;
                case 4: apply_sip_n<4, float, double>(g, x, y, eta, a64, z, b64, s); return;
                case 5: apply_sip_n<5, float, double>(g, x, y, eta, a64, z, b64, s); return;
                case 6: apply_sip_n<6, float, double>(g, x, y, eta, a64, z, b64, s); return;
                case 7: apply_sip_n<7, float, double>(g, x, y, eta, a64, z, b64, s); return;
                default: throw Error(SIP_ERR_INVALID_ARG, "unsupported polynomial degree");
            }
        }
    }
    if (v != APPLY_TILE &&
        launch_apply_sip_elem<T>(N, g, x, y, eta, alpha, z, beta, v != APPLY_ELEM1, s))
        return;
    switch (N) {
        case 2: apply_sip_n<2, T>(g, x, y, eta, alpha, z, beta, s); break;
        case 3: apply_sip_n<3, T>(g, x, y, eta, alpha, z, beta, s); break;
        case 4: apply_sip_n<4, T>(g, x, y, eta, alpha, z, beta, s); break;
        case 5: apply_sip_n<5, T>(g, x, y, eta, alpha, z, beta, s); break;
        case 6: apply_sip_n<6, T>(g, x, y, eta, alpha, z, beta, s); break;
        case 7: apply_sip_n<7, T>(g, x, y, eta, alpha, z, beta, s); break;
        default: throw Error(SIP_ERR_INVALID_ARG, "unsupported polynomial degree");
    }
}
template void launch_apply_sip<double>(int, const OpGeom&, const double*, double*, const double*,
                                       double, const double*, double, cudaStream_t);
template void launch_apply_sip<float>(int, const OpGeom&, const float*, float*, const float*,
                                      float, const float*, float, cudaStream_t);

template <typename T>
void launch_apply_B(int k, const OpGeom& g, const T* p, T* y, cudaStream_t s) {
    const size_t total = size_t(g.nx) * g.ny * 2 * (k + 1) * (k + 1);
    const unsigned blocks = unsigned((total + 255) / 256);
    switch (k + 1) {
#define SIP_B_CASE(NN_)                                                                    \
    case NN_: launch_k(k_apply_B<NN_, T>, blocks, 256, 0, s, make_bargs<NN_, T>(g, p, y)); break;
        SIP_B_CASE(2) SIP_B_CASE(3) SIP_B_CASE(4) SIP_B_CASE(5) SIP_B_CASE(6) SIP_B_CASE(7)
#undef SIP_B_CASE
        default: throw Error(SIP_ERR_INVALID_ARG, "unsupported polynomial degree");
    }
    SIP_CHECK_LAUNCH();
}
template void launch_apply_B<double>(int, const OpGeom&, const double*, double*, cudaStream_t);

template <typename T>
void launch_apply_Bt(int k, const OpGeom& g, const T* u, T* y, cudaStream_t s) {
    const size_t total = size_t(g.nx) * g.ny * k * k;
    const unsigned blocks = unsigned((total + 255) / 256);
    switch (k + 1) {
#define SIP_BT_CASE(NN_)                                                                   \
    case NN_: launch_k(k_apply_Bt<NN_, T>, blocks, 256, 0, s, make_bargs<NN_, T>(g, u, y)); break;
        SIP_BT_CASE(2) SIP_BT_CASE(3) SIP_BT_CASE(4) SIP_BT_CASE(5) SIP_BT_CASE(6) SIP_BT_CASE(7)
#undef SIP_BT_CASE
        default: throw Error(SIP_ERR_INVALID_ARG, "unsupported polynomial degree");
    }
    SIP_CHECK_LAUNCH();
}
template void launch_apply_Bt<double>(int, const OpGeom&, const double*, double*, cudaStream_t);

// Double-double instances (residual of iterative refinement): the tile
// kernel, B and B^T evaluate the same operator with the same FP64
// coefficients in ~106-bit arithmetic.
void launch_apply_sip_dd(int N, const OpGeom& g, const dd* x, dd* y, const dd* eta, const dd* z,
                         cudaStream_t s) {
    const dd one(1.0);
    switch (N) {
        case 2: apply_sip_n<2, dd>(g, x, y, eta, one, z, one, s); break;
        case 3: apply_sip_n<3, dd>(g, x, y, eta, one, z, one, s); break;
        case 4: apply_sip_n<4, dd>(g, x, y, eta, one, z, one, s); break;
        case 5: apply_sip_n<5, dd>(g, x, y, eta, one, z, one, s); break;
        case 6: apply_sip_n<6, dd>(g, x, y, eta, one, z, one, s); break;
        case 7: apply_sip_n<7, dd>(g, x, y, eta, one, z, one, s); break;
        default: throw Error(SIP_ERR_INVALID_ARG, "unsupported polynomial degree");
    }
}
template void launch_apply_B<dd>(int, const OpGeom&, const dd*, dd*, cudaStream_t);
template void launch_apply_Bt<dd>(int, const OpGeom&, const dd*, dd*, cudaStream_t);

void launch_rhs_body_force(int k, const OpGeom& g, const double* rho, double grav, double* f,
                           cudaStream_t s) {
    const int nb = 2 * (k + 1) * (k + 1);
    const size_t ne = size_t(g.nx) * g.ny;
    const size_t total = ne * nb;
    launch_k(k_rhs_body, unsigned((total + 255) / 256), 256, 0, s, rho, grav, 0.5 * g.hx * g.hy, nb, ne,
                                                             f);
    SIP_CHECK_LAUNCH();
}

void launch_rasterise(int nx, int ny, double lx, double ly, const double* shapes, int ns,
                      double eta_bg, double rho_bg, double* eta, double* rho, cudaStream_t s) {
    const int ne = nx * ny;
    launch_k(k_rasterise, (ne + 255) / 256, 256, 0, s, nx, ny, lx / nx, ly / ny, shapes, ns, eta_bg,
                                                 rho_bg, eta, rho);
    SIP_CHECK_LAUNCH();
}

// ------------------------------------------------- allocation-free rasteriser
// Device-side home of the inclusion records for sip_rasterise_inclusions_noalloc.
// Every GPU that loads this library holds it (SIP_NOALLOC_MAX_SHAPES records
// of 7 doubles, 224 KiB) until the process exits.  In host code the name
// below is only a host-side stand-in: its device address comes from
// cudaGetSymbolAddress, taken once per device.
static __device__ __align__(256) double g_noalloc_shapes[SIP_NOALLOC_MAX_SHAPES * 7];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the static record array on the current device; resolved
// on the first call per device (the caller made that device current).
double* noalloc_shapes_on(int device) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_shapes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error(SIP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        }
        g_noalloc_ptr[device] = static_cast<double*>(p);
    }
    return g_noalloc_ptr[device];
}

}  // namespace

}  // namespace sip

extern "C" sip_status sip_rasterise_inclusions_noalloc(sip_ctx* ctx, int nx, int ny, double lx,
                                                       double ly, const double* shapes_host,
                                                       int n_shapes, double eta_bg, double rho_bg,
                                                       double* eta_out, double* rho_out,
                                                       void* stream) {
    if (!ctx) return SIP_ERR_INVALID_ARG;
    try {
        using sip::require;
        require(nx >= 1 && ny >= 1 && std::isfinite(lx) && std::isfinite(ly) && lx > 0 && ly > 0,
                "bad mesh");
        require(n_shapes >= 0 && (n_shapes == 0 || shapes_host), "bad inclusion list");
        require(n_shapes <= SIP_NOALLOC_MAX_SHAPES,
                "sip_rasterise_inclusions_noalloc takes at most SIP_NOALLOC_MAX_SHAPES (4096) "
                "inclusion records");
        require(eta_out && rho_out, "null output");
        require(std::isfinite(eta_bg) && eta_bg > 0 && std::isfinite(rho_bg),
                "bad background material");
        for (int i = 0; i < n_shapes; ++i) {
            const double* s = shapes_host + 7 * i;
            for (int j = 0; j < 7; ++j) require(std::isfinite(s[j]), "non-finite inclusion record");
            require(s[0] == 0.0 || s[0] == 1.0, "unknown inclusion kind");
            require(s[0] != 0.0 || s[3] >= 0, "negative radius");
            require(s[5] >= eta_bg && s[6] >= rho_bg,
                    "inclusions must be at least as viscous and dense as the background");
        }
        require(ctx->device >= 0 && ctx->device < sip::kMaxDevices, "device index out of range");
        SIP_CUDA(cudaSetDevice(ctx->device));
        double* dev_shapes = sip::noalloc_shapes_on(ctx->device);
        const cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (n_shapes > 0)
            SIP_CUDA(cudaMemcpyAsync(dev_shapes, shapes_host, size_t(n_shapes) * 7 * sizeof(double),
                                     cudaMemcpyHostToDevice, s));
        sip::launch_rasterise(nx, ny, lx, ly, dev_shapes, n_shapes, eta_bg, rho_bg, eta_out,
                              rho_out, s);
        ctx->err.clear();
        return SIP_OK;
    } catch (const sip::Error& e) {
        ctx->err = e.what();
        return e.status;
    } catch (const std::exception& e) {
        ctx->err = e.what();
        return SIP_ERR_CUDA;
    }
}
