// Thread-per-element SIP apply for low degrees (N = k+1 <= 4).
//
// Same operator as k_apply_sip (eq. stiffness_form), organised so that the
// arithmetic is minimal: one thread owns one element's 2 N^2 coefficients in
// registers, the 1D reference tables are compile-time constants (so the zero
// entries of G = int l'l' and D = int l l' vanish from the unrolled code),
// traces at both ends of a line come from its even and odd parts
// (l_i(-1) = (-1)^i l_i(1)), and the contributions of two opposite faces are
// spread with one multiply-add per mode.  This matters most in FP64, whose
// pipe on GB300 is ~60x narrower than FP32.
//
// A CTA covers TX x TY elements.  Phase A: every element computes the
// traces (value and physical normal derivative, both components) on its four
// faces into shared memory, halo elements the one face that touches the
// tile, and the volume terms into registers.  Phase B: face vectors P, Q
// from own and neighbour traces, spread to the outputs, one write per mode.
#include "sip_face.cuh"
#include "sip_internal.h"

namespace sip {

namespace {

// ---- compile-time tables of the orthonormal Legendre basis ----------------
// Built by constant evaluation and stored as device constants; after loop
// unrolling every index is constant, so each entry becomes an immediate and
// the zero entries of G and D drop out of the code.
constexpr double csqrt_iter(double x, double g, int n) {
    return n == 0 ? g : csqrt_iter(x, 0.5 * (g + x / g), n - 1);
}
constexpr double csqrt(double x) { return x <= 0.0 ? 0.0 : csqrt_iter(x, x > 1.0 ? x : 1.0, 60); }

template <int N>
struct CTabs {
    double lp[N];     // l_i(+1)
    double dp[N];     // l_i'(+1)
    double G[N][N];   // int l_a' l_b'
    double D[N][N];   // int l_p l_q'
};

template <int N>
constexpr CTabs<N> build_ctabs() {
    CTabs<N> t{};
    for (int i = 0; i < N; ++i) {
        const double c = csqrt((2.0 * i + 1.0) / 2.0);
        t.lp[i] = c;
        t.dp[i] = c * i * (i + 1) / 2.0;
    }
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            const int m = a < b ? a : b;
            t.G[a][b] = ((a + b) % 2 == 0 && m >= 1) ? t.lp[a] * t.lp[b] * m * (m + 1) : 0.0;
            t.D[a][b] = (b > a && (b - a) % 2 == 1) ? 2.0 * t.lp[a] * t.lp[b] : 0.0;
        }
    return t;
}

template <int N>
__device__ constexpr CTabs<N> kT = build_ctabs<N>();

constexpr int TX = 32, TY = 2, TXY = TX * TY;
constexpr int NHALO = 2 * TX + 2 * TY;

template <typename T>
struct ElemArgs {
    const T* x;
    T* y;
    const T* eta;
    const T* z;
    T alpha, beta;
    int nx, ny;
    T two_over_hx, two_over_hy;
    T c2hy_hx, chx_hy, c2hx_hy, chy_hx;
    FaceGeo<T> fgx, fgy;
    int bc[4];
    T pen_x, pen_y;
};

// Traces of one element on face F (0 left, 1 right, 2 bottom, 3 top):
// out[0][c][m] = value, out[1][c][m] = physical normal derivative d/dx_d.
template <int N, typename T>
__device__ __forceinline__ void face_traces(const T (&u)[2][N][N], int F, T two_over_h,
                                            T* out /* [2][2][N] */) {
    const bool plus = (F & 1) != 0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int m = 0; m < N; ++m) {
            T ev = T(0), od = T(0), evd = T(0), odd = T(0);
#pragma unroll
            for (int q = 0; q < N; ++q) {
                const T uq = F < 2 ? u[c][m][q] : u[c][q][m];   // q along the normal
                if (q % 2 == 0) {
                    ev += T(kT<N>.lp[q]) * uq;
                    if (q > 0) evd += T(kT<N>.dp[q]) * uq;
                } else {
                    od += T(kT<N>.lp[q]) * uq;
                    odd += T(kT<N>.dp[q]) * uq;
                }
            }
            // l_q(-1) = (-1)^q l_q(1),  l_q'(-1) = -(-1)^q l_q'(1)
            out[0 * 2 * N + c * N + m] = plus ? ev + od : ev - od;
            out[1 * 2 * N + c * N + m] = (plus ? evd + odd : odd - evd) * two_over_h;
        }
}

template <int N, typename T>
__global__ void __launch_bounds__(TXY) k_apply_elem(const ElemArgs<T> a) {
    constexpr int TR = 4 * N;                 // [2 val/der][2 comp][N] per face
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // own element, all four faces: s_tr[TXY][4][TR]; halo: s_halo[NHALO][TR]
    T (*s_tr)[4][TR] = reinterpret_cast<T (*)[4][TR]>(smem_raw);
    T (*s_halo)[TR] = reinterpret_cast<T (*)[TR]>(smem_raw + sizeof(T) * TXY * 4 * TR);
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int ex0 = blockIdx.x * TX, ey0 = blockIdx.y * TY;
    const int ex = ex0 + tx, ey = ey0 + ty;
    const int nx = a.nx, ny = a.ny;
    const bool active = ex < nx && ey < ny;
    constexpr int NB = 2 * N * N;

    // ---- phase A: halo traces (one face per halo element)
    for (int h = threadIdx.x; h < NHALO; h += TXY) {
        int hx, hy, F;   // halo element and the face of it that touches the tile
        if (h < TX) { hx = ex0 + h; hy = ey0 - 1; F = 3; }                    // below: its top
        else if (h < 2 * TX) { hx = ex0 + h - TX; hy = ey0 + TY; F = 2; }     // above: its bottom
        else if (h < 2 * TX + TY) { hx = ex0 - 1; hy = ey0 + h - 2 * TX; F = 1; }   // left: its right
        else { hx = ex0 + TX; hy = ey0 + h - 2 * TX - TY; F = 0; }            // right: its left
        if (hx >= 0 && hx < nx && hy >= 0 && hy < ny) {
            T uh[2][N][N];
            const T* src = a.x + (size_t(hy) * nx + hx) * NB;
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int j = 0; j < N; ++j)
#pragma unroll
                    for (int i = 0; i < N; ++i) uh[c][j][i] = src[c * N * N + j * N + i];
            face_traces<N, T>(uh, F, F < 2 ? a.two_over_hx : a.two_over_hy, s_halo[h]);
        }
    }
    // ---- phase A: own traces and the volume terms
    T y[2][N][N];
    T etaK = T(0);
    if (active) {
        T u[2][N][N];
        const T* src = a.x + (size_t(ey) * nx + ex) * NB;
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int j = 0; j < N; ++j)
#pragma unroll
                for (int i = 0; i < N; ++i) u[c][j][i] = src[c * N * N + j * N + i];
        etaK = a.eta[size_t(ey) * nx + ex];
#pragma unroll
        for (int F = 0; F < 4; ++F)
            face_traces<N, T>(u, F, F < 2 ? a.two_over_hx : a.two_over_hy, s_tr[threadIdx.x][F]);
        // volume: eta_K [ 2(hy/hx) G_x + (hx/hy) G_y + cross ] on u_x, and
        //         eta_K [ 2(hx/hy) G_y + (hy/hx) G_x + cross ] on u_y
#pragma unroll
        for (int b = 0; b < N; ++b)
#pragma unroll
            for (int av = 0; av < N; ++av) {
                T gx0 = T(0), gx1 = T(0), gy0 = T(0), gy1 = T(0);
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    if (kT<N>.G[av][i] != 0.0) {
                        gx0 += T(kT<N>.G[av][i]) * u[0][b][i];
                        gx1 += T(kT<N>.G[av][i]) * u[1][b][i];
                    }
                    if (kT<N>.G[b][i] != 0.0) {
                        gy0 += T(kT<N>.G[b][i]) * u[0][i][av];
                        gy1 += T(kT<N>.G[b][i]) * u[1][i][av];
                    }
                }
                y[0][b][av] = a.c2hy_hx * gx0 + a.chx_hy * gy0;
                y[1][b][av] = a.chy_hx * gx1 + a.c2hx_hy * gy1;
            }
        // cross terms: W_x[j][a] = sum_i D[a][i] u_y[j][i]; y_x[b][a] += sum_j D[j][b] W_x[j][a]
        //              W_y[b][i] = sum_j D[b][j] u_x[j][i]; y_y[b][a] += sum_i D[i][a] W_y[b][i]
        T w[N][N];
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
            for (int av = 0; av < N; ++av) {
                T s = T(0);
#pragma unroll
                for (int i = 0; i < N; ++i)
                    if (kT<N>.D[av][i] != 0.0) s += T(kT<N>.D[av][i]) * u[1][j][i];
                w[j][av] = s;
            }
#pragma unroll
        for (int b = 0; b < N; ++b)
#pragma unroll
            for (int av = 0; av < N; ++av) {
#pragma unroll
                for (int j = 0; j < N; ++j)
                    if (kT<N>.D[j][b] != 0.0) y[0][b][av] += T(kT<N>.D[j][b]) * w[j][av];
            }
#pragma unroll
        for (int b = 0; b < N; ++b)
#pragma unroll
            for (int i = 0; i < N; ++i) {
                T s = T(0);
#pragma unroll
                for (int j = 0; j < N; ++j)
                    if (kT<N>.D[b][j] != 0.0) s += T(kT<N>.D[b][j]) * u[0][j][i];
                w[b][i] = s;
            }
#pragma unroll
        for (int b = 0; b < N; ++b)
#pragma unroll
            for (int av = 0; av < N; ++av) {
#pragma unroll
                for (int i = 0; i < N; ++i)
                    if (kT<N>.D[i][av] != 0.0) y[1][b][av] += T(kT<N>.D[i][av]) * w[b][i];
                y[0][b][av] *= etaK;
                y[1][b][av] *= etaK;
            }
    }
    __syncthreads();
    if (!active) return;

    // ---- phase B: faces, in opposite pairs (left/right, bottom/top)
    T Dm[N * N];
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
        for (int q = 0; q < N; ++q) Dm[p * N + q] = T(kT<N>.D[p][q]);
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
        T PQ[2][2][2][N];   // [face lo/hi][P/Q][c][m]
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int F = 2 * dir + side;
            const T* own = s_tr[threadIdx.x][F];
            const T* nbr = nullptr;
            T etaN = T(0);
            int kind;
            const bool has_nbr = dir == 0 ? (side == 0 ? ex > 0 : ex < nx - 1)
                                          : (side == 0 ? ey > 0 : ey < ny - 1);
            if (has_nbr) {
                kind = 0;
                const int nxi = ex + (dir == 0 ? (side == 0 ? -1 : 1) : 0);
                const int nyi = ey + (dir == 1 ? (side == 0 ? -1 : 1) : 0);
                etaN = a.eta[size_t(nyi) * nx + nxi];
                const int ltx = nxi - ex0, lty = nyi - ey0;
                if (ltx >= 0 && ltx < TX && lty >= 0 && lty < TY) {
                    nbr = s_tr[lty * TX + ltx][F ^ 1];
                } else if (dir == 1) {
                    nbr = s_halo[(side == 0 ? 0 : TX) + tx];
                } else {
                    nbr = s_halo[2 * TX + (side == 0 ? 0 : TY) + ty];
                }
            } else {
                kind = 1 + a.bc[F];
                nbr = own;   // unused by the boundary formulas
            }
            const T eta_e = kind == 0 ? (etaK > etaN ? etaK : etaN) : etaK;
            const T pen = dir == 0 ? a.pen_x : a.pen_y;
            const T sigma = pen * eta_e * (kind == 0 ? T(1) : T(2));
            const T s = side == 0 ? T(-1) : T(1);
            const FaceGeo<T>& fg = dir == 0 ? a.fgx : a.fgy;
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int m = 0; m < N; ++m) {
                    T P, Q;
                    face_pq<N, T>(kind, c, m, dir, s, fg, etaK, etaN, sigma, own, own + 2 * N, nbr,
                                  nbr + 2 * N, Dm, P, Q);
                    PQ[side][0][c][m] = P;
                    PQ[side][1][c][m] = Q;
                }
        }
        // spread: test mode q along the normal, m along the face;
        // q even: l_q(1) (P_hi + P_lo) + l_q'(1) (Q_hi - Q_lo)
        // q odd : l_q(1) (P_hi - P_lo) + l_q'(1) (Q_hi + Q_lo)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int m = 0; m < N; ++m) {
                const T pp = PQ[1][0][c][m] + PQ[0][0][c][m];
                const T pm = PQ[1][0][c][m] - PQ[0][0][c][m];
                const T qp = PQ[1][1][c][m] + PQ[0][1][c][m];
                const T qm = PQ[1][1][c][m] - PQ[0][1][c][m];
#pragma unroll
                for (int q = 0; q < N; ++q) {
                    T add = q % 2 == 0 ? T(kT<N>.lp[q]) * pp : T(kT<N>.lp[q]) * pm;
                    if (q > 0) add += q % 2 == 0 ? T(kT<N>.dp[q]) * qm : T(kT<N>.dp[q]) * qp;
                    if (dir == 0)
                        y[c][m][q] += add;
                    else
                        y[c][q][m] += add;
                }
            }
    }
    T* dst = a.y + (size_t(ey) * nx + ex) * NB;
    const T* zz = a.z ? a.z + (size_t(ey) * nx + ex) * NB : nullptr;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int o = c * N * N + j * N + i;
                T v = a.alpha * y[c][j][i];
                if (zz) v += a.beta * zz[o];
                dst[o] = v;
            }
}

template <int N, typename T>
void apply_elem_n(const OpGeom& g, const T* x, T* y, const T* eta, T alpha, const T* z, T beta,
                  cudaStream_t s) {
    ElemArgs<T> a;
    a.x = x;
    a.y = y;
    a.eta = eta;
    a.z = z;
    a.alpha = alpha;
    a.beta = beta;
    a.nx = g.nx;
    a.ny = g.ny;
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
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY);
    const size_t smem = sizeof(T) * (size_t(TXY) * 4 + NHALO) * 4 * N;
    static const bool attr_set = [smem] {   // once per process, thread-safe
        SIP_CUDA(cudaFuncSetAttribute(k_apply_elem<N, T>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        return true;
    }();
    (void)attr_set;
    k_apply_elem<N, T><<<grid, TXY, smem, s>>>(a);
    SIP_CHECK_LAUNCH();
}

}  // namespace

template <typename T>
bool launch_apply_sip_elem(int N, const OpGeom& g, const T* x, T* y, const T* eta, T alpha,
                           const T* z, T beta, cudaStream_t s) {
    switch (N) {
        case 2: apply_elem_n<2, T>(g, x, y, eta, alpha, z, beta, s); return true;
        case 3: apply_elem_n<3, T>(g, x, y, eta, alpha, z, beta, s); return true;
        case 4: apply_elem_n<4, T>(g, x, y, eta, alpha, z, beta, s); return true;
        default: return false;
    }
}
template bool launch_apply_sip_elem<double>(int, const OpGeom&, const double*, double*,
                                            const double*, double, const double*, double,
                                            cudaStream_t);
template bool launch_apply_sip_elem<float>(int, const OpGeom&, const float*, float*, const float*,
                                           float, const float*, float, cudaStream_t);

}  // namespace sip
