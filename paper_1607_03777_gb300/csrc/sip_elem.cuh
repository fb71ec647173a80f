// Device helpers shared by the element-wise SIP apply kernels (included
// by apply_elem.cu and apply_stage.cu): compile-time 1D tables of the
// orthonormal Legendre basis, the kernel argument block, face traces and the
// volume terms of one velocity component (eq. stiffness_form).
#pragma once

#include "sip_face.cuh"
#include "sip_internal.h"

namespace sip {

// Kernel arguments of the element kernels (shared by translation units).
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
    T* r1;   // component-split kernel: write only the Q^2_1 modes (i, j < 2) here
};

template <typename T>
ElemArgs<T> make_elem_args(const OpGeom& g, const T* x, T* y, const T* eta, T alpha, const T* z,
                           T beta) {
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
    a.r1 = nullptr;
    return a;
}

// Staged-tile apply (apply_stage.cu): TS = storage, TC = arithmetic precision.
template <typename TS, typename TC>
struct StageArgs {
    ElemArgs<TC> c;              // scalars in the arithmetic precision (pointers unused)
    const TS* x;
    TS* y;
    const TS* eta;
    const TS* z;
    TS* r1;                      // non-null: write only the Q^2_1 modes of the result here
    const unsigned char* skip;   // tiles left to the other launch (null: none)
    const int* tiles;            // tile ids of a list launch
    int ntx;                     // tiles per mesh row
    long long n_total;           // entries of x
};

// Many staged applies in one launch (split tiles of 32 x 2 elements): CTA b
// applies args[items[b].x] on tile items[b].y; active (may be null) masks
// members.  N <= 6.
template <typename TS, typename TC>
void launch_apply_stage_batch(int N, const StageArgs<TS, TC>* args, const int2* items,
                              int n_items, const int* active, bool vec, cudaStream_t s);
template <typename TS, typename TC>
StageArgs<TS, TC> stage_args(const OpGeom& g, const TS* x, TS* y, const TS* eta, double alpha,
                             const TS* z, double beta, TS* r1, int N);

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

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

__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }

// Face vectors P, Q of test component C (every tangential mode m) for one
// interior face of K with normal direction dir on side `side` (0: minus, 1:
// plus): the interior case of face_pq with its scalar factors gathered per
// face, no branches on the face kind.  own / nbr: trace records [val c0 |
// val c1 | der c0 | der c1] (N each) of K and of the neighbour.
template <int N, typename T, int C>
__device__ __forceinline__ void face_interior_comp(int dir, int side, const FaceGeo<T>& fg, T pen,
                                                   T etaK, T etaN, const T* own, const T* nbr,
                                                   T* P, T* Q) {
    const int nc = dir, tc = 1 - dir;   // normal / tangential component
    const T s = side ? T(1) : T(-1);
    const T kP = pen * (etaK > etaN ? etaK : etaN) * fg.half_ht;
    if (C == nc) {
        // flux of the normal derivative, symmetry term through the tangential
        // derivative of the jump, penalty
        const T kA = -s * fg.half_ht * etaK, kB = -s * fg.half_ht * etaN;
        const T kC = T(-0.5) * s * etaK, kQ = -s * etaK * fg.ht_over_hn;
        T wt[N];
#pragma unroll
        for (int mm = 0; mm < N; ++mm) wt[mm] = own[tc * N + mm] - nbr[tc * N + mm];
#pragma unroll
        for (int m = 0; m < N; ++m) {
            T dtw = T(0);
#pragma unroll
            for (int mm = 0; mm < N; ++mm)
                if (kT<N>.D[mm][m] != 0.0) dtw = fmat(T(kT<N>.D[mm][m]), wt[mm], dtw);
            const T wn = own[nc * N + m] - nbr[nc * N + m];
            T p = kA * own[2 * N + nc * N + m];
            p = fmat(kB, nbr[2 * N + nc * N + m], p);
            p = fmat(kC, dtw, p);
            P[m] = fmat(kP, wn, p);
            Q[m] = kQ * wn;
        }
    } else {
        // shear flux with the tangential derivative of the normal component
        // on both sides, penalty
        const T kA2 = T(-0.5) * s * fg.half_ht * etaK, kB2 = T(-0.5) * s * fg.half_ht * etaN;
        const T kC = T(-0.5) * s * etaK, kF = T(-0.5) * s * etaN;
        const T kQ = -s * etaK * fg.half_ht_over_hn;
#pragma unroll
        for (int m = 0; m < N; ++m) {
            T svo = T(0), svn = T(0);
#pragma unroll
            for (int mm = 0; mm < N; ++mm)
                if (kT<N>.D[m][mm] != 0.0) {
                    svo = fmat(T(kT<N>.D[m][mm]), own[nc * N + mm], svo);
                    svn = fmat(T(kT<N>.D[m][mm]), nbr[nc * N + mm], svn);
                }
            const T wt = own[tc * N + m] - nbr[tc * N + m];
            T t = kA2 * own[2 * N + tc * N + m];
            t = fmat(kB2, nbr[2 * N + tc * N + m], t);
            t = fmat(kC, svo, t);
            t = fmat(kF, svn, t);
            P[m] = fmat(kP, wt, t);
            Q[m] = kQ * wt;
        }
    }
}

// Spread the face vectors of the two faces with normal direction dir into
// one component's result: test mode q along the normal, m along the face;
// the even / odd parts of l_q(+-1) and l_q'(+-1) combine the two faces.
template <int N, typename T>
__device__ __forceinline__ void spread_faces(int dir, const T (&P)[2][N], const T (&Q)[2][N],
                                             T (&y)[N][N]) {
#pragma unroll
    for (int m = 0; m < N; ++m) {
        const T pp = P[1][m] + P[0][m], pm = P[1][m] - P[0][m];
        const T qp = Q[1][m] + Q[0][m], qm = Q[1][m] - Q[0][m];
#pragma unroll
        for (int q = 0; q < N; ++q) {
            const T a = q % 2 == 0 ? pp : pm, b = q % 2 == 0 ? qm : qp;
            if (dir == 0) {
                y[m][q] = fmat(T(kT<N>.lp[q]), a, y[m][q]);
                if (q > 0) y[m][q] = fmat(T(kT<N>.dp[q]), b, y[m][q]);
            } else {
                y[q][m] = fmat(T(kT<N>.lp[q]), a, y[q][m]);
                if (q > 0) y[q][m] = fmat(T(kT<N>.dp[q]), b, y[q][m]);
            }
        }
    }
}

constexpr int TX = 32, TY = 2, TXY = TX * TY;
constexpr int NHALO = 2 * TX + 2 * TY;


// Traces of one element on face F (0 left, 1 right, 2 bottom, 3 top):
// out[0][c][m] = value, out[1][c][m] = physical normal derivative d/dx_d.
template <int N, typename T>
__device__ __forceinline__ void face_traces(const T (&u)[2][N][N], int F, T two_over_h,
                                            T* out /* [2][2][N] */) {
    const bool plus = (F & 1) != 0;
    T dps[N];   // l_q'(+1) times 2 / h: physical derivative
#pragma unroll
    for (int q = 0; q < N; ++q) dps[q] = T(kT<N>.dp[q]) * two_over_h;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int m = 0; m < N; ++m) {
            T ev = T(0), od = T(0), evd = T(0), odd = T(0);
#pragma unroll
            for (int q = 0; q < N; ++q) {
                const T uq = F < 2 ? u[c][m][q] : u[c][q][m];   // q along the normal
                if (q % 2 == 0) {
                    ev = fmat(T(kT<N>.lp[q]), uq, ev);
                    if (q > 0) evd = fmat(dps[q], uq, evd);
                } else {
                    od = fmat(T(kT<N>.lp[q]), uq, od);
                    odd = fmat(dps[q], uq, odd);
                }
            }
            // l_q(-1) = (-1)^q l_q(1),  l_q'(-1) = -(-1)^q l_q'(1)
            out[0 * 2 * N + c * N + m] = plus ? ev + od : ev - od;
            out[1 * 2 * N + c * N + m] = plus ? evd + odd : odd - evd;
        }
}

// Component c only of face_traces (c uniform within a warp).
template <int N, typename T>
__device__ __forceinline__ void face_traces_comp(const T (&u)[2][N][N], int F, int c,
                                                 T two_over_h, T* out /* [2][2][N] */) {
    const bool plus = (F & 1) != 0;
    T dps[N];   // l_q'(+1) times 2 / h: physical derivative
#pragma unroll
    for (int q = 0; q < N; ++q) dps[q] = T(kT<N>.dp[q]) * two_over_h;
#pragma unroll
    for (int m = 0; m < N; ++m) {
        T ev = T(0), od = T(0), evd = T(0), odd = T(0);
#pragma unroll
        for (int q = 0; q < N; ++q) {
            const T uq = F < 2 ? u[c][m][q] : u[c][q][m];
            if (q % 2 == 0) {
                ev = fmat(T(kT<N>.lp[q]), uq, ev);
                if (q > 0) evd = fmat(dps[q], uq, evd);
            } else {
                od = fmat(T(kT<N>.lp[q]), uq, od);
                odd = fmat(dps[q], uq, odd);
            }
        }
        out[0 * 2 * N + c * N + m] = plus ? ev + od : ev - od;
        out[1 * 2 * N + c * N + m] = plus ? evd + odd : odd - evd;
    }
}

// 16-byte vector accesses to one element's coefficients.  A thread reads a
// whole element (2 N^2 contiguous values), so scalar loads cost one L1
// wavefront per value and warp; 16-byte loads cut that by 2 (FP64) or 4
// (FP32).  Usable when an element and a component block are multiples of 16
// bytes (N = 2, 4) and the vectors are 16-byte aligned (checked at launch).
template <typename T> struct Vec16;
template <> struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
    __device__ static double get(const double2& v, int i) { return i == 0 ? v.x : v.y; }
    __device__ static double2 make(const double* p) { return make_double2(p[0], p[1]); }
};
template <> struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
    __device__ static float get(const float4& v, int i) {
        return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
    }
    __device__ static float4 make(const float* p) { return make_float4(p[0], p[1], p[2], p[3]); }
};

template <int N, typename T>
constexpr bool vec_ok() {
    return (N * N * sizeof(T)) % 16 == 0;
}

// Work of one component C (compile-time, so the register arrays stay in
// registers) in phase A: own traces of component C and the volume terms of y_C.
template <int N, typename T, int C>
__device__ __forceinline__ void elem2_phase_a(const ElemArgs<T>& a, const T (&u)[2][N][N], T etaK,
                                              T* tr, T (&y)[N][N]) {
#pragma unroll
    for (int F = 0; F < 4; ++F)
        face_traces_comp<N, T>(u, F, C, F < 2 ? a.two_over_hx : a.two_over_hy, tr + F * 4 * N);
    const T sx = etaK * (C == 0 ? a.c2hy_hx : a.chy_hx);   // weight of G along x on u_C
    const T sy = etaK * (C == 0 ? a.chx_hy : a.c2hx_hy);   // weight of G along y on u_C
    T Gx[N][N], Gy[N][N], De[N][N];   // scaled tables (zero entries never read)
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
        for (int q = 0; q < N; ++q) {
            Gx[p][q] = kT<N>.G[p][q] != 0.0 ? sx * T(kT<N>.G[p][q]) : T(0);
            Gy[p][q] = kT<N>.G[p][q] != 0.0 ? sy * T(kT<N>.G[p][q]) : T(0);
            De[p][q] = kT<N>.D[p][q] != 0.0 ? etaK * T(kT<N>.D[p][q]) : T(0);
        }
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
        for (int av = 0; av < N; ++av) {
            T acc = T(0);
#pragma unroll
            for (int i = 0; i < N; ++i) {
                if (kT<N>.G[av][i] != 0.0) acc = fmat(Gx[av][i], u[C][b][i], acc);
                if (kT<N>.G[b][i] != 0.0) acc = fmat(Gy[b][i], u[C][i][av], acc);
            }
            y[b][av] = acc;
        }
    T w[N][N];
    if (C == 0) {
        // y_x[b][a] += eta_K sum_j D[j][b] sum_i D[a][i] u_y[j][i]
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
            for (int av = 0; av < N; ++av) {
                T t = T(0);
#pragma unroll
                for (int i = 0; i < N; ++i)
                    if (kT<N>.D[av][i] != 0.0) t = fmat(T(kT<N>.D[av][i]), u[1][j][i], t);
                w[j][av] = t;
            }
#pragma unroll
        for (int b = 0; b < N; ++b)
#pragma unroll
            for (int av = 0; av < N; ++av)
#pragma unroll
                for (int j = 0; j < N; ++j)
                    if (kT<N>.D[j][b] != 0.0) y[b][av] = fmat(De[j][b], w[j][av], y[b][av]);
    } else {
        // y_y[b][a] += eta_K sum_i D[i][a] sum_j D[b][j] u_x[j][i]
#pragma unroll
        for (int b = 0; b < N; ++b)
#pragma unroll
            for (int i = 0; i < N; ++i) {
                T t = T(0);
#pragma unroll
                for (int j = 0; j < N; ++j)
                    if (kT<N>.D[b][j] != 0.0) t = fmat(T(kT<N>.D[b][j]), u[0][j][i], t);
                w[b][i] = t;
            }
#pragma unroll
        for (int b = 0; b < N; ++b)
#pragma unroll
            for (int av = 0; av < N; ++av)
#pragma unroll
                for (int i = 0; i < N; ++i)
                    if (kT<N>.D[i][av] != 0.0) y[b][av] = fmat(De[i][av], w[b][i], y[b][av]);
    }
}


}  // namespace

}  // namespace sip
