// Thread-per-element SIP apply for low degrees (N = k+1 <= 6).
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
#include "sip_elem.cuh"
#include "sip_face.cuh"
#include "sip_internal.h"
#include "sip_parity.cuh"

namespace sip {

namespace {

template <int N, typename T>
__global__ void __launch_bounds__(TXY) k_apply_elem(const ElemArgs<T> a) {
    grid_dep_wait();
    constexpr int TR = 4 * N;                 // [2 val/der][2 comp][N] per face
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // own element, all four faces: s_tr[TXY][4 TR + 1]; halo: s_halo[NHALO][TR + 1]
    // (odd row strides: lanes of a warp hit distinct banks)
    T (*s_tr)[4 * TR + 1] = reinterpret_cast<T (*)[4 * TR + 1]>(smem_raw);
    T (*s_halo)[TR + 1] =
        reinterpret_cast<T (*)[TR + 1]>(smem_raw + sizeof(T) * TXY * (4 * TR + 1));
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
            face_traces<N, T>(u, F, F < 2 ? a.two_over_hx : a.two_over_hy,
                              s_tr[threadIdx.x] + F * TR);
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
            const T* own = s_tr[threadIdx.x] + F * TR;
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
                    nbr = s_tr[lty * TX + ltx] + (F ^ 1) * TR;
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

// Component-split variant: one warp = one velocity component of 32
// consecutive elements of a row (warps 2r and 2r+1 share row r of the tile),
// so every element is served by two threads and twice as many warps keep the
// narrow FP64 pipe busy.  The component is uniform within a warp: no
// divergence.  Each thread reads both components (the volume cross terms and
// the face terms couple them), writes its component's traces to shared memory
// and computes its component's outputs.
constexpr int TY2 = 2;                        // tile rows
constexpr int T2THREADS = 64 * TY2;           // 2 warps per tile row
constexpr int NHALO2 = 2 * TX + 2 * TY2;

template <int N, typename T, bool VEC>
__device__ __forceinline__ void load_elem(const T* __restrict__ src, T (&u)[2][N][N]) {
    constexpr int NN = N * N;
    if constexpr (VEC && vec_ok<N, T>()) {
        using V = Vec16<T>;
        const typename V::type* s = reinterpret_cast<const typename V::type*>(src);
#pragma unroll
        for (int k = 0; k < 2 * NN / V::n; ++k) {
            const typename V::type v = __ldg(s + k);
#pragma unroll
            for (int t = 0; t < V::n; ++t) {
                const int f = k * V::n + t;
                u[f / NN][(f % NN) / N][f % N] = V::get(v, t);
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int j = 0; j < N; ++j)
#pragma unroll
                for (int i = 0; i < N; ++i) u[c][j][i] = src[c * NN + j * N + i];
    }
}

// dst[j][i] = alpha y[j][i] (+ beta zz[j][i]) over one component block;
// the same values also go to sres (shared memory) when it is not null
template <int N, typename T, bool VEC>
__device__ __forceinline__ void store_comp(T* dst, const T* zz, T alpha, T beta,
                                           const T (&y)[N][N], T* sres) {
    if constexpr (VEC && vec_ok<N, T>()) {
        using V = Vec16<T>;
        typename V::type* d = reinterpret_cast<typename V::type*>(dst);
#pragma unroll
        for (int k = 0; k < N * N / V::n; ++k) {
            T v[V::n];
            if (zz) {
                const typename V::type zv = __ldg(reinterpret_cast<const typename V::type*>(zz) + k);
#pragma unroll
                for (int t = 0; t < V::n; ++t) {
                    const int f = k * V::n + t;
                    v[t] = alpha * y[f / N][f % N] + beta * V::get(zv, t);
                }
            } else {
#pragma unroll
                for (int t = 0; t < V::n; ++t) {
                    const int f = k * V::n + t;
                    v[t] = alpha * y[f / N][f % N];
                }
            }
            d[k] = V::make(v);
            if (sres) {
#pragma unroll
                for (int t = 0; t < V::n; ++t) sres[k * V::n + t] = v[t];
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
            for (int i = 0; i < N; ++i) {
                T v = alpha * y[j][i];
                if (zz) v += beta * zz[j * N + i];
                dst[j * N + i] = v;
                if (sres) sres[j * N + i] = v;
            }
    }
}

// Phase B of component C: face vectors from own and neighbour traces, spread
// into y_C, written out.
template <int N, typename T, int C, bool VEC>
__device__ __forceinline__ void elem2_phase_b(const ElemArgs<T>& a, int ex, int ey, int ex0, int ey0,
                                              int tx, int ty, T etaK, T (*s_tr)[16 * N + 1],
                                              T (*s_halo)[4 * N + 1], int el, T (&y)[N][N],
                                              T* sres = nullptr) {
    constexpr int NB = 2 * N * N;
    const int nx = a.nx, ny = a.ny;
    T Dm[N * N];
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
        for (int q = 0; q < N; ++q) Dm[p * N + q] = T(kT<N>.D[p][q]);
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
        T P[2][N], Q[2][N];   // [face lo/hi][m]
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int F = 2 * dir + side;
            const T* own = s_tr[el] + F * 4 * N;
            const T* nbr = own;
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
                if (ltx >= 0 && ltx < TX && lty >= 0 && lty < TY2)
                    nbr = s_tr[lty * TX + ltx] + (F ^ 1) * 4 * N;
                else if (dir == 1)
                    nbr = s_halo[(side == 0 ? 0 : TX) + tx];
                else
                    nbr = s_halo[2 * TX + (side == 0 ? 0 : TY2) + ty];
            } else {
                kind = 1 + a.bc[F];
            }
            const T eta_e = kind == 0 ? (etaK > etaN ? etaK : etaN) : etaK;
            const T pen = dir == 0 ? a.pen_x : a.pen_y;
            const T sigma = pen * eta_e * (kind == 0 ? T(1) : T(2));
            const T s = side == 0 ? T(-1) : T(1);
            const FaceGeo<T>& fg = dir == 0 ? a.fgx : a.fgy;
            if (kind == 0) {
                face_interior_comp<N, T, C>(dir, side, fg, pen, etaK, etaN, own, nbr, P[side],
                                            Q[side]);
            } else {
#pragma unroll
                for (int m = 0; m < N; ++m)
                    face_pq<N, T>(kind, C, m, dir, s, fg, etaK, etaN, sigma, own, own + 2 * N, nbr,
                                  nbr + 2 * N, Dm, P[side][m], Q[side][m]);
            }
        }
        spread_faces<N, T>(dir, P, Q, y);
    }
    const T* zz = a.z ? a.z + (size_t(ey) * nx + ex) * NB + C * N * N : nullptr;
    if (a.r1) {   // residual restricted to the Q^2_1 modes (p-transfer R = P^T)
        T* d1 = a.r1 + (size_t(ey) * nx + ex) * 8 + C * 4;
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                T v = a.alpha * y[j][i];
                if (zz) v += a.beta * zz[j * N + i];
                d1[j * 2 + i] = v;
            }
        return;
    }
    T* dst = a.y + (size_t(ey) * nx + ex) * NB + C * N * N;
    store_comp<N, T, VEC>(dst, zz, a.alpha, a.beta, y, sres);
}

// Thread roles of the component-split tile: warps 2r and 2r+1 serve
// velocity components 0 and 1 of the 32 elements of tile row r.
struct Elem2Ids {
    int warp, lane, ty, c, tx, el, ex0, ey0, ex, ey;
    bool active;
    __device__ Elem2Ids(int nx, int ny) {
        warp = threadIdx.x / 32;
        lane = threadIdx.x % 32;
        ty = warp / 2;
        c = warp % 2;
        tx = lane;
        el = ty * TX + tx;
        ex0 = blockIdx.x * TX;
        ey0 = blockIdx.y * TY2;
        ex = ex0 + tx;
        ey = ey0 + ty;
        active = ex < nx && ey < ny;
    }
};

// Phase A of the component-split tile: halo traces (both components of the
// face touching the tile) and, for an active thread, its component's own
// traces and volume terms (into y).  Ends with the CTA barrier.
template <int N, typename T, bool VEC>
__device__ __forceinline__ void elem2_phase_a_all(const ElemArgs<T>& a, const Elem2Ids& id,
                                                  T (*s_tr)[16 * N + 1], T (*s_halo)[4 * N + 1],
                                                  T (&y)[N][N], T& etaK) {
    constexpr int NB = 2 * N * N;
    const int nx = a.nx, ny = a.ny;
    for (int h = threadIdx.x; h < NHALO2; h += T2THREADS) {
        int hx, hy, F;
        if (h < TX) { hx = id.ex0 + h; hy = id.ey0 - 1; F = 3; }
        else if (h < 2 * TX) { hx = id.ex0 + h - TX; hy = id.ey0 + TY2; F = 2; }
        else if (h < 2 * TX + TY2) { hx = id.ex0 - 1; hy = id.ey0 + h - 2 * TX; F = 1; }
        else { hx = id.ex0 + TX; hy = id.ey0 + h - 2 * TX - TY2; F = 0; }
        if (hx >= 0 && hx < nx && hy >= 0 && hy < ny) {
            T uh[2][N][N];
            load_elem<N, T, VEC>(a.x + (size_t(hy) * nx + hx) * NB, uh);
            face_traces<N, T>(uh, F, F < 2 ? a.two_over_hx : a.two_over_hy, s_halo[h]);
        }
    }
    etaK = T(0);
    if (id.active) {
        T u[2][N][N];
        load_elem<N, T, VEC>(a.x + (size_t(id.ey) * nx + id.ex) * NB, u);
        etaK = a.eta[size_t(id.ey) * nx + id.ex];
        if (id.c == 0)
            elem2_phase_a<N, T, 0>(a, u, etaK, s_tr[id.el], y);
        else
            elem2_phase_a<N, T, 1>(a, u, etaK, s_tr[id.el], y);
    }
    __syncthreads();
}

template <int N, typename T, bool VEC>
__global__ void __launch_bounds__(T2THREADS) k_apply_elem2(const ElemArgs<T> a) {
    grid_dep_wait();
    constexpr int TR = 4 * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // [TX*TY2][4 TR + 1] and [NHALO2][TR + 1]: odd row strides, conflict-free banks
    T (*s_tr)[4 * TR + 1] = reinterpret_cast<T (*)[4 * TR + 1]>(smem_raw);
    T (*s_halo)[TR + 1] =
        reinterpret_cast<T (*)[TR + 1]>(smem_raw + sizeof(T) * TX * TY2 * (4 * TR + 1));
    const Elem2Ids id(a.nx, a.ny);
    T y[N][N];
    T etaK;
    elem2_phase_a_all<N, T, VEC>(a, id, s_tr, s_halo, y, etaK);
    if (!id.active) return;
    if (id.c == 0)
        elem2_phase_b<N, T, 0, VEC>(a, id.ex, id.ey, id.ex0, id.ey0, id.tx, id.ty, etaK, s_tr,
                                    s_halo, id.el, y);
    else
        elem2_phase_b<N, T, 1, VEC>(a, id.ex, id.ey, id.ex0, id.ey0, id.tx, id.ty, etaK, s_tr,
                                    s_halo, id.el, y);
}

// Element-block Jacobi / Chebyshev update of the fused smoother step.
template <typename T>
struct BJArgs {
    const int* emap;        // class (< 0: -(mask+1)) or unique slot of each element
    const T* cls_inv;       // reference inverses by boundary mask, scaled by 1/eta_K
    const int* cls_sym;     // their reflection-symmetry types (null: dense)
    const T* uniq_inv;      // inverses of the unique blocks
    const T* eta_inv;       // 1/eta_K
    const T* d_old;         // previous direction (null when c1 == 0 and !pend)
    T* d_new;               // new direction
    T* yv;                  // iterate to update (null: no update)
    T c1, c2;
    int pend;               // add d_old to the iterate too (its update was deferred)
};

// One p-level Chebyshev step of the element-block Jacobi smoother (Sec. 6)
// in one launch:
//   r = z - A x,  d_new = c1 d_old + c2 M^{-1} r,  yv += [pend] d_old + d_new.
// The operator part is k_apply_elem2's (alpha = -1, beta = 1, output r; z
// may alias r); the residual blocks of the tile are also kept in shared
// memory, where each warp then applies the block inverses of its elements
// (lane = row, columns of the symmetric inverse read coalesced).  x must not
// alias d_new or yv: other tiles read x while this one writes.
template <int N, typename T, bool VEC>
__global__ void __launch_bounds__(T2THREADS) k_cheb_elem2(const ElemArgs<T> a, const BJArgs<T> b) {
    grid_dep_wait();
    constexpr int TR = 4 * N;
    constexpr int NB = 2 * N * N;
    static_assert(NB <= 32, "one warp lane per block row");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T (*s_tr)[4 * TR + 1] = reinterpret_cast<T (*)[4 * TR + 1]>(smem_raw);
    T (*s_halo)[TR + 1] =
        reinterpret_cast<T (*)[TR + 1]>(smem_raw + sizeof(T) * TX * TY2 * (4 * TR + 1));
    // residual blocks, row stride NB + 1
    T* s_res = reinterpret_cast<T*>(smem_raw + sizeof(T) * (TX * TY2 * (4 * TR + 1) +
                                                            NHALO2 * (TR + 1)));
    const Elem2Ids id(a.nx, a.ny);
    T y[N][N];
    T etaK;
    elem2_phase_a_all<N, T, VEC>(a, id, s_tr, s_halo, y, etaK);
    if (id.active) {
        T* sres = s_res + id.el * (NB + 1) + id.c * N * N;
        if (id.c == 0)
            elem2_phase_b<N, T, 0, VEC>(a, id.ex, id.ey, id.ex0, id.ey0, id.tx, id.ty, etaK, s_tr,
                                        s_halo, id.el, y, sres);
        else
            elem2_phase_b<N, T, 1, VEC>(a, id.ex, id.ey, id.ex0, id.ey0, id.tx, id.ty, etaK, s_tr,
                                        s_halo, id.el, y, sres);
    }
    __syncthreads();
    // block inverses: warp w takes elements w, w + NW, ...; ILP of them at a
    // time so that their independent column loads overlap
    constexpr int NW = T2THREADS / 32;
    constexpr int PER = TX * TY2 / NW;
    constexpr int ILP = 4;
    static_assert(PER % ILP == 0, "whole rounds of ILP elements per warp");
    const int row = id.lane;
#pragma unroll 1
    for (int base = 0; base < PER; base += ILP) {
        const T* Mk[ILP];
        T sc[ILP];
        size_t ek[ILP];
        int e2k[ILP];
        int symk[ILP];
        bool ok[ILP];
#pragma unroll
        for (int k = 0; k < ILP; ++k) {
            const int e2 = id.warp + NW * (base + k);
            const int gx = id.ex0 + e2 % TX, gy = id.ey0 + e2 / TX;
            e2k[k] = e2;
            ok[k] = gx < a.nx && gy < a.ny;
            ek[k] = ok[k] ? size_t(gy) * a.nx + gx : 0;
            const int m = ok[k] ? b.emap[ek[k]] : -1;   // outside: any valid matrix, unused
            if (m < 0) {
                Mk[k] = b.cls_inv + size_t(-m - 1) * NB * NB;
                sc[k] = ok[k] ? b.eta_inv[ek[k]] : T(0);
                symk[k] = b.cls_sym ? b.cls_sym[-m - 1] : 0;
            } else {
                Mk[k] = b.uniq_inv + size_t(m) * NB * NB;
                sc[k] = T(1);
                symk[k] = 0;
            }
        }
        if (row < NB) {
            T acc[ILP];
#pragma unroll
            for (int k = 0; k < ILP; ++k)
                acc[k] = block_row_apply<N, T>(Mk[k], s_res + e2k[k] * (NB + 1), row, symk[k]);
#pragma unroll
            for (int k = 0; k < ILP; ++k) {
                if (!ok[k]) continue;
                const size_t o = ek[k] * NB + row;
                T v = b.c2 * sc[k] * acc[k];
                if (b.c1 != T(0)) v += b.c1 * b.d_old[o];
                b.d_new[o] = v;
                if (b.yv) b.yv[o] += b.pend ? b.d_old[o] + v : v;
            }
        }
    }
}

// dynamic shared memory of the component-split kernels (padded rows)
template <int N, typename T>
size_t elem2_smem(bool with_residual) {
    const size_t tile = size_t(TX) * TY2;
    size_t words = tile * (16 * N + 1) + size_t(NHALO2) * (4 * N + 1);
    if (with_residual) words += tile * (2 * N * N + 1);
    return sizeof(T) * words;
}

template <int N, typename T>
void apply_elem_n(const OpGeom& g, const T* x, T* y, const T* eta, T alpha, const T* z, T beta,
                  bool split, cudaStream_t s) {
    const ElemArgs<T> a = make_elem_args<T>(g, x, y, eta, alpha, z, beta);
    if (split) {
        dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY2 - 1) / TY2);
        const size_t smem = elem2_smem<N, T>(false);
        static const bool attr2 = [smem] {   // once per process, thread-safe
            SIP_CUDA(cudaFuncSetAttribute(k_apply_elem2<N, T, false>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
            SIP_CUDA(cudaFuncSetAttribute(k_apply_elem2<N, T, true>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
            return true;
        }();
        (void)attr2;
        if (vec_ok<N, T>() && aligned16(x) && aligned16(y) && (z == nullptr || aligned16(z)))
            launch_k(k_apply_elem2<N, T, true>, grid, T2THREADS, smem, s, a);
        else
            launch_k(k_apply_elem2<N, T, false>, grid, T2THREADS, smem, s, a);
        SIP_CHECK_LAUNCH();
        return;
    }
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY);
    const size_t smem = sizeof(T) * (size_t(TXY) * (16 * N + 1) + size_t(NHALO) * (4 * N + 1));
    static const bool attr_set = [smem] {   // once per process, thread-safe
        SIP_CUDA(cudaFuncSetAttribute(k_apply_elem<N, T>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        return true;
    }();
    (void)attr_set;
    launch_k(k_apply_elem<N, T>, grid, TXY, smem, s, a);
    SIP_CHECK_LAUNCH();
}

template <int N, typename T>
void residual_restrict_n(const OpGeom& g, const T* y, const T* b, const T* eta, T* r1,
                         cudaStream_t s) {
    ElemArgs<T> a = make_elem_args<T>(g, y, nullptr, eta, T(-1), b, T(1));
    a.r1 = r1;
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY2 - 1) / TY2);
    const size_t smem = elem2_smem<N, T>(false);
    static const bool attr = [smem] {   // once per process, thread-safe
        SIP_CUDA(cudaFuncSetAttribute(k_apply_elem2<N, T, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        SIP_CUDA(cudaFuncSetAttribute(k_apply_elem2<N, T, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        return true;
    }();
    (void)attr;
    if (vec_ok<N, T>() && aligned16(y) && aligned16(b))
        launch_k(k_apply_elem2<N, T, true>, grid, T2THREADS, smem, s, a);
    else
        launch_k(k_apply_elem2<N, T, false>, grid, T2THREADS, smem, s, a);
    SIP_CHECK_LAUNCH();
}

template <int N, typename T>
void cheb_elem_n(const OpGeom& g, const T* x, const T* z, T* r, const T* eta, const BJArgs<T>& b,
                 cudaStream_t s) {
    const ElemArgs<T> a = make_elem_args<T>(g, x, r, eta, T(-1), z, T(1));
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY2 - 1) / TY2);
    const size_t smem = elem2_smem<N, T>(true);
    static const bool attr = [smem] {   // once per process, thread-safe
        SIP_CUDA(cudaFuncSetAttribute(k_cheb_elem2<N, T, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        SIP_CUDA(cudaFuncSetAttribute(k_cheb_elem2<N, T, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        return true;
    }();
    (void)attr;
    if (vec_ok<N, T>() && aligned16(x) && aligned16(r) && aligned16(z))
        launch_k(k_cheb_elem2<N, T, true>, grid, T2THREADS, smem, s, a, b);
    else
        launch_k(k_cheb_elem2<N, T, false>, grid, T2THREADS, smem, s, a, b);
    SIP_CHECK_LAUNCH();
}


}  // namespace

bool cheb_elem_available(int N) { return N >= 2 && N <= 4; }

template <typename T>
bool launch_residual_restrict_elem(int N, const OpGeom& g, const T* y, const T* b, const T* eta,
                                   T* r1, cudaStream_t s) {
    if (!cheb_elem_available(N)) return false;
    switch (N) {
        case 2: residual_restrict_n<2, T>(g, y, b, eta, r1, s); break;
        case 3: residual_restrict_n<3, T>(g, y, b, eta, r1, s); break;
        default: residual_restrict_n<4, T>(g, y, b, eta, r1, s); break;
    }
    return true;
}
template bool launch_residual_restrict_elem<double>(int, const OpGeom&, const double*,
                                                    const double*, const double*, double*,
                                                    cudaStream_t);
template bool launch_residual_restrict_elem<float>(int, const OpGeom&, const float*, const float*,
                                                   const float*, float*, cudaStream_t);

template <typename T>
bool launch_cheb_elem(int N, const OpGeom& g, const T* x, const T* z, T* r, const T* eta,
                      const int* emap, const T* cls_inv, const int* cls_sym, const T* uniq_inv,
                      const T* eta_inv, const T* d_old, T* d_new, T* yv, T c1, T c2, bool pend,
                      cudaStream_t s) {
    if (!cheb_elem_available(N)) return false;
    BJArgs<T> b;
    b.emap = emap;
    b.cls_inv = cls_inv;
    b.cls_sym = cls_sym;
    b.uniq_inv = uniq_inv;
    b.eta_inv = eta_inv;
    b.d_old = d_old;
    b.d_new = d_new;
    b.yv = yv;
    b.c1 = c1;
    b.c2 = c2;
    b.pend = pend ? 1 : 0;
    switch (N) {
        case 2: cheb_elem_n<2, T>(g, x, z, r, eta, b, s); break;
        case 3: cheb_elem_n<3, T>(g, x, z, r, eta, b, s); break;
        default: cheb_elem_n<4, T>(g, x, z, r, eta, b, s); break;
    }
    return true;
}
template bool launch_cheb_elem<double>(int, const OpGeom&, const double*, const double*, double*,
                                       const double*, const int*, const double*, const int*,
                                       const double*, const double*, const double*, double*,
                                       double*, double, double, bool, cudaStream_t);
template bool launch_cheb_elem<float>(int, const OpGeom&, const float*, const float*, float*,
                                      const float*, const int*, const float*, const int*,
                                      const float*, const float*, const float*, float*, float*,
                                      float, float, bool, cudaStream_t);

template <typename T>
bool launch_apply_sip_elem(int N, const OpGeom& g, const T* x, T* y, const T* eta, T alpha,
                           const T* z, T beta, bool split, cudaStream_t s) {
    switch (N) {
        case 2: apply_elem_n<2, T>(g, x, y, eta, alpha, z, beta, split, s); return true;
        case 3: apply_elem_n<3, T>(g, x, y, eta, alpha, z, beta, split, s); return true;
        case 4: apply_elem_n<4, T>(g, x, y, eta, alpha, z, beta, split, s); return true;
        case 5: apply_elem_n<5, T>(g, x, y, eta, alpha, z, beta, split, s); return true;
        case 6: apply_elem_n<6, T>(g, x, y, eta, alpha, z, beta, split, s); return true;
        default: return false;
    }
}
template bool launch_apply_sip_elem<double>(int, const OpGeom&, const double*, double*,
                                            const double*, double, const double*, double, bool,
                                            cudaStream_t);
template bool launch_apply_sip_elem<float>(int, const OpGeom&, const float*, float*, const float*,
                                           float, const float*, float, bool, cudaStream_t);

}  // namespace sip
