// Face terms of the SIP form (eq. stiffness_form) in 1D modal form, shared by
// the operator apply and the element-block (smoother) construction.
#pragma once

namespace sip {

// Geometric factors of the faces with one normal direction (precomputed on
// the host: no division on the device).  h_t = face length, h_n = element
// size along the normal.
template <typename T>
struct FaceGeo {
    T half_ht;          // h_t / 2 (face Jacobian)
    T two_over_ht;      // d/d(tangent) of a reference mode
    T ht_over_hn;
    T half_ht_over_hn;
};

template <typename T>
__host__ __device__ inline FaceGeo<T> make_face_geo(double hn, double ht) {
    FaceGeo<T> g;
    g.half_ht = T(0.5 * ht);
    g.two_over_ht = T(2.0 / ht);
    g.ht_over_hn = T(ht / hn);
    g.half_ht_over_hn = T(0.5 * ht / hn);
    return g;
}

// Face vectors P, Q (test component c, tangential mode m) of one face of K:
// the test mode (q along the normal, m along the face) receives
// l_q(s) P + l_q'(s) Q.
// kind: 0 interior, else 1 + sip_bc of the boundary side (1 Navier,
// 2 Neumann, 3 Dirichlet).  Arrays are indexed [comp][m]; nc / tc are the
// normal / tangential component; s = +-1 the outward normal sign; own / nbr
// traces (val) and physical normal derivatives (der).
template <int N, typename T>
__host__ __device__ __forceinline__ void face_pq(int kind, int c, int m, int nc, T s,
                                                 const FaceGeo<T>& fg, T etaK, T etaN, T sigma,
                                                 const T* vo, const T* dv, const T* vn,
                                                 const T* dn, const T* D, T& P, T& Q) {
    const int tc = 1 - nc;
    const T half_ht = fg.half_ht;
    P = T(0);
    Q = T(0);
    if (kind == 0) {  // interior
        if (c == nc) {
            T Fn = s * (etaK * dv[nc * N + m] + etaN * dn[nc * N + m]);
            T DTw = T(0);
#pragma unroll
            for (int mm = 0; mm < N; ++mm)
                if (D[mm * N + m] != T(0)) DTw += D[mm * N + m] * (vo[tc * N + mm] - vn[tc * N + mm]);
            T wn = vo[nc * N + m] - vn[nc * N + m];
            P = -half_ht * Fn - etaK * s * T(0.5) * DTw + sigma * half_ht * wn;
            Q = -etaK * s * fg.ht_over_hn * wn;
        } else {
            T tno = T(0), tnn = T(0);
#pragma unroll
            for (int mm = 0; mm < N; ++mm) {
                if (D[m * N + mm] != T(0)) {
                    tno += D[m * N + mm] * vo[nc * N + mm];
                    tnn += D[m * N + mm] * vn[nc * N + mm];
                }
            }
            tno *= fg.two_over_ht;
            tnn *= fg.two_over_ht;
            T Ft = s * T(0.5) * (etaK * (dv[tc * N + m] + tno) + etaN * (dn[tc * N + m] + tnn));
            T wt = vo[tc * N + m] - vn[tc * N + m];
            P = -half_ht * Ft + sigma * half_ht * wt;
            Q = -etaK * s * fg.half_ht_over_hn * wt;
        }
    } else if (kind == 1) {  // Navier: normal component only
        if (c == nc) {
            P = -etaK * s * T(2) * half_ht * dv[nc * N + m] + sigma * half_ht * vo[nc * N + m];
            Q = T(-2) * etaK * s * fg.ht_over_hn * vo[nc * N + m];
        }
    } else if (kind == 3) {  // Dirichlet extension: full vector, zero exterior trace
        if (c == nc) {
            T DTv = T(0);
#pragma unroll
            for (int mm = 0; mm < N; ++mm)
                if (D[mm * N + m] != T(0)) DTv += D[mm * N + m] * vo[tc * N + mm];
            P = -half_ht * (s * T(2) * etaK * dv[nc * N + m]) - etaK * s * DTv +
                sigma * half_ht * vo[nc * N + m];
            Q = T(-2) * etaK * s * fg.ht_over_hn * vo[nc * N + m];
        } else {
            T tno = T(0);
#pragma unroll
            for (int mm = 0; mm < N; ++mm)
                if (D[m * N + mm] != T(0)) tno += D[m * N + mm] * vo[nc * N + mm];
            tno *= fg.two_over_ht;
            T Ft = s * etaK * (dv[tc * N + m] + tno);
            P = -half_ht * Ft + sigma * half_ht * vo[tc * N + m];
            Q = -etaK * s * fg.ht_over_hn * vo[tc * N + m];
        }
    }
    // kind == 2: Neumann, natural condition, no face terms
}

}  // namespace sip
