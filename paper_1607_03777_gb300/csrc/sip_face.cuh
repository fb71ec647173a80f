// Face terms of the SIP form (eq. stiffness_form) in 1D modal form, shared by
// the operator apply and the element-block (smoother) construction.
#pragma once

namespace sip {

// Face vectors P, Q (test component c, tangential mode m) of one face of K.
// kind: 0 interior, else 1 + sip_bc of the boundary side (1 Navier,
// 2 Neumann, 3 Dirichlet).  Arrays are indexed [comp][m]; nc / tc are the normal /
// tangential component; s = +-1 the outward normal sign; own / nbr traces
// (val), physical normal derivatives (der).
template <int N, typename T>
__host__ __device__ __forceinline__ void face_pq(int kind, int c, int m, int nc, T s, T hn, T ht,
                                        T etaK, T etaN, T sigma, const T* vo, const T* dv,
                                        const T* vn, const T* dn, const T* D, T& P, T& Q) {
    const int tc = 1 - nc;
    const T half_ht = T(0.5) * ht;
    P = T(0);
    Q = T(0);
    if (kind == 0) {  // interior
        if (c == nc) {
            T Fn = s * (etaK * dv[nc * N + m] + etaN * dn[nc * N + m]);
            T DTw = T(0);
#pragma unroll
            for (int mm = 0; mm < N; ++mm) DTw += D[mm * N + m] * (vo[tc * N + mm] - vn[tc * N + mm]);
            T wn = vo[nc * N + m] - vn[nc * N + m];
            P = -half_ht * Fn - etaK * s * T(0.5) * DTw + sigma * half_ht * wn;
            Q = -etaK * s * (ht / hn) * wn;
        } else {
            T tno = T(0), tnn = T(0);
#pragma unroll
            for (int mm = 0; mm < N; ++mm) {
                tno += D[m * N + mm] * vo[nc * N + mm];
                tnn += D[m * N + mm] * vn[nc * N + mm];
            }
            tno *= T(2) / ht;
            tnn *= T(2) / ht;
            T Ft = s * T(0.5) * (etaK * (dv[tc * N + m] + tno) + etaN * (dn[tc * N + m] + tnn));
            T wt = vo[tc * N + m] - vn[tc * N + m];
            P = -half_ht * Ft + sigma * half_ht * wt;
            Q = -etaK * s * (half_ht / hn) * wt;
        }
    } else if (kind == 1) {  // Navier: normal component only
        if (c == nc) {
            P = -etaK * s * ht * dv[nc * N + m] + sigma * half_ht * vo[nc * N + m];
            Q = T(-2) * etaK * s * (ht / hn) * vo[nc * N + m];
        }
    } else if (kind == 3) {  // Dirichlet extension: full vector, zero exterior trace
        if (c == nc) {
            T DTv = T(0);
#pragma unroll
            for (int mm = 0; mm < N; ++mm) DTv += D[mm * N + m] * vo[tc * N + mm];
            P = -half_ht * (s * T(2) * etaK * dv[nc * N + m]) - etaK * s * DTv +
                sigma * half_ht * vo[nc * N + m];
            Q = T(-2) * etaK * s * (ht / hn) * vo[nc * N + m];
        } else {
            T tno = T(0);
#pragma unroll
            for (int mm = 0; mm < N; ++mm) tno += D[m * N + mm] * vo[nc * N + mm];
            tno *= T(2) / ht;
            T Ft = s * etaK * (dv[tc * N + m] + tno);
            P = -half_ht * Ft + sigma * half_ht * vo[tc * N + m];
            Q = -etaK * s * (ht / hn) * vo[tc * N + m];
        }
    }
    // kind == 2: Neumann, natural condition, no face terms
}


}  // namespace sip
