// Device helpers of the continuous-level operators, shared by the
// transfer / h-level kernels and their batched forms: the weights of the
// bilinear hats on the orthonormal Q_1 modes (P_cd, Sec. 6.1.2) and one row
// of the 9-point 2x2-block stencil.
#pragma once

#include "sip_internal.h"

namespace sip {

namespace {

constexpr double kInvSqrt2 = 0.70710678118654752440;   // int L_p l_0 for the two end hats
constexpr double kInvSqrt6 = 0.40824829046386301637;   // |int L_p l_1|

// weight of corner p (0 = low end, 1 = high end) on mode i of the 1D
// orthonormal basis: int L_p l_i over [-1, 1] with L_0 = (1-xi)/2, L_1 = (1+xi)/2
__device__ __forceinline__ double hatw(int i, int p) {
    return i == 0 ? kInvSqrt2 : (p == 0 ? -kInvSqrt6 : kInvSqrt6);
}

// Two consecutive values; one 2-word vector load when VEC (the launcher has
// checked that every such pair is 2-word aligned).
template <typename T, bool VEC>
__device__ __forceinline__ void ld2(const T* p, T& a, T& b) {
    if constexpr (VEC && sizeof(T) == 8) {
        const double2 v = *reinterpret_cast<const double2*>(p);
        a = v.x;
        b = v.y;
    } else if constexpr (VEC) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        a = v.x;
        b = v.y;
    } else {
        a = p[0];
        b = p[1];
    }
}

// Row c of vertex (vx, vy) of the 9-point 2x2-block stencil times x.
template <typename T, bool VEC>
__device__ __forceinline__ T stencil_row(int nvx, int nvy, int vx, int vy, int c, const T* sv,
                                         const T* __restrict__ x) {
    T acc = T(0);
    for (int dy = -1; dy <= 1; ++dy) {
        const int wy = vy + dy;
        if (wy < 0 || wy >= nvy) continue;
        for (int dx = -1; dx <= 1; ++dx) {
            const int wx = vx + dx;
            if (wx < 0 || wx >= nvx) continue;
            const int t = (dy + 1) * 3 + (dx + 1);
            T s0, s1, x0, x1;
            ld2<T, VEC>(sv + t * 4 + c * 2, s0, s1);
            ld2<T, VEC>(x + 2 * (size_t(wy) * nvx + wx), x0, x1);
            acc += s0 * x0 + s1 * x1;
        }
    }
    return acc;
}

}  // namespace

}  // namespace sip
