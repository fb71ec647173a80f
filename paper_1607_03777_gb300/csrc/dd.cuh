// Double-double arithmetic: a value is the unevaluated sum hi + lo of two
// doubles with |lo| <= ulp(hi) / 2, about 106 significant bits.  Used only to
// evaluate the Stokes residual b - K x beyond FP64 (iterative refinement of
// the FP64 solve); the generic operator kernels are instantiated with it.
//
// Building blocks (exact error-free transformations of IEEE doubles):
//   two_sum       s + e = a + b exactly (Knuth, TAOCP vol. 2, 4.2.2);
//   fast_two_sum  the same when |a| >= |b| (Dekker, Numer. Math. 18, 1971);
//   two_prod      p + e = a * b exactly, e from one fused multiply-add.
// Addition is the accurate double-double sum (both parts added with error
// terms, then renormalised), multiplication keeps the cross terms hi*lo; the
// relative error of each operation is a small multiple of 2^-104.
#pragma once

#include <cmath>

namespace sip {

struct dd {
    double hi, lo;
    __host__ __device__ dd() : hi(0.0), lo(0.0) {}
    __host__ __device__ dd(double h) : hi(h), lo(0.0) {}   // NOLINT: implicit by design
    __host__ __device__ dd(double h, double l) : hi(h), lo(l) {}
};

__host__ __device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    const double bv = s - a;
    e = (a - (s - bv)) + (b - bv);
}

__host__ __device__ __forceinline__ void fast_two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    e = b - (s - a);
}

__host__ __device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
    p = a * b;
    e = fma(a, b, -p);
}

__host__ __device__ __forceinline__ dd operator+(const dd& a, const dd& b) {
    double s, e, t, f;
    two_sum(a.hi, b.hi, s, e);
    two_sum(a.lo, b.lo, t, f);
    e += t;
    fast_two_sum(s, e, s, e);
    e += f;
    fast_two_sum(s, e, s, e);
    return dd(s, e);
}

__host__ __device__ __forceinline__ dd operator-(const dd& a) { return dd(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ dd operator-(const dd& a, const dd& b) { return a + (-b); }

__host__ __device__ __forceinline__ dd operator*(const dd& a, const dd& b) {
    double p, e;
    two_prod(a.hi, b.hi, p, e);
    e += a.hi * b.lo + a.lo * b.hi;
    fast_two_sum(p, e, p, e);
    return dd(p, e);
}

__host__ __device__ __forceinline__ dd& operator+=(dd& a, const dd& b) { return a = a + b; }
__host__ __device__ __forceinline__ dd& operator-=(dd& a, const dd& b) { return a = a - b; }
__host__ __device__ __forceinline__ dd& operator*=(dd& a, const dd& b) { return a = a * b; }

// comparisons of normalised values: by hi, then by lo
__host__ __device__ __forceinline__ bool operator<(const dd& a, const dd& b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__host__ __device__ __forceinline__ bool operator>(const dd& a, const dd& b) { return b < a; }
__host__ __device__ __forceinline__ bool operator==(const dd& a, const dd& b) {
    return a.hi == b.hi && a.lo == b.lo;
}
__host__ __device__ __forceinline__ bool operator!=(const dd& a, const dd& b) { return !(a == b); }

}  // namespace sip
