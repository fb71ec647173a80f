// Reflection parity of the element velocity modes, used to apply the
// element-block Jacobi inverses with fewer products.
//
// Reflecting x -> -x maps the velocity mode l_i(x) l_j(y) e_c to
// (-1)^(i + [c == 0]) times itself (u_x changes sign, l_i(-x) = (-1)^i l_i(x));
// reflecting y -> -y gives (-1)^(j + [c == 1]).  The viscous form is
// invariant under both reflections, and so is the diagonal block of an
// element whose two x-faces are of the same kind with the same penalty
// (both interior with eta_e = eta_K, or both boundary with the same
// condition), likewise in y.  Such a block, and its inverse, couples only
// modes of equal parity: with both symmetries it splits into four diagonal
// blocks (8 x 8 at k = 3 instead of 32 x 32, a quarter of the products),
// with one symmetry into two.
#pragma once

namespace sip {

template <int N>
struct ParityTabs {
    static constexpr int NB = 2 * N * N;
    int cls[NB];          // bit 0: x-parity, bit 1: y-parity of dof (c, j, i)
    int cnt[3][4];        // symmetry type t = 1 (x), 2 (y), 3 (both): size of group g
    int cols[3][4][NB];   // members of group g = cls & t, in dof order
};

template <int N>
constexpr ParityTabs<N> build_parity() {
    ParityTabs<N> p{};
    constexpr int NB = 2 * N * N;
    for (int q = 0; q < NB; ++q) {
        const int c = q / (N * N), j = (q / N) % N, i = q % N;
        p.cls[q] = ((i + (c == 0 ? 1 : 0)) & 1) | (((j + (c == 1 ? 1 : 0)) & 1) << 1);
    }
    for (int t = 1; t <= 3; ++t)
        for (int g = 0; g < 4; ++g) {
            int n = 0;
            for (int q = 0; q < NB; ++q)
                if ((p.cls[q] & t) == g) p.cols[t - 1][g][n++] = q;
            p.cnt[t - 1][g] = n;
        }
    return p;
}

template <int N>
__device__ constexpr ParityTabs<N> kParity = build_parity<N>();

// Row `row` of M^{-1} r for one element block (NB x NB, symmetric, read by
// columns so that lanes = rows coalesce); sym = symmetry type of the block
// (0: none, dense).  Skipped entries are zero by the reflection symmetry.
template <int N, typename T>
__device__ __forceinline__ T block_row_apply(const T* __restrict__ Minv, const T* rr, int row,
                                             int sym) {
    constexpr int NB = 2 * N * N;
    T acc = T(0);
    if (sym == 0) {
#pragma unroll 8
        for (int q = 0; q < NB; ++q) acc += Minv[q * NB + row] * rr[q];
    } else {
        const int g = kParity<N>.cls[row] & sym;
        const int n = kParity<N>.cnt[sym - 1][g];
        const int* cols = kParity<N>.cols[sym - 1][g];
#pragma unroll 4
        for (int k = 0; k < n; ++k) {
            const int q = cols[k];
            acc += Minv[q * NB + row] * rr[q];
        }
    }
    return acc;
}

}  // namespace sip
