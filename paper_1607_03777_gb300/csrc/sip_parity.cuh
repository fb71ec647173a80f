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

// Row `row` of M^{-1} r for one element block (NB x NB, symmetric, read by
// columns so that lanes = rows coalesce); sym = symmetry type of the block
// (0: none, dense).  Skipped entries are zero by the reflection symmetry.
// The members of the row's parity group are enumerated arithmetically (no
// table reads): mode (c, j, i) has x-parity (i + [c = x]) & 1, so for each
// component the group's i (and, with the y-symmetry, j) run over one parity.
// TA: accumulation type (FP64 accumulation of an FP32 block keeps the small
// components of an ill-conditioned block's result, which FP32 sums cancel).
template <int N, typename T, typename TA = T>
__device__ __forceinline__ TA block_row_apply(const T* __restrict__ Minv, const T* rr, int row,
                                              int sym) {
    constexpr int NN = N * N;
    constexpr int NB = 2 * NN;
    TA acc = TA(0);
    if (sym == 0) {
#pragma unroll 8
        for (int q = 0; q < NB; ++q) acc += TA(Minv[q * NB + row]) * TA(rr[q]);
        return acc;
    }
    const int cr = row / NN, jr = (row / N) % N, ir = row % N;
    const int px = (ir + (cr == 0 ? 1 : 0)) & 1;
    const int py = (jr + (cr == 1 ? 1 : 0)) & 1;
    const bool sx = (sym & 1) != 0, sy = (sym & 2) != 0;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        // first i (j) of component c in the row's x- (y-) parity group
        const int i0 = sx ? (px ^ (c == 0 ? 1 : 0)) : 0;
        const int j0 = sy ? (py ^ (c == 1 ? 1 : 0)) : 0;
        const int di = sx ? 2 : 1, dj = sy ? 2 : 1;
#pragma unroll
        for (int b = 0; b < N; ++b) {
            const int j = j0 + b * dj;
            if (j >= N) break;
#pragma unroll
            for (int a = 0; a < N; ++a) {
                const int i = i0 + a * di;
                if (i >= N) break;
                const int q = c * NN + j * N + i;
                acc += TA(Minv[q * NB + row]) * TA(rr[q]);
            }
        }
    }
    return acc;
}

}  // namespace sip
