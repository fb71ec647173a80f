// Warp-row SIP apply (eq. stiffness_form) for FP32 vectors: the operator in
// the precision of the mixed-form V-cycle, where the apply moves little data
// per FLOP and every issued instruction counts.
//
// One thread owns one element and both of its velocity components; one warp
// owns one tile row of 32 elements; a CTA of four warps owns a 32 x 4 tile
// and loops over tiles (persistent grid, up to three CTAs per SM).  Per tile:
//   * the element blocks of the tile, of its left and right neighbours and
//     of the rows below and above are copied into shared memory with 16-byte
//     cp.async copies, no registers and no per-value index arithmetic on the
//     way (one stage buffer: the next tile's copies are issued as soon as
//     the current tile is done, and the other CTAs of the SM compute
//     meanwhile);
//   * each thread reads its element from shared memory (odd N: contiguous
//     blocks of 2 N^2 words, 8-byte reads free of bank conflicts; even N:
//     padded slots, 16-byte reads free of bank conflicts), forms the value
//     and normal-derivative traces of its four faces and the volume terms;
//   * the traces of the left and right neighbours come by warp shuffle, those
//     of the rows below and above through shared memory, those of the halo
//     elements from a few threads of each warp;
//   * the face terms are added and the result goes back through the same
//     shared-memory slots to coalesced 16-byte global stores.
// Global traffic is the algorithmic one plus the halo re-reads, which L2
// serves.  x must not overlap y; z may equal y.
#include <algorithm>

#include "sip_elem.cuh"
#include "sip_face.cuh"
#include "sip_internal.h"

namespace sip {

namespace {

constexpr int WTX = 32;           // elements per tile row: the lanes of a warp
constexpr int WTY = 4;            // tile rows: the warps of a CTA
constexpr int WNT = WTX * WTY;    // threads per CTA
constexpr unsigned FULL = 0xffffffffu;

// NBUF stage buffers (the launched kernel uses one; the helpers below read
// only the members that do not depend on NBUF)
template <int N, int NBUF = 1>
struct WarpLayout {
    static constexpr int NN = N * N;
    static constexpr int NB = 2 * NN;               // floats per element
    static constexpr int EB = 4 * NB;               // bytes per element (8 N^2)
    static constexpr bool PAD = N % 2 == 0;         // EB a multiple of 32 bytes
    static constexpr int CPE = EB / 16;             // 16-byte chunks per element (even N)
    static constexpr int SLOT = PAD ? EB + 16 : EB; // bytes between staged elements
    static constexpr int SW = WTX + 2;              // staged elements per row
    static constexpr int SH = WTY + 2;              // staged rows
    // odd N: a row is copied as the aligned 16-byte chunks covering it, so
    // its first element sits 0 or 8 bytes into the row buffer
    static constexpr int ROWB = PAD ? SW * SLOT : (16 + SW * EB + 15) / 16 * 16;
    static constexpr int BUFB = SH * ROWB;          // one stage buffer
    static constexpr int TRS = 4 * N + 2;           // floats per trace record (TRS / 2 odd)
    static constexpr int NHALO = 2 * WTX + 2 * WTY; // halo faces of a tile
    static constexpr int OFF_ETA = NBUF * BUFB;
    static constexpr int OFF_REC = OFF_ETA + (NBUF * SH * SW * 4 + 15) / 16 * 16;
    static constexpr int OFF_HALO = OFF_REC + 2 * WTY * WTX * TRS * 4;
    static constexpr int BYTES = OFF_HALO + NHALO * TRS * 4;
    static constexpr int MINB = NBUF == 1 ? (BYTES + 1024 <= 75 * 1024 ? 3 : 2)
                                          : (BYTES + 1024 <= 114 * 1024 ? 2 : 1);
    static_assert(NHALO % WTY == 0, "halo faces split evenly over the warps");
    static_assert(NHALO / WTY <= 32, "one halo face per lane");
};

struct WarpArgs {
    ElemArgs<float> c;   // scalars (its pointers unused)
    const float* x;
    float* y;
    const float* eta;
    const float* z;
    long long n_total;   // floats of x
    int ntx, ntiles;
    int bulk;            // y = A x (alpha 1, no z): aligned rows leave as bulk copies
    const unsigned char* skip;   // split-precision tiles (32 x 2) written by another launch
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(unsigned dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(unsigned dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}
// 4 bytes, zero-filled when n == 0 (src is not read then)
__device__ __forceinline__ void cp_async4z(unsigned dst, const void* src, int n) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(n)
                 : "memory");
}
// bulk shared -> global copies of finished output rows (async proxy)
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_store(void* gdst, unsigned ssrc, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gdst),
                 "r"(ssrc), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
// returns once this thread's bulk copies have read their shared-memory source
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Byte offset of staged element j (0 = the left neighbour column) in the row
// buffer of mesh row ey (odd N: the row's shift of 0 or 8 bytes, from the
// parity of the row's first staged element ey nx + ex0 - 1).
template <int N>
__device__ __forceinline__ int elem_off(int ey, int nx, int ex0, int j) {
    using L = WarpLayout<N>;
    if constexpr (L::PAD) {
        return j * L::SLOT;
    } else {
        return (((ey & nx) ^ (ex0 - 1)) & 1) * 8 + j * L::EB;   // EB = 8 mod 16
    }
}

// Issue the copies of tile (ex0, ey0) into one stage buffer.  Stage row r is
// mesh row ey0 - 1 + r and holds its elements ex0 - 1 .. ex0 + 32 that lie in
// the mesh (the corners of the first and last rows are copied but never
// read; rows outside the mesh are not copied and never read).  Each half of
// a stage row, with its viscosities, goes to one warp (three halves per
// warp); the chunk loops are unrolled with immediate offsets.
template <int N>
__device__ __forceinline__ void warp_stage(const WarpArgs& a, int ex0, int ey0,
                                           unsigned char* buf, float* seta) {
    using L = WarpLayout<N>;
    static_assert((2 * L::SH) % WTY == 0, "stage half-rows split evenly over the warps");
    static_assert(L::SW % 2 == 0 && L::SW / 2 <= 32, "one viscosity per lane and half-row");
    const int nx = a.c.nx, ny = a.c.ny;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int elo = max(ex0 - 1, 0), ehi = min(ex0 + WTX + 1, nx);   // every stage row
    const unsigned sbuf = smem_u32(buf);
    const char* xb = reinterpret_cast<const char*>(a.x);
#pragma unroll 1
    for (int hr = warp; hr < 2 * L::SH; hr += WTY) {
        const int r = hr >> 1, half = hr & 1;
        const int ey = ey0 - 1 + r;
        const bool row_in = ey >= 0 && ey < ny;   // uniform over the warp
        const long long row = (long long)ey * nx;
        if (lane < L::SW / 2) {   // viscosities of stage columns half * SW / 2 + lane
            const int c = half * (L::SW / 2) + lane, ex = ex0 - 1 + c;
            const bool in = row_in && ex >= 0 && ex < nx;
            cp_async4z(smem_u32(seta + r * L::SW + c), in ? a.eta + (row + ex) : a.eta, in ? 4 : 0);
        }
        if (!row_in) continue;
        const unsigned srow = sbuf + r * L::ROWB;
        if constexpr (L::PAD) {
            // whole element slots, the row's elements split into two halves
            const int ne = ehi - elo;
            const int e_lo = half ? (ne + 1) / 2 : 0, e_hi = half ? ne : (ne + 1) / 2;
            const int nch = (e_hi - e_lo) * L::CPE;
            const char* g = xb + (row + elo + e_lo) * L::EB;
            const unsigned d0 = srow + (elo - (ex0 - 1) + e_lo) * L::SLOT;
            if constexpr (32 % L::CPE == 0) {
                constexpr int EPI = 32 / L::CPE;                 // elements per iteration
                constexpr int MAXC = ((L::SW + 1) / 2) * L::CPE; // chunks of a half, at most
                const char* gp = g + 16 * lane;
                const unsigned dp = d0 + (lane / L::CPE) * L::SLOT + 16 * (lane % L::CPE);
#pragma unroll
                for (int i = 0; i < (MAXC + 31) / 32; ++i)
                    if (lane + 32 * i < nch) cp_async16(dp + i * EPI * L::SLOT, gp + 512 * i);
            } else {
                for (int q = lane; q < nch; q += 32) {
                    const int e = q / L::CPE, sub = q - e * L::CPE;
                    cp_async16(d0 + e * L::SLOT + 16 * sub, g + 16LL * q);
                }
            }
        } else {
            // the aligned 16-byte chunks covering the row, split into two halves
            const long long anchor = (row + ex0 - 1) * L::EB;   // bytes, may be negative
            const long long gs = (row + elo) * L::EB, ge = (row + ehi) * L::EB;
            const long long g16 = gs & ~15LL;
            const int nall = int((ge - g16 + 15) >> 4);
            const int c_lo = half ? nall / 2 : 0, c_hi = half ? nall : nall / 2;
            const bool tail8 = g16 + 16LL * nall > a.n_total * 4;   // x ends 8 bytes into it
            const long long gq = g16 + 16LL * (c_lo + lane);
            const char* gp = xb + gq;
            const unsigned dp = srow + unsigned(int(anchor & 15)) + unsigned(gq - anchor);
            const int nq = c_hi - c_lo;
            constexpr int MAXC = (L::ROWB / 16 + 1) / 2 + 1;      // chunks of a half, at most
#pragma unroll
            for (int i = 0; i < (MAXC + 31) / 32; ++i) {
                const int q = lane + 32 * i;
                if (q < nq) {
                    if (tail8 && c_lo + q == nall - 1)
                        cp_async8(dp + 512 * i, gp + 512 * i);
                    else
                        cp_async16(dp + 512 * i, gp + 512 * i);
                }
            }
        }
    }
}

// Element block from shared memory (8-byte aligned for odd N, 16 for even).
template <int N>
__device__ __forceinline__ void load_elem(const unsigned char* p, float (&u)[2][N][N]) {
    constexpr int NN = N * N;
    if constexpr (N % 2 == 0) {
        const float4* v = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int q = 0; q < 2 * NN / 4; ++q) {
            const float4 w = v[q];
            const float ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int f = 4 * q + t;
                u[f / NN][(f % NN) / N][f % N] = ww[t];
            }
        }
    } else {
        const float2* v = reinterpret_cast<const float2*>(p);
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            const float2 w = v[q];
            const int f0 = 2 * q, f1 = 2 * q + 1;
            u[f0 / NN][(f0 % NN) / N][f0 % N] = w.x;
            u[f1 / NN][(f1 % NN) / N][f1 % N] = w.y;
        }
    }
}

template <int N>
__device__ __forceinline__ void store_elem(unsigned char* p, const float (&y)[2][N][N]) {
    constexpr int NN = N * N;
    if constexpr (N % 2 == 0) {
        float4* v = reinterpret_cast<float4*>(p);
#pragma unroll
        for (int q = 0; q < 2 * NN / 4; ++q) {
            float ww[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int f = 4 * q + t;
                ww[t] = y[f / NN][(f % NN) / N][f % N];
            }
            v[q] = make_float4(ww[0], ww[1], ww[2], ww[3]);
        }
    } else {
        float2* v = reinterpret_cast<float2*>(p);
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            const int f0 = 2 * q, f1 = 2 * q + 1;
            v[q] = make_float2(y[f0 / NN][(f0 % NN) / N][f0 % N], y[f1 / NN][(f1 % NN) / N][f1 % N]);
        }
    }
}

// Traces of both faces with normal direction DIR (0: x, faces left/right;
// 1: y, faces bottom/top), both components: record [val c0 | val c1 |
// der c0 | der c1] (N each; der = physical normal derivative).  The even and
// odd parts along the normal are shared by the two faces.
template <int N, int DIR>
__device__ __forceinline__ void dir_traces(const float (&u)[2][N][N], float two_over_h,
                                           float (&lo)[4 * N], float (&hi)[4 * N]) {
    float dps[N];   // l_q'(+1) times 2 / h: physical derivative
#pragma unroll
    for (int q = 0; q < N; ++q) dps[q] = float(kT<N>.dp[q]) * two_over_h;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int m = 0; m < N; ++m) {
            float ev = 0.f, od = 0.f, evd = 0.f, odd = 0.f;
#pragma unroll
            for (int q = 0; q < N; ++q) {
                const float uq = DIR == 0 ? u[c][m][q] : u[c][q][m];   // q along the normal
                if (q % 2 == 0) {
                    ev = fmaf(float(kT<N>.lp[q]), uq, ev);
                    if (q > 0) evd = fmaf(dps[q], uq, evd);
                } else {
                    od = fmaf(float(kT<N>.lp[q]), uq, od);
                    odd = fmaf(dps[q], uq, odd);
                }
            }
            // l_q(-1) = (-1)^q l_q(1),  l_q'(-1) = -(-1)^q l_q'(1)
            lo[c * N + m] = ev - od;
            hi[c * N + m] = ev + od;
            lo[2 * N + c * N + m] = odd - evd;
            hi[2 * N + c * N + m] = evd + odd;
        }
}

// Volume terms of component C times eta_K (the same 1D Kronecker form as the
// component-split kernels: G along x and y on u_C, D x D cross terms), every
// scalar factor folded into the few nonzero table entries first.
template <int N, int C>
__device__ __forceinline__ void volume_comp(const ElemArgs<float>& a, const float (&u)[2][N][N],
                                            float etaK, float (&y)[N][N]) {
    const float sx = etaK * (C == 0 ? a.c2hy_hx : a.chy_hx);   // weight of G along x on u_C
    const float sy = etaK * (C == 0 ? a.chx_hy : a.c2hx_hy);   // weight of G along y on u_C
    float Gx[N][N], Gy[N][N], De[N][N];   // scaled tables (zero entries never read)
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
        for (int q = 0; q < N; ++q) {
            Gx[p][q] = kT<N>.G[p][q] != 0.0 ? sx * float(kT<N>.G[p][q]) : 0.f;
            Gy[p][q] = kT<N>.G[p][q] != 0.0 ? sy * float(kT<N>.G[p][q]) : 0.f;
            De[p][q] = kT<N>.D[p][q] != 0.0 ? etaK * float(kT<N>.D[p][q]) : 0.f;
        }
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
        for (int av = 0; av < N; ++av) {
            float acc = 0.f;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                if (kT<N>.G[av][i] != 0.0) acc = fmaf(Gx[av][i], u[C][b][i], acc);
                if (kT<N>.G[b][i] != 0.0) acc = fmaf(Gy[b][i], u[C][i][av], acc);
            }
            y[b][av] = acc;
        }
    float w[N][N];
    if constexpr (C == 0) {
        // y_x[b][a] += eta_K sum_j D[j][b] sum_i D[a][i] u_y[j][i]
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
            for (int av = 0; av < N; ++av) {
                float t = 0.f;
#pragma unroll
                for (int i = 0; i < N; ++i)
                    if (kT<N>.D[av][i] != 0.0) t = fmaf(float(kT<N>.D[av][i]), u[1][j][i], t);
                w[j][av] = t;
            }
#pragma unroll
        for (int b = 0; b < N; ++b)
#pragma unroll
            for (int av = 0; av < N; ++av)
#pragma unroll
                for (int j = 0; j < N; ++j)
                    if (kT<N>.D[j][b] != 0.0) y[b][av] = fmaf(De[j][b], w[j][av], y[b][av]);
    } else {
        // y_y[b][a] += eta_K sum_i D[i][a] sum_j D[b][j] u_x[j][i]
#pragma unroll
        for (int b = 0; b < N; ++b)
#pragma unroll
            for (int i = 0; i < N; ++i) {
                float t = 0.f;
#pragma unroll
                for (int j = 0; j < N; ++j)
                    if (kT<N>.D[b][j] != 0.0) t = fmaf(float(kT<N>.D[b][j]), u[0][j][i], t);
                w[b][i] = t;
            }
#pragma unroll
        for (int b = 0; b < N; ++b)
#pragma unroll
            for (int av = 0; av < N; ++av)
#pragma unroll
                for (int i = 0; i < N; ++i)
                    if (kT<N>.D[i][av] != 0.0) y[b][av] = fmaf(De[i][av], w[b][i], y[b][av]);
    }
}

// Face vectors of one face of K with normal direction DIR on side `side`,
// any kind (face_pq): the case of boundary faces and ragged tiles.
template <int N, int DIR>
__device__ __forceinline__ void face_general(const ElemArgs<float>& a, int side, bool nb, float etaK,
                                          float etaN, const float* own, const float* nbr, float* P,
                                          float* Q) {
    const FaceGeo<float>& fg = DIR == 0 ? a.fgx : a.fgy;
    const float pen = DIR == 0 ? a.pen_x : a.pen_y;
    float Dm[N * N];
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
        for (int q = 0; q < N; ++q) Dm[p * N + q] = float(kT<N>.D[p][q]);
    const int kind = nb ? 0 : 1 + a.bc[2 * DIR + side];
    const float eN = nb ? etaN : 0.f;
    const float sigma = pen * (nb ? fmaxf(etaK, eN) : 2.f * etaK);
    const float s = side == 0 ? -1.f : 1.f;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int m = 0; m < N; ++m)
            face_pq<N, float>(kind, c, m, DIR, s, fg, etaK, eN, sigma, own, own + 2 * N, nbr,
                              nbr + 2 * N, Dm, P[c * N + m], Q[c * N + m]);
}

// Face terms of the two faces with normal direction DIR, both components,
// spread into y (test mode q along the normal, m along the face).  A side
// whose faces are interior for the whole warp takes face_interior; otherwise
// face_pq with the face's kind (boundary kinds, ragged tiles).  nb_lo /
// nb_hi: the face has a neighbour element.
template <int N, int DIR>
__device__ __forceinline__ void flux_dir(const ElemArgs<float>& a, bool nb_lo, bool nb_hi,
                                         float etaK, float eta_lo, float eta_hi,
                                         const float (&own_lo)[4 * N], const float (&own_hi)[4 * N],
                                         const float (&nbr_lo)[4 * N], const float (&nbr_hi)[4 * N],
                                         float (&y)[2][N][N]) {
    const FaceGeo<float>& fg = DIR == 0 ? a.fgx : a.fgy;
    const float pen = DIR == 0 ? a.pen_x : a.pen_y;
    float P[2][2][N], Q[2][2][N];   // [comp][side][m]
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const bool nb = side == 0 ? nb_lo : nb_hi;
        const float etaN = side == 0 ? eta_lo : eta_hi;
        const float(&own)[4 * N] = side == 0 ? own_lo : own_hi;
        const float(&nbr)[4 * N] = side == 0 ? nbr_lo : nbr_hi;
        if (__all_sync(FULL, nb)) {   // every lane of the warp is active here
            face_interior_comp<N, float, 0>(DIR, side, fg, pen, etaK, etaN, own, nbr, P[0][side],
                                            Q[0][side]);
            face_interior_comp<N, float, 1>(DIR, side, fg, pen, etaK, etaN, own, nbr, P[1][side],
                                            Q[1][side]);
        } else {
            float tp[2 * N], tq[2 * N];
            face_general<N, DIR>(a, side, nb, etaK, etaN, own, nbr, tp, tq);
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int m = 0; m < N; ++m) {
                    P[c][side][m] = tp[c * N + m];
                    Q[c][side][m] = tq[c * N + m];
                }
        }
    }
    spread_faces<N, float>(DIR, P[0], Q[0], y[0]);
    spread_faces<N, float>(DIR, P[1], Q[1], y[1]);
}

template <int N>
__device__ __forceinline__ void load_rec(const float* p, float (&r)[4 * N]) {
    const float2* v = reinterpret_cast<const float2*>(p);
#pragma unroll
    for (int q = 0; q < 2 * N; ++q) {
        const float2 w = v[q];
        r[2 * q] = w.x;
        r[2 * q + 1] = w.y;
    }
}
template <int N>
__device__ __forceinline__ void store_rec(float* p, const float (&r)[4 * N]) {
    float2* v = reinterpret_cast<float2*>(p);
#pragma unroll
    for (int q = 0; q < 2 * N; ++q) v[q] = make_float2(r[2 * q], r[2 * q + 1]);
}

// One tile (ex0, ey0) from stage buffer buf: y = alpha A x + beta z.
template <int N>
__device__ __forceinline__ void warp_tile(const WarpArgs& a, int ex0, int ey0, unsigned char* buf,
                                          const float* seta, float* rec, float* halo) {
    using L = WarpLayout<N>;
    const ElemArgs<float>& c = a.c;
    const int nx = c.nx, ny = c.ny;
    const int r = threadIdx.x / 32, l = threadIdx.x % 32;
    const int ex = ex0 + l, ey = ey0 + r;

    // halo faces: the face of each outside neighbour that touches the tile
    // (18 per warp: lanes 0..17)
    {
        const int h = r * (L::NHALO / WTY) + l;
        if (l < L::NHALO / WTY) {
            int sr, j, F;
            if (h < WTX) { sr = 0; j = h + 1; F = 3; }                           // below: its top
            else if (h < 2 * WTX) { sr = L::SH - 1; j = h - WTX + 1; F = 2; }    // above: its bottom
            else if (h < 2 * WTX + WTY) { sr = h - 2 * WTX + 1; j = 0; F = 1; }  // left: its right
            else { sr = h - 2 * WTX - WTY + 1; j = L::SW - 1; F = 0; }           // right: its left
            const int hx = ex0 - 1 + j, hy = ey0 - 1 + sr;
            if (hx >= 0 && hx < nx && hy >= 0 && hy < ny) {
                float uh[2][N][N];
                load_elem<N>(buf + sr * L::ROWB + elem_off<N>(hy, nx, ex0, j), uh);
                face_traces<N, float>(uh, F, F < 2 ? c.two_over_hx : c.two_over_hy,
                                      halo + h * L::TRS);
            }
        }
    }
    const bool active = ex < nx && ey < ny;
    unsigned char* mine = buf + (r + 1) * L::ROWB + elem_off<N>(ey, nx, ex0, l + 1);
    float u[2][N][N];
    if (active) {
        load_elem<N>(mine, u);
    } else {
#pragma unroll
        for (int cc = 0; cc < 2; ++cc)
#pragma unroll
            for (int j = 0; j < N; ++j)
#pragma unroll
                for (int i = 0; i < N; ++i) u[cc][j][i] = 0.f;
    }
    const float etaK = seta[(r + 1) * L::SW + l + 1];
    float* rec_bot = rec + (0 * WTY + r) * WTX * L::TRS + l * L::TRS;   // own bottom face
    float* rec_top = rec + (1 * WTY + r) * WTX * L::TRS + l * L::TRS;   // own top face
    {
        float bo[4 * N], to[4 * N];
        dir_traces<N, 1>(u, c.two_over_hy, bo, to);
        store_rec<N>(rec_bot, bo);
        store_rec<N>(rec_top, to);
    }
    float y[2][N][N];
    volume_comp<N, 0>(c, u, etaK, y[0]);
    volume_comp<N, 1>(c, u, etaK, y[1]);
    float xl[4 * N], xr[4 * N];
    dir_traces<N, 0>(u, c.two_over_hx, xl, xr);
    __syncthreads();   // records and halo faces written

    {   // faces with x-normal: neighbour traces by shuffle, halo columns at the ends
        float nl[4 * N], nr[4 * N];
#pragma unroll
        for (int k = 0; k < 4 * N; ++k) {
            nl[k] = __shfl_up_sync(FULL, xr[k], 1);
            nr[k] = __shfl_down_sync(FULL, xl[k], 1);
        }
        if (l == 0) load_rec<N>(halo + (2 * WTX + r) * L::TRS, nl);
        if (l == WTX - 1) load_rec<N>(halo + (2 * WTX + WTY + r) * L::TRS, nr);
        const float eta_l = seta[(r + 1) * L::SW + l];
        const float eta_r = seta[(r + 1) * L::SW + l + 2];
        flux_dir<N, 0>(c, ex > 0, ex < nx - 1, etaK, eta_l, eta_r, xl, xr, nl, nr, y);
    }
    {   // faces with y-normal: records of the rows below and above
        float ob[4 * N], ot[4 * N], nb[4 * N], nt[4 * N];
        load_rec<N>(rec_bot, ob);
        load_rec<N>(rec_top, ot);
        load_rec<N>(r > 0 ? rec + (1 * WTY + r - 1) * WTX * L::TRS + l * L::TRS
                          : halo + l * L::TRS, nb);
        load_rec<N>(r < WTY - 1 ? rec + (0 * WTY + r + 1) * WTX * L::TRS + l * L::TRS
                                : halo + (WTX + l) * L::TRS, nt);
        const float eta_b = seta[r * L::SW + l + 1];
        const float eta_t = seta[(r + 2) * L::SW + l + 1];
        flux_dir<N, 1>(c, ey > 0, ey < ny - 1, etaK, eta_b, eta_t, ob, ot, nb, nt, y);
    }

    // result: into the element's own slot, then the warp's row out, as bulk
    // copies (y = A x on aligned rows) or as 16-byte chunks alpha y + beta z
    if (active) store_elem<N>(mine, y);
    if (ey >= ny) return;   // uniform over the warp
    if (a.skip && a.skip[size_t(ey >> 1) * a.ntx + (ex0 / WTX)]) return;   // the FP64 launch's row
    const int ehi = min(ex0 + WTX, nx);
    const long long row = (long long)ey * nx;
    char* yb = reinterpret_cast<char*>(a.y);
    if (a.bulk) {
        if constexpr (L::PAD) {
            if (active) {   // each element's slot (16-byte aligned, EB a multiple of 32)
                fence_async_smem();
                bulk_store(yb + (row + ex) * L::EB, smem_u32(mine), L::EB);
                bulk_commit();
            }
            return;
        } else {
            const long long gs = (row + ex0) * L::EB, ge = (row + ehi) * L::EB;
            if (((gs | ge) & 15) == 0) {   // uniform over the warp
                fence_async_smem();
                __syncwarp();
                if (l == 0) {
                    bulk_store(yb + gs,
                               smem_u32(buf + (r + 1) * L::ROWB + elem_off<N>(ey, nx, ex0, 1)),
                               unsigned(ge - gs));
                    bulk_commit();
                }
                return;
            }
        }
    }
    __syncwarp();
    const unsigned char* srow = buf + (r + 1) * L::ROWB;
    const float alpha = c.alpha, beta = c.beta;
    const char* zb = reinterpret_cast<const char*>(a.z);
    if constexpr (L::PAD && 32 % L::CPE == 0) {
        constexpr int EPI = 32 / L::CPE;
        const int nch = (ehi - ex0) * L::CPE;
        const long long g0 = (row + ex0) * L::EB + 16 * l;
        const unsigned char* sp = srow + (l / L::CPE + 1) * L::SLOT + 16 * (l % L::CPE);
#pragma unroll
        for (int i = 0; i < L::CPE; ++i) {
            if (l + 32 * i >= nch) break;
            float4 v = *reinterpret_cast<const float4*>(sp + i * EPI * L::SLOT);
            const long long g = g0 + 512 * i;
            if (zb) {
                const float4 zv = __ldg(reinterpret_cast<const float4*>(zb + g));
                v = make_float4(fmaf(alpha, v.x, beta * zv.x), fmaf(alpha, v.y, beta * zv.y),
                                fmaf(alpha, v.z, beta * zv.z), fmaf(alpha, v.w, beta * zv.w));
            } else {
                v = make_float4(alpha * v.x, alpha * v.y, alpha * v.z, alpha * v.w);
            }
            *reinterpret_cast<float4*>(yb + g) = v;
        }
    } else if constexpr (L::PAD) {
        const int nch = (ehi - ex0) * L::CPE;
        const long long g0 = (row + ex0) * L::EB;
        for (int q = l; q < nch; q += 32) {
            const int e = q / L::CPE, sub = q - e * L::CPE;
            float4 v = *reinterpret_cast<const float4*>(srow + (e + 1) * L::SLOT + 16 * sub);
            const long long g = g0 + 16LL * q;
            if (zb) {
                const float4 zv = __ldg(reinterpret_cast<const float4*>(zb + g));
                v = make_float4(fmaf(alpha, v.x, beta * zv.x), fmaf(alpha, v.y, beta * zv.y),
                                fmaf(alpha, v.z, beta * zv.z), fmaf(alpha, v.w, beta * zv.w));
            } else {
                v = make_float4(alpha * v.x, alpha * v.y, alpha * v.z, alpha * v.w);
            }
            *reinterpret_cast<float4*>(yb + g) = v;
        }
    } else {
        const long long anchor = (row + ex0 - 1) * L::EB;
        const long long gs = (row + ex0) * L::EB, ge = (row + ehi) * L::EB;
        const long long g16 = gs & ~15LL;
        const int nch = int((ge - g16 + 15) >> 4);
        const bool head8 = g16 != gs, tail8 = (ge & 15) != 0;
        const unsigned char* sp = srow + int(anchor & 15) + int(g16 - anchor) + 16 * l;
        const long long gl = g16 + 16 * l;
        constexpr int MAXC = (WTX * L::EB + 16) / 16 + 1;   // chunks of a row, at most
#pragma unroll
        for (int i = 0; i < (MAXC + 31) / 32; ++i) {
            const int q = l + 32 * i;
            if (q >= nch) break;
            const long long g = gl + 512 * i;
            if ((head8 && q == 0) || (tail8 && q == nch - 1)) {
                // an 8-byte half at either end of a row with an odd start
                const int off = (head8 && q == 0) ? 8 : 0;
                const float2 v = *reinterpret_cast<const float2*>(sp + 512 * i + off);
                float2 w;
                if (zb) {
                    const float2 zv = __ldg(reinterpret_cast<const float2*>(zb + g + off));
                    w = make_float2(fmaf(alpha, v.x, beta * zv.x), fmaf(alpha, v.y, beta * zv.y));
                } else {
                    w = make_float2(alpha * v.x, alpha * v.y);
                }
                *reinterpret_cast<float2*>(yb + g + off) = w;
            } else {
                float4 v = *reinterpret_cast<const float4*>(sp + 512 * i);
                if (zb) {
                    const float4 zv = __ldg(reinterpret_cast<const float4*>(zb + g));
                    v = make_float4(fmaf(alpha, v.x, beta * zv.x), fmaf(alpha, v.y, beta * zv.y),
                                    fmaf(alpha, v.z, beta * zv.z), fmaf(alpha, v.w, beta * zv.w));
                } else {
                    v = make_float4(alpha * v.x, alpha * v.y, alpha * v.z, alpha * v.w);
                }
                *reinterpret_cast<float4*>(yb + g) = v;
            }
        }
    }
}

// Persistent CTAs: tile t = blockIdx.x + i gridDim.x, staged NBUF tiles ahead.
template <int N, int NBUF>
__global__ void __launch_bounds__(WNT, (WarpLayout<N, NBUF>::MINB)) k_apply_warp(const WarpArgs a) {
    using L = WarpLayout<N, NBUF>;
    grid_dep_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* seta0 = reinterpret_cast<float*>(smem_raw + L::OFF_ETA);
    float* rec = reinterpret_cast<float*>(smem_raw + L::OFF_REC);
    float* halo = reinterpret_cast<float*>(smem_raw + L::OFF_HALO);
    const int G = int(gridDim.x);
#pragma unroll 1
    for (int s = 0; s < NBUF; ++s) {
        const int ts = int(blockIdx.x) + s * G;
        if (ts < a.ntiles)
            warp_stage<N>(a, (ts % a.ntx) * WTX, (ts / a.ntx) * WTY, smem_raw + s * L::BUFB,
                          seta0 + s * L::SH * L::SW);
        cp_commit();
    }
#pragma unroll 1
    for (int it = 0, t = int(blockIdx.x); t < a.ntiles; ++it, t += G) {
        const int b = NBUF == 1 ? 0 : (it & 1);
        if constexpr (NBUF == 1) cp_wait0(); else cp_wait1();   // this thread's copies of tile t
        __syncthreads();   // everyone's
        warp_tile<N>(a, (t % a.ntx) * WTX, (t / a.ntx) * WTY, smem_raw + b * L::BUFB,
                     seta0 + b * L::SH * L::SW, rec, halo);
        bulk_wait_read();  // this thread's bulk output copies have left buffer b
        __syncthreads();   // buffer b, records and halo faces free
        const int tn = t + NBUF * G;
        if (tn < a.ntiles)
            warp_stage<N>(a, (tn % a.ntx) * WTX, (tn / a.ntx) * WTY, smem_raw + b * L::BUFB,
                          seta0 + b * L::SH * L::SW);
        cp_commit();
    }
}

int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    SIP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] == 0) {
        int n = 0;
        SIP_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        cached[dev] = n;   // benign race: every writer stores the same value
    }
    return cached[dev];
}

template <int N, int NBUF>
void warp_apply_nb(const OpGeom& g, const float* x, float* y, const float* eta, float alpha,
                   const float* z, float beta, const unsigned char* skip, cudaStream_t s) {
    using L = WarpLayout<N, NBUF>;
    WarpArgs a;
    a.c = make_elem_args<float>(g, nullptr, nullptr, nullptr, alpha, nullptr, beta);
    a.x = x;
    a.y = y;
    a.eta = eta;
    a.z = z;
    a.n_total = (long long)g.nx * g.ny * L::NB;
    a.ntx = (g.nx + WTX - 1) / WTX;
    a.ntiles = a.ntx * ((g.ny + WTY - 1) / WTY);
    a.bulk = (alpha == 1.f && z == nullptr) ? 1 : 0;
    a.skip = skip;
    static const bool attr = [] {   // once per process, thread-safe
        SIP_CUDA(cudaFuncSetAttribute(k_apply_warp<N, NBUF>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(L::BYTES)));
        return true;
    }();
    (void)attr;
    const int grid = std::min(a.ntiles, L::MINB * sm_count());
    launch_k(k_apply_warp<N, NBUF>, dim3(unsigned(grid)), dim3(WNT), size_t(L::BYTES), s, a);
    SIP_CHECK_LAUNCH();
}

// One stage buffer and three CTAs per SM where shared memory admits them:
// with the loads of one CTA overlapping the arithmetic of the others this
// measured as fast as a double buffer with two CTAs per SM, or faster (k = 3).
template <int N>
void warp_apply_n(const OpGeom& g, const float* x, float* y, const float* eta, float alpha,
                  const float* z, float beta, const unsigned char* skip, cudaStream_t s) {
    warp_apply_nb<N, 1>(g, x, y, eta, alpha, z, beta, skip, s);
}

}  // namespace

bool launch_apply_sip_warp(int N, const OpGeom& g, const float* x, float* y, const float* eta,
                           float alpha, const float* z, float beta, const unsigned char* skip,
                           cudaStream_t s) {
    if (g.n_hi > 0 && !skip) return false;   // split precision: this launch needs the flags
    if (!aligned16(x) || !aligned16(y) || (z && !aligned16(z))) return false;
    if (g.nx < 1 || g.ny < 1) return false;
    switch (N) {
        case 2: warp_apply_n<2>(g, x, y, eta, alpha, z, beta, skip, s); return true;
        case 3: warp_apply_n<3>(g, x, y, eta, alpha, z, beta, skip, s); return true;
        case 4: warp_apply_n<4>(g, x, y, eta, alpha, z, beta, skip, s); return true;
        case 5: warp_apply_n<5>(g, x, y, eta, alpha, z, beta, skip, s); return true;
        case 6: warp_apply_n<6>(g, x, y, eta, alpha, z, beta, skip, s); return true;
        default: return false;
    }
}

}  // namespace sip
