// Batched inner solves: the inner Krylov solves (Sec. 5-6: the viscous block
// solved by CG, or flexible CG for the FP32 V-cycle, preconditioned by one
// hp-multigrid V-cycle, Algorithm 1) of many independent Stokes problems of
// different mesh sizes, degrees and viscosity fields advance together in one
// CUDA graph.  Every stage of the V-cycle and of the Krylov iteration is one
// launch over a work list of (member, tile / element group / chunk) items,
// one launch per polynomial degree for the element kernels: the number of
// launches per stage does not grow with the number of problems.  The loop
// runs on the device (a `while` conditional node) until every member has met
// its stopping test or the iteration cap; a member that has stopped skips the
// rest of the loop.
//
// The outer Krylov method of each problem keeps running on its own host
// thread and stream (run_solve); where it asks for an inner solve, the
// thread waits at a rendezvous until every problem of the group still
// solving has asked, and the last one to arrive launches the batched loop
// for all of them.  So the problems move through their outer iterations in
// lockstep, and the device sees one batched inner solve per outer step.
//
// Same arithmetic as the single-problem loop (inner_graph.cu) except the
// blocking of the dot products (a fixed number of partial sums per member,
// deterministic), so a batched solve equals the same solve alone to rounding.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <mutex>

#include "sip_elem.cuh"
#include "sip_level.cuh"
#include "sip_solver.h"

namespace sip {

namespace {

constexpr int kMaxLv = 12;   // continuous levels of a member (h-levels 0..L)
constexpr int kMaxSt = 8;    // Chebyshev steps per smoothing
constexpr int kParts = 64;   // partial sums per member of a dot product
constexpr int kChunk = 256;  // entries per CTA of the vector kernels

// Device-resident description of one member: the buffers of its V-cycle
// (precision T) and of its inner Krylov iteration (FP64).
template <typename T>
struct BMember {
    int N, nx, ny, L;   // degree + 1, mesh, coarsest continuous level
    long long ne, n_u;
    T *vin, *vout, *pr, *pd, *r1, *e1;
    int hnx[kMaxLv], hny[kMaxLv];   // elements per side of continuous level l
    long long hn[kMaxLv];           // its unknowns, 2 (hnx + 1)(hny + 1)
    const T* S[kMaxLv];
    const T* dinv[kMaxLv];
    T* hb[kMaxLv];
    T* hx[kMaxLv];
    T* hr[kMaxLv];
    T* hd[kMaxLv];
    T* hd2[kMaxLv];
    T hc1[kMaxLv][kMaxSt], hc2[kMaxLv][kMaxSt];   // Chebyshev coefficients per level, step
    const T* cinv;
    int nc;
    double *r, *d, *q, *z;   // inner Krylov vectors
};

// Krylov state of one member; t / y are set per round.
struct BState {
    const double* t;
    double* y;
    double nt, rz, dq, alpha, beta, rr;
    int it, status, want;
};

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[32];
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    v = warp_sum(v);
    if (lane == 0) ws[w] = v;
    __syncthreads();
    v = threadIdx.x < blockDim.x / 32 ? ws[lane] : 0.0;
    if (w == 0) v = warp_sum(v);
    __syncthreads();
    return v;
}

// member m's sum of its kParts partials (one CTA per member)
__device__ __forceinline__ double member_sum(const double* partial, int m) {
    const double v = threadIdx.x < kParts ? partial[size_t(m) * kParts + threadIdx.x] : 0.0;
    return block_sum(v);
}

// ---- element-vector kernels: items (member, chunk of kChunk entries)

// which vector of the p-level a kernel reads / writes
enum PVec { V_IN, V_OUT, V_PR, V_PD, V_R1, V_E1 };
template <typename T>
__device__ __forceinline__ T* pvec(const BMember<T>& b, int v) {
    switch (v) {
        case V_IN: return b.vin;
        case V_OUT: return b.vout;
        case V_PR: return b.pr;
        case V_PD: return b.pd;
        case V_R1: return b.r1;
        default: return b.e1;
    }
}

// dst = src over n_u entries (T)
template <typename T>
__global__ void k_b_copy(const BMember<T>* __restrict__ mb, const int2* __restrict__ items,
                         const int* __restrict__ act, int src, int dst) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    if (!act[it.x]) return;
    const BMember<T>& b = mb[it.x];
    const long long g = (long long)it.y * kChunk + threadIdx.x;
    if (g >= b.n_u) return;
    pvec(b, dst)[g] = pvec(b, src)[g];
}

// vin = (T) r   (the V-cycle input, rounded to its precision)
template <typename T>
__global__ void k_b_r_to_vin(const BMember<T>* __restrict__ mb, const int2* __restrict__ items,
                             const int* __restrict__ act) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    if (!act[it.x]) return;
    const BMember<T>& b = mb[it.x];
    const long long g = (long long)it.y * kChunk + threadIdx.x;
    if (g >= b.n_u) return;
    b.vin[g] = T(b.r[g]);
}

// e1 -> y: y += P e1 (hierarchical injection of the Q_1 modes); items over ne * 8
template <typename T>
__global__ void k_b_prolong_add(const BMember<T>* __restrict__ mb, const int2* __restrict__ items,
                                const int* __restrict__ act) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    if (!act[it.x]) return;
    const BMember<T>& b = mb[it.x];
    const long long g = (long long)it.y * kChunk + threadIdx.x;
    if (g >= b.ne * 8) return;
    const int N = b.N;
    const long long e = g / 8;
    const int l = int(g % 8), c = l / 4, j = (l / 2) % 2, i = l % 2;
    b.vout[e * 2 * N * N + c * N * N + j * N + i] += b.e1[g];
}

// R_dc: level-0 vertex values from the element Q_1 residual r1; items over hn[0]
template <typename T>
__global__ void k_b_rdc(const BMember<T>* __restrict__ mb, const int2* __restrict__ items,
                        const int* __restrict__ act) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    if (!act[it.x]) return;
    const BMember<T>& b = mb[it.x];
    const long long g = (long long)it.y * kChunk + threadIdx.x;
    if (g >= b.hn[0]) return;
    const int nx = b.nx, ny = b.ny;
    const int c = int(g % 2);
    const long long v = g / 2;
    const int vx = int(v % (nx + 1)), vy = int(v / (nx + 1));
    double acc = 0.0;
    for (int q = 0; q < 2; ++q) {
        const int ey = vy - q;
        if (ey < 0 || ey >= ny) continue;
        for (int p = 0; p < 2; ++p) {
            const int ex = vx - p;
            if (ex < 0 || ex >= nx) continue;
            const T* re = b.r1 + ((long long)ey * nx + ex) * 8 + c * 4;
            for (int j = 0; j < 2; ++j)
                for (int i = 0; i < 2; ++i) acc += hatw(i, p) * hatw(j, q) * double(re[j * 2 + i]);
        }
    }
    b.hb[0][g] = T(acc);
}

// P_cd: element Q_1 coefficients e1 from the level-0 vertex values; items over ne * 8
template <typename T>
__global__ void k_b_pcd(const BMember<T>* __restrict__ mb, const int2* __restrict__ items,
                        const int* __restrict__ act) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    if (!act[it.x]) return;
    const BMember<T>& b = mb[it.x];
    const long long g = (long long)it.y * kChunk + threadIdx.x;
    if (g >= b.ne * 8) return;
    const int nx = b.nx;
    const long long e = g / 8;
    const int l = int(g % 8), c = l / 4, j = (l / 2) % 2, i = l % 2;
    const int ex = int(e % nx), ey = int(e / nx);
    const T* v = b.hx[0];
    double acc = 0.0;
    for (int q = 0; q < 2; ++q)
        for (int p = 0; p < 2; ++p)
            acc += hatw(i, p) * hatw(j, q) *
                   double(v[2 * ((long long)(ey + q) * (nx + 1) + ex + p) + c]);
    b.e1[g] = T(acc);
}

// ---- continuous levels: items (member, chunk) over the unknowns of level lv

// first Chebyshev step from zero: r = b, d = c2 D^{-1} b, x = d
template <typename T>
__global__ void k_b_hfirst(const BMember<T>* __restrict__ mb, const int2* __restrict__ items,
                           const int* __restrict__ act, int lv) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    if (!act[it.x]) return;
    const BMember<T>& b = mb[it.x];
    const long long g = (long long)it.y * kChunk + threadIdx.x;
    if (g >= b.hn[lv]) return;
    const T bv = b.hb[lv][g];
    const T v = b.hc2[lv][0] * b.dinv[lv][g] * bv;
    b.hr[lv][g] = bv;
    b.hd[lv][g] = v;
    b.hx[lv][g] = v;
}

// first step from a non-zero iterate, x update deferred: r = b - S x, d = c2 D^{-1} r
template <typename T>
__global__ void k_b_hstart(const BMember<T>* __restrict__ mb, const int2* __restrict__ items,
                           const int* __restrict__ act, int lv) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    if (!act[it.x]) return;
    const BMember<T>& b = mb[it.x];
    const long long g = (long long)it.y * kChunk + threadIdx.x;
    if (g >= b.hn[lv]) return;
    const int nvx = b.hnx[lv] + 1, nvy = b.hny[lv] + 1;
    const int c = int(g % 2);
    const long long v = g / 2;
    const T acc = stencil_row<T, false>(nvx, nvy, int(v % nvx), int(v / nvx), c,
                                        b.S[lv] + v * 36, b.hx[lv]);
    const T rn = b.hb[lv][g] - acc;
    b.hr[lv][g] = rn;
    b.hd[lv][g] = b.hc2[lv][0] * b.dinv[lv][g] * rn;
}

// step st >= 1: r -= S d_old; d_new = c1 d_old + c2 D^{-1} r; x += d_new (+ d_old if pend)
template <typename T>
__global__ void k_b_hstep(const BMember<T>* __restrict__ mb, const int2* __restrict__ items,
                          const int* __restrict__ act, int lv, int st, int pend) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    if (!act[it.x]) return;
    const BMember<T>& b = mb[it.x];
    const long long g = (long long)it.y * kChunk + threadIdx.x;
    if (g >= b.hn[lv]) return;
    const T* d_old = (st % 2 == 1) ? b.hd[lv] : b.hd2[lv];
    T* d_new = (st % 2 == 1) ? b.hd2[lv] : b.hd[lv];
    const int nvx = b.hnx[lv] + 1, nvy = b.hny[lv] + 1;
    const int c = int(g % 2);
    const long long v = g / 2;
    const T acc = stencil_row<T, false>(nvx, nvy, int(v % nvx), int(v / nvx), c,
                                        b.S[lv] + v * 36, d_old);
    const T rn = b.hr[lv][g] - acc;
    b.hr[lv][g] = rn;
    const T dn = b.hc1[lv][st] * d_old[g] + b.hc2[lv][st] * b.dinv[lv][g] * rn;
    d_new[g] = dn;
    b.hx[lv][g] += pend ? d_old[g] + dn : dn;
}

// r = b - S x on level lv
template <typename T>
__global__ void k_b_hresid(const BMember<T>* __restrict__ mb, const int2* __restrict__ items,
                           const int* __restrict__ act, int lv) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    if (!act[it.x]) return;
    const BMember<T>& b = mb[it.x];
    const long long g = (long long)it.y * kChunk + threadIdx.x;
    if (g >= b.hn[lv]) return;
    const int nvx = b.hnx[lv] + 1, nvy = b.hny[lv] + 1;
    const int c = int(g % 2);
    const long long v = g / 2;
    const T acc = stencil_row<T, false>(nvx, nvy, int(v % nvx), int(v / nvx), c,
                                        b.S[lv] + v * 36, b.hx[lv]);
    b.hr[lv][g] = b.hb[lv][g] - acc;
}

// b_{lv+1} = R_h r_lv (items over the unknowns of level lv + 1)
template <typename T>
__global__ void k_b_rh(const BMember<T>* __restrict__ mb, const int2* __restrict__ items,
                       const int* __restrict__ act, int lv) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    if (!act[it.x]) return;
    const BMember<T>& b = mb[it.x];
    const long long g = (long long)it.y * kChunk + threadIdx.x;
    if (g >= b.hn[lv + 1]) return;
    const int nxc = b.hnx[lv + 1], nyc = b.hny[lv + 1];
    const int nfx = 2 * nxc + 1, nfy = 2 * nyc + 1;
    const int c = int(g % 2);
    const long long v = g / 2;
    const int I = int(v % (nxc + 1)), J = int(v / (nxc + 1));
    const T* rf = b.hr[lv];
    T acc = T(0);
    for (int dy = -1; dy <= 1; ++dy) {
        const int fy = 2 * J + dy;
        if (fy < 0 || fy >= nfy) continue;
        const T wy = dy == 0 ? T(1) : T(0.5);
        for (int dx = -1; dx <= 1; ++dx) {
            const int fx = 2 * I + dx;
            if (fx < 0 || fx >= nfx) continue;
            const T wx = dx == 0 ? T(1) : T(0.5);
            acc += wx * wy * rf[2 * ((long long)fy * nfx + fx) + c];
        }
    }
    b.hb[lv + 1][g] = acc;
}

// x_lv += P_h x_{lv+1} (items over the unknowns of level lv)
template <typename T>
__global__ void k_b_ph_add(const BMember<T>* __restrict__ mb, const int2* __restrict__ items,
                           const int* __restrict__ act, int lv) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    if (!act[it.x]) return;
    const BMember<T>& b = mb[it.x];
    const long long g = (long long)it.y * kChunk + threadIdx.x;
    if (g >= b.hn[lv]) return;
    const int nxc = b.hnx[lv + 1];
    const int nfx = 2 * nxc + 1;
    const T* xc = b.hx[lv + 1];
    const int c = int(g % 2);
    const long long v = g / 2;
    const int fx = int(v % nfx), fy = int(v / nfx);
    const int ix0 = fx / 2, ix1 = (fx + 1) / 2, iy0 = fy / 2, iy1 = (fy + 1) / 2;
    const T wx = (fx % 2) ? T(0.5) : T(1), wy = (fy % 2) ? T(0.5) : T(1);
    const long long rc = nxc + 1;
    T acc;
    if (fx % 2 == 0 && fy % 2 == 0) {
        acc = xc[2 * (iy0 * rc + ix0) + c];
    } else if (fy % 2 == 0) {
        acc = wx * (xc[2 * (iy0 * rc + ix0) + c] + xc[2 * (iy0 * rc + ix1) + c]);
    } else if (fx % 2 == 0) {
        acc = wy * (xc[2 * (iy0 * rc + ix0) + c] + xc[2 * (iy1 * rc + ix0) + c]);
    } else {
        acc = wx * wy * (xc[2 * (iy0 * rc + ix0) + c] + xc[2 * (iy0 * rc + ix1) + c] +
                         xc[2 * (iy1 * rc + ix0) + c] + xc[2 * (iy1 * rc + ix1) + c]);
    }
    b.hx[lv][g] += acc;
}

// coarsest level of every member: x_L = C^{-1} b_L (dense inverse), one warp
// per row; items (member, group of 8 rows)
template <typename T>
__global__ void k_b_coarse(const BMember<T>* __restrict__ mb, const int2* __restrict__ items,
                           const int* __restrict__ act) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    if (!act[it.x]) return;
    const BMember<T>& b = mb[it.x];
    const int row = it.y * 8 + threadIdx.x / 32, lane = threadIdx.x % 32;
    const int n = b.nc;
    if (row >= n) return;
    const T* M = b.cinv + size_t(row) * n;
    const T* x = b.hb[b.L];
    T acc = T(0);
    for (int j = lane; j < n; j += 32) acc += M[j] * x[j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) b.hx[b.L][row] = acc;
}

// ---- inner Krylov kernels (FP64): items (member, part) of kParts per member
// for the reductions, (member, chunk) for the updates

// r = t, y = 0, d = 0; partials of t.t.  Members that do not want a solve
// this round are skipped (want read from the state).
template <typename T>
__global__ void __launch_bounds__(kChunk) k_b_init(const BMember<T>* __restrict__ mb,
                                                   const BState* __restrict__ st,
                                                   const int2* __restrict__ items,
                                                   double* partial) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    const BMember<T>& b = mb[it.x];
    const BState& s = st[it.x];
    double acc = 0.0;
    if (s.want) {
        for (long long g = (long long)it.y * kChunk + threadIdx.x; g < b.n_u;
             g += (long long)kParts * kChunk) {
            const double v = s.t[g];
            acc += v * v;
            b.r[g] = v;
            s.y[g] = 0.0;
            b.d[g] = 0.0;
        }
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[size_t(it.x) * kParts + it.y] = acc;
}

__global__ void __launch_bounds__(kChunk) k_b_init_final(BState* st, int* act,
                                                         const double* partial) {
    grid_dep_wait();
    const int m = blockIdx.x;
    const double s = member_sum(partial, m);
    if (threadIdx.x == 0) {
        BState& x = st[m];
        const double nt = sqrt(s);
        x.nt = nt;
        x.rr = nt;
        x.rz = 0.0;
        x.it = 0;
        x.status = isfinite(nt) ? 0 : 1;
        act[m] = (x.want && isfinite(nt) && nt > 0.0) ? 1 : 0;
    }
}

// z = widen(vout); partials of (flexible ? z.q : r.z)
template <typename T>
__global__ void __launch_bounds__(kChunk) k_b_dot_z(const BMember<T>* __restrict__ mb,
                                                    const int2* __restrict__ items,
                                                    const int* __restrict__ act, int flexible,
                                                    double* partial) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    double acc = 0.0;
    if (act[it.x]) {
        const BMember<T>& b = mb[it.x];
        const double* w = flexible ? b.q : b.r;
        for (long long g = (long long)it.y * kChunk + threadIdx.x; g < b.n_u;
             g += (long long)kParts * kChunk) {
            const double z = double(b.vout[g]);
            b.z[g] = z;
            acc += z * w[g];
        }
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[size_t(it.x) * kParts + it.y] = acc;
}

// PCG: beta = rz_new / rz (0 on the first pass), rz = rz_new;
// FCG(1): beta = -(z.q) / (d.q) (stored so that d = z + beta d)
__global__ void __launch_bounds__(kChunk) k_b_beta_final(BState* st, const int* act,
                                                         const double* partial, int flexible) {
    grid_dep_wait();
    const int m = blockIdx.x;
    if (!act[m]) return;
    const double s = member_sum(partial, m);
    if (threadIdx.x == 0) {
        BState& x = st[m];
        if (flexible) {
            x.beta = x.it == 0 ? 0.0 : -(s / x.dq);
        } else {
            x.beta = x.it == 0 ? 0.0 : s / x.rz;
            x.rz = s;
        }
    }
}

// d = z + beta d
template <typename T>
__global__ void k_b_dir(const BMember<T>* __restrict__ mb, const BState* __restrict__ st,
                        const int2* __restrict__ items, const int* __restrict__ act) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    if (!act[it.x]) return;
    const BMember<T>& b = mb[it.x];
    const long long g = (long long)it.y * kChunk + threadIdx.x;
    if (g >= b.n_u) return;
    b.d[g] = b.z[g] + st[it.x].beta * b.d[g];
}

// partials of d.q (first half) and d.r (second half, flexible only)
template <typename T>
__global__ void __launch_bounds__(kChunk) k_b_dot_dq(const BMember<T>* __restrict__ mb,
                                                     const int2* __restrict__ items,
                                                     const int* __restrict__ act, int nmem,
                                                     int flexible, double* partial) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    double a1 = 0.0, a2 = 0.0;
    if (act[it.x]) {
        const BMember<T>& b = mb[it.x];
        for (long long g = (long long)it.y * kChunk + threadIdx.x; g < b.n_u;
             g += (long long)kParts * kChunk) {
            const double dv = b.d[g];
            a1 += dv * b.q[g];
            if (flexible) a2 += dv * b.r[g];
        }
    }
    a1 = block_sum(a1);
    a2 = block_sum(a2);
    if (threadIdx.x == 0) {
        partial[size_t(it.x) * kParts + it.y] = a1;
        partial[(size_t(nmem) + it.x) * kParts + it.y] = a2;
    }
}

// PCG: alpha = rz / (d.q); FCG: dq = d.q, alpha = (d.r) / dq
__global__ void __launch_bounds__(kChunk) k_b_alpha_final(BState* st, const int* act,
                                                          const double* partial, int nmem,
                                                          int flexible) {
    grid_dep_wait();
    const int m = blockIdx.x;
    if (!act[m]) return;
    const double dq = member_sum(partial, m);
    const double dr = member_sum(partial, nmem + m);
    if (threadIdx.x == 0) {
        BState& x = st[m];
        if (flexible) {
            x.dq = dq;
            x.alpha = dr / dq;
        } else {
            x.alpha = x.rz / dq;
        }
    }
}

// y += alpha d; r -= alpha q; partials of r.r
template <typename T>
__global__ void __launch_bounds__(kChunk) k_b_update(const BMember<T>* __restrict__ mb,
                                                     const BState* __restrict__ st,
                                                     const int2* __restrict__ items,
                                                     const int* __restrict__ act, double* partial) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    double acc = 0.0;
    if (act[it.x]) {
        const BMember<T>& b = mb[it.x];
        const double a = st[it.x].alpha;
        double* y = st[it.x].y;
        for (long long g = (long long)it.y * kChunk + threadIdx.x; g < b.n_u;
             g += (long long)kParts * kChunk) {
            y[g] += a * b.d[g];
            const double rv = b.r[g] - a * b.q[g];
            b.r[g] = rv;
            acc += rv * rv;
        }
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[size_t(it.x) * kParts + it.y] = acc;
}

// end of a pass of member m: counter, stopping test ||r|| < rtol ||t|| or
// the cap; a member that stops leaves the loop
__global__ void __launch_bounds__(kChunk) k_b_ctl_final(BState* st, int* act,
                                                        const double* partial, double rtol,
                                                        int maxit) {
    grid_dep_wait();
    const int m = blockIdx.x;
    if (!act[m]) return;
    const double s = member_sum(partial, m);
    if (threadIdx.x == 0) {
        BState& x = st[m];
        const double rr = sqrt(s);
        const int it = x.it + 1;
        x.it = it;
        x.rr = rr;
        if (!isfinite(rr)) x.status = 1;
        const bool more = isfinite(rr) && !(rr < rtol * x.nt) && it < maxit;
        act[m] = more ? 1 : 0;
    }
}

// loop condition: some member still iterating
__global__ void k_b_any(const int* act, int nmem, cudaGraphConditionalHandle h) {
    grid_dep_wait();
    int any = 0;
    for (int m = threadIdx.x; m < nmem; m += blockDim.x) any |= act[m];
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

inline int ceil_div(long long a, long long b) { return int((a + b - 1) / b); }

// device copy of a host vector (kept alive by the owner)
template <typename V>
void upload(DeviceBuffer& buf, const std::vector<V>& v, cudaStream_t s) {
    buf.alloc(std::max<size_t>(1, v.size()) * sizeof(V));
    if (!v.empty())
        SIP_CUDA(cudaMemcpyAsync(buf.ptr, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice, s));
}

struct Cheb {
    double theta, delta, sigma;
    Cheb(double lo, double hi) : theta(0.5 * (hi + lo)), delta(0.5 * (hi - lo)), sigma(theta / delta) {}
};

// coefficients (c1, c2) of the Chebyshev steps of Multigrid::smooth_p / smooth_h
void cheb_coefs(double lo, double hi, int steps, double* c1, double* c2) {
    const Cheb ch(lo, hi);
    double rho = 1.0 / ch.sigma;
    c1[0] = 0.0;
    c2[0] = 1.0 / ch.theta;
    for (int st = 1; st < steps; ++st) {
        const double rn = 1.0 / (2.0 * ch.sigma - rho);
        c1[st] = rn * rho;
        c2[st] = 2.0 * rn / ch.delta;
        rho = rn;
    }
}

}  // namespace

// ---------------------------------------------------------------- engine
// One batched inner loop for a fixed group of problems of one V-cycle
// precision T.  Built once per group (tables, work lists, the graph).
template <typename T>
struct BatchEngine {
    std::vector<sip_problem*> probs;
    int nmem = 0;
    bool flexible = false;
    double rtol = 0.0;
    int maxit = 0;
    int steps_p = 0, steps_h = 0;
    DeviceBuffer d_mem, d_state, d_act, d_partial;
    // per degree N: apply role tables (V-cycle precision, plus the FP64-
    // arithmetic tiles of split members) and their work lists
    struct Group {
        int N = 0;
        DeviceBuffer a_dec, a_res, a_r1, a_dec_hi, a_res_hi, a_r1_hi, a_q;
        DeviceBuffer it_lo, it_hi, it_all, it_bj;
        int n_lo = 0, n_hi = 0, n_all = 0, n_bj = 0;
        std::vector<DeviceBuffer> bj;   // block-Jacobi tables: [0] first step pre, [1] first step post, [1 + st] step st
    };
    std::vector<Group> groups;
    // work lists of the vector kernels
    DeviceBuffer it_u, it_parts, it_q1, it_v0, it_coarse;
    int n_u_items = 0, n_parts = 0, n_q1 = 0, n_v0 = 0, n_coarse = 0;
    std::vector<DeviceBuffer> it_lv, it_lv1;   // level l (members with l < L), level l + 1 of those
    std::vector<int> n_lv, n_lv1;
    int max_L = 0;
    bool vec = true;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;
    int64_t body_kernels = 0, top_kernels = 0;
    std::vector<BState> hstate;   // host mirror (pinned copy below)
    BState* pin = nullptr;

    ~BatchEngine() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        if (pin) cudaFreeHost(pin);
    }

    Multigrid<T>& mg(sip_problem* P);
    void build(cudaStream_t s);
    void capture_vcycle(cudaStream_t s);
    void capture_body(cudaStream_t s, cudaGraphConditionalHandle h);
    // one round: the listed members solve A y_m = t_m; returns iterations
    // per member (-1: breakdown)
    void round(const std::vector<const double*>& t, const std::vector<double*>& y,
               const std::vector<int>& want, std::vector<int>& its);
};

template <>
Multigrid<float>& BatchEngine<float>::mg(sip_problem* P) { return *P->mg32; }
template <>
Multigrid<double>& BatchEngine<double>::mg(sip_problem* P) { return *P->mg64; }

template <typename T>
void BatchEngine<T>::build(cudaStream_t s) {
    nmem = int(probs.size());
    std::vector<BMember<T>> hm(nmem);
    std::vector<int2> items_u, items_parts, items_q1, items_v0, items_coarse;
    max_L = 0;
    for (int m = 0; m < nmem; ++m) {
        sip_problem* P = probs[m];
        Multigrid<T>& G = mg(P);
        Workspace& W = *P->ws;
        for (DeviceBuffer* b : {&W.cg_r, &W.cg_d, &W.cg_q, &W.cg_z}) b->alloc(size_t(P->n_u) * sizeof(double));
        BMember<T>& b = hm[m];
        b.N = P->n;
        b.nx = P->desc.nx;
        b.ny = P->desc.ny;
        b.L = int(G.h.size()) - 1;
        b.ne = P->ne;
        b.n_u = P->n_u;
        b.vin = G.vin.template as<T>();
        b.vout = G.vout.template as<T>();
        b.pr = G.pr.template as<T>();
        b.pd = G.pd.template as<T>();
        b.r1 = G.r1.template as<T>();
        b.e1 = G.e1.template as<T>();
        require(b.L >= 1 && b.L < kMaxLv, "batched solve: needs 1 to 11 h-coarsenings");
        for (int l = 0; l <= b.L; ++l) {
            HLevel<T>& H = G.h[l];
            b.hnx[l] = H.nx;
            b.hny[l] = H.ny;
            b.hn[l] = (long long)H.n;
            b.S[l] = H.S.template as<T>();
            b.dinv[l] = H.dinv.template as<T>();
            b.hb[l] = H.b.template as<T>();
            b.hx[l] = H.x.template as<T>();
            b.hr[l] = H.r.template as<T>();
            b.hd[l] = H.d.template as<T>();
            b.hd2[l] = H.d2.template as<T>();
            double c1[kMaxSt], c2[kMaxSt];
            cheb_coefs(P->desc.cheb_lo * H.lmax, P->desc.cheb_hi * H.lmax, steps_h, c1, c2);
            for (int st = 0; st < kMaxSt; ++st) {
                b.hc1[l][st] = T(st < steps_h ? c1[st] : 0.0);
                b.hc2[l][st] = T(st < steps_h ? c2[st] : 0.0);
            }
        }
        b.cinv = G.cinv.template as<T>();
        b.nc = G.nc;
        b.r = W.cg_r.template as<double>();
        b.d = W.cg_d.template as<double>();
        b.q = W.cg_q.template as<double>();
        b.z = W.cg_z.template as<double>();
        max_L = std::max(max_L, b.L);
        for (int c = 0; c < ceil_div(b.n_u, kChunk); ++c) items_u.push_back({m, c});
        for (int c = 0; c < kParts; ++c) items_parts.push_back({m, c});
        for (int c = 0; c < ceil_div(b.ne * 8, kChunk); ++c) items_q1.push_back({m, c});
        for (int c = 0; c < ceil_div(b.hn[0], kChunk); ++c) items_v0.push_back({m, c});
        for (int c = 0; c < ceil_div(b.nc, 8); ++c) items_coarse.push_back({m, c});
        for (const void* p : {static_cast<const void*>(b.vin), static_cast<const void*>(b.vout),
                              static_cast<const void*>(b.pr), static_cast<const void*>(b.pd),
                              static_cast<const void*>(b.r), static_cast<const void*>(b.d),
                              static_cast<const void*>(b.q)})
            vec = vec && aligned16(p);
    }
    it_lv.clear();
    it_lv1.clear();
    it_lv.resize(max_L);
    it_lv1.resize(max_L);
    n_lv.assign(max_L, 0);
    n_lv1.assign(max_L, 0);
    for (int l = 0; l < max_L; ++l) {
        std::vector<int2> a, b1;
        for (int m = 0; m < nmem; ++m) {
            if (l >= hm[m].L) continue;
            for (int c = 0; c < ceil_div(hm[m].hn[l], kChunk); ++c) a.push_back({m, c});
            for (int c = 0; c < ceil_div(hm[m].hn[l + 1], kChunk); ++c) b1.push_back({m, c});
        }
        upload(it_lv[l], a, s);
        upload(it_lv1[l], b1, s);
        n_lv[l] = int(a.size());
        n_lv1[l] = int(b1.size());
    }
    upload(d_mem, hm, s);
    upload(it_u, items_u, s);
    upload(it_parts, items_parts, s);
    upload(it_q1, items_q1, s);
    upload(it_v0, items_v0, s);
    upload(it_coarse, items_coarse, s);
    n_u_items = int(items_u.size());
    n_parts = int(items_parts.size());
    n_q1 = int(items_q1.size());
    n_v0 = int(items_v0.size());
    n_coarse = int(items_coarse.size());
    d_state.alloc(size_t(nmem) * sizeof(BState));
    d_act.alloc(size_t(nmem) * sizeof(int));
    SIP_CUDA(cudaMemsetAsync(d_act.ptr, 0, size_t(nmem) * sizeof(int), s));
    d_partial.alloc(size_t(2) * nmem * kParts * sizeof(double));
    if (!pin) {
        if (cudaMallocHost(&pin, size_t(nmem) * sizeof(BState)) != cudaSuccess) {
            cudaGetLastError();
            pin = nullptr;
            throw Error(SIP_ERR_OOM, "pinned host allocation failed");
        }
    }
    // element kernels, per degree
    groups.clear();
    for (int N = 2; N <= 6; ++N) {
        std::vector<int> ms;
        for (int m = 0; m < nmem; ++m)
            if (probs[m]->n == N) ms.push_back(m);
        if (ms.empty()) continue;
        Group g;
        g.N = N;
        std::vector<StageArgs<T, T>> dec(nmem), res(nmem), r1(nmem);
        std::vector<StageArgs<T, double>> dech(nmem), resh(nmem), r1h(nmem);
        std::vector<StageArgs<double, double>> qa(nmem);
        std::vector<int2> lo, hi, all, bjit;
        const int nbj = steps_p + 1;
        std::vector<std::vector<BJBatchArgs<T>>> bjt(nbj, std::vector<BJBatchArgs<T>>(nmem));
        for (int m : ms) {
            sip_problem* P = probs[m];
            Multigrid<T>& G = mg(P);
            const BMember<T>& b = hm[m];
            const T* eta = sizeof(T) == 4 ? reinterpret_cast<const T*>(P->eta_f.ptr)
                                          : reinterpret_cast<const T*>(P->eta_d.ptr);
            const T* eta_inv = sizeof(T) == 4 ? reinterpret_cast<const T*>(P->eta_inv_f.ptr)
                                              : reinterpret_cast<const T*>(P->eta_inv_d.ptr);
            dec[m] = stage_args<T, T>(P->geom, b.pd, b.pr, eta, -1.0, b.pr, 1.0, nullptr, N);
            res[m] = stage_args<T, T>(P->geom, b.vout, b.pr, eta, -1.0, b.vin, 1.0, nullptr, N);
            r1[m] = stage_args<T, T>(P->geom, b.vout, nullptr, eta, -1.0, b.vin, 1.0, b.r1, N);
            if constexpr (sizeof(T) == 4) {
                dech[m] = stage_args<T, double>(P->geom, b.pd, b.pr, eta, -1.0, b.pr, 1.0, nullptr, N);
                resh[m] = stage_args<T, double>(P->geom, b.vout, b.pr, eta, -1.0, b.vin, 1.0, nullptr, N);
                r1h[m] = stage_args<T, double>(P->geom, b.vout, nullptr, eta, -1.0, b.vin, 1.0, b.r1, N);
            }
            qa[m] = stage_args<double, double>(P->geom, b.d, b.q, P->eta_d.template as<double>(), 1.0,
                                               nullptr, 0.0, nullptr, N);
            const int nt = split_tile_count(b.nx, b.ny);
            std::vector<unsigned char> flag(size_t(nt), 0);
            if (sizeof(T) == 4 && G.n_hi > 0) {
                SIP_CUDA(cudaMemcpyAsync(flag.data(), G.hi_flag.ptr, size_t(nt), cudaMemcpyDeviceToHost, s));
                SIP_CUDA(cudaStreamSynchronize(s));
            }
            for (int t = 0; t < nt; ++t) {
                (flag[t] ? hi : lo).push_back({m, t});
                all.push_back({m, t});
            }
            const int eb = bj_group(N);
            for (int c = 0; c < ceil_div(b.ne, eb); ++c) bjit.push_back({m, c});
            double c1[kMaxSt], c2[kMaxSt];
            cheb_coefs(P->desc.cheb_lo * G.lmax_p, P->desc.cheb_hi * G.lmax_p, steps_p, c1, c2);
            for (int k = 0; k < nbj; ++k) {
                const int st = k < 2 ? 0 : k - 1;
                BJBatchArgs<T>& a = bjt[k][m];
                a.ne = int(b.ne);
                a.r = b.pr;
                a.out = b.pd;
                a.x = b.vout;
                a.emap = G.emap.template as<int>();
                a.cls_inv = G.cls_inv.template as<T>();
                a.cls_sym = G.cls_sym.template as<int>();
                a.uniq_inv = G.uniq_inv.template as<T>();
                a.eta_inv = eta_inv;
                a.uniq_hi = G.bj_hi();
                a.uniq_inv64 = G.bj_inv64();
                a.c1 = T(c1[st]);
                a.c2 = T(c2[st]);
                a.x_zero = k == 0 ? 1 : 0;
            }
        }
        upload(g.a_dec, dec, s);
        upload(g.a_res, res, s);
        upload(g.a_r1, r1, s);
        upload(g.a_dec_hi, dech, s);
        upload(g.a_res_hi, resh, s);
        upload(g.a_r1_hi, r1h, s);
        upload(g.a_q, qa, s);
        upload(g.it_lo, lo, s);
        upload(g.it_hi, hi, s);
        upload(g.it_all, all, s);
        upload(g.it_bj, bjit, s);
        g.n_lo = int(lo.size());
        g.n_hi = int(hi.size());
        g.n_all = int(all.size());
        g.n_bj = int(bjit.size());
        g.bj.resize(nbj);
        for (int k = 0; k < nbj; ++k) upload(g.bj[k], bjt[k], s);
        groups.push_back(std::move(g));
    }
    SIP_CUDA(cudaStreamSynchronize(s));   // host staging vectors are released on return
}

template <typename T>
void BatchEngine<T>::capture_vcycle(cudaStream_t s) {
    const BMember<T>* mb = d_mem.template as<BMember<T>>();
    const int* act = d_act.template as<int>();
    const int2* iu = it_u.template as<int2>();
    auto apply = [&](int role) {   // 0: pr -= A pd, 1: pr = vin - A vout, 2: r1 = R(vin - A vout)
        for (Group& g : groups) {
            DeviceBuffer& lo = role == 0 ? g.a_dec : (role == 1 ? g.a_res : g.a_r1);
            DeviceBuffer& hi = role == 0 ? g.a_dec_hi : (role == 1 ? g.a_res_hi : g.a_r1_hi);
            launch_apply_stage_batch<T, T>(g.N, lo.template as<StageArgs<T, T>>(), g.it_lo.template as<int2>(),
                                           g.n_lo, act, vec, s);
            if constexpr (sizeof(T) == 4)
                launch_apply_stage_batch<T, double>(g.N, hi.template as<StageArgs<T, double>>(),
                                                    g.it_hi.template as<int2>(), g.n_hi, act, vec, s);
        }
    };
    auto bj = [&](int k) {
        for (Group& g : groups)
            launch_bj_apply_batch<T>(g.N, g.bj[k].template as<BJBatchArgs<T>>(), g.it_bj.template as<int2>(), g.n_bj,
                                     act, s);
    };
    auto smooth = [&](bool zero) {
        if (zero) {
            launch_k(k_b_copy<T>, dim3(unsigned(n_u_items)), kChunk, 0, s, mb, iu, act, int(V_IN),
                     int(V_PR));
            SIP_CHECK_LAUNCH();
            bj(0);
        } else {
            apply(1);
            bj(1);
        }
        for (int st = 1; st < steps_p; ++st) {
            apply(0);
            bj(1 + st);
        }
    };
    auto hsmooth = [&](int l, bool zero) {
        const dim3 grid = dim3(unsigned(n_lv[l]));
        if (zero)
            launch_k(k_b_hfirst<T>, grid, kChunk, 0, s, mb, it_lv[l].template as<int2>(), act, l);
        else
            launch_k(k_b_hstart<T>, grid, kChunk, 0, s, mb, it_lv[l].template as<int2>(), act, l);
        SIP_CHECK_LAUNCH();
        for (int st = 1; st < steps_h; ++st) {
            launch_k(k_b_hstep<T>, grid, kChunk, 0, s, mb, it_lv[l].template as<int2>(), act, l, st,
                     (!zero && st == 1) ? 1 : 0);
            SIP_CHECK_LAUNCH();
        }
    };
    // Algorithm 1: pre-smoothing from y = 0, restricted residual, coarse
    // correction through the continuous levels, prolongation, post-smoothing
    smooth(true);
    apply(2);
    launch_k(k_b_rdc<T>, dim3(unsigned(n_v0)), kChunk, 0, s, mb, it_v0.template as<int2>(), act);
    SIP_CHECK_LAUNCH();
    for (int l = 0; l < max_L; ++l) {   // members with l < L go one level down
        hsmooth(l, true);
        launch_k(k_b_hresid<T>, dim3(unsigned(n_lv[l])), kChunk, 0, s, mb, it_lv[l].template as<int2>(),
                 act, l);
        SIP_CHECK_LAUNCH();
        launch_k(k_b_rh<T>, dim3(unsigned(n_lv1[l])), kChunk, 0, s, mb, it_lv1[l].template as<int2>(),
                 act, l);
        SIP_CHECK_LAUNCH();
    }
    launch_k(k_b_coarse<T>, dim3(unsigned(n_coarse)), kChunk, 0, s, mb, it_coarse.template as<int2>(), act);
    SIP_CHECK_LAUNCH();
    for (int l = max_L - 1; l >= 0; --l) {
        launch_k(k_b_ph_add<T>, dim3(unsigned(n_lv[l])), kChunk, 0, s, mb, it_lv[l].template as<int2>(),
                 act, l);
        SIP_CHECK_LAUNCH();
        hsmooth(l, false);
    }
    launch_k(k_b_pcd<T>, dim3(unsigned(n_q1)), kChunk, 0, s, mb, it_q1.template as<int2>(), act);
    SIP_CHECK_LAUNCH();
    launch_k(k_b_prolong_add<T>, dim3(unsigned(n_q1)), kChunk, 0, s, mb, it_q1.template as<int2>(), act);
    SIP_CHECK_LAUNCH();
    smooth(false);
}

template <typename T>
void BatchEngine<T>::capture_body(cudaStream_t s, cudaGraphConditionalHandle h) {
    const BMember<T>* mb = d_mem.template as<BMember<T>>();
    BState* st = d_state.template as<BState>();
    int* act = d_act.template as<int>();
    double* part = d_partial.template as<double>();
    const int2* iu = it_u.template as<int2>();
    const int2* ip = it_parts.template as<int2>();
    const int fl = flexible ? 1 : 0;
    launch_k(k_b_r_to_vin<T>, dim3(unsigned(n_u_items)), kChunk, 0, s, mb, iu,
             static_cast<const int*>(act));
    SIP_CHECK_LAUNCH();
    capture_vcycle(s);
    launch_k(k_b_dot_z<T>, dim3(unsigned(n_parts)), kChunk, 0, s, mb, ip,
             static_cast<const int*>(act), fl, part);
    SIP_CHECK_LAUNCH();
    launch_k(k_b_beta_final, dim3(unsigned(nmem)), kChunk, 0, s, st, static_cast<const int*>(act),
             static_cast<const double*>(part), fl);
    SIP_CHECK_LAUNCH();
    launch_k(k_b_dir<T>, dim3(unsigned(n_u_items)), kChunk, 0, s, mb,
             static_cast<const BState*>(st), iu, static_cast<const int*>(act));
    SIP_CHECK_LAUNCH();
    for (Group& g : groups)
        launch_apply_stage_batch<double, double>(g.N, g.a_q.template as<StageArgs<double, double>>(),
                                                 g.it_all.template as<int2>(), g.n_all, act, vec, s);
    launch_k(k_b_dot_dq<T>, dim3(unsigned(n_parts)), kChunk, 0, s, mb, ip,
             static_cast<const int*>(act), nmem, fl, part);
    SIP_CHECK_LAUNCH();
    launch_k(k_b_alpha_final, dim3(unsigned(nmem)), kChunk, 0, s, st, static_cast<const int*>(act),
             static_cast<const double*>(part), nmem, fl);
    SIP_CHECK_LAUNCH();
    launch_k(k_b_update<T>, dim3(unsigned(n_parts)), kChunk, 0, s, mb,
             static_cast<const BState*>(st), ip, static_cast<const int*>(act), part);
    SIP_CHECK_LAUNCH();
    launch_k(k_b_ctl_final, dim3(unsigned(nmem)), kChunk, 0, s, st, act,
             static_cast<const double*>(part), rtol, maxit);
    SIP_CHECK_LAUNCH();
    launch_k(k_b_any, 1, 256, 0, s, static_cast<const int*>(act), nmem, h);
    SIP_CHECK_LAUNCH();
}

template <typename T>
void BatchEngine<T>::round(const std::vector<const double*>& t, const std::vector<double*>& y,
                           const std::vector<int>& want, std::vector<int>& its) {
    PdlOffScope pdl_off;   // plain launches inside the conditional graph
    if (!cs) SIP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    if (!exec) {
        SIP_CUDA(cudaStreamSynchronize(cs));
        const int64_t before = launch_counter();
        cudaGraph_t g = nullptr;
        SIP_CUDA(cudaGraphCreate(&g, 0));
        graph = g;
        cudaGraphConditionalHandle h;
        SIP_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
        SIP_CUDA(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        try {
            launch_k(k_b_init<T>, dim3(unsigned(n_parts)), kChunk, 0, cs,
                     static_cast<const BMember<T>*>(d_mem.template as<BMember<T>>()),
                     static_cast<const BState*>(d_state.template as<BState>()),
                     static_cast<const int2*>(it_parts.template as<int2>()), d_partial.template as<double>());
            SIP_CHECK_LAUNCH();
            launch_k(k_b_init_final, dim3(unsigned(nmem)), kChunk, 0, cs, d_state.template as<BState>(),
                     d_act.template as<int>(), static_cast<const double*>(d_partial.template as<double>()));
            SIP_CHECK_LAUNCH();
            launch_k(k_b_any, 1, 256, 0, cs, static_cast<const int*>(d_act.template as<int>()), nmem, h);
            SIP_CHECK_LAUNCH();
        } catch (const Error&) {
            e = cudaErrorUnknown;
        }
        top_kernels = launch_counter() - before;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t nloop = nullptr;
        if (e == cudaSuccess) {
            cudaStreamCaptureStatus cst;
            const cudaGraphNode_t* deps = nullptr;
            size_t ndeps = 0;
            e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
            if (e == cudaSuccess) e = cudaGraphAddNode(&nloop, g, deps, nullptr, ndeps, &cp);
            if (e == cudaSuccess)
                e = cudaStreamUpdateCaptureDependencies(cs, &nloop, nullptr, 1,
                                                        cudaStreamSetCaptureDependencies);
        }
        cudaGraph_t gout = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(cs, &gout);
        SIP_CUDA(e);
        SIP_CUDA(ee);
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        SIP_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
        const int64_t b0 = launch_counter();
        try {
            capture_body(cs, h);
        } catch (...) {
            cudaGraph_t tmp;
            cudaStreamEndCapture(cs, &tmp);
            launch_counter() = before;
            throw;
        }
        body_kernels = launch_counter() - b0;
        cudaGraph_t body_out;
        SIP_CUDA(cudaStreamEndCapture(cs, &body_out));
        launch_counter() = before;
        SIP_CUDA(cudaGraphInstantiate(&exec, g, 0));
    }
    for (int m = 0; m < nmem; ++m) {
        pin[m] = BState{};
        pin[m].t = t[m];
        pin[m].y = y[m];
        pin[m].want = want[m];
    }
    SIP_CUDA(cudaMemcpyAsync(d_state.ptr, pin, size_t(nmem) * sizeof(BState), cudaMemcpyHostToDevice, cs));
    SIP_CUDA(cudaGraphLaunch(exec, cs));
    SIP_CUDA(cudaMemcpyAsync(pin, d_state.ptr, size_t(nmem) * sizeof(BState), cudaMemcpyDeviceToHost, cs));
    SIP_CUDA(cudaStreamSynchronize(cs));
    its.assign(nmem, 0);
    int passes = 0;
    for (int m = 0; m < nmem; ++m) {
        its[m] = pin[m].status != 0 ? -1 : pin[m].it;
        passes = std::max(passes, pin[m].it);
    }
    launch_counter() += top_kernels + body_kernels * passes;
}

template struct BatchEngine<float>;
template struct BatchEngine<double>;

// ---------------------------------------------------------------- rendezvous
struct BatchCollector {
    std::mutex mu;
    std::condition_variable cv;
    std::vector<sip_problem*> probs;
    std::vector<int> index_of_thread;
    int registered = 0;   // members still solving
    int waiting = 0;
    int64_t round_no = 0;
    bool launching = false;
    bool mixed = false;
    double rtol = 0.0;
    int maxit = 0;
    std::vector<const double*> t;
    std::vector<double*> y;
    std::vector<int> want, its;
    std::string err;
    sip_status err_st = SIP_OK;
    std::unique_ptr<BatchEngine<float>> e32;
    std::unique_ptr<BatchEngine<double>> e64;

    int inner(sip_problem* P, const double* tt, double* yy, cudaStream_t s);
    void leave(sip_problem* P);
    void launch_round();   // called with mu held by the last arriving thread
};

BatchCollector*& batch_collector() {
    static thread_local BatchCollector* c = nullptr;
    return c;
}

namespace {
int member_index(const BatchCollector& c, const sip_problem* P) {
    for (size_t i = 0; i < c.probs.size(); ++i)
        if (c.probs[i] == P) return int(i);
    return -1;
}
}  // namespace

void BatchCollector::launch_round() {
    launching = true;
    std::vector<int> out;
    try {
        const cudaStream_t s0 = nullptr;
        (void)s0;
        if (mixed) {
            if (!e32) {
                e32 = std::make_unique<BatchEngine<float>>();
                e32->probs = probs;
                e32->flexible = true;
                e32->rtol = rtol;
                e32->maxit = maxit;
                e32->steps_p = probs[0]->desc.cheb_steps_p;
                e32->steps_h = probs[0]->desc.cheb_steps_h;
                cudaStream_t bs;
                SIP_CUDA(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
                e32->cs = bs;
                e32->build(bs);
            }
            e32->round(t, y, want, out);
        } else {
            if (!e64) {
                e64 = std::make_unique<BatchEngine<double>>();
                e64->probs = probs;
                e64->flexible = false;
                e64->rtol = rtol;
                e64->maxit = maxit;
                e64->steps_p = probs[0]->desc.cheb_steps_p;
                e64->steps_h = probs[0]->desc.cheb_steps_h;
                cudaStream_t bs;
                SIP_CUDA(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
                e64->cs = bs;
                e64->build(bs);
            }
            e64->round(t, y, want, out);
        }
    } catch (const Error& e) {
        err = e.what();
        err_st = e.status;
        out.assign(probs.size(), -2);
    } catch (const std::exception& e) {
        err = e.what();
        err_st = SIP_ERR_CUDA;
        out.assign(probs.size(), -2);
    }
    its = out;
    std::fill(want.begin(), want.end(), 0);
    waiting = 0;
    ++round_no;
    launching = false;
    cv.notify_all();
}

int BatchCollector::inner(sip_problem* P, const double* tt, double* yy, cudaStream_t s) {
    SIP_CUDA(cudaStreamSynchronize(s));   // t is ready; y may be written by the batch
    std::unique_lock<std::mutex> lk(mu);
    const int m = member_index(*this, P);
    require(m >= 0, "batched inner solve: unknown problem");
    t[m] = tt;
    y[m] = yy;
    want[m] = 1;
    ++waiting;
    const int64_t my_round = round_no;
    if (waiting == registered) {
        launch_round();
    } else {
        cv.wait(lk, [&] { return round_no != my_round; });
    }
    const int it = its[m];
    if (it == -2) throw Error(err_st, err);
    if (it < 0) throw Error(SIP_ERR_BREAKDOWN, "non-finite inner residual");
    return it;
}

void BatchCollector::leave(sip_problem* P) {
    (void)P;
    std::unique_lock<std::mutex> lk(mu);
    --registered;
    if (waiting > 0 && waiting == registered && !launching) launch_round();
}

// inner solve through the group's rendezvous when this thread is a member of
// a batched group (sets *used), else nothing
int batched_inner(sip_problem* P, const double* t, double* y, cudaStream_t s, bool* used) {
    BatchCollector* c = batch_collector();
    *used = c != nullptr;
    if (!c) return 0;
    return c->inner(P, t, y, s);
}

BatchCollector* make_collector(const std::vector<sip_problem*>& probs, bool mixed, double rtol,
                               int maxit) {
    auto* c = new BatchCollector();
    c->probs = probs;
    c->registered = int(probs.size());
    c->mixed = mixed;
    c->rtol = rtol;
    c->maxit = std::max(1, std::min(maxit, 100000));
    c->t.assign(probs.size(), nullptr);
    c->y.assign(probs.size(), nullptr);
    c->want.assign(probs.size(), 0);
    c->its.assign(probs.size(), 0);
    return c;
}

void free_collector(BatchCollector* c) { delete c; }
void collector_leave(BatchCollector* c, sip_problem* P) { c->leave(P); }
int64_t collector_rounds(const BatchCollector* c) { return c->round_no; }

}  // namespace sip
