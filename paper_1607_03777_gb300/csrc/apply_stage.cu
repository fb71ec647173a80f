// Staged-tile SIP apply (eq. stiffness_form) for the memory-bound
// precisions, and the split-precision form of the FP32 operator.
//
// Same operator and the same component-split thread roles as k_apply_elem2
// (warps 2r and 2r+1 serve the two velocity components of the 32 elements of
// tile row r), with a different data path.  The element blocks of a tile of
// STX x TYS elements, the left and right neighbours of each tile row and the
// tile rows below and above are first copied into shared memory: one tile row
// with its two neighbours is one contiguous span of x, which the whole CTA
// reads with consecutive 16-byte loads (every sector fully used) and scatters
// into a padded layout (odd element stride: lane-per-element reads are free
// of bank conflicts).  The viscosities of the same elements are staged beside
// them.  Traces and volume terms are then computed from shared memory; the
// output blocks are gathered in shared memory and written back as consecutive
// 16-byte stores, the beta z term read the same way.  Global traffic is the
// algorithmic one plus the re-reads of the halo rows, which L2 serves.
//
// Storage and arithmetic precision are separate template parameters (TS,
// TC).  The mixed-precision V-cycle keeps its vectors in FP32 but must not
// evaluate the operator in FP32 where the viscosity is far above the
// smallest one: there, a nearly rigid motion of a stiff inclusion (large
// coefficients, eta_K times a small strain) is cancelled in the volume and
// penalty terms, and FP32 rounding of that cancellation (eps_32 eta_K |u|)
// swamps the residual of the soft medium.  Such tiles (any element of the
// tile or its halo with eta >= ratio x min eta) are listed at set-up and
// evaluated by a second launch in FP64 arithmetic on the same FP32 data
// (rounding the inputs to FP32 is harmless; only the cancellation is not);
// the FP32 launch skips them.
#include "sip_elem.cuh"
#include "sip_face.cuh"
#include "sip_internal.h"

namespace sip {

namespace {

constexpr int STX = 32;      // elements per tile row
constexpr int SPLIT_TYS = 2; // tile rows of the split-precision launches
static_assert(STX == 32 && SPLIT_TYS == 2,
              "the warp-row kernel reads the split-precision flags of 32 x 2 tiles");
constexpr size_t kMaxSmem = 227 * 1024;   // dynamic shared memory of one CTA

template <int N, typename TS, typename TC, int TYS>
struct StageLayout {
    static constexpr int NB = 2 * N * N;
    static constexpr int XS = NB + 1;       // odd element stride (NB is even)
    static constexpr int XW = STX + 2;      // staged elements per row
    static constexpr int XH = TYS + 2;      // staged rows
    static constexpr int NT = 64 * TYS;     // two warps per tile row
    static constexpr int NHALO = 2 * STX + 2 * TYS;
    static constexpr int TRW = 16 * N + 1;  // own traces of one element, all four faces
    static constexpr int HW = 4 * N + 1;    // the one face of a halo element
    // Region 0 holds in turn the staged input blocks, the own traces and the
    // output blocks (each phase ends at a barrier with its data read or in
    // registers): one region instead of three, so more CTAs fit an SM.
    static constexpr size_t X_BYTES = size_t(XH) * XW * XS * sizeof(TS);
    static constexpr size_t TR_BYTES = size_t(STX) * TYS * TRW * sizeof(TC);
    static constexpr size_t OUT_BYTES = size_t(TYS) * STX * XS * sizeof(TC);
    static constexpr size_t R0_BYTES =
        X_BYTES > TR_BYTES ? (X_BYTES > OUT_BYTES ? X_BYTES : OUT_BYTES)
                           : (TR_BYTES > OUT_BYTES ? TR_BYTES : OUT_BYTES);
    static constexpr size_t ETA_OFF = (R0_BYTES + 15) / 16 * 16;
    static constexpr size_t H_OFF = ETA_OFF + (size_t(XH) * XW * sizeof(TC) + 15) / 16 * 16;
    static constexpr size_t BYTES = H_OFF + size_t(NHALO) * HW * sizeof(TC);
    // CTAs per SM asked of the register allocator: as many as the shared
    // memory admits (1 KB reserved per CTA), unless that leaves a thread
    // fewer registers than the element's arrays need without spilling
    static constexpr int REG_FLOOR =
        sizeof(TC) == 8 ? (N <= 4 ? 128 : (N == 5 ? 168 : 255)) : (N <= 5 ? 80 : 128);
    static constexpr int SMEM_FIT = int((228 * 1024) / (BYTES + 1024));
    static constexpr int REG_FIT = 65536 / (NT * REG_FLOOR);
    static constexpr int MIN_BLOCKS =
        (SMEM_FIT < REG_FIT ? SMEM_FIT : REG_FIT) > 1 ? (SMEM_FIT < REG_FIT ? SMEM_FIT : REG_FIT)
                                                      : 1;
};

// Copy the tile's staged element blocks and viscosities into shared memory.
// Stage row r is mesh row ey0 - 1 + r, stage column c mesh column ex0 - 1 + c.
// The first and last stage rows hold only the STX elements below / above the
// tile (their face traces are all that is needed); corners and elements
// outside the mesh stay unset and are never read.
template <int N, typename TS, typename TC, int TYS, bool VEC>
__device__ __forceinline__ void stage_tile(const StageArgs<TS, TC>& a, int ex0, int ey0, TS* sx,
                                           TC* seta) {
    using L = StageLayout<N, TS, TC, TYS>;
    constexpr int NB = L::NB;
    const int nx = a.c.nx, ny = a.c.ny;
    for (int q = threadIdx.x; q < L::XH * L::XW; q += L::NT) {
        const int r = q / L::XW, c = q % L::XW;
        const int ey = ey0 - 1 + r, ex = ex0 - 1 + c;
        seta[q] = (ey >= 0 && ey < ny && ex >= 0 && ex < nx) ? TC(a.eta[size_t(ey) * nx + ex])
                                                             : TC(0);
    }
    constexpr int V = VEC ? 16 / int(sizeof(TS)) : 1;
    constexpr int CPR = (L::XW * NB + V - 1) / V + 1;   // chunks per stage row (bound)
    constexpr int QT = L::XH * CPR;
    constexpr int BATCH = 8;                             // loads in flight per thread
#pragma unroll 1
    for (int q0 = 0; q0 < QT; q0 += BATCH * L::NT) {
        TS v[BATCH][V];
        // per chunk: its first entry and the staged row's valid range, as
        // offsets from the row's stage origin (element ex0 - 1): 32-bit
        int rel0[BATCH], rlo[BATCH], rhi[BATCH], srow[BATCH];
        bool ok[BATCH];
#pragma unroll
        for (int b = 0; b < BATCH; ++b) {
            const int q = q0 + b * L::NT + int(threadIdx.x);
            const int r = q / CPR, c = q % CPR;
            const int ey = ey0 - 1 + r;
            ok[b] = false;
            rel0[b] = rlo[b] = rhi[b] = srow[b] = 0;
            long long gfirst = 0;
            if (q < QT && ey >= 0 && ey < ny) {
                const bool edge = r == 0 || r == L::XH - 1;
                const int elo = edge ? ex0 : max(ex0 - 1, 0);
                const int ehi = edge ? min(ex0 + STX, nx) : min(ex0 + STX + 1, nx);
                const long long row = (long long)ey * nx;
                const long long gbase = (row + ex0 - 1) * NB;
                const long long glo = (row + elo) * NB;
                gfirst = (glo / V + c) * V;
                rel0[b] = int(gfirst - gbase);
                rlo[b] = (elo - (ex0 - 1)) * NB;
                rhi[b] = (ehi - (ex0 - 1)) * NB;
                srow[b] = r;
                ok[b] = elo < ehi && rel0[b] < rhi[b];
            }
            if (!ok[b]) continue;
            if constexpr (VEC) {
                if (gfirst + V <= a.n_total) {
                    using VV = Vec16<TS>;
                    const typename VV::type w =
                        __ldg(reinterpret_cast<const typename VV::type*>(a.x + gfirst));
#pragma unroll
                    for (int t = 0; t < V; ++t) v[b][t] = VV::get(w, t);
                    continue;
                }
            }
#pragma unroll
            for (int t = 0; t < V; ++t) v[b][t] = gfirst + t < a.n_total ? a.x[gfirst + t] : TS(0);
        }
#pragma unroll
        for (int b = 0; b < BATCH; ++b) {
            if (!ok[b]) continue;
            TS* row = sx + srow[b] * L::XW * L::XS;
#pragma unroll
            for (int t = 0; t < V; ++t) {
                const int rel = rel0[b] + t;
                if (rel >= rlo[b] && rel < rhi[b]) {
                    const int el = rel / NB;   // rel >= 0 here
                    row[el * L::XS + (rel - el * NB)] = v[b][t];
                }
            }
        }
    }
}

// Phase B of component C on the staged tile: face vectors from own and
// neighbour traces (neighbour viscosities from the stage), spread into y_C;
// with a.r1, alpha y + beta z of its Q^2_1 modes go straight to r1.
template <int N, typename TS, typename TC, int C, int TYS>
__device__ __forceinline__ void stage_phase_b(const StageArgs<TS, TC>& a, int ex, int ey, int tx,
                                              int ty, TC etaK, const TC* seta, const TC* s_tr,
                                              const TC* s_halo, TC (&y)[N][N]) {
    using L = StageLayout<N, TS, TC, TYS>;
    constexpr int NB = L::NB;
    const int nx = a.c.nx, ny = a.c.ny;
    const int el = ty * STX + tx;
    TC Dm[N * N];
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
        for (int q = 0; q < N; ++q) Dm[p * N + q] = TC(kT<N>.D[p][q]);
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
        TC P[2][N], Q[2][N];   // [face lo/hi][m]
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int F = 2 * dir + side;
            const TC* own = s_tr + el * L::TRW + F * 4 * N;
            const TC* nbr = own;
            TC etaN = TC(0);
            int kind;
            const bool has_nbr = dir == 0 ? (side == 0 ? ex > 0 : ex < nx - 1)
                                          : (side == 0 ? ey > 0 : ey < ny - 1);
            if (has_nbr) {
                kind = 0;
                const int ltx = tx + (dir == 0 ? (side == 0 ? -1 : 1) : 0);
                const int lty = ty + (dir == 1 ? (side == 0 ? -1 : 1) : 0);
                etaN = seta[(lty + 1) * L::XW + ltx + 1];
                if (ltx >= 0 && ltx < STX && lty >= 0 && lty < TYS)
                    nbr = s_tr + (lty * STX + ltx) * L::TRW + (F ^ 1) * 4 * N;
                else if (dir == 1)
                    nbr = s_halo + ((side == 0 ? 0 : STX) + tx) * L::HW;
                else
                    nbr = s_halo + (2 * STX + (side == 0 ? 0 : TYS) + ty) * L::HW;
            } else {
                kind = 1 + a.c.bc[F];
            }
            const TC eta_e = kind == 0 ? (etaK > etaN ? etaK : etaN) : etaK;
            const TC pen = dir == 0 ? a.c.pen_x : a.c.pen_y;
            const TC sigma = pen * eta_e * (kind == 0 ? TC(1) : TC(2));
            const TC s = side == 0 ? TC(-1) : TC(1);
            const FaceGeo<TC>& fg = dir == 0 ? a.c.fgx : a.c.fgy;
            if (kind == 0) {
                face_interior_comp<N, TC, C>(dir, side, fg, pen, etaK, etaN, own, nbr, P[side],
                                             Q[side]);
            } else {
#pragma unroll
                for (int m = 0; m < N; ++m)
                    face_pq<N, TC>(kind, C, m, dir, s, fg, etaK, etaN, sigma, own, own + 2 * N,
                                   nbr, nbr + 2 * N, Dm, P[side][m], Q[side][m]);
            }
        }
        spread_faces<N, TC>(dir, P, Q, y);
    }
    if (a.r1) {   // residual restricted to the Q^2_1 modes (p-transfer R = P^T)
        const TS* zz = a.z ? a.z + (size_t(ey) * nx + ex) * NB + C * N * N : nullptr;
        TS* d1 = a.r1 + (size_t(ey) * nx + ex) * 8 + C * 4;
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                TC v = a.c.alpha * y[j][i];
                if (zz) v += a.c.beta * TC(zz[j * N + i]);
                d1[j * 2 + i] = TS(v);
            }
    }
}

// Write the tile's output blocks from shared memory: y = alpha (A x) + beta z
// over each tile row's contiguous span; 16-byte accesses inside the span,
// single words where a vector would reach into a neighbouring tile's span.
template <int N, typename TS, typename TC, int TYS, bool VEC>
__device__ __forceinline__ void stage_store(const StageArgs<TS, TC>& a, int ex0, int ey0,
                                            const TC* sy) {
    using L = StageLayout<N, TS, TC, TYS>;
    constexpr int NB = L::NB;
    constexpr int V = VEC ? 16 / int(sizeof(TS)) : 1;
    constexpr int CPR = (STX * NB + V - 1) / V + 1;
    constexpr int QT = TYS * CPR;
    const int nx = a.c.nx, ny = a.c.ny;
    const int ehi = min(ex0 + STX, nx);
    const TC alpha = a.c.alpha, beta = a.c.beta;
    for (int q = threadIdx.x; q < QT; q += L::NT) {
        const int r = q / CPR, c = q % CPR;
        const int ey = ey0 + r;
        if (ey >= ny) continue;
        const long long g0 = ((long long)ey * nx + ex0) * NB;
        const int span = (ehi - ex0) * NB;            // entries of this tile row
        const long long gf = (g0 / V + c) * V;
        const int rel0 = int(gf - g0);                 // may be negative (before the span)
        if (rel0 >= span) continue;
        const TC* srow = sy + r * STX * L::XS;
        if constexpr (VEC) {
            if (rel0 >= 0 && rel0 + V <= span) {
                using VV = Vec16<TS>;
                TS w[V];
                if (a.z) {
                    const typename VV::type zv =
                        __ldg(reinterpret_cast<const typename VV::type*>(a.z + gf));
#pragma unroll
                    for (int t = 0; t < V; ++t) {
                        const int rel = rel0 + t, el = rel / NB;
                        w[t] = TS(alpha * srow[el * L::XS + (rel - el * NB)] +
                                  beta * TC(VV::get(zv, t)));
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < V; ++t) {
                        const int rel = rel0 + t, el = rel / NB;
                        w[t] = TS(alpha * srow[el * L::XS + (rel - el * NB)]);
                    }
                }
                *reinterpret_cast<typename VV::type*>(a.y + gf) = VV::make(w);
                continue;
            }
        }
#pragma unroll
        for (int t = 0; t < V; ++t) {
            const int rel = rel0 + t;
            if (rel < 0 || rel >= span) continue;
            const int el = rel / NB;
            TC w = alpha * srow[el * L::XS + (rel - el * NB)];
            if (a.z) w += beta * TC(a.z[gf + t]);
            a.y[gf + t] = TS(w);
        }
    }
}

// The whole apply of tile (bx, by) by one CTA.
template <int N, typename TS, typename TC, int TYS, bool VEC>
__device__ __forceinline__ void stage_body(const StageArgs<TS, TC>& a, int bx, int by) {
    using L = StageLayout<N, TS, TC, TYS>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TS* sx = reinterpret_cast<TS*>(smem_raw);       // region 0: staged inputs,
    TC* s_tr = reinterpret_cast<TC*>(smem_raw);     // then own traces,
    TC* sy = reinterpret_cast<TC*>(smem_raw);       // then output blocks
    TC* seta = reinterpret_cast<TC*>(smem_raw + L::ETA_OFF);
    TC* s_halo = reinterpret_cast<TC*>(smem_raw + L::H_OFF);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int ty = warp / 2, c = warp % 2, tx = lane;
    const int ex0 = bx * STX, ey0 = by * TYS;
    const int ex = ex0 + tx, ey = ey0 + ty;
    const int nx = a.c.nx, ny = a.c.ny;
    const bool active = ex < nx && ey < ny;
    stage_tile<N, TS, TC, TYS, VEC>(a, ex0, ey0, sx, seta);
    __syncthreads();
    // halo traces: the face of each outside neighbour that touches the tile
    for (int h = threadIdx.x; h < L::NHALO; h += L::NT) {
        int lx, ly, F;
        if (h < STX) { lx = h + 1; ly = 0; F = 3; }                              // below: its top
        else if (h < 2 * STX) { lx = h - STX + 1; ly = L::XH - 1; F = 2; }       // above: its bottom
        else if (h < 2 * STX + TYS) { lx = 0; ly = h - 2 * STX + 1; F = 1; }     // left: its right
        else { lx = L::XW - 1; ly = h - 2 * STX - TYS + 1; F = 0; }              // right: its left
        const int hx = ex0 - 1 + lx, hy = ey0 - 1 + ly;
        if (hx >= 0 && hx < nx && hy >= 0 && hy < ny) {
            TC uh[2][N][N];
            const TS* src = sx + (ly * L::XW + lx) * L::XS;
#pragma unroll
            for (int cc = 0; cc < 2; ++cc)
#pragma unroll
                for (int j = 0; j < N; ++j)
#pragma unroll
                    for (int i = 0; i < N; ++i) uh[cc][j][i] = TC(src[cc * N * N + j * N + i]);
            face_traces<N, TC>(uh, F, F < 2 ? a.c.two_over_hx : a.c.two_over_hy,
                               s_halo + h * L::HW);
        }
    }
    TC u[2][N][N];
    TC etaK = TC(0);
    if (active) {
        const TS* src = sx + ((ty + 1) * L::XW + tx + 1) * L::XS;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc)
#pragma unroll
            for (int j = 0; j < N; ++j)
#pragma unroll
                for (int i = 0; i < N; ++i) u[cc][j][i] = TC(src[cc * N * N + j * N + i]);
        etaK = seta[(ty + 1) * L::XW + tx + 1];
    }
    __syncthreads();   // staged blocks read: region 0 takes the traces
    TC y[N][N];
    if (active) {
        TC* tr = s_tr + (ty * STX + tx) * L::TRW;
        if (c == 0)
            elem2_phase_a<N, TC, 0>(a.c, u, etaK, tr, y);
        else
            elem2_phase_a<N, TC, 1>(a.c, u, etaK, tr, y);
    }
    __syncthreads();
    if (active) {
        if (c == 0)
            stage_phase_b<N, TS, TC, 0, TYS>(a, ex, ey, tx, ty, etaK, seta, s_tr, s_halo, y);
        else
            stage_phase_b<N, TS, TC, 1, TYS>(a, ex, ey, tx, ty, etaK, seta, s_tr, s_halo, y);
    }
    if (a.r1) return;
    __syncthreads();   // traces read: region 0 takes the output blocks
    if (active) {
        TC* dst = sy + (ty * STX + tx) * L::XS + c * N * N;
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
            for (int i = 0; i < N; ++i) dst[j * N + i] = y[j][i];
    }
    __syncthreads();
    stage_store<N, TS, TC, TYS, VEC>(a, ex0, ey0, sy);
}

// One CTA per tile: a 2D grid over the mesh (tiles flagged in skip exit at
// once), or (LIST) a 1D grid over the tile ids in a.tiles.
template <int N, typename TS, typename TC, int TYS, bool VEC, bool LIST>
__global__ void __launch_bounds__(64 * TYS, (StageLayout<N, TS, TC, TYS>::MIN_BLOCKS))
    k_apply_stage(const StageArgs<TS, TC> a) {
    grid_dep_wait();
    int bx, by;
    if constexpr (LIST) {
        const int t = a.tiles[blockIdx.x];
        bx = t % a.ntx;
        by = t / a.ntx;
    } else {
        bx = blockIdx.x;
        by = blockIdx.y;
        if (a.skip && a.skip[size_t(by) * a.ntx + bx]) return;   // uniform over the CTA
    }
    stage_body<N, TS, TC, TYS, VEC>(a, bx, by);
}

// Many operators in one launch: CTA b applies the operator of member
// items[b].x (arguments args[items[b].x]) on its tile items[b].y (split
// tile numbering); members with active[m] == 0 are skipped.
template <int N, typename TS, typename TC, bool VEC>
__global__ void __launch_bounds__(64 * SPLIT_TYS, (StageLayout<N, TS, TC, SPLIT_TYS>::MIN_BLOCKS))
    k_apply_stage_batch(const StageArgs<TS, TC>* __restrict__ args, const int2* __restrict__ items,
                        const int* __restrict__ active) {
    grid_dep_wait();
    const int2 it = items[blockIdx.x];
    if (active && !active[it.x]) return;
    const StageArgs<TS, TC>& a = args[it.x];
    stage_body<N, TS, TC, SPLIT_TYS, VEC>(a, it.y % a.ntx, it.y / a.ntx);
}

template <int N, typename TS, typename TC>
void stage_batch_n(const StageArgs<TS, TC>* args, const int2* items, int n_items,
                   const int* active, bool vec, cudaStream_t s) {
    const size_t smem = StageLayout<N, TS, TC, SPLIT_TYS>::BYTES;
    static const bool attr = [smem] {   // once per process, thread-safe
        SIP_CUDA(cudaFuncSetAttribute(k_apply_stage_batch<N, TS, TC, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        SIP_CUDA(cudaFuncSetAttribute(k_apply_stage_batch<N, TS, TC, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        return true;
    }();
    (void)attr;
    if (vec)
        launch_k(k_apply_stage_batch<N, TS, TC, true>, dim3(unsigned(n_items)), 64 * SPLIT_TYS,
                 smem, s, args, items, active);
    else
        launch_k(k_apply_stage_batch<N, TS, TC, false>, dim3(unsigned(n_items)), 64 * SPLIT_TYS,
                 smem, s, args, items, active);
    SIP_CHECK_LAUNCH();
}

template <typename TS, typename TC>
StageArgs<TS, TC> make_stage_args(const OpGeom& g, const TS* x, TS* y, const TS* eta, double alpha,
                                  const TS* z, double beta, TS* r1, int N, int tys) {
    StageArgs<TS, TC> a;
    a.c = make_elem_args<TC>(g, nullptr, nullptr, nullptr, TC(alpha), nullptr, TC(beta));
    a.x = x;
    a.y = y;
    a.eta = eta;
    a.z = z;
    a.r1 = r1;
    a.skip = nullptr;
    a.tiles = nullptr;
    a.ntx = (g.nx + STX - 1) / STX;
    (void)tys;
    a.n_total = (long long)g.nx * g.ny * 2 * N * N;
    return a;
}

template <int N, typename TS, typename TC, int TYS, bool LIST>
void launch_stage(const StageArgs<TS, TC>& a, dim3 grid, bool vec, cudaStream_t s) {
    const size_t smem = StageLayout<N, TS, TC, TYS>::BYTES;
    static const bool attr = [smem] {   // once per process, thread-safe
        SIP_CUDA(cudaFuncSetAttribute(k_apply_stage<N, TS, TC, TYS, false, LIST>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        SIP_CUDA(cudaFuncSetAttribute(k_apply_stage<N, TS, TC, TYS, true, LIST>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        return true;
    }();
    (void)attr;
    if (vec)
        launch_k(k_apply_stage<N, TS, TC, TYS, true, LIST>, grid, 64 * TYS, smem, s, a);
    else
        launch_k(k_apply_stage<N, TS, TC, TYS, false, LIST>, grid, 64 * TYS, smem, s, a);
    SIP_CHECK_LAUNCH();
}

inline bool vec_aligned(const void* x, const void* y, const void* z) {
    return aligned16(x) && (y == nullptr || aligned16(y)) && (z == nullptr || aligned16(z));
}

// Plain staged apply in one precision (TYS tile rows).
template <int N, typename T, int TYS>
void stage_plain(const OpGeom& g, const T* x, T* y, const T* eta, T alpha, const T* z, T beta,
                 T* r1, cudaStream_t s) {
    const StageArgs<T, T> a = make_stage_args<T, T>(g, x, y, eta, alpha, z, beta, r1, N, TYS);
    const dim3 grid((g.nx + STX - 1) / STX, (g.ny + TYS - 1) / TYS);
    launch_stage<N, T, T, TYS, false>(a, grid, vec_aligned(x, y, z), s);
}

// A second stream of this host thread on the current device, with a fork
// and a join event: the two launches of the split-precision apply write
// disjoint tiles and run side by side (in a captured graph: two parallel
// kernel nodes).
struct ForkStream {
    int dev = -1;
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    void release() {
        if (s) cudaStreamDestroy(s);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        s = nullptr;
        fork = join = nullptr;
    }
    ~ForkStream() { release(); }   // errors at process teardown are ignored
};

ForkStream& fork_stream() {
    thread_local ForkStream f;
    int dev = 0;
    SIP_CUDA(cudaGetDevice(&dev));
    if (f.dev != dev || !f.s) {
        f.release();
        SIP_CUDA(cudaStreamCreateWithFlags(&f.s, cudaStreamNonBlocking));
        SIP_CUDA(cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming));
        SIP_CUDA(cudaEventCreateWithFlags(&f.join, cudaEventDisableTiming));
        f.dev = dev;
    }
    return f;
}

// Split-precision FP32 apply: FP32 arithmetic on the tiles not flagged in
// g.hi_flag, FP64 arithmetic on the g.n_hi tiles of g.hi_tiles.  The FP64
// launch has few CTAs and runs at the FP64 pipe's rate; the FP32 launch
// fills the SMs beside it on a second stream.
template <int N>
void stage_split(const OpGeom& g, const float* x, float* y, const float* eta, float alpha,
                 const float* z, float beta, float* r1, cudaStream_t s) {
    const bool vec = vec_aligned(x, y, z);
    ForkStream& f = fork_stream();
    StageArgs<float, double> hi =
        make_stage_args<float, double>(g, x, y, eta, alpha, z, beta, r1, N, SPLIT_TYS);
    hi.tiles = g.hi_tiles;
    SIP_CUDA(cudaEventRecord(f.fork, s));
    SIP_CUDA(cudaStreamWaitEvent(f.s, f.fork, 0));
    launch_stage<N, float, double, SPLIT_TYS, true>(hi, dim3(unsigned(g.n_hi)), vec, f.s);
    SIP_CUDA(cudaEventRecord(f.join, f.s));
    // the unflagged tiles: the warp-row kernel (y = alpha A x + beta z), else
    // (residual restricted to the Q^2_1 modes) the staged kernel
    if (r1 || !launch_apply_sip_warp(N, g, x, y, eta, alpha, z, beta, g.hi_flag, s)) {
        StageArgs<float, float> lo =
            make_stage_args<float, float>(g, x, y, eta, alpha, z, beta, r1, N, SPLIT_TYS);
        lo.skip = g.hi_flag;
        const dim3 grid((g.nx + STX - 1) / STX, (g.ny + SPLIT_TYS - 1) / SPLIT_TYS);
        launch_stage<N, float, float, SPLIT_TYS, false>(lo, grid, vec, s);
    }
    SIP_CUDA(cudaStreamWaitEvent(s, f.join, 0));
}

template <int N, typename T>
void stage_dispatch(const OpGeom& g, const T* x, T* y, const T* eta, T alpha, const T* z, T beta,
                    T* r1, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (g.n_hi > 0 && g.hi_tiles && g.hi_flag) {
            stage_split<N>(g, x, y, eta, alpha, z, beta, r1, s);
            return;
        }
    }
    if constexpr (StageLayout<N, T, T, 4>::BYTES <= kMaxSmem) {
        if (g.stage_rows[sizeof(T) == 4 ? 1 : 0] == 4) {
            stage_plain<N, T, 4>(g, x, y, eta, alpha, z, beta, r1, s);
            return;
        }
    }
    stage_plain<N, T, 2>(g, x, y, eta, alpha, z, beta, r1, s);
}

// ---- set-up: tiles that need FP64 arithmetic in the FP32 operator
__global__ void k_eta_min(size_t n, const double* eta, double* out) {
    grid_dep_wait();
    __shared__ double sm[32];
    double m = 1e300;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) m = fmin(m, eta[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_down_sync(0xffffffffu, m, o));
    if (threadIdx.x % 32 == 0) sm[threadIdx.x / 32] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < blockDim.x / 32 ? sm[threadIdx.x] : 1e300;
        for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_down_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) *out = m;
    }
}

// flag[t] = 1 when an element of split tile t or of its one-element halo has
// eta >= ratio x min eta; the flagged tiles are appended to list.
__global__ void k_mark_hi(int nx, int ny, int ntx, int nty, const double* eta, const double* emin,
                          double ratio, unsigned char* flag, int* list, int* count) {
    grid_dep_wait();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntx * nty) return;
    const int bx = t % ntx, by = t / ntx;
    const double thr = ratio * *emin;
    bool hi = false;
    for (int ey = max(by * SPLIT_TYS - 1, 0); ey <= min(by * SPLIT_TYS + SPLIT_TYS, ny - 1); ++ey)
        for (int ex = max(bx * STX - 1, 0); ex <= min(bx * STX + STX, nx - 1); ++ex)
            hi = hi || eta[size_t(ey) * nx + ex] >= thr;
    flag[t] = hi ? 1 : 0;
    if (hi) list[atomicAdd(count, 1)] = t;
}

}  // namespace

void split_fork_prepare() { (void)fork_stream(); }

int split_tile_count(int nx, int ny) {
    return ((nx + STX - 1) / STX) * ((ny + SPLIT_TYS - 1) / SPLIT_TYS);
}

int mark_hi_tiles(int nx, int ny, const double* eta, double ratio, unsigned char* flag, int* list,
                  int* scratch, cudaStream_t s) {
    const int ntx = (nx + STX - 1) / STX, nty = (ny + SPLIT_TYS - 1) / SPLIT_TYS;
    const int nt = ntx * nty;
    double* emin = reinterpret_cast<double*>(scratch);   // scratch: 2 doubles + 1 int
    int* count = reinterpret_cast<int*>(scratch + 4);
    SIP_CUDA(cudaMemsetAsync(count, 0, sizeof(int), s));
    launch_k(k_eta_min, 1, 1024, 0, s, size_t(nx) * ny, eta, emin);
    SIP_CHECK_LAUNCH();
    launch_k(k_mark_hi, unsigned((nt + 255) / 256), 256, 0, s, nx, ny, ntx, nty, eta,
             static_cast<const double*>(emin), ratio, flag, list, count);
    SIP_CHECK_LAUNCH();
    int n = 0;
    SIP_CUDA(cudaMemcpyAsync(&n, count, sizeof(int), cudaMemcpyDeviceToHost, s));
    SIP_CUDA(cudaStreamSynchronize(s));
    return n;
}

template <typename TS, typename TC>
void launch_apply_stage_batch(int N, const StageArgs<TS, TC>* args, const int2* items,
                              int n_items, const int* active, bool vec, cudaStream_t s) {
    if (n_items <= 0) return;
    switch (N) {
        case 2: stage_batch_n<2, TS, TC>(args, items, n_items, active, vec, s); break;
        case 3: stage_batch_n<3, TS, TC>(args, items, n_items, active, vec, s); break;
        case 4: stage_batch_n<4, TS, TC>(args, items, n_items, active, vec, s); break;
        case 5: stage_batch_n<5, TS, TC>(args, items, n_items, active, vec, s); break;
        case 6: stage_batch_n<6, TS, TC>(args, items, n_items, active, vec, s); break;
        default: throw Error(SIP_ERR_INVALID_ARG, "batched apply: degree above 5");
    }
}
template void launch_apply_stage_batch<float, float>(int, const StageArgs<float, float>*,
                                                     const int2*, int, const int*, bool,
                                                     cudaStream_t);
template void launch_apply_stage_batch<float, double>(int, const StageArgs<float, double>*,
                                                      const int2*, int, const int*, bool,
                                                      cudaStream_t);
template void launch_apply_stage_batch<double, double>(int, const StageArgs<double, double>*,
                                                       const int2*, int, const int*, bool,
                                                       cudaStream_t);

template <typename TS, typename TC>
StageArgs<TS, TC> stage_args(const OpGeom& g, const TS* x, TS* y, const TS* eta, double alpha,
                             const TS* z, double beta, TS* r1, int N) {
    return make_stage_args<TS, TC>(g, x, y, eta, alpha, z, beta, r1, N, SPLIT_TYS);
}
template StageArgs<float, float> stage_args<float, float>(const OpGeom&, const float*, float*,
                                                          const float*, double, const float*,
                                                          double, float*, int);
template StageArgs<float, double> stage_args<float, double>(const OpGeom&, const float*, float*,
                                                            const float*, double, const float*,
                                                            double, float*, int);
template StageArgs<double, double> stage_args<double, double>(const OpGeom&, const double*,
                                                              double*, const double*, double,
                                                              const double*, double, double*,
                                                              int);

template <typename T>
bool launch_apply_sip_stage(int N, const OpGeom& g, const T* x, T* y, const T* eta, T alpha,
                            const T* z, T beta, T* r1, cudaStream_t s) {
    switch (N) {
        case 2: stage_dispatch<2, T>(g, x, y, eta, alpha, z, beta, r1, s); return true;
        case 3: stage_dispatch<3, T>(g, x, y, eta, alpha, z, beta, r1, s); return true;
        case 4: stage_dispatch<4, T>(g, x, y, eta, alpha, z, beta, r1, s); return true;
        case 5: stage_dispatch<5, T>(g, x, y, eta, alpha, z, beta, r1, s); return true;
        case 6: stage_dispatch<6, T>(g, x, y, eta, alpha, z, beta, r1, s); return true;
        default: return false;
    }
}
template bool launch_apply_sip_stage<double>(int, const OpGeom&, const double*, double*,
                                             const double*, double, const double*, double,
                                             double*, cudaStream_t);
template bool launch_apply_sip_stage<float>(int, const OpGeom&, const float*, float*,
                                            const float*, float, const float*, float, float*,
                                            cudaStream_t);

}  // namespace sip
