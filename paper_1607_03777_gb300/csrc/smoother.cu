// Element-block Jacobi smoother of the p-level (Sec. 6): the diagonal blocks
// M_K of A, their inverses, and the fused block-Jacobi / Chebyshev update.
//
// M_K depends on the element only through eta_K, the face kinds and the
// face penalties.  When eta_K is at least the viscosity of every face
// neighbour, all face penalties of K use eta_e = eta_K and M_K = eta_K M_ref,
// where M_ref depends only on which sides of K lie on the boundary (a 4-bit
// mask).  Such elements share one reference inverse per mask, scaled by
// 1/eta_K; the remaining ("unique") elements get their own inverse.
#include "sip_face.cuh"
#include "sip_internal.h"
#include "sip_parity.cuh"
#include "sip_solver.h"

namespace sip {

namespace {

template <int N>
struct BlockArgs {
    const int* spec;       // >= 0: element index; < 0: -(mask+1) reference block
    const double* eta;
    int nx, ny;
    double hx, hy;
    int bc[4];
    double pen_x, pen_y;
    Tab1D<N, double> tab;
};

// Entry M[r][s] of the element block: the local operator (neighbour
// coefficients zero) applied to the unit vector s, row r.
template <int N>
__device__ double block_entry(int r, int s, double etaK, const int kind[4], const double sig[4],
                              double hx, double hy, const Tab1D<N, double>& tb) {
    constexpr int NN = N * N;
    const int a = r % N, b = (r / N) % N, c = r / NN;
    const int i = s % N, j = (s / N) % N, c2 = s / NN;
    const double* G = tb.G;
    const double* D = tb.D;
    double vol = 0.0;
    if (c == 0) {
        if (c2 == 0) {
            if (b == j) vol += 2.0 * hy / hx * G[a * N + i];
            if (a == i) vol += hx / hy * G[b * N + j];
        } else {
            vol += D[j * N + b] * D[a * N + i];
        }
    } else {
        if (c2 == 1) {
            if (a == i) vol += 2.0 * hx / hy * G[b * N + j];
            if (b == j) vol += hy / hx * G[a * N + i];
        } else {
            vol += D[i * N + a] * D[b * N + j];
        }
    }
    double acc = etaK * vol;
    double vo[2 * N], dv[2 * N], zero[2 * N];
    for (int F = 0; F < 4; ++F) {
        const int d = F < 2 ? 0 : 1;
        const bool plus = (F % 2) == 1;
        const double sgn = plus ? 1.0 : -1.0;
        const double* l = plus ? tb.lp : tb.lm;
        const double* dl = plus ? tb.dp : tb.dm;
        for (int q = 0; q < 2 * N; ++q) vo[q] = dv[q] = zero[q] = 0.0;
        if (d == 0) {  // trace along y of mode (j, i): value l_i(s) at m = j
            vo[c2 * N + j] = l[i];
            dv[c2 * N + j] = 2.0 / hx * dl[i];
        } else {
            vo[c2 * N + i] = l[j];
            dv[c2 * N + i] = 2.0 / hy * dl[j];
        }
        const int mt = d == 0 ? b : a;   // test mode along the face
        const int qt = d == 0 ? a : b;   // test mode along the normal
        double P, Q;
        face_pq<N, double>(kind[F], c, mt, d, sgn, make_face_geo<double>(d == 0 ? hx : hy, d == 0 ? hy : hx), etaK, 0.0,
                           sig[F], vo, dv, zero, zero, D, P, Q);
        acc += l[qt] * P + dl[qt] * Q;
    }
    return acc;
}

// One CTA per block: build M in shared memory, invert it by Gauss-Jordan
// elimination (SPD: no pivoting needed), store M^{-1} as T.
template <int N, typename T>
__global__ void __launch_bounds__(256) k_build_blocks(const BlockArgs<N> a, T* out) {
    grid_dep_wait();
    constexpr int NB = 2 * N * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* M = reinterpret_cast<double*>(smem_raw);
    __shared__ double colk[NB];
    __shared__ double rowk[NB];
    const int sp = a.spec[blockIdx.x];
    double etaK;
    int kind[4];
    double sig[4];
    if (sp >= 0) {
        const int ex = sp % a.nx, ey = sp / a.nx;
        etaK = a.eta[sp];
        const int nbr[4] = {ex > 0 ? sp - 1 : -1, ex < a.nx - 1 ? sp + 1 : -1,
                            ey > 0 ? sp - a.nx : -1, ey < a.ny - 1 ? sp + a.nx : -1};
        for (int F = 0; F < 4; ++F) {
            const double pen = F < 2 ? a.pen_x : a.pen_y;
            if (nbr[F] >= 0) {
                kind[F] = 0;
                sig[F] = pen * fmax(etaK, a.eta[nbr[F]]);
            } else {
                kind[F] = 1 + a.bc[F];
                sig[F] = 2.0 * pen * etaK;
            }
        }
    } else {
        const int mask = -sp - 1;
        etaK = 1.0;
        for (int F = 0; F < 4; ++F) {
            const double pen = F < 2 ? a.pen_x : a.pen_y;
            const bool bnd = (mask >> F) & 1;
            kind[F] = bnd ? 1 + a.bc[F] : 0;
            sig[F] = bnd ? 2.0 * pen : pen;
        }
    }
    for (int q = threadIdx.x; q < NB * NB; q += blockDim.x)
        M[q] = block_entry<N>(q / NB, q % NB, etaK, kind, sig, a.hx, a.hy, a.tab);
    __syncthreads();
    for (int k = 0; k < NB; ++k) {
        const double piv = 1.0 / M[k * NB + k];
        for (int q = threadIdx.x; q < NB; q += blockDim.x) {
            colk[q] = M[q * NB + k];
            rowk[q] = M[k * NB + q];
        }
        __syncthreads();
        for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) {
            const int i = q / NB, j = q % NB;
            if (i == k && j == k)
                M[q] = piv;
            else if (i == k)
                M[q] = rowk[j] * piv;
            else if (j == k)
                M[q] = -colk[i] * piv;
            else
                M[q] -= colk[i] * rowk[j] * piv;
        }
        __syncthreads();
    }
    T* o = out + size_t(blockIdx.x) * NB * NB;
    for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) o[q] = T(M[q]);
}

// Element classification: mask of boundary sides; class elements (eta_K not
// below any face neighbour) map to -(mask+1), the others get a slot in the
// unique list (order by atomic ticket; results do not depend on it).
__global__ void k_classify(int nx, int ny, const double* eta, int* emap, int* uniq_list,
                           int* n_uniq) {
    grid_dep_wait();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nx * ny) return;
    const int ex = e % nx, ey = e / nx;
    int mask = 0;
    bool cls = true;
    const double et = eta[e];
    if (ex == 0) mask |= 1; else cls = cls && et >= eta[e - 1];
    if (ex == nx - 1) mask |= 2; else cls = cls && et >= eta[e + 1];
    if (ey == 0) mask |= 4; else cls = cls && et >= eta[e - nx];
    if (ey == ny - 1) mask |= 8; else cls = cls && et >= eta[e + nx];
    if (cls) {
        emap[e] = -(mask + 1);
    } else {
        const int slot = atomicAdd(n_uniq, 1);
        uniq_list[slot] = e;
        emap[e] = slot;
    }
}

// out = c2 * M_K^{-1} r_K (+ c1 * out_old); if x: x = (x_zero ? 0 : x) + out.
// EB elements per CTA, the residual blocks staged in shared memory; thread
// (element, row r) reads column r of the symmetric inverse (coalesced).
// Unique blocks flagged in uniq_hi (may be null) are applied in FP64 from
// their FP64 inverses (uniq_inv64): rounding an ill-conditioned inverse to
// FP32, or summing its products in FP32, loses the small components of the
// result.
template <int N, typename T>
__device__ __forceinline__ void bj_body(int e0, const BJBatchArgs<T>& a) {
    constexpr int NB = 2 * N * N;
    constexpr int EB = (256 / NB) > 0 ? (256 / NB) : 1;
    static_assert(EB * NB <= 256, "one (element, row) per thread");
    __shared__ T sr[EB * NB];
    __shared__ const T* s_minv[EB];
    __shared__ T s_scale[EB];
    __shared__ int s_sym[EB];   // symmetry type; -1: dense, FP64 inverse
    __shared__ const double* s_m64[EB];
    const int ne = a.ne;
    const int cnt = min(EB, ne - e0) * NB;
    // every load that does not depend on another is issued before the
    // barrier: the residual block, the element's block pointer and scale,
    // the previous direction and iterate
    const int q = threadIdx.x;
    const bool act = q < cnt;
    const size_t o = size_t(e0) * NB + q;
    if (act) sr[q] = a.r[o];
    if (q < EB && e0 + q < ne) {
        const int e = e0 + q;
        const int m = a.emap[e];
        if (m < 0) {
            s_minv[q] = a.cls_inv + size_t(-m - 1) * NB * NB;
            s_scale[q] = a.eta_inv[e];
            s_sym[q] = a.cls_sym ? a.cls_sym[-m - 1] : 0;
        } else {
            s_minv[q] = a.uniq_inv + size_t(m) * NB * NB;
            s_scale[q] = T(1);
            const bool hi = a.uniq_hi && a.uniq_hi[m] && a.uniq_inv64;
            s_sym[q] = hi ? -1 : 0;
            s_m64[q] = hi ? a.uniq_inv64 + size_t(m) * NB * NB : nullptr;
        }
    }
    const T c1 = a.c1, c2 = a.c2;
    const T out_old = (act && c1 != T(0)) ? a.out[o] : T(0);
    const T x_old = (act && a.x && !a.x_zero) ? a.x[o] : T(0);
    __syncthreads();
    if (!act) return;
    const int el = q / NB, row = q % NB;
    T acc;
    if constexpr (sizeof(T) == 4) {
        if (s_sym[el] < 0) {
            const double* M = s_m64[el];
            const T* rr = sr + el * NB;
            double a64 = 0.0;
#pragma unroll 8
            for (int q2 = 0; q2 < NB; ++q2) a64 += M[q2 * NB + row] * double(rr[q2]);
            acc = T(a64);
        } else {
            acc = block_row_apply<N, T>(s_minv[el], sr + el * NB, row, s_sym[el]);
        }
    } else {
        acc = block_row_apply<N, T>(s_minv[el], sr + el * NB, row, s_sym[el] < 0 ? 0 : s_sym[el]);
    }
    T v = c2 * s_scale[el] * acc;
    if (c1 != T(0)) v += c1 * out_old;
    a.out[o] = v;
    if (a.x) a.x[o] = a.x_zero ? v : x_old + v;
}

template <int N, typename T>
__global__ void __launch_bounds__(256) k_bj_apply(const BJBatchArgs<T> a) {
    grid_dep_wait();
    constexpr int NB = 2 * N * N;
    constexpr int EB = (256 / NB) > 0 ? (256 / NB) : 1;
    bj_body<N, T>(blockIdx.x * EB, a);
}

// Many block-Jacobi applies in one launch: CTA b serves member items[b].x
// (arguments args[items[b].x]), element group items[b].y; members with
// active[m] == 0 are skipped.
template <int N, typename T>
__global__ void __launch_bounds__(256) k_bj_apply_batch(const BJBatchArgs<T>* __restrict__ args,
                                                        const int2* __restrict__ items,
                                                        const int* __restrict__ active) {
    grid_dep_wait();
    constexpr int NB = 2 * N * N;
    constexpr int EB = (256 / NB) > 0 ? (256 / NB) : 1;
    const int2 it = items[blockIdx.x];
    if (active && !active[it.x]) return;
    bj_body<N, T>(it.y * EB, args[it.x]);
}

template <int N>
BlockArgs<N> make_block_args(const OpGeom& g, const int* spec, const double* eta) {
    BlockArgs<N> a;
    a.spec = spec;
    a.eta = eta;
    a.nx = g.nx;
    a.ny = g.ny;
    a.hx = g.hx;
    a.hy = g.hy;
    for (int i = 0; i < 4; ++i) a.bc[i] = g.bc[i];
    a.pen_x = g.pen_x;
    a.pen_y = g.pen_y;
    a.tab = make_tab<N, double>();
    return a;
}

template <int N, typename T>
void build_blocks_n(const OpGeom& g, const int* spec, int count, const double* eta, T* out,
                    cudaStream_t s) {
    if (count == 0) return;
    constexpr int NB = 2 * N * N;
    const size_t smem = size_t(NB) * NB * sizeof(double);
    SIP_CUDA(cudaFuncSetAttribute(k_build_blocks<N, T>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    launch_k(k_build_blocks<N, T>, count, 256, smem, s, make_block_args<N>(g, spec, eta), out);
    SIP_CHECK_LAUNCH();
}

template <int N, typename T>
void bj_apply_n(int ne, const T* r, T* out, T* x, const int* emap, const T* cls_inv,
                const int* cls_sym, const T* uniq_inv, const T* eta, T c1, T c2, bool x_zero,
                const unsigned char* uniq_hi, const double* uniq_inv64, cudaStream_t s) {
    constexpr int NB = 2 * N * N;
    constexpr int EB = (256 / NB) > 0 ? (256 / NB) : 1;
    const int blocks = (ne + EB - 1) / EB;
    const BJBatchArgs<T> a{ne, r, out, x, emap, cls_inv, cls_sym, uniq_inv, eta, uniq_hi,
                           uniq_inv64, c1, c2, x_zero ? 1 : 0};
    launch_k(k_bj_apply<N, T>, blocks, 256, 0, s, a);
    SIP_CHECK_LAUNCH();
}

template <int N, typename T>
void bj_batch_n(const BJBatchArgs<T>* args, const int2* items, int n_items, const int* active,
                cudaStream_t s) {
    launch_k(k_bj_apply_batch<N, T>, dim3(unsigned(n_items)), 256, 0, s, args, items, active);
    SIP_CHECK_LAUNCH();
}

}  // namespace

void launch_classify(int nx, int ny, const double* eta, int* emap, int* uniq_list, int* n_uniq,
                     cudaStream_t s) {
    const int ne = nx * ny;
    launch_k(k_classify, (ne + 255) / 256, 256, 0, s, nx, ny, eta, emap, uniq_list, n_uniq);
    SIP_CHECK_LAUNCH();
}

template <typename T>
void launch_build_blocks(int N, const OpGeom& g, const int* spec, int count, const double* eta,
                         T* out, cudaStream_t s) {
    switch (N) {
        case 2: build_blocks_n<2, T>(g, spec, count, eta, out, s); break;
        case 3: build_blocks_n<3, T>(g, spec, count, eta, out, s); break;
        case 4: build_blocks_n<4, T>(g, spec, count, eta, out, s); break;
        case 5: build_blocks_n<5, T>(g, spec, count, eta, out, s); break;
        case 6: build_blocks_n<6, T>(g, spec, count, eta, out, s); break;
        case 7: build_blocks_n<7, T>(g, spec, count, eta, out, s); break;
        default: throw Error(SIP_ERR_INVALID_ARG, "unsupported polynomial degree");
    }
}
template void launch_build_blocks<double>(int, const OpGeom&, const int*, int, const double*,
                                          double*, cudaStream_t);
template void launch_build_blocks<float>(int, const OpGeom&, const int*, int, const double*,
                                         float*, cudaStream_t);

template <typename T>
void launch_bj_apply(int N, int ne, const T* r, T* out, T* x, const int* emap, const T* cls_inv,
                     const int* cls_sym, const T* uniq_inv, const T* eta, T c1, T c2, bool x_zero,
                     cudaStream_t s, const unsigned char* uniq_hi, const double* uniq_inv64) {
    switch (N) {
        case 2: bj_apply_n<2, T>(ne, r, out, x, emap, cls_inv, cls_sym, uniq_inv, eta, c1, c2, x_zero, uniq_hi, uniq_inv64, s); break;
        case 3: bj_apply_n<3, T>(ne, r, out, x, emap, cls_inv, cls_sym, uniq_inv, eta, c1, c2, x_zero, uniq_hi, uniq_inv64, s); break;
        case 4: bj_apply_n<4, T>(ne, r, out, x, emap, cls_inv, cls_sym, uniq_inv, eta, c1, c2, x_zero, uniq_hi, uniq_inv64, s); break;
        case 5: bj_apply_n<5, T>(ne, r, out, x, emap, cls_inv, cls_sym, uniq_inv, eta, c1, c2, x_zero, uniq_hi, uniq_inv64, s); break;
        case 6: bj_apply_n<6, T>(ne, r, out, x, emap, cls_inv, cls_sym, uniq_inv, eta, c1, c2, x_zero, uniq_hi, uniq_inv64, s); break;
        case 7: bj_apply_n<7, T>(ne, r, out, x, emap, cls_inv, cls_sym, uniq_inv, eta, c1, c2, x_zero, uniq_hi, uniq_inv64, s); break;
        default: throw Error(SIP_ERR_INVALID_ARG, "unsupported polynomial degree");
    }
}
template void launch_bj_apply<double>(int, int, const double*, double*, double*, const int*,
                                      const double*, const int*, const double*, const double*,
                                      double, double, bool, cudaStream_t, const unsigned char*,
                                      const double*);
template void launch_bj_apply<float>(int, int, const float*, float*, float*, const int*,
                                     const float*, const int*, const float*, const float*, float,
                                     float, bool, cudaStream_t, const unsigned char*,
                                     const double*);

int bj_group(int N) {
    const int nb = 2 * N * N;
    return (256 / nb) > 0 ? (256 / nb) : 1;
}

template <typename T>
void launch_bj_apply_batch(int N, const BJBatchArgs<T>* args, const int2* items, int n_items,
                           const int* active, cudaStream_t s) {
    if (n_items <= 0) return;
    switch (N) {
        case 2: bj_batch_n<2, T>(args, items, n_items, active, s); break;
        case 3: bj_batch_n<3, T>(args, items, n_items, active, s); break;
        case 4: bj_batch_n<4, T>(args, items, n_items, active, s); break;
        case 5: bj_batch_n<5, T>(args, items, n_items, active, s); break;
        case 6: bj_batch_n<6, T>(args, items, n_items, active, s); break;
        case 7: bj_batch_n<7, T>(args, items, n_items, active, s); break;
        default: throw Error(SIP_ERR_INVALID_ARG, "unsupported polynomial degree");
    }
}
template void launch_bj_apply_batch<double>(int, const BJBatchArgs<double>*, const int2*, int,
                                            const int*, cudaStream_t);
template void launch_bj_apply_batch<float>(int, const BJBatchArgs<float>*, const int2*, int,
                                           const int*, cudaStream_t);

// uniq_hi[s] = 1 when the unique block of slot s belongs to an element whose
// largest face-neighbour viscosity is at least ratio times its own: the
// blocks whose condition grows with that contrast.
__global__ void k_mark_uniq_hi(int nx, int ny, const int* list, const int* n_uniq,
                               const double* eta, double ratio, unsigned char* flag) {
    grid_dep_wait();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= *n_uniq) return;
    const int e = list[s], ex = e % nx, ey = e / nx;
    double m = 0.0;
    if (ex > 0) m = fmax(m, eta[e - 1]);
    if (ex < nx - 1) m = fmax(m, eta[e + 1]);
    if (ey > 0) m = fmax(m, eta[e - nx]);
    if (ey < ny - 1) m = fmax(m, eta[e + nx]);
    flag[s] = m >= ratio * eta[e] ? 1 : 0;
}

void launch_mark_uniq_hi(int nx, int ny, const int* list, const int* n_uniq_dev, int n_uniq,
                         const double* eta, double ratio, unsigned char* flag, cudaStream_t s) {
    if (n_uniq <= 0) return;
    launch_k(k_mark_uniq_hi, unsigned((n_uniq + 255) / 256), 256, 0, s, nx, ny, list, n_uniq_dev,
             eta, ratio, flag);
    SIP_CHECK_LAUNCH();
}

}  // namespace sip
