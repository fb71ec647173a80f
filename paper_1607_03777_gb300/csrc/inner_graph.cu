// Inner Krylov solve of the block preconditioner (Sec. 5: the viscous block
// solved to a relative tolerance by CG -- or GCR, Sec. 7.3 -- preconditioned
// with one hp-multigrid V-cycle) as ONE CUDA graph launch per solve: the iteration is a device-side `while`
// conditional node, the stopping test (||r|| < rtol ||t|| or the iteration
// cap) is taken by a one-block kernel at the end of every pass, and alpha,
// beta, the norms and the counter stay in device memory.  No host round trip
// happens inside the loop.
//
// The arithmetic is that of the host-driven loop step for step (same
// kernels' blocking, same reduction order), so the iterates are identical.
// The loop ends by construction: the control kernel runs once per pass,
// increments the counter unconditionally and clears the condition once the
// counter reaches the cap, which the host clamps to [1, 100000].
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "sip_solver.h"

namespace sip {

namespace {

constexpr int kRB = 304;   // reduction blocks (2 x 152 SMs), fixed: deterministic sums
constexpr int kRT = 256;

struct PcgState {
    const double* t;   // right-hand side (set before each launch)
    double* y;         // iterate (set before each launch)
    double nt, rz, alpha, beta, rr, dq, nz0, nz;
    int it, status;    // status 0 ok, 1 non-finite (or a GCR direction with A z = 0)
    int cnt;           // GCR: directions stored in the current cycle
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

__device__ __forceinline__ double final_sum(const double* partial) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < kRB; i += blockDim.x) acc += partial[i];
    return block_sum(acc);
}

__global__ void k_set(PcgState* st, const double* t, double* y) {
    grid_dep_wait();
    st->t = t;
    st->y = y;
}

// r = t, y = 0, d = 0; partial sums of t.t
__global__ void __launch_bounds__(kRT) k_init(size_t n, PcgState* st, double* r, double* d,
                                              double* partial) {
    grid_dep_wait();
    const double* t = st->t;
    double* y = st->y;
    double acc = 0.0;
    for (size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n;
         g += size_t(gridDim.x) * blockDim.x) {
        const double v = t[g];
        acc += v * v;
        r[g] = v;
        y[g] = 0.0;
        d[g] = 0.0;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kRT) k_init_final(PcgState* st, const double* partial,
                                                    cudaGraphConditionalHandle h) {
    grid_dep_wait();
    const double s = final_sum(partial);
    if (threadIdx.x == 0) {
        const double nt = sqrt(s);
        st->nt = nt;
        st->rr = nt;
        st->rz = 0.0;
        st->it = 0;
        st->cnt = 0;
        st->status = isfinite(nt) ? 0 : 1;
        cudaGraphSetConditional(h, (isfinite(nt) && nt > 0.0) ? 1u : 0u);
    }
}

// partial sums of r.z, with z = widen(zs) stored into zd when zd != nullptr
template <typename Tz>
__global__ void __launch_bounds__(kRT) k_dot_rz(size_t n, const double* __restrict__ r,
                                                const Tz* __restrict__ zs, double* zd,
                                                double* partial) {
    grid_dep_wait();
    double acc = 0.0;
    for (size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n;
         g += size_t(gridDim.x) * blockDim.x) {
        const double z = double(zs[g]);
        if (zd) zd[g] = z;
        acc += r[g] * z;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// beta = rz_new / rz (0 on the first pass); rz = rz_new
__global__ void __launch_bounds__(kRT) k_beta_final(PcgState* st, const double* partial) {
    grid_dep_wait();
    const double s = final_sum(partial);
    if (threadIdx.x == 0) {
        st->beta = st->it == 0 ? 0.0 : s / st->rz;
        st->rz = s;
    }
}

// d = z + beta d
__global__ void k_dir(size_t n, const double* __restrict__ z, double* d, const PcgState* st) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= n) return;
    d[g] = z[g] + st->beta * d[g];
}

__global__ void __launch_bounds__(kRT) k_dot(size_t n, const double* __restrict__ a,
                                             const double* __restrict__ b, double* partial) {
    grid_dep_wait();
    double acc = 0.0;
    for (size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n;
         g += size_t(gridDim.x) * blockDim.x)
        acc += a[g] * b[g];
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// alpha = rz / (d.q)
__global__ void __launch_bounds__(kRT) k_alpha_final(PcgState* st, const double* partial) {
    grid_dep_wait();
    const double s = final_sum(partial);
    if (threadIdx.x == 0) st->alpha = st->rz / s;
}

// y += alpha d; r -= alpha q; partial sums of r.r
__global__ void __launch_bounds__(kRT) k_update_rr(size_t n, const double* __restrict__ d,
                                                   const double* __restrict__ q, double* r,
                                                   const PcgState* st, double* partial) {
    grid_dep_wait();
    const double a = st->alpha;
    double* y = st->y;
    double acc = 0.0;
    for (size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n;
         g += size_t(gridDim.x) * blockDim.x) {
        y[g] += a * d[g];
        const double rv = r[g] - a * q[g];
        r[g] = rv;
        acc += rv * rv;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// ---- flexible CG, FCG(1) (Notay, SIAM J. Sci. Comput. 22, 2000): the
// direction is A-orthogonalised against the previous one explicitly,
//   beta = <z_{k+1}, q_k> / <d_k, q_k>,  d_{k+1} = z_{k+1} - beta d_k,
//   alpha = <d_k, r_k> / <d_k, q_k>,
// which equals PCG in exact arithmetic with a fixed SPD preconditioner and
// tolerates a preconditioner that varies slightly between applications
// (the FP32 V-cycle of the mixed form).

// partial sums of z.q, with z = widen(zs) stored into zd when zd != nullptr
template <typename Tz>
__global__ void __launch_bounds__(kRT) k_dot_zq(size_t n, const double* __restrict__ q,
                                                const Tz* __restrict__ zs, double* zd,
                                                double* partial) {
    grid_dep_wait();
    double acc = 0.0;
    for (size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n;
         g += size_t(gridDim.x) * blockDim.x) {
        const double z = double(zs[g]);
        if (zd) zd[g] = z;
        acc += z * q[g];
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// stored as -beta so that k_dir (d = z + beta d) forms z - beta d
__global__ void __launch_bounds__(kRT) k_beta_fcg_final(PcgState* st, const double* partial) {
    grid_dep_wait();
    const double s = final_sum(partial);
    if (threadIdx.x == 0) st->beta = st->it == 0 ? 0.0 : -(s / st->dq);
}

// partial sums of d.q (partial[0..kRB)) and d.r (partial[kRB..2kRB))
__global__ void __launch_bounds__(kRT) k_dot_dq_dr(size_t n, const double* __restrict__ d,
                                                   const double* __restrict__ q,
                                                   const double* __restrict__ r,
                                                   double* partial) {
    grid_dep_wait();
    double a1 = 0.0, a2 = 0.0;
    for (size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n;
         g += size_t(gridDim.x) * blockDim.x) {
        const double dv = d[g];
        a1 += dv * q[g];
        a2 += dv * r[g];
    }
    a1 = block_sum(a1);
    a2 = block_sum(a2);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = a1;
        partial[kRB + blockIdx.x] = a2;
    }
}

__global__ void __launch_bounds__(kRT) k_alpha_fcg_final(PcgState* st, const double* partial) {
    grid_dep_wait();
    const double dq = final_sum(partial);
    const double dr = final_sum(partial + kRB);
    if (threadIdx.x == 0) {
        st->dq = dq;
        st->alpha = dr / dq;
    }
}

// End of one pass: counter, stopping test, loop condition.
__global__ void __launch_bounds__(kRT) k_ctl_final(PcgState* st, const double* partial,
                                                   double rtol, int maxit,
                                                   cudaGraphConditionalHandle h) {
    grid_dep_wait();
    const double s = final_sum(partial);
    if (threadIdx.x == 0) {
        const double rr = sqrt(s);
        const int it = st->it + 1;
        st->it = it;
        st->rr = rr;
        if (!isfinite(rr)) st->status = 1;
        const bool more = isfinite(rr) && !(rr < rtol * st->nt) && it < maxit;
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
}

// ---- stopping on the preconditioned residual ||V r|| (the default test of
// PETSc's CG, which the paper ran): the V-cycle moves to the end of the pass,
// so that the test sees the z it produces; one V-cycle of the initial
// residual precedes the loop.

// partial sums of z.z (partial[0..kRB)) and z.w (partial[kRB..2kRB)), with
// z = widen(zs) stored into zd when zd != nullptr; w = r (PCG) or q (FCG)
template <typename Tz>
__global__ void __launch_bounds__(kRT) k_dot_zz_zw(size_t n, const double* __restrict__ w,
                                                   const Tz* __restrict__ zs, double* zd,
                                                   double* partial) {
    grid_dep_wait();
    double a1 = 0.0, a2 = 0.0;
    for (size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n;
         g += size_t(gridDim.x) * blockDim.x) {
        const double z = double(zs[g]);
        if (zd) zd[g] = z;
        a1 += z * z;
        a2 += w[g] * z;
    }
    a1 = block_sum(a1);
    a2 = block_sum(a2);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = a1;
        partial[kRB + blockIdx.x] = a2;
    }
}

// after z_0 = V(r_0): ||z_0||, rz = r.z (PCG), beta = 0, first condition
__global__ void __launch_bounds__(kRT) k_pn_first_final(PcgState* st, const double* partial,
                                                        cudaGraphConditionalHandle h) {
    grid_dep_wait();
    const double zz = final_sum(partial);
    const double zw = final_sum(partial + kRB);
    if (threadIdx.x == 0) {
        const double nz0 = sqrt(zz);
        st->nz0 = nz0;
        st->nz = nz0;
        st->rz = zw;
        st->beta = 0.0;
        if (!isfinite(nz0)) st->status = 1;
        const bool go = st->status == 0 && st->nt > 0.0 && nz0 > 0.0;
        cudaGraphSetConditional(h, go ? 1u : 0u);
    }
}

// end of a pass: counter, test ||z|| < rtol ||z_0||, the next beta
// (PCG: rz_new / rz; FCG, stored negated: -(z.q) / (d.q)), loop condition
__global__ void __launch_bounds__(kRT) k_pn_ctl_final(PcgState* st, const double* partial,
                                                      double rtol, int maxit, int flexible,
                                                      cudaGraphConditionalHandle h) {
    grid_dep_wait();
    const double zz = final_sum(partial);
    const double zw = final_sum(partial + kRB);
    if (threadIdx.x == 0) {
        const double nz = sqrt(zz);
        const int it = st->it + 1;
        st->it = it;
        st->nz = nz;
        if (flexible) {
            st->beta = -(zw / st->dq);
        } else {
            st->beta = zw / st->rz;
            st->rz = zw;
        }
        if (!isfinite(nz)) st->status = 1;
        const bool more = isfinite(nz) && !(nz < rtol * st->nz0) && it < maxit;
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
}


// ---- GCR (Eisenstat, Elman & Schultz, SIAM J. Numer. Anal. 20, 1983),
// restarted after m directions, flexible; the method the paper ran for the
// viscous block of the six-inclusion problem (Sec. 7.3).  A pass: z = V(r),
// q = A z; q is orthogonalised against the stored q_i with the same
// combination applied to z (classical Gram-Schmidt, twice), the pair is
// written to slot cnt of the direction arrays Zs, Qs ([m][n] each), then
// alpha = <r, q> / <q, q>, y += alpha z, r -= alpha q.  The stopping test is
// ||r|| < rtol ||t||.  The number of stored pairs is read on the device, so
// one captured body serves every pass.

constexpr int kGcrMax = 64;   // restart length cap (coefficients in shared memory)

// partial sums <q, Qs[i]> for i < cnt into partial[i * kRB + block]; q is the
// fixed buffer (first pass) or slot cnt itself (second pass, q == nullptr)
__global__ void __launch_bounds__(kRT) k_gcr_mdot(size_t n, const double* __restrict__ q,
                                                  const double* __restrict__ Qs,
                                                  const PcgState* st, double* partial) {
    grid_dep_wait();
    const int cnt = st->cnt;
    const double* qv = q ? q : Qs + size_t(cnt) * n;
    for (int i0 = 0; i0 < cnt; i0 += 4) {
        const int nb = min(4, cnt - i0);
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        const double* Q0 = Qs + size_t(i0) * n;
        for (size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n;
             g += size_t(gridDim.x) * blockDim.x) {
            const double v = qv[g];
#pragma unroll
            for (int l = 0; l < 4; ++l)
                if (l < nb) a[l] += v * Q0[size_t(l) * n + g];
        }
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            if (l < nb) {   // nb is uniform over the block: the barriers inside are safe
                const double t = block_sum(a[l]);
                if (threadIdx.x == 0) partial[size_t(i0 + l) * kRB + blockIdx.x] = t;
            }
        }
    }
}

// beta_i = <q, q_i> / <q_i, q_i>, block i per coefficient
__global__ void __launch_bounds__(kRT) k_gcr_coef_final(const PcgState* st, const double* partial,
                                                        const double* qq, double* beta) {
    grid_dep_wait();
    const int i = blockIdx.x;
    if (i >= st->cnt) return;   // uniform over the block
    const double s = final_sum(partial + size_t(i) * kRB);
    if (threadIdx.x == 0) beta[i] = s / qq[i];
}

// Qs[cnt] = q - sum_i beta_i Qs[i], Zs[cnt] = z - sum_i beta_i Zs[i] (q, z the
// fixed buffers on the first pass; slot cnt in place on the second, z ==
// nullptr).  On the last pass also the partial sums of <q, q> and <r, q>.
__global__ void __launch_bounds__(kRT) k_gcr_orth(size_t n, const double* __restrict__ z,
                                                  const double* __restrict__ q, double* Zs,
                                                  double* Qs, const double* __restrict__ r,
                                                  const PcgState* st, const double* beta,
                                                  int last, double* partial) {
    grid_dep_wait();
    __shared__ double sb[kGcrMax];
    const int cnt = st->cnt;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) sb[i] = beta[i];
    __syncthreads();
    double* zo = Zs + size_t(cnt) * n;
    double* qo = Qs + size_t(cnt) * n;
    const double* zi = z ? z : zo;
    const double* qi = q ? q : qo;
    double a1 = 0.0, a2 = 0.0;
    for (size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n;
         g += size_t(gridDim.x) * blockDim.x) {
        double zv = zi[g], qv = qi[g];
        for (int i = 0; i < cnt; ++i) {
            const double b = sb[i];
            zv -= b * Zs[size_t(i) * n + g];
            qv -= b * Qs[size_t(i) * n + g];
        }
        zo[g] = zv;
        qo[g] = qv;
        if (last) {
            a1 += qv * qv;
            a2 += r[g] * qv;
        }
    }
    if (last) {
        a1 = block_sum(a1);
        a2 = block_sum(a2);
        if (threadIdx.x == 0) {
            partial[blockIdx.x] = a1;
            partial[kRB + blockIdx.x] = a2;
        }
    }
}

// alpha = <r, q> / <q, q>; <q, q> kept for the later coefficients
__global__ void __launch_bounds__(kRT) k_gcr_alpha_final(PcgState* st, const double* partial,
                                                         double* qq) {
    grid_dep_wait();
    const double qn = final_sum(partial);
    const double rq = final_sum(partial + kRB);
    if (threadIdx.x == 0) {
        const int cnt = st->cnt;
        qq[cnt] = qn;
        if (!(qn > 0.0) || !isfinite(qn) || !isfinite(rq)) {
            st->status = 1;
            st->alpha = 0.0;
        } else {
            st->alpha = rq / qn;
        }
    }
}

// y += alpha Zs[cnt]; r -= alpha Qs[cnt]; partial sums of r.r
__global__ void __launch_bounds__(kRT) k_gcr_step(size_t n, const double* __restrict__ Zs,
                                                  const double* __restrict__ Qs, double* r,
                                                  const PcgState* st, double* partial) {
    grid_dep_wait();
    const double a = st->alpha;
    const int cnt = st->cnt;
    const double* zc = Zs + size_t(cnt) * n;
    const double* qc = Qs + size_t(cnt) * n;
    double* y = st->y;
    double acc = 0.0;
    for (size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n;
         g += size_t(gridDim.x) * blockDim.x) {
        y[g] += a * zc[g];
        const double rv = r[g] - a * qc[g];
        r[g] = rv;
        acc += rv * rv;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// end of a GCR pass: counter, next slot (restart after m), stopping test
__global__ void __launch_bounds__(kRT) k_gcr_ctl_final(PcgState* st, const double* partial,
                                                       double rtol, int maxit, int m,
                                                       cudaGraphConditionalHandle h) {
    grid_dep_wait();
    const double s = final_sum(partial);
    if (threadIdx.x == 0) {
        const double rr = sqrt(s);
        const int it = st->it + 1;
        st->it = it;
        st->rr = rr;
        const int c = st->cnt + 1;
        st->cnt = c == m ? 0 : c;
        if (!isfinite(rr)) st->status = 1;
        const bool more = st->status == 0 && !(rr < rtol * st->nt) && it < maxit;
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
}

inline unsigned nblk(size_t n) { return unsigned((n + 255) / 256); }

}  // namespace

struct InnerLoop {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;
    DeviceBuffer state, partial;
    HostScalars hs;             // pinned read-back of the state
    bool mixed = false;
    bool flexible = false;
    bool pnorm = false;   // stop on the preconditioned residual
    int gcr = 0;          // GCR restart length (0: a CG variant)
    const void* gcr_buf = nullptr;
    DeviceBuffer gcr_coef;   // beta[kGcrMax], <q_i, q_i>[kGcrMax]
    double rtol = -1.0;
    int maxit = -1;
    int gen = -1;
    const void* mg = nullptr;
    int64_t top_kernels = 0, body_kernels = 0;

    ~InnerLoop() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
    }
};

void InnerLoopDeleter::operator()(InnerLoop* p) const { delete p; }

namespace {

// One pass of the loop body, captured into the conditional node's graph.
void capture_body(sip_problem* P, Workspace& W, InnerLoop& L, cudaGraphConditionalHandle h,
                  cudaStream_t cs) {
    const size_t n_u = size_t(P->n_u);
    double* r = W.cg_r.as<double>();
    double* d = W.cg_d.as<double>();
    double* q = W.cg_q.as<double>();
    double* z = W.cg_z.as<double>();
    double* part = L.partial.as<double>();
    PcgState* st = L.state.as<PcgState>();
    // z = V(r) with the scalar of the direction update: r.z (PCG) or z.q (FCG)
    if (L.mixed) {
        Multigrid<float>& mg = *P->mg32;
        float* vin = mg.vin.as<float>();
        float* vout = mg.vout.as<float>();
        launch_cast<double, float>(n_u, r, vin, cs);
        mg.vcycle_on(vin, vout, cs);
        if (L.flexible)
            launch_k(k_dot_zq<float>, kRB, kRT, 0, cs, n_u, q, vout, z, part);
        else
            launch_k(k_dot_rz<float>, kRB, kRT, 0, cs, n_u, r, vout, z, part);
        SIP_CHECK_LAUNCH();
    } else {
        Multigrid<double>& mg = *P->mg64;
        mg.vcycle_on(r, z, cs);
        if (L.flexible)
            launch_k(k_dot_zq<double>, kRB, kRT, 0, cs, n_u, q, z, nullptr, part);
        else
            launch_k(k_dot_rz<double>, kRB, kRT, 0, cs, n_u, r, z, nullptr, part);
        SIP_CHECK_LAUNCH();
    }
    if (L.flexible)
        launch_k(k_beta_fcg_final, 1, kRT, 0, cs, st, part);
    else
        launch_k(k_beta_final, 1, kRT, 0, cs, st, part);
    SIP_CHECK_LAUNCH();
    launch_k(k_dir, nblk(n_u), 256, 0, cs, n_u, z, d, st);
    SIP_CHECK_LAUNCH();
    launch_apply_sip<double>(P->n, P->geom, d, q, P->eta_d.as<double>(), 1.0, nullptr, 0.0, cs);
    if (L.flexible) {
        launch_k(k_dot_dq_dr, kRB, kRT, 0, cs, n_u, d, q, r, part);
        SIP_CHECK_LAUNCH();
        launch_k(k_alpha_fcg_final, 1, kRT, 0, cs, st, part);
        SIP_CHECK_LAUNCH();
    } else {
        launch_k(k_dot, kRB, kRT, 0, cs, n_u, d, q, part);
        SIP_CHECK_LAUNCH();
        launch_k(k_alpha_final, 1, kRT, 0, cs, st, part);
        SIP_CHECK_LAUNCH();
    }
    launch_k(k_update_rr, kRB, kRT, 0, cs, n_u, d, q, r, st, part);
    SIP_CHECK_LAUNCH();
    launch_k(k_ctl_final, 1, kRT, 0, cs, st, part, L.rtol, L.maxit, h);
    SIP_CHECK_LAUNCH();
}

// z = V(r) (z stored in FP64) with the partial sums of z.z and z.w
void vcycle_dots(sip_problem* P, Workspace& W, InnerLoop& L, const double* w, cudaStream_t cs) {
    const size_t n_u = size_t(P->n_u);
    double* r = W.cg_r.as<double>();
    double* z = W.cg_z.as<double>();
    double* part = L.partial.as<double>();
    if (L.mixed) {
        Multigrid<float>& mg = *P->mg32;
        float* vin = mg.vin.as<float>();
        float* vout = mg.vout.as<float>();
        launch_cast<double, float>(n_u, r, vin, cs);
        mg.vcycle_on(vin, vout, cs);
        launch_k(k_dot_zz_zw<float>, kRB, kRT, 0, cs, n_u, w, vout, z, part);
    } else {
        P->mg64->vcycle_on(r, z, cs);
        launch_k(k_dot_zz_zw<double>, kRB, kRT, 0, cs, n_u, w, z, nullptr, part);
    }
    SIP_CHECK_LAUNCH();
}

// One pass of the preconditioned-norm loop: d = z + beta d, q = A d, alpha,
// y += alpha d, r -= alpha q, z = V(r), test ||z||.
void capture_body_pnorm(sip_problem* P, Workspace& W, InnerLoop& L, cudaGraphConditionalHandle h,
                        cudaStream_t cs) {
    const size_t n_u = size_t(P->n_u);
    double* r = W.cg_r.as<double>();
    double* d = W.cg_d.as<double>();
    double* q = W.cg_q.as<double>();
    double* z = W.cg_z.as<double>();
    double* part = L.partial.as<double>();
    PcgState* st = L.state.as<PcgState>();
    launch_k(k_dir, nblk(n_u), 256, 0, cs, n_u, z, d, st);
    SIP_CHECK_LAUNCH();
    launch_apply_sip<double>(P->n, P->geom, d, q, P->eta_d.as<double>(), 1.0, nullptr, 0.0, cs);
    if (L.flexible) {
        launch_k(k_dot_dq_dr, kRB, kRT, 0, cs, n_u, d, q, r, part);
        SIP_CHECK_LAUNCH();
        launch_k(k_alpha_fcg_final, 1, kRT, 0, cs, st, part);
    } else {
        launch_k(k_dot, kRB, kRT, 0, cs, n_u, d, q, part);
        SIP_CHECK_LAUNCH();
        launch_k(k_alpha_final, 1, kRT, 0, cs, st, part);
    }
    SIP_CHECK_LAUNCH();
    launch_k(k_update_rr, kRB, kRT, 0, cs, n_u, d, q, r, st, part);
    SIP_CHECK_LAUNCH();
    vcycle_dots(P, W, L, L.flexible ? q : r, cs);
    launch_k(k_pn_ctl_final, 1, kRT, 0, cs, st, part, L.rtol, L.maxit, L.flexible ? 1 : 0, h);
    SIP_CHECK_LAUNCH();
}

// One GCR pass (see the kernels above).
void capture_body_gcr(sip_problem* P, Workspace& W, InnerLoop& L, cudaGraphConditionalHandle h,
                      cudaStream_t cs) {
    const size_t n_u = size_t(P->n_u);
    double* r = W.cg_r.as<double>();
    double* q = W.cg_q.as<double>();
    double* z = W.cg_z.as<double>();
    double* Zs = W.gcr_z.as<double>();
    double* Qs = W.gcr_q.as<double>();
    double* part = L.partial.as<double>();
    double* beta = L.gcr_coef.as<double>();
    double* qq = beta + kGcrMax;
    PcgState* st = L.state.as<PcgState>();
    if (L.mixed) {
        Multigrid<float>& mg = *P->mg32;
        float* vin = mg.vin.as<float>();
        float* vout = mg.vout.as<float>();
        launch_cast<double, float>(n_u, r, vin, cs);
        mg.vcycle_on(vin, vout, cs);
        launch_cast<float, double>(n_u, vout, z, cs);
    } else {
        P->mg64->vcycle_on(r, z, cs);
    }
    launch_apply_sip<double>(P->n, P->geom, z, q, P->eta_d.as<double>(), 1.0, nullptr, 0.0, cs);
    for (int pass = 0; pass < 2; ++pass) {
        const bool first = pass == 0;
        launch_k(k_gcr_mdot, kRB, kRT, 0, cs, n_u, first ? static_cast<const double*>(q) : nullptr,
                 static_cast<const double*>(Qs), static_cast<const PcgState*>(st), part);
        SIP_CHECK_LAUNCH();
        launch_k(k_gcr_coef_final, unsigned(L.gcr), kRT, 0, cs, static_cast<const PcgState*>(st),
                 static_cast<const double*>(part), static_cast<const double*>(qq), beta);
        SIP_CHECK_LAUNCH();
        launch_k(k_gcr_orth, kRB, kRT, 0, cs, n_u, first ? static_cast<const double*>(z) : nullptr,
                 first ? static_cast<const double*>(q) : nullptr, Zs, Qs,
                 static_cast<const double*>(r), static_cast<const PcgState*>(st),
                 static_cast<const double*>(beta), first ? 0 : 1, part);
        SIP_CHECK_LAUNCH();
    }
    launch_k(k_gcr_alpha_final, 1, kRT, 0, cs, st, static_cast<const double*>(part), qq);
    SIP_CHECK_LAUNCH();
    launch_k(k_gcr_step, kRB, kRT, 0, cs, n_u, static_cast<const double*>(Zs),
             static_cast<const double*>(Qs), r, static_cast<const PcgState*>(st), part);
    SIP_CHECK_LAUNCH();
    launch_k(k_gcr_ctl_final, 1, kRT, 0, cs, st, static_cast<const double*>(part), L.rtol, L.maxit,
             L.gcr, h);
    SIP_CHECK_LAUNCH();
}

void build_loop(sip_problem* P, Workspace& W, InnerLoop& L, cudaStream_t s) {
    // plain launches inside the graph that holds the conditional node
    PdlOffScope pdl_off;
    if (L.exec) {
        SIP_CUDA(cudaGraphExecDestroy(L.exec));
        L.exec = nullptr;
    }
    if (L.graph) {
        SIP_CUDA(cudaGraphDestroy(L.graph));
        L.graph = nullptr;
    }
    if (!L.cs) SIP_CUDA(cudaStreamCreateWithFlags(&L.cs, cudaStreamNonBlocking));
    SIP_CUDA(cudaStreamSynchronize(s));   // buffers allocated on s are ready
    const size_t n_u = size_t(P->n_u);
    const int64_t before = launch_counter();
    cudaGraph_t g = nullptr;
    SIP_CUDA(cudaGraphCreate(&g, 0));
    L.graph = g;
    cudaGraphConditionalHandle h;
    SIP_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    // pre-loop part (r = t, y = 0, d = 0, ||t||, first condition), then the
    // while node after it
    SIP_CUDA(cudaStreamBeginCaptureToGraph(L.cs, g, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal));
    launch_k(k_init, kRB, kRT, 0, L.cs, n_u, L.state.as<PcgState>(), W.cg_r.as<double>(),
                                  W.cg_d.as<double>(), L.partial.as<double>());
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        launch_k(k_init_final, 1, kRT, 0, L.cs, L.state.as<PcgState>(), L.partial.as<double>(), h);
        e = cudaGetLastError();
    }
    int64_t pre_kernels = 2;
    if (e == cudaSuccess && L.pnorm && !L.gcr) {   // z_0 = V(r_0), its norm, before the loop
        const int64_t c0 = launch_counter();
        try {
            vcycle_dots(P, W, L, W.cg_r.as<double>(), L.cs);
            launch_k(k_pn_first_final, 1, kRT, 0, L.cs, L.state.as<PcgState>(),
                     L.partial.as<double>(), h);
            SIP_CHECK_LAUNCH();
        } catch (const Error&) {
            e = cudaErrorUnknown;
        }
        pre_kernels += launch_counter() - c0;
    }
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
        e = cudaStreamGetCaptureInfo(L.cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
        if (e == cudaSuccess) e = cudaGraphAddNode(&nloop, g, deps, nullptr, ndeps, &cp);
        if (e == cudaSuccess)
            e = cudaStreamUpdateCaptureDependencies(L.cs, &nloop, nullptr, 1,
                                                    cudaStreamSetCaptureDependencies);
    }
    cudaGraph_t gout = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(L.cs, &gout);
    SIP_CUDA(e);
    SIP_CUDA(ee);
    L.top_kernels = pre_kernels;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    SIP_CUDA(cudaStreamBeginCaptureToGraph(L.cs, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal));
    const int64_t b0 = launch_counter();
    try {
        if (L.gcr)
            capture_body_gcr(P, W, L, h, L.cs);
        else if (L.pnorm)
            capture_body_pnorm(P, W, L, h, L.cs);
        else
            capture_body(P, W, L, h, L.cs);
    } catch (...) {
        cudaGraph_t tmp;
        cudaStreamEndCapture(L.cs, &tmp);
        launch_counter() = before;
        throw;
    }
    L.body_kernels = launch_counter() - b0;
    cudaGraph_t body_out;
    SIP_CUDA(cudaStreamEndCapture(L.cs, &body_out));
    launch_counter() = before;
    SIP_CUDA(cudaGraphInstantiate(&L.exec, g, 0));
}

}  // namespace

int inner_pcg_graph(sip_problem* P, Workspace& W, bool mixed, bool flexible, bool pnorm,
                    const double* t, double* y, double rtol, int maxit, cudaStream_t s,
                    int gcr_restart) {
    maxit = std::max(1, std::min(maxit, 100000));
    const size_t n_u = size_t(P->n_u);
    for (DeviceBuffer* b : {&W.cg_r, &W.cg_d, &W.cg_q, &W.cg_z}) b->alloc(n_u * sizeof(double));
    if (!W.loop) W.loop.reset(new InnerLoop());
    InnerLoop& L = *W.loop;
    static_assert(sizeof(PcgState) <= 256 * sizeof(double), "state fits the pinned block");
    if (gcr_restart < 0 || gcr_restart > kGcrMax) throw Error(SIP_ERR_INVALID_ARG, "GCR restart");
    L.state.alloc(sizeof(PcgState));
    L.partial.alloc(size_t(std::max(2, gcr_restart)) * kRB * sizeof(double));
    if (gcr_restart) {
        W.gcr_z.alloc(size_t(gcr_restart) * n_u * sizeof(double));
        W.gcr_q.alloc(size_t(gcr_restart) * n_u * sizeof(double));
        L.gcr_coef.alloc(2 * kGcrMax * sizeof(double));
    }
    const void* mg = mixed ? static_cast<const void*>(P->mg32.get())
                           : static_cast<const void*>(P->mg64.get());
    const int gen = mixed ? P->mg32->setup_gen : P->mg64->setup_gen;
    const void* gbuf = gcr_restart ? W.gcr_z.ptr : nullptr;
    if (!L.exec || L.mixed != mixed || L.flexible != flexible || L.pnorm != pnorm ||
        L.gcr != gcr_restart || L.gcr_buf != gbuf || L.rtol != rtol ||
        L.maxit != maxit || L.gen != gen || L.mg != mg) {
        L.mixed = mixed;
        L.flexible = flexible;
        L.pnorm = pnorm;
        L.gcr = gcr_restart;
        L.gcr_buf = gbuf;
        L.rtol = rtol;
        L.maxit = maxit;
        L.gen = gen;
        L.mg = mg;
        build_loop(P, W, L, s);
    }
    launch_k(k_set, 1, 1, 0, s, L.state.as<PcgState>(), t, y);
    SIP_CHECK_LAUNCH();
    SIP_CUDA(cudaGraphLaunch(L.exec, s));
    SIP_CUDA(cudaMemcpyAsync(L.hs.p, L.state.ptr, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    SIP_CUDA(cudaStreamSynchronize(s));
    const PcgState& hs = *reinterpret_cast<const PcgState*>(L.hs.p);
    launch_counter() += L.top_kernels + L.body_kernels * hs.it;
    if (hs.status != 0)
        throw Error(SIP_ERR_BREAKDOWN, gcr_restart ? "inner GCR breakdown (non-finite or A z = 0)"
                                                   : "non-finite inner residual");
    return hs.it;
}

}  // namespace sip
