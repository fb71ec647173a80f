// Kernel-schedule autotuner.  Instances of the batched and served forms
// differ in mesh size, degree and precision, and no single kernel shape wins
// everywhere: the component-split apply (two threads per element) hides the
// narrow FP64 pipe's latency on small meshes, the one-thread-per-element
// apply issues fewer loads on large ones, the shared-memory tile kernel
// covers every degree, and the staged-tile kernel (element blocks copied
// through shared memory with coalesced 16-byte accesses, 2 or 4 tile rows)
// suits the memory-bound FP32 operator, as does the warp-row kernel (one
// thread per element, one warp per tile row, cp.async staging; FP32 only).  So each problem times the candidates on its own mesh
// the first time it is set up and keeps the fastest:
//   * the apply kernel, per precision the problem runs in;
//   * the p-level smoother step: one fused launch (apply + block-Jacobi +
//     Chebyshev update) against the apply and block-Jacobi launches.
// Choices are cached per (degree, precision, mesh), so every problem of one
// shape in a process runs the same kernels (a solve gives the same bits
// alone and inside a batch).  SIP_AUTOTUNE=0 keeps the defaults.
#include <cuda_runtime.h>

#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "sip_solver.h"

namespace sip {

namespace {

template <typename T> const T* eta_vec(sip_problem* P);
template <> const double* eta_vec<double>(sip_problem* P) { return P->eta_d.as<double>(); }
template <> const float* eta_vec<float>(sip_problem* P) { return P->eta_f.as<float>(); }
template <typename T> const T* eta_inv_vec(sip_problem* P);
template <> const double* eta_inv_vec<double>(sip_problem* P) { return P->eta_inv_d.as<double>(); }
template <> const float* eta_inv_vec<float>(sip_problem* P) { return P->eta_inv_f.as<float>(); }

bool autotune_on() {
    static const bool on = [] {
        const char* v = std::getenv("SIP_AUTOTUNE");
        return !(v && std::string(v) == "0");
    }();
    return on;
}

using Key = std::tuple<int, int, int, int, int>;   // what, N, word size, nx, ny

std::mutex& cache_mu() {
    static std::mutex m;
    return m;
}
std::map<Key, int>& cache() {
    static std::map<Key, int> c;
    return c;
}

bool cached(const Key& k, int& v) {
    std::lock_guard<std::mutex> lk(cache_mu());
    auto it = cache().find(k);
    if (it == cache().end()) return false;
    v = it->second;
    return true;
}

void store(const Key& k, int v) {
    std::lock_guard<std::mutex> lk(cache_mu());
    cache().emplace(k, v);
}

// mean device time of one call of f on stream s (2 warm-up calls, reps timed)
template <class F>
double time_ms(F&& f, cudaStream_t s, int reps) {
    cudaEvent_t e0, e1;
    SIP_CUDA(cudaEventCreate(&e0));
    SIP_CUDA(cudaEventCreate(&e1));
    f();
    f();
    SIP_CUDA(cudaEventRecord(e0, s));
    for (int i = 0; i < reps; ++i) f();
    SIP_CUDA(cudaEventRecord(e1, s));
    SIP_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    SIP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return double(ms) / reps;
}

template <typename T>
void tune_apply_t(sip_problem* P, cudaStream_t s) {
    const int t = sizeof(T) == 4 ? 1 : 0;
    if (P->pin_apply[t] > 0) {   // pinned: code 5 = staged with 4 tile rows
        P->geom.variant[t] = P->pin_apply[t] == 5 ? int(APPLY_STAGE) : P->pin_apply[t];
        P->geom.stage_rows[t] = P->pin_apply[t] == 5 ? 4 : 2;
        return;
    }
    const Key key{0, P->n, int(sizeof(T)), P->desc.nx, P->desc.ny};
    int best = APPLY_AUTO;   // variant + 16 x stage rows
    if (!cached(key, best)) {
        const size_t n_u = size_t(P->n_u);
        DeviceBuffer x, y;
        x.alloc(n_u * sizeof(T));
        y.alloc(n_u * sizeof(T));
        SIP_CUDA(cudaMemsetAsync(x.ptr, 0, n_u * sizeof(T), s));
        const T* eta = eta_vec<T>(P);
        double tbest = 1e300;
        const int64_t launches = launch_counter();
        const int saved_rows = P->geom.stage_rows[t];
        for (int cand : {int(APPLY_ELEM2), int(APPLY_ELEM1), int(APPLY_TILE),
                         int(APPLY_STAGE) + 16 * 2, int(APPLY_STAGE) + 16 * 4,
                         sizeof(T) == 4 ? int(APPLY_WARP) : -1}) {
            if (cand < 0) continue;
            P->geom.variant[t] = cand % 16;
            P->geom.stage_rows[t] = cand / 16 ? cand / 16 : saved_rows;
            const double ms = time_ms(
                [&] {
                    launch_apply_sip<T>(P->n, P->geom, x.as<T>(), y.as<T>(), eta, T(1), nullptr,
                                        T(0), s);
                },
                s, 5);
            if (ms < tbest) {
                tbest = ms;
                best = cand;
            }
        }
        P->geom.stage_rows[t] = saved_rows;
        launch_counter() = launches;
        store(key, best);
    }
    P->geom.variant[t] = best % 16;
    if (best / 16) P->geom.stage_rows[t] = best / 16;
}

}  // namespace

void tune_apply(sip_problem* P, cudaStream_t s) {
    if (P->n > 6) return;   // one kernel exists above degree 5
    if (!autotune_on()) {
        for (int t = 0; t < 2; ++t)
            if (P->pin_apply[t] > 0) {
                P->geom.variant[t] = P->pin_apply[t] == 5 ? int(APPLY_STAGE) : P->pin_apply[t];
                P->geom.stage_rows[t] = P->pin_apply[t] == 5 ? 4 : 2;
            }
        return;
    }
    tune_apply_t<double>(P, s);
    if (P->desc.precision != SIP_PREC_FP64) tune_apply_t<float>(P, s);
}

template <typename T>
void Multigrid<T>::tune_smoother(cudaStream_t s) {
    const int t = sizeof(T) == 4 ? 1 : 0;
    if (P->pin_fused[t] >= 0) {
        P->geom.fused[t] = P->pin_fused[t];
        return;
    }
    if (!autotune_on() || !cheb_elem_available(N) || !pd2.ptr) return;
    const Key key{1, N, int(sizeof(T)), P->desc.nx, P->desc.ny};
    int fused = 1;
    if (!cached(key, fused)) {
        T* b = pb.template as<T>();
        T* r = pr.template as<T>();
        T* d = pd.template as<T>();
        T* d2 = pd2.template as<T>();
        T* y = vout.template as<T>();
        for (T* v : {b, r, d, d2, y}) SIP_CUDA(cudaMemsetAsync(v, 0, n_u * sizeof(T), s));
        const T* eta = eta_vec<T>(P);
        const T* einv = eta_inv_vec<T>(P);
        const int* em = emap.template as<int>();
        const T* ci = cls_inv.template as<T>();
        const T* ui = uniq_inv.template as<T>();
        const int* csym = cls_sym.template as<int>();
        const int64_t launches = launch_counter();
        const double t_fused = time_ms(
            [&] {
                launch_cheb_elem<T>(N, P->geom, d, r, r, eta, em, ci, csym, ui, einv, d, d2, y,
                                    T(0.5), T(0.5), false, s);
            },
            s, 5);
        const double t_split = time_ms(
            [&] {
                launch_apply_sip<T>(N, P->geom, d, r, eta, T(-1), r, T(1), s);
                launch_bj_apply<T>(N, int(ne), r, d2, y, em, ci, csym, ui, einv, T(0.5), T(0.5),
                                   false, s);
            },
            s, 5);
        launch_counter() = launches;
        fused = t_fused <= t_split ? 1 : 0;
        store(key, fused);
    }
    P->geom.fused[t] = fused;
}

template void Multigrid<double>::tune_smoother(cudaStream_t);
template void Multigrid<float>::tune_smoother(cudaStream_t);

}  // namespace sip
