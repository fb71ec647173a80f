// Krylov vector kernels: deterministic dot products (fixed two-stage tree,
// FP64 accumulation for FP32 data too), the multi-dot / multi-axpy of
// classical Gram-Schmidt, and the fused PCG updates whose scalars stay in
// device memory (no host round trip inside an iteration).
#include "sip_internal.h"

namespace sip {

namespace {

constexpr int kRedBlocks = 304;   // 2 x 152 SMs; fixed so sums are deterministic
constexpr int kRedThreads = 256;

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

// partial[blockIdx.y][blockIdx.x] = sum over the block's strided range of x_y . w
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_mdot_partial(size_t n, const T* __restrict__ V, size_t ldv,
                                                    const T* __restrict__ w, double* partial) {
    grid_dep_wait();
    const T* x = V + blockIdx.y * ldv;
    double acc = 0.0;
    for (size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n; g += size_t(gridDim.x) * blockDim.x)
        acc += double(x[g]) * double(w[g]);
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kRedThreads) k_final_sum(int parts, const double* partial, double* out) {
    grid_dep_wait();
    double acc = 0.0;
    for (int i = threadIdx.x; i < parts; i += blockDim.x) acc += partial[blockIdx.x * parts + i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

// w += sign * sum_i h_i V_i
template <typename T>
__global__ void k_maxpy(int m, size_t n, const T* __restrict__ V, size_t ldv, const double* __restrict__ h,
                        double sign, T* w) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= n) return;
    double acc = 0.0;
    for (int i = 0; i < m; ++i) acc += h[i] * double(V[i * ldv + g]);
    w[g] = T(double(w[g]) + sign * acc);
}

// y += alpha x, r -= alpha w with alpha = num / den (device scalars)
template <typename T>
__global__ void k_pcg_update(size_t n, const T* __restrict__ d, const T* __restrict__ q, T* y, T* r,
                             const double* num, const double* den) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const T a = T(*num / *den);
    y[g] += a * d[g];
    r[g] -= a * q[g];
}

// d = z + (num / den) d
template <typename T>
__global__ void k_pcg_dir(size_t n, const T* __restrict__ z, T* d, const double* num, const double* den) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= n) return;
    d[g] = z[g] + T(*num / *den) * d[g];
}

// v = v / sqrt(*s2) (the scale rounded to T, as a host-side axpby would)
template <typename T>
__global__ void k_scale_inv_sqrt(size_t n, const double* __restrict__ s2, T* v) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= n) return;
    v[g] = T(1.0 / sqrt(*s2)) * v[g];
}

template <typename T>
__global__ void k_axpby(size_t n, T a, const T* __restrict__ x, T b, T* y) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= n) return;
    y[g] = a * x[g] + (b == T(0) ? T(0) : b * y[g]);
}

// y = x * scale[i] (element-wise scale vector)
template <typename T>
__global__ void k_vmul(size_t n, const T* __restrict__ x, const T* __restrict__ s, T* y) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g < n) y[g] = x[g] * s[g];
}

template <typename Ti, typename To>
__global__ void k_cast(size_t n, const Ti* __restrict__ a, To* __restrict__ b) {
    grid_dep_wait();
    const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g < n) b[g] = To(a[g]);
}

// zero-mean projection of the constant pressure: subtract mean of p[e][0][0]
__global__ void k_sub_mode0(size_t ne, int mp, double* p, const double* sum) {
    grid_dep_wait();
    const size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < ne) p[e * mp] -= *sum / double(ne);
}

template <typename T>
__global__ void k_sum_mode0_partial(size_t ne, int mp, const T* __restrict__ p, double* partial) {
    grid_dep_wait();
    double acc = 0.0;
    for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < ne; e += size_t(gridDim.x) * blockDim.x)
        acc += double(p[e * mp]);
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

inline unsigned nblk(size_t n, int t = 256) { return unsigned((n + t - 1) / t); }

}  // namespace

size_t reduction_workspace_doubles(int max_vectors) { return size_t(kRedBlocks) * max_vectors; }

template <typename T>
void launch_mdot(int m, size_t n, const T* V, size_t ldv, const T* w, double* out, double* ws,
                 cudaStream_t s) {
    if (m <= 0) return;
    dim3 grid(kRedBlocks, m);
    launch_k(k_mdot_partial<T>, grid, kRedThreads, 0, s, n, V, ldv, w, ws);
    SIP_CHECK_LAUNCH();
    launch_k(k_final_sum, m, kRedThreads, 0, s, kRedBlocks, ws, out);
    SIP_CHECK_LAUNCH();
}

template <typename T>
void launch_dot(size_t n, const T* x, const T* y, double* out, double* ws, cudaStream_t s) {
    launch_mdot<T>(1, n, x, 0, y, out, ws, s);
}

template <typename T>
void launch_maxpy(int m, size_t n, const T* V, size_t ldv, const double* h, double sign, T* w,
                  cudaStream_t s) {
    if (m <= 0) return;
    launch_k(k_maxpy<T>, nblk(n), 256, 0, s, m, n, V, ldv, h, sign, w);
    SIP_CHECK_LAUNCH();
}

template <typename T>
void launch_pcg_update(size_t n, const T* d, const T* q, T* y, T* r, const double* num,
                       const double* den, cudaStream_t s) {
    launch_k(k_pcg_update<T>, nblk(n), 256, 0, s, n, d, q, y, r, num, den);
    SIP_CHECK_LAUNCH();
}

template <typename T>
void launch_pcg_dir(size_t n, const T* z, T* d, const double* num, const double* den,
                    cudaStream_t s) {
    launch_k(k_pcg_dir<T>, nblk(n), 256, 0, s, n, z, d, num, den);
    SIP_CHECK_LAUNCH();
}

template <typename T>
void launch_scale_inv_sqrt(size_t n, const double* s2, T* v, cudaStream_t s) {
    launch_k(k_scale_inv_sqrt<T>, nblk(n), 256, 0, s, n, s2, v);
    SIP_CHECK_LAUNCH();
}

template <typename T>
void launch_axpby(size_t n, T a, const T* x, T b, T* y, cudaStream_t s) {
    launch_k(k_axpby<T>, nblk(n), 256, 0, s, n, a, x, b, y);
    SIP_CHECK_LAUNCH();
}

template <typename T>
void launch_vmul(size_t n, const T* x, const T* sc, T* y, cudaStream_t s) {
    launch_k(k_vmul<T>, nblk(n), 256, 0, s, n, x, sc, y);
    SIP_CHECK_LAUNCH();
}

template <typename Ti, typename To>
void launch_cast(size_t n, const Ti* a, To* b, cudaStream_t s) {
    launch_k(k_cast<Ti, To>, nblk(n), 256, 0, s, n, a, b);
    SIP_CHECK_LAUNCH();
}

void launch_zero_mean_pressure(size_t ne, int mp, double* p, double* ws, cudaStream_t s) {
    launch_k(k_sum_mode0_partial<double>, kRedBlocks, kRedThreads, 0, s, ne, mp, p, ws);
    SIP_CHECK_LAUNCH();
    launch_k(k_final_sum, 1, kRedThreads, 0, s, kRedBlocks, ws, ws + kRedBlocks);
    SIP_CHECK_LAUNCH();
    launch_k(k_sub_mode0, nblk(ne), 256, 0, s, ne, mp, p, ws + kRedBlocks);
    SIP_CHECK_LAUNCH();
}

#define SIP_INST(T)                                                                              \
    template void launch_mdot<T>(int, size_t, const T*, size_t, const T*, double*, double*,     \
                                 cudaStream_t);                                                  \
    template void launch_dot<T>(size_t, const T*, const T*, double*, double*, cudaStream_t);    \
    template void launch_maxpy<T>(int, size_t, const T*, size_t, const double*, double, T*,     \
                                  cudaStream_t);                                                 \
    template void launch_pcg_update<T>(size_t, const T*, const T*, T*, T*, const double*,       \
                                       const double*, cudaStream_t);                             \
    template void launch_pcg_dir<T>(size_t, const T*, T*, const double*, const double*,         \
                                    cudaStream_t);                                               \
    template void launch_axpby<T>(size_t, T, const T*, T, T*, cudaStream_t);                    \
    template void launch_scale_inv_sqrt<T>(size_t, const double*, T*, cudaStream_t);             \
    template void launch_vmul<T>(size_t, const T*, const T*, T*, cudaStream_t);
SIP_INST(double)
SIP_INST(float)
#undef SIP_INST
template void launch_cast<double, float>(size_t, const double*, float*, cudaStream_t);
template void launch_cast<float, double>(size_t, const float*, double*, cudaStream_t);
template void launch_cast<double, double>(size_t, const double*, double*, cudaStream_t);

}  // namespace sip
