// Vector kernels of the quasi-Newton step (Alg. 1 with Alg. 4-6) over the per-slot dual
// variables in tile layout (padding slots carry var = kNoVar and stay 0 in every vector).
//
// * subgradient (Alg. 1, first line): per slot 1 iff its min-marginal difference is
//   negative, i.e. every minimising assignment of the BDD sets the variable to 1 (App. A.5);
// * dot products in FP64 with per-block partial sums in a fixed order (the host adds the
//   partials in block order), so the L-BFGS scalars (Alg. 5) are deterministic;
// * dual-feasible projection (Alg. 1, third line): d^j_i -= mean over i's slots, through the
//   rank-indexed sectors the averaging uses (no atomics);
// * trial / step lambda + gamma d in double-float, like every other lambda update.
#include "device_util.cuh"
#include "kernels.h"

namespace disco {
namespace {

using namespace dev;

constexpr int kDotBlocks = 608;  // 4 per SM
constexpr int kDotThreads = 256;

inline unsigned grid_of(int64_t n) {
    const int64_t g = (n + 255) / 256;
    return unsigned(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

__global__ void k_sign(const float* __restrict__ mm, const uint32_t* __restrict__ var, int64_t n, float* __restrict__ g) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        g[i] = (var[i] != kNoVar && mm[i] < 0.0f) ? 1.0f : 0.0f;
}

__global__ void __launch_bounds__(kDotThreads) k_dot(const float* __restrict__ a, const float* __restrict__ b, int64_t n,
                                                     double* __restrict__ partial) {
    __shared__ double red[kDotThreads / 32];
    double x = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        x += double(a[i]) * double(b[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kDotThreads / 32; ++w) t += red[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void k_axpy(float* __restrict__ y, float a, const float* __restrict__ x, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] += a * x[i];
}

__global__ void k_scale(float* __restrict__ x, float a, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        x[i] *= a;
}

__global__ void k_sub(const float* __restrict__ a, const float* __restrict__ b, int64_t n, float* __restrict__ out) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = a[i] - b[i];
}

__global__ void k_to_table(const float* __restrict__ x, const uint32_t* __restrict__ var,
                           const uint32_t* __restrict__ desc, int64_t n, float* __restrict__ tab) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t v = var[i];
        if (v != kNoVar) tab[size_t(v) * kAccStride + decode(desc[i]).rank] = x[i];
    }
}

__global__ void k_sub_mean(float* __restrict__ x, const uint32_t* __restrict__ var, const uint32_t* __restrict__ desc,
                           int64_t n, const float* __restrict__ tab) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t v = var[i];
        if (v == kNoVar) continue;
        const int deg = decode(desc[i]).deg;
        float s = 0.0f;
        for (int r = 0; r < deg; ++r) s += tab[size_t(v) * kAccStride + r];
        x[i] -= s / float(deg);
    }
}

// out = lambda + gamma d (double-float); out may alias lambda.
__global__ void k_step(const float* lam, const float* lam_lo, const float* __restrict__ d, float gamma,
                       const uint32_t* __restrict__ var, int64_t n, float* out, float* out_lo) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        if (var[i] == kNoVar) continue;
        const df r = df_add_f(df{lam[i], lam_lo[i]}, gamma * d[i]);
        out[i] = r.hi;
        out_lo[i] = r.lo;
    }
}

// s = (lambda + pend) - old, in double-float, rounded to FP32.
__global__ void k_delta(const float* __restrict__ lam, const float* __restrict__ lam_lo,
                        const long long* __restrict__ msum, float inv, const float* __restrict__ old,
                        const float* __restrict__ old_lo, const uint32_t* __restrict__ var,
                        const uint32_t* __restrict__ desc, int64_t n, float* __restrict__ s) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t v = var[i];
        if (v == kNoVar) {
            s[i] = 0.0f;
            continue;
        }
        const df t = df_add(df{lam[i], lam_lo[i]}, fx_mean(msum[v], decode(desc[i]).deg, inv));
        const df r = df_add(t, df{-old[i], -old_lo[i]});
        s[i] = r.hi + r.lo;
    }
}

}  // namespace

cudaError_t launch_qn_sign(const float* mm, const uint32_t* var, int64_t n, float* g, cudaStream_t s) {
    k_sign<<<grid_of(n), 256, 0, s>>>(mm, var, n, g);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

int qn_dot_blocks() { return kDotBlocks; }

cudaError_t launch_qn_dot(const float* a, const float* b, int64_t n, double* partial, cudaStream_t s) {
    k_dot<<<kDotBlocks, kDotThreads, 0, s>>>(a, b, n, partial);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_qn_axpy(float* y, float a, const float* x, int64_t n, cudaStream_t s) {
    k_axpy<<<grid_of(n), 256, 0, s>>>(y, a, x, n);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_qn_scale(float* x, float a, int64_t n, cudaStream_t s) {
    k_scale<<<grid_of(n), 256, 0, s>>>(x, a, n);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_qn_sub(const float* a, const float* b, int64_t n, float* out, cudaStream_t s) {
    k_sub<<<grid_of(n), 256, 0, s>>>(a, b, n, out);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_qn_project(float* x, const uint32_t* var, const uint32_t* desc, int64_t n, float* tab,
                              cudaStream_t s) {
    k_to_table<<<grid_of(n), 256, 0, s>>>(x, var, desc, n, tab);
    k_sub_mean<<<grid_of(n), 256, 0, s>>>(x, var, desc, n, tab);
    g_launches.fetch_add(2, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_qn_step(const float* lam, const float* lam_lo, const float* d, float gamma, const uint32_t* var,
                           int64_t n, float* out, float* out_lo, cudaStream_t s) {
    k_step<<<grid_of(n), 256, 0, s>>>(lam, lam_lo, d, gamma, var, n, out, out_lo);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_qn_delta(const float* lam, const float* lam_lo, const long long* msum, float inv, const float* old,
                            const float* old_lo, const uint32_t* var, const uint32_t* desc, int64_t n, float* s_out,
                            cudaStream_t s) {
    k_delta<<<grid_of(n), 256, 0, s>>>(lam, lam_lo, msum, inv, old, old_lo, var, desc, n, s_out);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace disco
