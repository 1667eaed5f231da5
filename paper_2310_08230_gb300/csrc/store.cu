// Device-side construction of the BDD store's tile layout (the slot arrays the half-pass
// kernels stream): the host uploads each instance's slot arrays in canonical order (segment
// by segment, layer by layer) and one record per segment; these kernels scatter the layers
// into the layer-major warp tiles.
#include "device_util.cuh"
#include "kernels.h"

namespace disco {
namespace {

// One thread per segment, in tile order: consecutive threads are the lanes of one tile, so
// every layer's stores of a warp fill one 128-byte line of each array.
__global__ void k_layout(const int64_t* __restrict__ seg_canon, const int32_t* __restrict__ seg_len,
                         const int64_t* __restrict__ seg_pos, const uint32_t* __restrict__ seg_vb, int64_t nseg,
                         const int32_t* __restrict__ cvar, const uint32_t* __restrict__ cdesc,
                         const float* __restrict__ clam, const float* __restrict__ clam_lo, uint32_t* __restrict__ var,
                         uint32_t* __restrict__ desc, float* __restrict__ lam, float* __restrict__ lam_lo,
                         int64_t* __restrict__ canon_pos) {
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < nseg; k += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c0 = seg_canon[k], p0 = seg_pos[k];
        const uint32_t vb = seg_vb[k];
        const int n = seg_len[k];
        for (int l = 0; l < n; ++l) {
            const int64_t c = c0 + l, p = p0 + int64_t(l) * 32;
            var[p] = vb + uint32_t(cvar[c]);
            desc[p] = cdesc[c];
            lam[p] = clam[c];
            lam_lo[p] = clam_lo[c];
            canon_pos[c] = p;
        }
    }
}

// out[v] = the instance whose variables [base[i], base[i + 1]) hold v.
__global__ void k_instance_of(const int64_t* __restrict__ base, int32_t ni, int64_t n, int32_t* __restrict__ out) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        int lo = 0, hi = ni - 1;  // the last i with base[i] <= v
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (base[mid] <= v) lo = mid;
            else hi = mid - 1;
        }
        out[v] = lo;
    }
}

__global__ void k_vpos(const uint32_t* __restrict__ var, const uint32_t* __restrict__ desc, int64_t n,
                       int32_t* __restrict__ vpos) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t v = var[i];
        if (v != kNoVar) vpos[size_t(v) * kAccStride + ((desc[i] >> 22) & 7u)] = int32_t(i);
    }
}

// One thread per variable: its deg slot masses in rank order, summed and divided in
// double-float exactly as the half-pass kernels form a deferred mean from a sector. The
// degree and the 32-byte position sector load together, and every mass gather issues before
// the sum, so a variable waits on two memory round trips, not 2 + deg.
__global__ void k_reduce(const int32_t* __restrict__ vpos, const float* __restrict__ m, const uint8_t* __restrict__ deg,
                         int64_t n, float2* __restrict__ pend) {
    using namespace dev;
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        const int4* qp = reinterpret_cast<const int4*>(vpos + size_t(v) * kAccStride);
        const int4 q0 = qp[0], q1 = qp[1];
        const int dg = deg[v];
        if (dg < 2) {  // every internal variable has 2 or more slots
            pend[v] = make_float2(0.0f, 0.0f);
            continue;
        }
        const int q[kAccStride] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
        float x[kAccStride];
#pragma unroll
        for (int r = 0; r < kAccStride; ++r) x[r] = r < dg ? m[q[r]] : 0.0f;
        df s = df_add_f(df{x[0], 0.0f}, x[1]);
#pragma unroll
        for (int r = 2; r < kAccStride; ++r)
            if (r < dg) s = df_add_f(s, x[r]);
        const df p = df_div_i(s, dg);
        pend[v] = make_float2(p.hi, p.lo);
    }
}

__global__ void k_scatter_back(const int32_t* __restrict__ vpos, const float* __restrict__ m,
                               const uint8_t* __restrict__ deg, int64_t n, float* __restrict__ acc) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x)
        for (int r = 0; r < deg[v]; ++r) acc[size_t(v) * kAccStride + r] = m[vpos[size_t(v) * kAccStride + r]];
}

inline unsigned grid_for(int64_t n, int block) {
    const int64_t g = (n + block - 1) / block;
    return unsigned(g < 1 ? 1 : (g > 152 * 64 ? 152 * 64 : g));
}

}  // namespace

cudaError_t launch_layout(const int64_t* seg_canon, const int32_t* seg_len, const int64_t* seg_pos,
                          const uint32_t* seg_vb, int64_t nseg, const int32_t* cvar, const uint32_t* cdesc,
                          const float* clam, const float* clam_lo, uint32_t* var, uint32_t* desc, float* lam,
                          float* lam_lo, int64_t* canon_pos, cudaStream_t s) {
    if (nseg <= 0) return cudaSuccess;
    k_layout<<<grid_for(nseg, 128), 128, 0, s>>>(seg_canon, seg_len, seg_pos, seg_vb, nseg, cvar, cdesc, clam, clam_lo,
                                                   var, desc, lam, lam_lo, canon_pos);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_vpos(const uint32_t* var, const uint32_t* desc, int64_t nslots, int32_t* vpos, cudaStream_t s) {
    if (nslots <= 0) return cudaSuccess;
    k_vpos<<<grid_for(nslots, 256), 256, 0, s>>>(var, desc, nslots, vpos);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const int32_t* vpos, const float* slot_mass, const uint8_t* deg, int64_t nint, float2* pend,
                          cudaStream_t s) {
    if (nint <= 0) return cudaSuccess;
    k_reduce<<<grid_for(nint, 256), 256, 0, s>>>(vpos, slot_mass, deg, nint, pend);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_scatter_back(const int32_t* vpos, const float* slot_mass, const uint8_t* deg, int64_t nint,
                                float* acc, cudaStream_t s) {
    if (nint <= 0) return cudaSuccess;
    k_scatter_back<<<grid_for(nint, 256), 256, 0, s>>>(vpos, slot_mass, deg, nint, acc);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_instance_of(const int64_t* base, int32_t ni, int64_t n, int32_t* out, cudaStream_t s) {
    if (n <= 0 || ni <= 0) return cudaSuccess;
    k_instance_of<<<grid_for(n, 256), 256, 0, s>>>(base, ni, n, out);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace disco
