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

cudaError_t launch_instance_of(const int64_t* base, int32_t ni, int64_t n, int32_t* out, cudaStream_t s) {
    if (n <= 0 || ni <= 0) return cudaSuccess;
    k_instance_of<<<grid_for(n, 256), 256, 0, s>>>(base, ni, n, out);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace disco
