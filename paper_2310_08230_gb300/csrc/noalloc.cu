// disco_candidates_noalloc: the candidate mask of disco_candidates computed without
// allocating any memory, host or device.
//
// Who needs this: callers that must not allocate while they run — code that works inside
// a fixed device-memory budget handed out by another allocator (a framework's caching
// pool that owns all free memory, where a stray cudaMalloc can fail or fragment it),
// latency-critical loops where an allocation's implicit synchronisation is not
// acceptable, and callers that assemble work into a pre-planned memory layout. They pass
// device inputs and outputs; every temporary lives in one file-scope device array of fixed
// size that the library owns for the lifetime of the process.
//
// Limits (checked, DISCO_ERR_INVALID_ARG beyond them): at most kMaxVerts vertices and
// kMaxTris triangles per mesh, 1 <= k <= kMaxK. The array is kScratchInts int32 (about
// 3.75 MiB) and is held on every device that loads the library until the process exits.
//
// Sharing: every call on a device uses the same array, and it keeps the contents of the
// last call; whatever must start at zero is cleared by the call itself. Two calls whose
// GPU work overlaps (different streams, or different host threads on one device) race on
// the array and give undefined masks: serialise them.
//
// Set-up: the first call on a device resolves the array's device address with
// cudaGetSymbolAddress (with that device current) and caches it; make that first call
// before any stream capture. A cudaDeviceReset invalidates the cached address: after one,
// this entry point must not be called again in the same process.
#include <cfloat>
#include <mutex>

#include "../../include/disco.h"
#include "kernels.h"

namespace {

constexpr int kMaxVerts = 16384;
constexpr int kMaxTris = 32768;
constexpr int kMaxK = 32;
constexpr int kMaxDevices = 64;

// Layout (int32 units): top-k picks, then per mesh: triangles, incidence offsets,
// incidence list, fill cursors.
constexpr size_t kTopkInts = size_t(kMaxVerts) * kMaxK;
constexpr size_t kTriInts = size_t(kMaxTris) * 3;
constexpr size_t kPtrInts = size_t(kMaxVerts) + 64;  // nv + 1 offsets, padded to 256 bytes
constexpr size_t kIncInts = size_t(kMaxTris) * 3;
constexpr size_t kCurInts = size_t(kMaxVerts);
constexpr size_t kMeshInts = kTriInts + kPtrInts + kIncInts + kCurInts;
constexpr size_t kScratchInts = kTopkInts + 2 * kMeshInts;

static __device__ __align__(256) int32_t g_scratch[kScratchInts];

std::mutex g_mutex;
int32_t* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (resolved once per device).
int scratch_address(int32_t** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return DISCO_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return DISCO_ERR_CUDA;
        }
        g_addr[dev] = static_cast<int32_t*>(p);
    }
    *out = g_addr[dev];
    return DISCO_OK;
}

__global__ void k_count(const int32_t* __restrict__ T, int n3, int32_t* count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x) atomicAdd(count + T[i], 1);
}

// Exclusive prefix sum of count[0..n) into ptr[0..n], one block; cursor = ptr[0..n).
// count and cursor may be the same array: each thread reads its chunk before writing it.
__global__ void k_scan(const int32_t* count, int n, int32_t* ptr, int32_t* cursor) {
    __shared__ int32_t part[1024];
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(n, b + per);
    int32_t s = 0;
    for (int i = b; i < e; ++i) s += count[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t run = 0;
        for (int t = 0; t < int(blockDim.x); ++t) {
            const int32_t x = part[t];
            part[t] = run;
            run += x;
        }
        ptr[n] = run;
    }
    __syncthreads();
    int32_t run = part[threadIdx.x];
    for (int i = b; i < e; ++i) {
        const int32_t c = count[i];
        ptr[i] = run;
        cursor[i] = run;
        run += c;
    }
}

__global__ void k_fill(const int32_t* __restrict__ T, int nt, int32_t* cursor, int32_t* inc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * nt; i += gridDim.x * blockDim.x)
        inc[atomicAdd(cursor + T[i], 1)] = i / 3;
}

// k smallest entries of every column of d (ties to the lower row), one warp per column; the
// same rule as the row kernel (k_topk_rows): only finite entries are picked, a missing pick
// is written as -1.
__global__ void k_topk_cols(const float* __restrict__ d, int rows, int cols, int k, int32_t* __restrict__ idx) {
    const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (col >= cols) return;
    float pv = -FLT_MAX;
    int pi = -1;
    for (int t = 0; t < k; ++t) {
        float bv = FLT_MAX;
        int bi = 0x7fffffff;
        for (int r = lane; r < rows; r += 32) {
            const float x = d[size_t(r) * cols + col];
            const bool after = (x > pv) || (x == pv && r > pi);
            if (after && ((x < bv) || (x == bv && r < bi))) { bv = x; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if ((ov < bv) || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (lane == 0) idx[size_t(col) * k + t] = bi == 0x7fffffff ? -1 : bi;
        pv = bv;
        pi = bi;
    }
}

// For every pick c of row r: mark c and every vertex of every triangle incident to c
// (together: the closed 1-ring of c) on the other mesh.
__global__ void k_mark(const int32_t* __restrict__ topk, int rows, int k, const int32_t* __restrict__ ptr,
                       const int32_t* __restrict__ inc, const int32_t* __restrict__ T, int nvy, bool transposed,
                       uint8_t* allowed) {
    const int r = blockIdx.x;
    if (r >= rows) return;
    for (int t = threadIdx.y; t < k; t += blockDim.y) {
        const int c = topk[size_t(r) * k + t];
        if (c < 0) continue;  // fewer than k finite entries
        const size_t self = transposed ? size_t(c) * nvy + r : size_t(r) * nvy + c;
        if (threadIdx.x == 0) allowed[self] = 1;
        for (int j = ptr[c] + threadIdx.x; j < ptr[c + 1]; j += blockDim.x) {
            const int tri = inc[j];
            for (int q = 0; q < 3; ++q) {
                const int o = T[3 * tri + q];
                if (!transposed) allowed[size_t(r) * nvy + o] = 1;
                else allowed[size_t(o) * nvy + r] = 1;
            }
        }
    }
}

bool is_device(const void* p) {
    cudaPointerAttributes at;
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int disco_candidates_noalloc(const float* d, int32_t nvx, int32_t nvy, int32_t k, const disco_mesh* X,
                                        const disco_mesh* Y, uint8_t* allowed, void* stream) {
    if (!d || !allowed || !X || !Y || !X->T || !Y->T || X->nv != nvx || Y->nv != nvy || nvx < 1 || nvy < 1 ||
        X->nt < 1 || Y->nt < 1) {
        return DISCO_ERR_INVALID_ARG;
    }
    if (nvx > kMaxVerts || nvy > kMaxVerts || X->nt > kMaxTris || Y->nt > kMaxTris || k < 1 || k > kMaxK ||
        k > nvx || k > nvy) {
        return DISCO_ERR_INVALID_ARG;
    }
    for (const disco_mesh* m : {X, Y})
        for (int64_t i = 0; i < int64_t(m->nt) * 3; ++i)
            if (m->T[i] < 0 || m->T[i] >= m->nv) {
                return DISCO_ERR_INVALID_ARG;
            }
    if (!is_device(d) || !is_device(allowed)) {
        return DISCO_ERR_INVALID_ARG;
    }
    int32_t* base = nullptr;
    if (scratch_address(&base) != DISCO_OK) {
        return DISCO_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t* topk = base;
    int32_t* mesh[2] = {base + kTopkInts, base + kTopkInts + kMeshInts};
    const disco_mesh* ms[2] = {X, Y};
    cudaError_t e = cudaMemsetAsync(allowed, 0, size_t(nvx) * nvy, s);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        int32_t* T = mesh[i];
        int32_t* ptr = T + kTriInts;
        int32_t* inc = ptr + kPtrInts;
        int32_t* cur = inc + kIncInts;
        const int nv = ms[i]->nv, nt = ms[i]->nt;
        e = cudaMemcpyAsync(T, ms[i]->T, size_t(nt) * 3 * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(cur, 0, size_t(nv) * sizeof(int32_t), s);
        if (e == cudaSuccess) {
            k_count<<<(3 * nt + 255) / 256, 256, 0, s>>>(T, 3 * nt, cur);
            k_scan<<<1, 1024, 0, s>>>(cur, nv, ptr, cur);
            k_fill<<<(3 * nt + 255) / 256, 256, 0, s>>>(T, nt, cur, inc);
            disco::g_launches.fetch_add(3, std::memory_order_relaxed);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = disco::launch_topk_rows(d, nvx, nvy, k, topk, s);
    if (e == cudaSuccess) {
        const int32_t* TY = mesh[1];
        k_mark<<<nvx, dim3(8, 8), 0, s>>>(topk, nvx, k, TY + kTriInts, TY + kTriInts + kPtrInts, TY, nvy, false,
                                          allowed);
        k_topk_cols<<<(nvy + 7) / 8, 256, 0, s>>>(d, nvx, nvy, k, topk);
        const int32_t* TX = mesh[0];
        k_mark<<<nvy, dim3(8, 8), 0, s>>>(topk, nvy, k, TX + kTriInts, TX + kTriInts + kPtrInts, TX, nvy, true,
                                          allowed);
        disco::g_launches.fetch_add(3, std::memory_order_relaxed);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        return DISCO_ERR_CUDA;
    }
    return DISCO_OK;
}
