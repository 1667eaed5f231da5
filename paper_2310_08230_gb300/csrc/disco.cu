// C ABI of the solver (include/disco.h): device store, pass scheduling, rounding loop.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <thread>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/disco.h"
#include "kernels.h"
#include "plan.h"

using namespace disco;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

#define CK(call)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? DISCO_ERR_OOM : DISCO_ERR_CUDA,                 \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                              \
    } while (0)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct WidthClass {
    int W;
    int tile0, tile_end;
};

// Stream-ordered device memory from one library pool per device that keeps freed memory
// (release threshold = max), so building and freeing many handles does not go back to the
// driver each time.
cudaError_t pool_for(int dev, cudaMemPool_t* out) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaError_t e = cudaMemPoolCreate(&pools[dev], &props);
        if (e != cudaSuccess) return e;
        uint64_t thr = UINT64_MAX;
        e = cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &thr);
        if (e != cudaSuccess) return e;
    }
    *out = pools[dev];
    return cudaSuccess;
}

int host_threads(const disco_opts& o) {
    return o.host_threads > 0 ? o.host_threads : int(std::max(1u, std::thread::hardware_concurrency()));
}

}  // namespace

struct disco_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // the width groups after the first run on `side`, concurrently with the first (a fork /
    // join per pass; captured into the iteration graphs as a parallel branch)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // averaging state (kernels.h, KArgs): three rotating buffers of one fixed-point sum per
    // variable. msum[phase] is the buffer the next update pass writes (all zero between
    // passes), msum[(phase + 2) % 3] holds the current state (the sums of the last update
    // pass: each variable's deferred mean is its sum / deg).
    long long* msum[3] = {nullptr, nullptr, nullptr};
    int phase = 0;
    FxScale fx{};
    uint32_t* status = nullptr;    // device status word (kStatus* bits)
    uint32_t* h_status = nullptr;  // pinned copy, read at synchronisation points
    disco_opts opts{};
    std::vector<Plan> plans;              // one per instance
    std::vector<int64_t> var_base;        // internal variable offset per instance (n + 1)
    std::vector<int64_t> slot_base;       // canonical slot offset per instance (n + 1)
    std::vector<int64_t> elem_base;       // matching-element offset per instance (n + 1)
    std::vector<int32_t> inst_tile_ptr;   // tiles of instance i: inst_tiles[ptr[i] .. ptr[i+1])
    std::vector<WidthClass> classes;
    int64_t ntiles = 0, nslots_tile = 0, nnodes_tile = 0, nint = 0;
    // device buffers
    TileInfo* tiles = nullptr;
    // locality tile order: the same tiles with the region blocks of each launch group in
    // reverse order, for the backward passes (they start where the forward pass ended, on
    // averaging sectors still in L2); null in the length order
    TileInfo* tiles_bwd = nullptr;
    uint32_t* var = nullptr;
    uint32_t* desc = nullptr;
    float* lam = nullptr;
    float* lam_lo = nullptr;
    float* lam0 = nullptr;         // lambda^0 (high / low), the start of disco_record
    float* lam0_lo = nullptr;
    float* F = nullptr;
    float* B = nullptr;
    double* tile_sum = nullptr;
    double* scalar = nullptr;      // per instance: lower bound
    double* consts = nullptr;      // per instance: presolve constant
    int32_t* d_inst_tile_ptr = nullptr;
    int32_t* d_inst_tiles = nullptr;
    int64_t* canon_pos = nullptr;  // canonical slot -> tile slot
    uint8_t* deg = nullptr;
    uint8_t* state = nullptr;
    uint8_t* trial = nullptr;
    uint32_t* reach = nullptr;
    uint8_t* sup = nullptr;
    float* mm_var = nullptr;
    float* mm_slot = nullptr;
    float* tmp = nullptr;          // nslots floats (canonical-order staging)
    int* counters = nullptr;       // 4 per instance
    int32_t* var_inst = nullptr;   // instance of every internal variable
    int* h_counters = nullptr;     // pinned, 4 per instance
    double* h_scalar = nullptr;    // pinned, one per instance
    int64_t device_bytes = 0;
    int64_t iterations = 0;
    double upload_ms = 0.0;
    int64_t n_inst() const { return int64_t(plans.size()); }
    int64_t nslots() const { return slot_base.back(); }
    int64_t nelems() const { return elem_base.back(); }
    bool has_b = false;
    std::vector<void*> allocations;
    int geometry = 2;              // warps per block of the fused MMA half-passes
    bool tuned = false;            // autotuner done (or off)
    // opts.graph_iters iterations, replayed as a block; one graph per averaging phase at which
    // it starts (the kernel arguments name the three sum buffers in rotation)
    cudaGraphExec_t iter_graph[3] = {nullptr, nullptr, nullptr};
    int64_t graph_launches[3] = {0, 0, 0};  // kernels in one replay
    bool graph_failed = false;     // the stream could not be captured: launch plainly
    // ---- differentiation (disco_record / disco_grad)
    struct Snap {  // the dual state at an iteration boundary, or the inputs of one half-pass
        float* lam = nullptr;
        float* lam_lo = nullptr;
        long long* msum = nullptr; // checkpoint: the averaging sums the next pass reads
        float2* pend = nullptr;    // tape: the deferred means the pass added (per variable)
        float* nodes = nullptr;    // checkpoint: node costs of the other direction; tape: the
                                   // node costs the pass stored (the next pass's input)
        int phase = 0;             // checkpoint: the averaging phase it was taken at
    };
    std::vector<Snap> checkpoints, tape;
    Snap final_state;
    int32_t rec_iters = -1, rec_every = 0;
    float* lbar = nullptr;         // adjoint per slot
    float* mub[2] = {nullptr, nullptr};  // adjoint sectors of the deferred means
    float* rbar = nullptr;         // per variable: adjoint of each removed mass (from mub)
    float2* pend_tmp = nullptr;    // per variable: deferred means of a checkpoint or the final state
    float* Fbar = nullptr;         // adjoints of the stored node costs
    float* Bbar = nullptr;
    float* cbar = nullptr;         // adjoint per internal variable
    // ---- quasi-Newton steps (Alg. 1 with Alg. 4-6)
    int qn_m = 0;                  // L-BFGS memory
    float* qn_g = nullptr;         // subgradient at the start of a call
    float* qn_g2 = nullptr;        // subgradient after its MMA iterations
    float* qn_d = nullptr;         // direction
    float* qn_old = nullptr;       // lambda at the start of a call (high / low)
    float* qn_old_lo = nullptr;
    float* qn_tr = nullptr;        // trial lambda + gamma d
    float* qn_tr_lo = nullptr;
    float* qn_tab = nullptr;       // rank sectors for the projection
    std::vector<float*> qn_S, qn_Y;  // m + 1 buffers; qn_order lists the stored pairs, oldest first
    std::vector<int> qn_order;
    std::vector<double> qn_sy, qn_yy;
    int qn_spare = 0;
    double* qn_part = nullptr;     // per-block dot partials (device) and their pinned copy
    double* qn_hpart = nullptr;
    double qn_gamma = 1e-3, qn_dmin = 0.0, qn_Estart = 0.0;
    int64_t qn_calls = 0;

    template <class T>
    int alloc(T** p, int64_t n) {
        size_t bytes = size_t(std::max<int64_t>(n, 1)) * sizeof(T);
        cudaMemPool_t pool;
        cudaError_t e = pool_for(device, &pool);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), bytes, pool, stream);
        if (e != cudaSuccess) return fail(DISCO_ERR_OOM, std::string("device allocation: ") + cudaGetErrorString(e));
        allocations.push_back(*p);
        device_bytes += int64_t(bytes);
        return DISCO_OK;
    }

    long long* msum_rd() const { return msum[(phase + 2) % 3]; }

    KArgs args(const WidthClass& c, bool backward = false) {
        KArgs a{};
        a.tiles = backward && tiles_bwd ? tiles_bwd : tiles;
        a.tile0 = c.tile0;
        a.tile_end = c.tile_end;
        a.var = var;
        a.desc = desc;
        a.lam = lam;
        a.lam_lo = lam_lo;
        a.F = F;
        a.B = B;
        a.msum_rd = msum[(phase + 2) % 3];
        a.msum_wr = msum[phase];
        a.msum_zero = msum[(phase + 1) % 3];
        a.fx = fx;
        a.status = status;
        a.nslots = nslots_tile;
        a.nnodes = nnodes_tile;
        a.nvars = nint;
        a.state = state;
        a.omega = opts.omega;
        a.mm_slot = mm_slot;
        a.mm_var = mm_var;
        a.tile_sum = tile_sum;
        a.reach = reach;
        a.sup_var = sup;
        return a;
    }

    // One pass over every width class (an update pass moves the averaging phase on). The
    // groups touch disjoint tiles, slots and per-variable entries and share only commuting
    // integer atomics, so they run concurrently and the results do not depend on it.
    int pass(Pass p) {
        const bool bwd = p == Pass::BwdMMA || p == Pass::BwdMMARound || p == Pass::BwdMM || p == Pass::BwdReset;
        if (classes.size() > 1 && side) {
            CK(cudaEventRecord(ev_fork, stream));
            CK(cudaStreamWaitEvent(side, ev_fork, 0));
            CK(launch_pass(p, classes[0].W, args(classes[0], bwd), stream, geometry));
            for (size_t c = 1; c < classes.size(); ++c) CK(launch_pass(p, classes[c].W, args(classes[c], bwd), side, geometry));
            CK(cudaEventRecord(ev_join, side));
            CK(cudaStreamWaitEvent(stream, ev_join, 0));
        } else {
            for (const WidthClass& c : classes) CK(launch_pass(p, c.W, args(c, bwd), stream, geometry));
        }
        if (p == Pass::FwdMMA || p == Pass::BwdMMA || p == Pass::FwdMMARound || p == Pass::BwdMMARound)
            phase = (phase + 1) % 3;
        return DISCO_OK;
    }

    // The averaging state set to "no deferred mass": every sum zero.
    int clear_sums() {
        for (long long* m : msum) CK(cudaMemsetAsync(m, 0, size_t(nint) * sizeof(long long), stream));
        return DISCO_OK;
    }

    // Queues a copy of the device status word to h_status on the handle's stream;
    // check_status() reads it once the stream has been synchronised and turns a set bit into
    // an error. The word is then cleared, so that the handle stays usable.
    int fetch_status() {
        CK(cudaMemcpyAsync(h_status, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
        return DISCO_OK;
    }
    int check_status() {
        const uint32_t st = *h_status;
        if (!st) return DISCO_OK;
        *h_status = 0;
        CK(cudaMemsetAsync(status, 0, sizeof(uint32_t), stream));
        if (st & kStatusBounds)
            return fail(DISCO_ERR_INTERNAL, "bounds check: a kernel index fell outside its array (access skipped)");
        return fail(DISCO_ERR_RANGE, "a removed mass left the fixed-point range of the averaging sums (costs too "
                                     "large for normalize_costs = 0, or the dual diverged)");
    }

    ~disco_handle() {
        for (cudaGraphExec_t g : iter_graph)
            if (g) cudaGraphExecDestroy(g);
        for (void* p : allocations) cudaFreeAsync(p, stream);
        if (stream) cudaStreamSynchronize(stream);
        if (h_counters) cudaFreeHost(h_counters);
        if (h_scalar) cudaFreeHost(h_scalar);
        if (h_status) cudaFreeHost(h_status);
        if (side) {
            cudaStreamSynchronize(side);
            cudaStreamDestroy(side);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (qn_hpart) cudaFreeHost(qn_hpart);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

int copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
    return DISCO_OK;
}

// Reads n elements of a host-or-device array into a host vector.
template <class T>
int to_host(const T* src, size_t n, pod_vector<T>* out) {
    out->resize(n);  // no zero fill: the copy writes every element
    if (is_device_ptr(src)) {
        CK(cudaMemcpy(out->data(), src, n * sizeof(T), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(out->data(), src, n * sizeof(T));
    }
    return DISCO_OK;
}

// Register widths of the tile classes: a segment goes to the narrowest class that holds its
// widest layer (per-layer work grows with the class width, not with the layer's width).
constexpr int kWidthClasses[] = {2, 4, 6, 8, 16, 32};

// The fused kernels instantiate widths 2, 4 and 6; launch_pass has 8, 16 and 32.
constexpr bool classes_have_kernels() {
    for (int c : kWidthClasses)
        if (c != 2 && c != 4 && c != 6 && c != 8 && c != 16 && c != 32) return false;
    return true;
}
static_assert(classes_have_kernels(), "every width class needs a kernel instantiation");

// Tile order for table locality (opts.tile_order == 2, see upload): segments per block.
constexpr int64_t kLocalityBlock = 4096;

int width_class(int w) {
    for (int c : kWidthClasses)
        if (w <= c) return c;
    return kMaxWidth;
}

int upload(disco_handle* h) {
    Trace tr;
    tr.scope = "upload";
    const int64_t ni = h->n_inst();
    const int nth = host_threads(h->opts);
    h->var_base.assign(size_t(ni) + 1, 0);
    h->slot_base.assign(size_t(ni) + 1, 0);
    h->elem_base.assign(size_t(ni) + 1, 0);
    for (int64_t i = 0; i < ni; ++i) {
        const Plan& P = h->plans[i];
        h->var_base[i + 1] = h->var_base[i] + P.n_free + P.n_aux;
        h->slot_base[i + 1] = h->slot_base[i] + int64_t(P.slot_var.size());
        h->elem_base[i + 1] = h->elem_base[i] + P.nvars;
    }
    h->nint = h->var_base[ni];
    if (h->nint >= (int64_t(1) << 32) - 1) return fail(DISCO_ERR_INVALID_ARG, "build: too many variables");
    // Every internal variable lies in 2 to 7 BDD segments: the descriptor holds the degree in
    // 3 bits, and a variable in one segment would have been fixed by the presolve (a row with
    // one free variable forces it). The deferred mean divides by it.
    for (int64_t i = 0; i < ni; ++i) {
        uint8_t lo = 255, hi = 0;  // a min / max reduction (vectorised), then the message
        for (uint8_t dg : h->plans[i].deg) {
            lo = std::min(lo, dg);
            hi = std::max(hi, dg);
        }
        if (!h->plans[i].deg.empty() && (lo < 2 || hi > 7))
            return fail(DISCO_ERR_INVALID_ARG, "build: an internal variable lies in " + std::to_string(int(lo < 2 ? lo : hi)) +
                                                   " segments (2 to 7 expected)");
    }
    // Fixed-point grid of the averaging sums: 2^-F with 2^(32 - F) >= the largest |cost| (at
    // least 2^-20), so one mass may reach 2^10 times the largest cost before the kernels flag
    // it (the sums stay below 2^45 grid units), and the grid is about 2e-10 of the largest cost.
    {
        double cmax = 0.0;  // the compiler's largest element cost of each instance (costs are >= 0)
        for (int64_t i = 0; i < ni; ++i) cmax = std::max(cmax, h->plans[i].cost_max);
        int e = 0;
        std::frexp(std::max(cmax, std::ldexp(1.0, -20)), &e);  // cmax < 2^e
        e = std::min(e, 100);  // 2^F and 2^(42 - F) stay normal FP32 numbers
        const int F = 32 - e;
        h->fx = FxScale{std::ldexp(1.0f, F), std::ldexp(1.0f, -F), std::ldexp(1.0f, 42 - F)};
    }
    tr.mark("degrees, grid");
    // ---- tiles: per instance, segments grouped by width class, longest first; a tile never
    // mixes instances (its bound sum belongs to one instance). Counting sorts by (class,
    // length), then the tiles by (launch group, length): both stable.
    struct TileSeg {
        int32_t inst;
        int64_t seg;
    };
    auto class_index = [](int W) { return W; };  // classes are at most 32 wide
    std::vector<TileInfo> tiles;
    std::vector<int64_t> tile_first;  // first entry of the tile's segments in `order`
    std::vector<int32_t> tile_count, tile_inst;
    std::vector<int64_t> tile_block;  // locality order: each tile's block (global id)
    std::vector<TileSeg> order;
    int maxL = 1;
    for (int64_t i = 0; i < ni; ++i) maxL = std::max(maxL, h->plans[i].max_layers);
    // Locality order (opts.tile_order == 2): segments are ordered by the region of their row (closedness rows by the
    // X vertex of their bucket, X projection rows beside their triangle's smallest vertex, Y
    // projection rows last), cut into blocks of kLocalityBlock, each block sorted by width
    // class and length, and tiles follow the blocks: the warps running together then hold
    // most of the slots of the variables they touch. It served half-passes that gathered and
    // scattered whole per-variable sectors; with 8-byte per-variable means they run faster in
    // the default order, by width class and length over the whole instance. Instances are ordered in
    // parallel, then concatenated in instance order.
    const bool locality = h->opts.tile_order == 2;
    auto launch_group = [](int W) { return W <= kFusedMaxW ? 0 : W <= 8 ? 1 : W <= 16 ? 2 : 3; };
    struct InstTiles {
        std::vector<int64_t> seg;  // the instance's segments in tile order
        std::vector<TileInfo> tiles;
        std::vector<int64_t> first;  // into seg
        std::vector<int32_t> count;
        std::vector<int32_t> block;  // locality order: the block each tile belongs to
    };
    std::vector<InstTiles> per(static_cast<size_t>(ni));
    parallel_tasks(ni, nth, [&](int64_t i) {
        const Plan& P = h->plans[i];
        InstTiles& R = per[size_t(i)];
        const int64_t nseg = int64_t(P.segs.size());
        R.seg.resize(size_t(nseg));
        auto cut_tiles = [&](int64_t k0, int64_t k1) {  // tiles of one run; none straddles a class
            for (int64_t k = k0; k < k1;) {
                const int W = width_class(P.segs[R.seg[k]].max_width);
                const int L = P.segs[R.seg[k]].n_layers;
                const int64_t first = k;
                int q = 0;
                while (q < 32 && k < k1 && width_class(P.segs[R.seg[k]].max_width) == W) ++q, ++k;
                R.tiles.push_back(TileInfo{0, 0, L, W});
                R.first.push_back(first);
                R.count.push_back(q);
            }
        };
        if (locality) {
            // stable counting sort by (launch group, region of the segment's row), so that the
            // closedness and X projection rows of one X neighbourhood are adjacent
            const int64_t nreg = int64_t(P.nvx) + P.n_projy;
            std::vector<int64_t> rcnt(size_t(4 * nreg) + 1, 0);
            auto rkey = [&](const Segment& sg) {
                return size_t(launch_group(width_class(sg.max_width))) * size_t(nreg) + size_t(P.row_region[size_t(sg.row)]);
            };
            for (const Segment& sg : P.segs) ++rcnt[rkey(sg) + 1];
            for (size_t q = 1; q < rcnt.size(); ++q) rcnt[q] += rcnt[q - 1];
            int64_t gstart[5];
            for (int g = 0; g <= 4; ++g) gstart[g] = rcnt[size_t(g) * size_t(nreg)];
            for (int64_t k = 0; k < nseg; ++k) R.seg[size_t(rcnt[rkey(P.segs[k])]++)] = k;
            std::vector<uint64_t> key;
            int32_t nblk = 0;
            for (int g = 0; g < 4; ++g)
                for (int64_t b0 = gstart[g]; b0 < gstart[g + 1]; b0 += kLocalityBlock) {
                    const int64_t b1 = std::min(gstart[g + 1], b0 + kLocalityBlock);
                    // (class, length descending, position): unique keys, so the order is fixed
                    key.resize(size_t(b1 - b0));
                    for (int64_t k = b0; k < b1; ++k) {
                        const Segment& sg = P.segs[R.seg[k]];
                        key[size_t(k - b0)] = uint64_t(width_class(sg.max_width)) << 48 |
                                              uint64_t(maxL - sg.n_layers) << 24 | uint64_t(k - b0);
                    }
                    std::sort(key.begin(), key.end());
                    std::vector<int64_t> tmp(R.seg.begin() + b0, R.seg.begin() + b1);
                    for (int64_t k = b0; k < b1; ++k) R.seg[k] = tmp[size_t(key[size_t(k - b0)] & 0xFFFFFFu)];
                    const size_t t_before = R.tiles.size();
                    cut_tiles(b0, b1);  // tiles never straddle a block
                    R.block.resize(R.tiles.size());
                    for (size_t t = t_before; t < R.tiles.size(); ++t) R.block[t] = nblk;
                    ++nblk;
                }
        } else {
            // stable counting sort by (class ascending, length descending): per-chunk counts,
            // offsets in (key, chunk) order, scatter; chunks in parallel for a single instance
            // (a batch orders its instances in parallel instead)
            const size_t nkey = size_t(kMaxWidth + 1) * (maxL + 1);
            const int nch = ni > 1 ? 1 : std::max(1, std::min<int>(nth, int(nseg / 16384) + 1));
            std::vector<uint32_t> key(static_cast<size_t>(nseg));
            std::vector<std::vector<int64_t>> cnt(size_t(nch), std::vector<int64_t>(nkey, 0));
            parallel_chunks(nseg, nch, [&](int c, int64_t k0, int64_t k1) {
                for (int64_t k = k0; k < k1; ++k) {
                    const Segment& sg = P.segs[k];
                    key[size_t(k)] = uint32_t(size_t(class_index(width_class(sg.max_width))) * (maxL + 1) +
                                              size_t(maxL - sg.n_layers));
                    ++cnt[size_t(c)][key[size_t(k)]];
                }
            });
            int64_t run = 0;
            for (size_t b = 0; b < nkey; ++b)
                for (int c = 0; c < nch; ++c) {
                    const int64_t x = cnt[size_t(c)][b];
                    cnt[size_t(c)][b] = run;
                    run += x;
                }
            // the keys travel with the segments, so that the tiles are cut from them in order
            std::vector<uint32_t> skey(static_cast<size_t>(nseg));
            parallel_chunks(nseg, nch, [&](int c, int64_t k0, int64_t k1) {
                for (int64_t k = k0; k < k1; ++k) {
                    const int64_t pos = cnt[size_t(c)][key[size_t(k)]]++;
                    R.seg[size_t(pos)] = k;
                    skey[size_t(pos)] = key[size_t(k)];
                }
            });
            const uint32_t kl = uint32_t(maxL + 1);  // key = class * (maxL + 1) + maxL - length
            for (int64_t k = 0; k < nseg;) {
                const uint32_t W = skey[size_t(k)] / kl;
                const int L = maxL - int(skey[size_t(k)] % kl);
                const int64_t first = k;
                int q = 0;
                while (q < 32 && k < nseg && skey[size_t(k)] / kl == W) ++q, ++k;
                R.tiles.push_back(TileInfo{0, 0, L, int(W)});
                R.first.push_back(first);
                R.count.push_back(q);
            }
        }
    });
    {
        std::vector<int64_t> soff(size_t(ni) + 1, 0), toff(size_t(ni) + 1, 0);
        for (int64_t i = 0; i < ni; ++i) {
            soff[size_t(i) + 1] = soff[size_t(i)] + int64_t(per[size_t(i)].seg.size());
            toff[size_t(i) + 1] = toff[size_t(i)] + int64_t(per[size_t(i)].tiles.size());
        }
        order.resize(size_t(soff[size_t(ni)]));
        tiles.resize(size_t(toff[size_t(ni)]));
        tile_first.resize(tiles.size());
        tile_count.resize(tiles.size());
        tile_inst.resize(tiles.size());
        if (locality) tile_block.resize(tiles.size());
        std::vector<int64_t> boff(size_t(ni) + 1, 0);  // global block ids: instance by instance
        for (int64_t i = 0; i < ni; ++i)
            boff[size_t(i) + 1] = boff[size_t(i)] + (per[size_t(i)].block.empty() ? 0 : per[size_t(i)].block.back() + 1);
        parallel_tasks(ni, nth, [&](int64_t i) {
            InstTiles& R = per[size_t(i)];
            const int64_t so = soff[size_t(i)], to = toff[size_t(i)];
            for (size_t k = 0; k < R.seg.size(); ++k) order[size_t(so) + k] = TileSeg{int32_t(i), R.seg[k]};
            for (size_t t = 0; t < R.tiles.size(); ++t) {
                tiles[size_t(to) + t] = R.tiles[t];
                tile_first[size_t(to) + t] = so + R.first[t];
                tile_count[size_t(to) + t] = R.count[t];
                tile_inst[size_t(to) + t] = int32_t(i);
                if (locality) tile_block[size_t(to) + t] = boff[size_t(i)] + R.block[t];
            }
            InstTiles().seg.swap(R.seg);
        });
    }
    // classes up to kFusedMaxW share one launch, longest tiles first; wider ones launch on their own
    {
        // inside a launch group, pair by pair: the warps running at any moment then touch the
        // averaging tables of one or two pairs (L2-resident) instead of all of them; a pair's
        // tiles keep their order, longest first
        // (in locality order the blocks keep their order: the key has no length part)
        const size_t nlen = locality ? 1 : size_t(maxL + 1);
        std::vector<int64_t> cnt(size_t(4) * size_t(ni) * nlen + 1, 0);
        std::vector<size_t> perm(tiles.size());
        auto key = [&](size_t t) {
            return (size_t(launch_group(tiles[t].W)) * size_t(ni) + size_t(tile_inst[t])) * nlen +
                   (locality ? 0 : size_t(maxL - tiles[t].L));
        };
        for (size_t t = 0; t < tiles.size(); ++t) ++cnt[key(t) + 1];
        for (size_t k = 1; k < cnt.size(); ++k) cnt[k] += cnt[k - 1];
        for (size_t t = 0; t < tiles.size(); ++t) perm[size_t(cnt[key(t)]++)] = t;
        std::vector<TileInfo> t2(tiles.size());
        std::vector<int64_t> f2(tiles.size()), b2(tile_block.size());
        std::vector<int32_t> c2(tiles.size()), i2(tiles.size());
        for (size_t k = 0; k < perm.size(); ++k) {
            t2[k] = tiles[perm[k]];
            f2[k] = tile_first[perm[k]];
            c2[k] = tile_count[perm[k]];
            i2[k] = tile_inst[perm[k]];
            if (locality) b2[k] = tile_block[perm[k]];
        }
        tiles.swap(t2);
        tile_first.swap(f2);
        tile_count.swap(c2);
        tile_inst.swap(i2);
        tile_block.swap(b2);
    }
    tr.mark("tile sort");
    h->classes.clear();
    int64_t slot_base = 0, node_base = 0;
    for (size_t t = 0; t < tiles.size(); ++t) {
        const int group = tiles[t].W <= kFusedMaxW ? 0 : tiles[t].W;
        if (h->classes.empty() || h->classes.back().W != group) h->classes.push_back(WidthClass{group, int(t), int(t)});
        h->classes.back().tile_end = int(t) + 1;
        tiles[t].slot_base = slot_base;
        tiles[t].node_base = node_base;
        slot_base += int64_t(tiles[t].L) * 32;
        node_base += int64_t(tiles[t].L + 1) * tiles[t].W * 32;
    }
    h->ntiles = int64_t(tiles.size());
    h->nslots_tile = slot_base;
    h->nnodes_tile = node_base;
    if (h->classes.size() > 1) {
        CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    }
    // backward order (locality only): inside each launch group, the runs of tiles of one block
    // in reverse order, each run's tiles (longest first) kept in order
    std::vector<TileInfo> tiles_bwd;
    if (locality) {
        tiles_bwd.reserve(tiles.size());
        for (const WidthClass& c : h->classes) {
            std::vector<std::pair<int, int>> runs;  // [begin, end) of each block's tiles
            for (int t = c.tile0; t < c.tile_end;) {
                int u = t + 1;
                while (u < c.tile_end && tile_block[size_t(u)] == tile_block[size_t(t)]) ++u;
                runs.emplace_back(t, u);
                t = u;
            }
            for (size_t r = runs.size(); r-- > 0;)
                for (int t = runs[r].first; t < runs[r].second; ++t) tiles_bwd.push_back(tiles[size_t(t)]);
        }
    }
    // tiles of each instance, in tile order (the bound sums them in this fixed order)
    h->inst_tile_ptr.assign(size_t(ni) + 1, 0);
    for (int32_t i : tile_inst) ++h->inst_tile_ptr[i + 1];
    for (int64_t i = 0; i < ni; ++i) h->inst_tile_ptr[i + 1] += h->inst_tile_ptr[i];
    std::vector<int32_t> inst_tiles(tiles.size());
    {
        std::vector<int32_t> pos(h->inst_tile_ptr.begin(), h->inst_tile_ptr.end() - 1);
        for (size_t t = 0; t < tiles.size(); ++t) inst_tiles[pos[tile_inst[t]]++] = int32_t(t);
    }
    const int64_t nslots = h->nslots();
    tr.mark("tile order");

    // one record per segment in tile order (canonical first slot, layers, tile slot, first
    // variable of its instance); the kernel k_layout scatters the canonical slot arrays
    const int64_t nseg_all = int64_t(order.size());
    pod_vector<int64_t> seg_canon(static_cast<size_t>(nseg_all)), seg_pos(static_cast<size_t>(nseg_all));
    pod_vector<int32_t> seg_len(static_cast<size_t>(nseg_all));
    pod_vector<uint32_t> seg_vb(static_cast<size_t>(nseg_all));
    parallel_chunks(int64_t(tiles.size()), nth, [&](int, int64_t t0, int64_t t1) {
        for (int64_t t = t0; t < t1; ++t)
            for (int lane = 0; lane < tile_count[t]; ++lane) {
                const int64_t k = tile_first[t] + lane;
                const TileSeg& ts = order[size_t(k)];
                const Segment& sg = h->plans[ts.inst].segs[ts.seg];
                seg_canon[k] = h->slot_base[ts.inst] + sg.first_slot;
                seg_len[k] = sg.n_layers;
                seg_pos[k] = tiles[t].slot_base + lane;
                seg_vb[k] = uint32_t(h->var_base[ts.inst]);
            }
    });
    std::vector<double> consts(static_cast<size_t>(ni));
    for (int64_t i = 0; i < ni; ++i) consts[i] = h->plans[i].constant;
    tr.mark("tile layout");
    int rc;
    if ((rc = h->alloc(&h->tiles, h->ntiles))) return rc;
    for (long long*& m : h->msum)
        if ((rc = h->alloc(&m, h->nint))) return rc;
    if ((rc = h->alloc(&h->status, 1))) return rc;
    if (locality && (rc = h->alloc(&h->tiles_bwd, h->ntiles))) return rc;
    if ((rc = h->alloc(&h->var, slot_base))) return rc;
    if ((rc = h->alloc(&h->desc, slot_base))) return rc;
    if ((rc = h->alloc(&h->lam, slot_base))) return rc;
    if ((rc = h->alloc(&h->lam_lo, slot_base))) return rc;
    if ((rc = h->alloc(&h->lam0, slot_base))) return rc;
    if ((rc = h->alloc(&h->lam0_lo, slot_base))) return rc;
    if ((rc = h->alloc(&h->F, node_base))) return rc;
    if ((rc = h->alloc(&h->B, node_base))) return rc;
    if ((rc = h->alloc(&h->tile_sum, h->ntiles))) return rc;
    if ((rc = h->alloc(&h->scalar, ni))) return rc;
    if ((rc = h->alloc(&h->consts, ni))) return rc;
    if ((rc = h->alloc(&h->d_inst_tile_ptr, ni + 1))) return rc;
    if ((rc = h->alloc(&h->d_inst_tiles, h->ntiles))) return rc;
    if ((rc = h->alloc(&h->canon_pos, nslots))) return rc;
    if ((rc = h->alloc(&h->deg, h->nint))) return rc;
    if ((rc = h->alloc(&h->state, h->nint))) return rc;
    if ((rc = h->alloc(&h->trial, h->nint))) return rc;
    if ((rc = h->alloc(&h->reach, slot_base))) return rc;
    if ((rc = h->alloc(&h->sup, h->nint * kAccStride))) return rc;
    if ((rc = h->alloc(&h->mm_var, h->nint * kAccStride))) return rc;
    if ((rc = h->alloc(&h->mm_slot, slot_base))) return rc;
    if ((rc = h->alloc(&h->tmp, std::max(nslots, h->nint)))) return rc;
    if ((rc = h->alloc(&h->counters, 4 * ni))) return rc;
    if ((rc = h->alloc(&h->var_inst, h->nint))) return rc;
    CK(cudaMallocHost(&h->h_counters, size_t(4 * std::max<int64_t>(ni, 1)) * sizeof(int)));
    CK(cudaMallocHost(&h->h_scalar, size_t(std::max<int64_t>(ni, 1)) * sizeof(double)));
    CK(cudaMallocHost(&h->h_status, sizeof(uint32_t)));
    *h->h_status = 0;
    tr.mark("allocations");
    cudaStream_t s = h->stream;
    // temporaries: canonical slot arrays, segment records, instance variable bases
    const size_t b_slots = size_t(nslots) * 4, b_segs = size_t(nseg_all) * 8, b_segs4 = size_t(nseg_all) * 4;
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t b_tmp = 4 * up(b_slots) + 2 * up(b_segs) + 2 * up(b_segs4) + up(size_t(ni + 1) * 8);
    char* tmp = nullptr;
    {
        cudaMemPool_t pool;
        cudaError_t e = pool_for(h->device, &pool);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&tmp), std::max<size_t>(b_tmp, 256), pool, s);
        if (e != cudaSuccess) return fail(DISCO_ERR_OOM, std::string("device allocation: ") + cudaGetErrorString(e));
    }
    char* q = tmp;
    auto carve = [&](size_t b) { char* r = q; q += up(b); return r; };
    int32_t* cvar = reinterpret_cast<int32_t*>(carve(b_slots));
    uint32_t* cdesc = reinterpret_cast<uint32_t*>(carve(b_slots));
    float* clam = reinterpret_cast<float*>(carve(b_slots));
    float* clam_lo = reinterpret_cast<float*>(carve(b_slots));
    int64_t* d_seg_canon = reinterpret_cast<int64_t*>(carve(b_segs));
    int64_t* d_seg_pos = reinterpret_cast<int64_t*>(carve(b_segs));
    int32_t* d_seg_len = reinterpret_cast<int32_t*>(carve(b_segs4));
    uint32_t* d_seg_vb = reinterpret_cast<uint32_t*>(carve(b_segs4));
    int64_t* d_var_base = reinterpret_cast<int64_t*>(carve(size_t(ni + 1) * 8));
    struct Release {  // the temporaries go back to the pool on every exit (stream-ordered)
        char* p;
        cudaStream_t s;
        ~Release() { cudaFreeAsync(p, s); }
    } release_tmp{tmp, s};
    rc = DISCO_OK;
    for (int64_t i = 0; i < ni && !rc; ++i) {
        const Plan& P = h->plans[i];
        const int64_t o = h->slot_base[i], n = int64_t(P.slot_var.size());
        (rc = copy_in(cvar + o, P.slot_var.data(), size_t(n) * 4, s)) || (rc = copy_in(cdesc + o, P.slot_desc.data(), size_t(n) * 4, s)) ||
            (rc = copy_in(clam + o, P.slot_lam0.data(), size_t(n) * 4, s)) ||
            (rc = copy_in(clam_lo + o, P.slot_lam0_lo.data(), size_t(n) * 4, s)) ||
            (rc = copy_in(h->deg + h->var_base[i], P.deg.data(), P.deg.size(), s));
    }
    if (!rc) {
        (rc = copy_in(d_seg_canon, seg_canon.data(), b_segs, s)) || (rc = copy_in(d_seg_pos, seg_pos.data(), b_segs, s)) ||
            (rc = copy_in(d_seg_len, seg_len.data(), b_segs4, s)) || (rc = copy_in(d_seg_vb, seg_vb.data(), b_segs4, s)) ||
            (rc = copy_in(d_var_base, h->var_base.data(), size_t(ni + 1) * 8, s)) ||
            (rc = copy_in(h->tiles, tiles.data(), tiles.size() * sizeof(TileInfo), s)) ||
            (locality && (rc = copy_in(h->tiles_bwd, tiles_bwd.data(), tiles_bwd.size() * sizeof(TileInfo), s)));
    }
    if (rc) return rc;
    // padding lanes and layers: no variable, zero descriptor and lambda
    CK(cudaMemsetAsync(h->var, 0xFF, size_t(slot_base) * 4, s));
    CK(cudaMemsetAsync(h->desc, 0, size_t(slot_base) * 4, s));
    CK(cudaMemsetAsync(h->lam, 0, size_t(slot_base) * 4, s));
    CK(cudaMemsetAsync(h->lam_lo, 0, size_t(slot_base) * 4, s));
    CK(launch_layout(d_seg_canon, d_seg_len, d_seg_pos, d_seg_vb, nseg_all, cvar, cdesc, clam, clam_lo, h->var, h->desc,
                     h->lam, h->lam_lo, h->canon_pos, s));
    CK(launch_instance_of(d_var_base, int32_t(ni), h->nint, h->var_inst, s));
    CK(cudaMemcpyAsync(h->lam0, h->lam, size_t(slot_base) * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->lam0_lo, h->lam_lo, size_t(slot_base) * 4, cudaMemcpyDeviceToDevice, s));
    if ((rc = copy_in(h->consts, consts.data(), consts.size() * 8, s))) return rc;
    if ((rc = copy_in(h->d_inst_tile_ptr, h->inst_tile_ptr.data(), h->inst_tile_ptr.size() * 4, s))) return rc;
    if ((rc = copy_in(h->d_inst_tiles, inst_tiles.data(), inst_tiles.size() * 4, s))) return rc;
    CK(cudaMemsetAsync(h->F, 0, size_t(node_base) * 4, s));
    CK(cudaMemsetAsync(h->B, 0, size_t(node_base) * 4, s));
    if ((rc = h->clear_sums())) return rc;
    h->phase = 0;
    CK(cudaMemsetAsync(h->status, 0, sizeof(uint32_t), s));
    CK(cudaMemsetAsync(h->state, 0, size_t(h->nint), s));
    CK(cudaStreamSynchronize(s));
    tr.mark("copies");
    return DISCO_OK;
}

// b of every node from the current lambda + pend (under the current fixings).
int reset_b(disco_handle* h) {
    int rc = h->pass(Pass::BwdReset);
    if (rc) return rc;
    h->has_b = true;
    return DISCO_OK;
}

int plain_iteration(disco_handle* h) {
    int rc;
    if ((rc = h->pass(Pass::FwdMMA))) return rc;
    if ((rc = h->pass(Pass::BwdMMA))) return rc;
    ++h->iterations;
    return DISCO_OK;
}

// Launch-geometry autotuner: every geometry runs the same per-lane arithmetic on the same
// tiles, so the results do not depend on the choice and the timed iterations are ordinary
// iterations. Each geometry runs kTrials iterations, timed with events on the handle's
// stream; the fastest single iteration wins.
constexpr int kGeometries[3] = {1, 2, 4};
constexpr int kTrials = 2;

int autotune(disco_handle* h, int* used) {
    cudaEvent_t ev[2];
    CK(cudaEventCreate(&ev[0]));
    CK(cudaEventCreate(&ev[1]));
    float best = 1e30f;
    int best_g = h->geometry, rc = DISCO_OK;
    for (int t = 0; t < kTrials && !rc; ++t)
        for (int g : kGeometries) {
            h->geometry = g;
            cudaEventRecord(ev[0], h->stream);
            if ((rc = plain_iteration(h))) break;
            cudaEventRecord(ev[1], h->stream);
            float ms = 0.0f;
            if (cudaEventSynchronize(ev[1]) != cudaSuccess || cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) {
                rc = fail(DISCO_ERR_CUDA, "autotune: event timing failed");
                break;
            }
            *used += 1;
            if (ms < best) {
                best = ms;
                best_g = g;
            }
        }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    h->geometry = best_g;
    h->tuned = true;
    return rc;
}

// Captures opts.graph_iters iterations, starting at the current averaging phase, into one
// executable graph (kernels only).
int capture_iterations(disco_handle* h) {
    const int G = h->opts.graph_iters;
    const int ph = h->phase;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        h->graph_failed = true;
        return DISCO_OK;
    }
    const int64_t before = g_launches.load();
    int rc = DISCO_OK;
    for (int t = 0; t < G && !rc; ++t) {
        rc = h->pass(Pass::FwdMMA);
        if (!rc) rc = h->pass(Pass::BwdMMA);
    }
    const cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    const int64_t captured = g_launches.load() - before;
    g_launches.fetch_sub(captured);  // recorded, not run
    h->phase = ph;
    if (rc || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        h->graph_failed = true;
        return DISCO_OK;
    }
    const cudaError_t ei = cudaGraphInstantiate(&h->iter_graph[ph], graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        h->iter_graph[ph] = nullptr;
        h->graph_failed = true;
        return DISCO_OK;
    }
    h->graph_launches[ph] = captured;
    return DISCO_OK;
}

// Dual iterations: forward and backward MMA half-passes. The averaging state stays in the
// rotating sum buffers between calls, so nothing is converted on entry or exit.
int run_iterations(disco_handle* h, int iters) {
    int rc;
    if (!h->has_b && (rc = reset_b(h))) return rc;
    int t = 0;
    if (iters > 0 && !h->tuned && h->opts.autotune && iters >= kTrials * 3) {
        int used = 0;
        if ((rc = autotune(h, &used))) return rc;
        t += used;
    }
    const int G = h->opts.graph_iters;
    if (G > 0 && (h->tuned || !h->opts.autotune)) {
        // the first time a block is replayed, the graphs of all three starting phases are
        // captured together (capturing runs nothing), so that no later call pays for one
        if (!h->graph_failed && iters - t >= G && !h->iter_graph[h->phase]) {
            const int ph0 = h->phase;
            for (int q = 0; q < 3 && !h->graph_failed; ++q) {
                h->phase = (ph0 + q) % 3;
                if (!h->iter_graph[h->phase] && (rc = capture_iterations(h))) {
                    h->phase = ph0;
                    return rc;
                }
            }
            h->phase = ph0;
        }
        while (!h->graph_failed && iters - t >= G) {
            if (!h->iter_graph[h->phase]) break;
            CK(cudaGraphLaunch(h->iter_graph[h->phase], h->stream));
            g_launches.fetch_add(h->graph_launches[h->phase], std::memory_order_relaxed);
            h->phase = (h->phase + 2 * G) % 3;
            h->iterations += G;
            t += G;
        }
    }
    for (; t < iters; ++t)
        if ((rc = plain_iteration(h))) return rc;
    return DISCO_OK;
}

// Per-instance lower bounds E(lambda + pend) + constant into h->h_scalar[0 .. n).
int lower_bounds(disco_handle* h) {
    int rc = h->pass(Pass::Lb);
    if (rc) return rc;
    CK(launch_sum_instances(h->tile_sum, h->d_inst_tile_ptr, h->d_inst_tiles, h->consts, h->n_inst(), h->scalar,
                            h->stream));
    CK(cudaMemcpyAsync(h->h_scalar, h->scalar, size_t(h->n_inst()) * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if ((rc = h->fetch_status())) return rc;
    CK(cudaStreamSynchronize(h->stream));
    return h->check_status();
}

// Sum of the instances' bounds (the bound of a single instance).
int lower_bound(disco_handle* h, double* lb) {
    int rc = lower_bounds(h);
    if (rc) return rc;
    double s = 0.0;
    for (int64_t i = 0; i < h->n_inst(); ++i) s += h->h_scalar[i];
    *lb = s;
    return DISCO_OK;
}

int check_handle(disco_handle* h) {
    if (!h) return fail(DISCO_ERR_INVALID_ARG, "null handle");
    CK(cudaSetDevice(h->device));
    return DISCO_OK;
}

int write_out(void* dst, const void* dev_src, size_t bytes, cudaStream_t s) {
    CK(cudaMemcpyAsync(dst, dev_src, bytes, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    return DISCO_OK;
}

}  // namespace

extern "C" {

int disco_default_opts(disco_opts* o) {
    if (!o) return fail(DISCO_ERR_INVALID_ARG, "null opts");
    std::memset(o, 0, sizeof(*o));
    o->omega = 0.5f;
    o->split_chunk = 0;
    o->lb_every = 20;
    o->conv_rel_tol = 1e-6;
    o->primal_rounds = 100;
    o->primal_inner_iters = 20;
    o->perturb_delta0 = 1e-3f;
    o->perturb_growth = 2.0f;
    o->tie_tau = 1e-6f;
    o->propagate_limit = 10000;
    o->device = 0;
    o->stream = nullptr;
    o->host_threads = 0;
    o->split_max_segments = 8;
    o->graph_iters = 10;
    o->autotune = 1;
    o->normalize_costs = 1;
    return DISCO_OK;
}

const char* disco_strerror(int code) {
    switch (code) {
        case DISCO_OK: return "ok";
        case DISCO_ERR_INVALID_ARG: return "invalid argument";
        case DISCO_ERR_NONMANIFOLD: return "mesh is not a closed, consistently oriented 2-manifold";
        case DISCO_ERR_GENUS_MISMATCH: return "meshes have different genus";
        case DISCO_ERR_INFEASIBLE: return "problem is infeasible";
        case DISCO_ERR_PRIMAL_FAILED: return "rounding did not reach a feasible solution";
        case DISCO_ERR_TIMEOUT: return "iteration limit reached";
        case DISCO_ERR_CUDA: return "CUDA error";
        case DISCO_ERR_OOM: return "out of memory";
        case DISCO_ERR_NOT_READY: return "call order violated";
        case DISCO_ERR_RANGE: return "a dual update left the range of the averaging sums";
        case DISCO_ERR_INTERNAL: return "a kernel index check failed (bounds-checking build)";
        default: return "unknown error";
    }
}

const char* disco_last_error(void) { return g_last_error.c_str(); }

int64_t disco_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"

namespace {

// Pair costs (norm = false) or distances (norm = true) from features that may be host or
// device arrays: host arrays are staged through one stream-ordered device buffer from the
// library's pool (returned to it on the same stream).
int pair_kernel(const char* what, const float* FX, const float* FY, int32_t nvx, int32_t nvy, int32_t dim, float* d,
                void* stream, bool norm) {
    if (!FX || !FY || !d || nvx <= 0 || nvy <= 0 || dim <= 0) return fail(DISCO_ERR_INVALID_ARG, std::string(what) + ": bad arguments");
    if (!is_device_ptr(d)) return fail(DISCO_ERR_INVALID_ARG, std::string(what) + ": d must be a device pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool hx = !is_device_ptr(FX), hy = !is_device_ptr(FY);
    if (!hx && !hy) {
        CK(launch_pair_costs(FX, FY, nvx, nvy, dim, d, s, norm));
        return DISCO_OK;
    }
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    CK(pool_for(dev, &pool));
    const size_t bx = size_t(nvx) * size_t(dim) * sizeof(float), by = size_t(nvy) * size_t(dim) * sizeof(float);
    float* buf = nullptr;
    CK(cudaMallocFromPoolAsync(reinterpret_cast<void**>(&buf), (hx ? bx : 0) + (hy ? by : 0), pool, s));
    const float* fx = FX;
    const float* fy = FY;
    cudaError_t e = cudaSuccess;
    if (hx) {
        e = cudaMemcpyAsync(buf, FX, bx, cudaMemcpyHostToDevice, s);
        fx = buf;
    }
    if (e == cudaSuccess && hy) {
        float* dst = buf + (hx ? size_t(nvx) * size_t(dim) : 0);
        e = cudaMemcpyAsync(dst, FY, by, cudaMemcpyHostToDevice, s);
        fy = dst;
    }
    if (e == cudaSuccess) e = launch_pair_costs(fx, fy, nvx, nvy, dim, d, s, norm);
    const cudaError_t ef = cudaFreeAsync(buf, s);
    if (e != cudaSuccess || ef != cudaSuccess)
        return fail(DISCO_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e != cudaSuccess ? e : ef));
    return DISCO_OK;
}

}  // namespace

extern "C" {

int disco_pair_costs(const float* FX, const float* FY, int32_t nvx, int32_t nvy, int32_t dim, float* d, void* stream) {
    return pair_kernel("pair_costs", FX, FY, nvx, nvy, dim, d, stream, false);
}

int disco_pair_distances(const float* FX, const float* FY, int32_t nvx, int32_t nvy, int32_t dim, float* d,
                         void* stream) {
    return pair_kernel("pair_distances", FX, FY, nvx, nvy, dim, d, stream, true);
}

int disco_candidates(const float* d, int32_t nvx, int32_t nvy, int32_t k, const disco_mesh* X, const disco_mesh* Y,
                     uint8_t* allowed, void* stream) {
    if (!d || !allowed || !X || !Y || !X->T || !Y->T || nvx != X->nv || nvy != Y->nv || k < 1 || k > 64 || k > nvx ||
        k > nvy)
        return fail(DISCO_ERR_INVALID_ARG, "candidates: bad arguments");
    if (!is_device_ptr(d) || !is_device_ptr(allowed))
        return fail(DISCO_ERR_INVALID_ARG, "candidates: d and allowed must be device pointers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // closed 1-rings as CSR (host -> device)
    auto rings = [](const disco_mesh* m, std::vector<int32_t>* ptr, std::vector<int32_t>* ring) {
        std::vector<std::vector<int32_t>> nb(m->nv);
        for (int v = 0; v < m->nv; ++v) nb[v].push_back(v);
        for (int t = 0; t < m->nt; ++t)
            for (int c = 0; c < 3; ++c) {
                int a = m->T[3 * t + c], b = m->T[3 * t + (c + 1) % 3];
                if (a < 0 || b < 0 || a >= m->nv || b >= m->nv) return false;
                nb[a].push_back(b);
                nb[b].push_back(a);
            }
        ptr->assign(1, 0);
        for (auto& x : nb) {
            std::sort(x.begin(), x.end());
            x.erase(std::unique(x.begin(), x.end()), x.end());
            ring->insert(ring->end(), x.begin(), x.end());
            ptr->push_back(int32_t(ring->size()));
        }
        return true;
    };
    std::vector<int32_t> px, rx, py, ry;
    if (!rings(X, &px, &rx) || !rings(Y, &py, &ry)) return fail(DISCO_ERR_INVALID_ARG, "candidates: bad mesh");
    int32_t *dpx, *drx, *dpy, *dry, *tk;
    float* dT;
    // temporaries from the library's pool (it keeps freed memory for the next call)
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    CK(pool_for(dev, &pool));
    auto palloc = [&](auto** p, size_t bytes) {
        return cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), std::max<size_t>(bytes, 4), pool, s);
    };
    CK(palloc(&dpx, px.size() * 4));
    CK(palloc(&drx, rx.size() * 4));
    CK(palloc(&dpy, py.size() * 4));
    CK(palloc(&dry, ry.size() * 4));
    CK(palloc(&tk, size_t(std::max(nvx, nvy)) * k * 4));
    CK(palloc(&dT, size_t(nvx) * nvy * 4));
    CK(cudaMemcpyAsync(dpx, px.data(), px.size() * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(drx, rx.data(), rx.size() * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dpy, py.data(), py.size() * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dry, ry.data(), ry.size() * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(allowed, 0, size_t(nvx) * nvy, s));
    CK(launch_topk_rows(d, nvx, nvy, k, tk, s));
    CK(launch_dilate(tk, nvx, k, dpy, dry, nvy, false, allowed, s));
    CK(launch_transpose(d, nvx, nvy, dT, s));
    CK(launch_topk_rows(dT, nvy, nvx, k, tk, s));
    CK(launch_dilate(tk, nvy, k, dpx, drx, nvy, true, allowed, s));
    CK(cudaFreeAsync(dpx, s));
    CK(cudaFreeAsync(drx, s));
    CK(cudaFreeAsync(dpy, s));
    CK(cudaFreeAsync(dry, s));
    CK(cudaFreeAsync(tk, s));
    CK(cudaFreeAsync(dT, s));
    CK(cudaStreamSynchronize(s));  // the host ring arrays die with this call
    return DISCO_OK;
}

}  // extern "C"

namespace {

// Builds a handle over n instances (host compiler per instance, one device store).
int build_handle(int32_t n, const disco_mesh* X, const disco_mesh* Y, const float* const* d,
                 const uint8_t* const* allowed, const disco_opts* opts, disco_handle** out) {
    if (!out || n < 1 || !X || !Y || !d) return fail(DISCO_ERR_INVALID_ARG, "build: null argument");
    *out = nullptr;
    for (int32_t i = 0; i < n; ++i)
        if (!X[i].T || !Y[i].T || !d[i]) return fail(DISCO_ERR_INVALID_ARG, "build: null mesh or cost array");
    disco_opts o;
    if (opts) o = *opts; else disco_default_opts(&o);
    if (!(o.omega > 0.0f && o.omega <= 1.0f) || o.split_chunk < 0 || o.split_max_segments < 0 || o.lb_every < 1 ||
        o.graph_iters < 0 || o.cost_model < 0 || o.cost_model > 1 || o.qn_memory < 0 || o.tile_order < 0 || o.tile_order > 2)
        return fail(DISCO_ERR_INVALID_ARG, "build: bad options");
    std::unique_ptr<disco_handle> h(new disco_handle());
    h->device = o.device;
    h->opts = o;
    CK(cudaSetDevice(o.device));
    if (o.stream) {
        h->stream = static_cast<cudaStream_t>(o.stream);
    } else {
        CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    // costs and masks on the host (they may be device arrays)
    Trace tr;
    std::vector<pod_vector<float>> hd(n);
    std::vector<pod_vector<uint8_t>> ha(n);
    int rc;
    for (int32_t i = 0; i < n; ++i) {
        const size_t npair = size_t(X[i].nv) * size_t(Y[i].nv);
        if ((rc = to_host(d[i], npair, &hd[i]))) return rc;
        if (allowed && allowed[i] && (rc = to_host(allowed[i], npair, &ha[i]))) return rc;
    }
    tr.mark("inputs to host");
    // one instance uses every host thread; several instances are compiled side by side
    const int hw = host_threads(o);
    const int outer = std::max(1, std::min<int>(n, hw));
    const int inner = std::max(1, hw / outer);
    h->plans.resize(size_t(n));
    std::vector<int> rcs(n, DISCO_OK);
    std::vector<std::string> errs(n);
    // one task per instance, largest first (by candidate pairs), taken dynamically by the
    // host threads, so that uneven pairs balance
    std::vector<int64_t> est(static_cast<size_t>(n), 1);
    if (n > 1)
        parallel_tasks(n, hw, [&](int64_t i) {
            const int64_t pairs = int64_t(X[i].nv) * Y[i].nv;
            est[i] = (allowed && allowed[i]) ? pairs - int64_t(std::count(ha[i].begin(), ha[i].end(), uint8_t(0))) : pairs;
        });
    std::vector<int32_t> order(static_cast<size_t>(n));
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return est[a] > est[b]; });
    // threads per pair (the plan does not depend on them; the largest pairs start first):
    // * no more pairs than threads: the threads in proportion to each pair's share of the
    //   work (1/hw of the total per thread), at least one, so that a large pair does not
    //   finish last on an even split;
    // * more pairs than threads: a pair holding more than half a thread's share would finish
    //   last on one thread, so it gets one thread per half share, up to 4.
    (void)inner;
    const double total = std::max<double>(1.0, double(std::accumulate(est.begin(), est.end(), int64_t(0))));
    parallel_chunks(n, n, [&](int c, int64_t, int64_t) {
        const int32_t i = order[c];
        const double share = double(est[i]) * hw / total;
        const int th = n <= hw ? std::max(1, std::min(hw, int(std::lround(share))))
                               : std::max(1, std::min(4, int(std::ceil(2.0 * share - 1e-9))));
        rcs[i] = build_plan(MeshIn{X[i].nv, X[i].nt, X[i].T, X[i].V}, MeshIn{Y[i].nv, Y[i].nt, Y[i].T, Y[i].V}, hd[i].data(),
                            (allowed && allowed[i]) ? ha[i].data() : nullptr, o.split_chunk, o.split_max_segments,
                            th, &h->plans[i], &errs[i], o.normalize_costs != 0, o.cost_model);
    });
    for (int32_t i = 0; i < n; ++i)
        if (rcs[i]) return fail(rcs[i], "build: instance " + std::to_string(i) + ": " + errs[i]);
    const auto tu = std::chrono::steady_clock::now();
    if ((rc = upload(h.get()))) return rc;
    h->upload_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tu).count();
    if (std::getenv("DISCO_TRACE")) std::fprintf(stderr, "disco build %-22s %8.2f ms\n", "device store upload", h->upload_ms);
    *out = h.release();
    return DISCO_OK;
}

void fill_info(const Plan& P, disco_info_t* info) {
    info->nvars += P.nvars;
    info->nrows += P.nrows;
    info->nvars_free += P.n_free;
    info->nvars_aux += P.n_aux;
    info->nbdds += int64_t(P.segs.size());
    info->nslots += int64_t(P.slot_var.size());
    info->nnodes += P.n_nodes;
    info->max_layers = std::max<int64_t>(info->max_layers, P.max_layers);
    info->max_width = std::max<int64_t>(info->max_width, P.max_width);
    info->constant += P.constant;
    info->build_ms = std::max(info->build_ms, P.build_ms);
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Quasi-Newton powered MMA (Alg. 1; L-BFGS memory Alg. 4, direction Alg. 5, step size
// Alg. 6). Readings, shared with the FP64 oracle: textbook L-BFGS on -E (y = g_k - g_{k+1},
// curvature test s^T y >= eps), the second loop's beta uses the running direction,
// FindStepSize starts from E_init = E(lambda), Delta_min = 1e-6 (E after the first call -
// E at its start) and 0 during the first call; the step is taken only if it raised the
// bound; eps = 1e-8, growth 1.1, shrink 0.8, K = 5 (the paper's values); first step 1e-3.
namespace {

constexpr double kQnEps = 1e-8, kQnGrow = 1.1, kQnShrink = 0.8;
constexpr int kQnK = 5;

int qn_init(disco_handle* h, int m) {
    if (h->qn_g) return DISCO_OK;
    h->qn_m = std::max(1, m);
    const int64_t n = h->nslots_tile;
    int rc;
    for (float** p : {&h->qn_g, &h->qn_g2, &h->qn_d, &h->qn_old, &h->qn_old_lo, &h->qn_tr, &h->qn_tr_lo})
        if ((rc = h->alloc(p, n))) return rc;
    if ((rc = h->alloc(&h->qn_tab, h->nint * kAccStride))) return rc;
    h->qn_S.assign(size_t(h->qn_m) + 1, nullptr);
    h->qn_Y.assign(size_t(h->qn_m) + 1, nullptr);
    for (int k = 0; k <= h->qn_m; ++k)
        if ((rc = h->alloc(&h->qn_S[k], n)) || (rc = h->alloc(&h->qn_Y[k], n))) return rc;
    h->qn_sy.assign(size_t(h->qn_m) + 1, 0.0);
    h->qn_yy.assign(size_t(h->qn_m) + 1, 0.0);
    h->qn_order.clear();
    h->qn_spare = 0;
    if ((rc = h->alloc(&h->qn_part, qn_dot_blocks()))) return rc;
    CK(cudaMallocHost(&h->qn_hpart, size_t(qn_dot_blocks()) * sizeof(double)));
    return DISCO_OK;
}

int qn_dot(disco_handle* h, const float* a, const float* b, double* out) {
    CK(launch_qn_dot(a, b, h->nslots_tile, h->qn_part, h->stream));
    CK(cudaMemcpyAsync(h->qn_hpart, h->qn_part, size_t(qn_dot_blocks()) * sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double x = 0.0;
    for (int k = 0; k < qn_dot_blocks(); ++k) x += h->qn_hpart[k];
    *out = x;
    return DISCO_OK;
}

// Per slot: 1 iff every minimising assignment of its BDD (on lambda + pend) sets the variable.
int qn_subgradient(disco_handle* h, float* g) {
    int rc;
    if ((rc = h->pass(Pass::FwdMM))) return rc;
    if ((rc = h->pass(Pass::BwdMM))) return rc;
    CK(launch_qn_sign(h->mm_slot, h->var, h->nslots_tile, g, h->stream));
    return DISCO_OK;
}

// E(lambda + gamma d) + constant (pend is 0 during the step search).
int qn_trial(disco_handle* h, double gamma, double* e) {
    CK(launch_qn_step(h->lam, h->lam_lo, h->qn_d, float(gamma), h->var, h->nslots_tile, h->qn_tr, h->qn_tr_lo,
                      h->stream));
    std::swap(h->lam, h->qn_tr);
    std::swap(h->lam_lo, h->qn_tr_lo);
    const int rc = lower_bound(h, e);
    std::swap(h->lam, h->qn_tr);
    std::swap(h->lam_lo, h->qn_tr_lo);
    return rc;
}

int qn_call(disco_handle* h, int mma_iters) {
    int rc;
    cudaStream_t s = h->stream;
    const int64_t n = h->nslots_tile;
    if ((rc = qn_init(h, h->opts.qn_memory > 0 ? h->opts.qn_memory : 5))) return rc;
    // lambda <- lambda + pend
    CK(launch_flush(h->var, h->desc, n, h->msum_rd(), h->fx.inv, h->lam, h->lam_lo, s));
    CK(cudaMemsetAsync(h->msum_rd(), 0, size_t(h->nint) * sizeof(long long), s));
    double E0;
    if ((rc = lower_bound(h, &E0))) return rc;
    if (h->qn_calls == 0) h->qn_Estart = E0;
    if ((rc = qn_subgradient(h, h->qn_g))) return rc;
    // d = H g (two loops), then the dual-feasible projection
    CK(cudaMemcpyAsync(h->qn_d, h->qn_g, size_t(n) * 4, cudaMemcpyDeviceToDevice, s));
    const int np = int(h->qn_order.size());
    std::vector<double> alpha(size_t(np), 0.0);
    for (int k = np - 1; k >= 0; --k) {
        const int b = h->qn_order[k];
        double sd;
        if ((rc = qn_dot(h, h->qn_S[b], h->qn_d, &sd))) return rc;
        alpha[k] = sd / h->qn_sy[b];
        CK(launch_qn_axpy(h->qn_d, float(-alpha[k]), h->qn_Y[b], n, s));
    }
    if (np > 0) {
        const int b = h->qn_order.back();
        CK(launch_qn_scale(h->qn_d, float(h->qn_sy[b] / h->qn_yy[b]), n, s));
    }
    for (int k = 0; k < np; ++k) {
        const int b = h->qn_order[k];
        double yd;
        if ((rc = qn_dot(h, h->qn_Y[b], h->qn_d, &yd))) return rc;
        CK(launch_qn_axpy(h->qn_d, float(alpha[k] - yd / h->qn_sy[b]), h->qn_S[b], n, s));
    }
    CK(launch_qn_project(h->qn_d, h->var, h->desc, n, h->qn_tab, s));
    // step size (Alg. 6)
    CK(cudaMemcpyAsync(h->qn_old, h->lam, size_t(n) * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->qn_old_lo, h->lam_lo, size_t(n) * 4, cudaMemcpyDeviceToDevice, s));
    double gamma = h->qn_gamma, gm = gamma, Em, e;
    if ((rc = qn_trial(h, gamma, &Em))) return rc;
    e = Em;
    for (int t = 0; t < kQnK; ++t) {
        gamma *= e <= E0 ? kQnShrink : kQnGrow;
        if ((rc = qn_trial(h, gamma, &e))) return rc;
        if (e >= Em) {
            gm = gamma;
            Em = e;
        }
        if (e - E0 >= h->qn_dmin) break;
    }
    if (Em > E0) CK(launch_qn_step(h->lam, h->lam_lo, h->qn_d, float(gm), h->var, n, h->lam, h->lam_lo, s));
    h->qn_gamma = gm;
    h->has_b = false;
    if ((rc = run_iterations(h, mma_iters))) return rc;
    // L-BFGS memory (Alg. 4): s = lambda_new - lambda_old, y = g_old - g_new
    if ((rc = qn_subgradient(h, h->qn_g2))) return rc;
    const int b = h->qn_spare;
    CK(launch_qn_delta(h->lam, h->lam_lo, h->msum_rd(), h->fx.inv, h->qn_old, h->qn_old_lo, h->var, h->desc, n,
                       h->qn_S[b], s));
    CK(launch_qn_sub(h->qn_g, h->qn_g2, n, h->qn_Y[b], s));
    double sy, yy;
    if ((rc = qn_dot(h, h->qn_S[b], h->qn_Y[b], &sy))) return rc;
    if (sy >= kQnEps) {
        if ((rc = qn_dot(h, h->qn_Y[b], h->qn_Y[b], &yy))) return rc;
        h->qn_sy[b] = sy;
        h->qn_yy[b] = yy;
        h->qn_order.push_back(b);
        if (int(h->qn_order.size()) > h->qn_m) {
            h->qn_spare = h->qn_order.front();
            h->qn_order.erase(h->qn_order.begin());
        } else {
            h->qn_spare = int(h->qn_order.size());  // buffers 0..m are used in order at first
        }
    }
    ++h->qn_calls;
    if (h->qn_calls == 1) {
        double lb;
        if ((rc = lower_bound(h, &lb))) return rc;
        h->qn_dmin = 1e-6 * (lb - h->qn_Estart);
    }
    return DISCO_OK;
}

}  // namespace

extern "C" {

int disco_build(const disco_mesh* X, const disco_mesh* Y, const float* d, const uint8_t* allowed, const disco_opts* opts,
                disco_handle** out) {
    if (!X || !Y || !d) return fail(DISCO_ERR_INVALID_ARG, "build: null argument");
    const float* dd[1] = {d};
    const uint8_t* aa[1] = {allowed};
    return build_handle(1, X, Y, dd, aa, opts, out);
}

int disco_build_batch(int32_t n, const disco_mesh* X, const disco_mesh* Y, const float* const* d,
                      const uint8_t* const* allowed, const disco_opts* opts, disco_handle** out) {
    return build_handle(n, X, Y, d, allowed, opts, out);
}

int disco_batch_size(disco_handle* h, int32_t* n) {
    if (!h || !n) return fail(DISCO_ERR_INVALID_ARG, "batch_size: null argument");
    *n = int32_t(h->n_inst());
    return DISCO_OK;
}

int disco_lower_bounds(disco_handle* h, double* lb, int32_t n) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!lb || n < h->n_inst()) return fail(DISCO_ERR_INVALID_ARG, "lower_bounds: output too small");
    if ((rc = lower_bounds(h))) return rc;
    for (int64_t i = 0; i < h->n_inst(); ++i) lb[i] = h->h_scalar[i];
    return DISCO_OK;
}

int disco_instance_info(disco_handle* h, int32_t i, disco_info_t* info) {
    if (!h || !info || i < 0 || i >= h->n_inst()) return fail(DISCO_ERR_INVALID_ARG, "instance_info: bad argument");
    std::memset(info, 0, sizeof(*info));
    const Plan& P = h->plans[i];
    fill_info(P, info);
    info->ntiles = h->inst_tile_ptr[i + 1] - h->inst_tile_ptr[i];
    info->iterations = h->iterations;
    info->bytes_per_iter = 2 * (8 * P.n_nodes + 20 * info->nslots + 8 * (P.n_free + P.n_aux));
    return DISCO_OK;
}

int disco_point_map(disco_handle* h, const uint8_t* x, int64_t nvars, int32_t* pairs, int64_t capacity,
                    int64_t* count) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (h->n_inst() != 1 || !x || !count || nvars < h->plans[0].nvars)
        return fail(DISCO_ERR_INVALID_ARG, "point_map: single-instance handle and a full x required");
    const Plan& P = h->plans[0];
    std::vector<int64_t> keys;
    for (int64_t e = 0; e < P.nvars; ++e)
        if (x[e])
            for (int v = 0; v < 3; ++v) keys.push_back(int64_t(P.vm[3 * e + v]) * P.nvy + P.vn[3 * e + v]);
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    *count = int64_t(keys.size());
    if (int64_t(keys.size()) > capacity || (!pairs && !keys.empty()))
        return fail(DISCO_ERR_INVALID_ARG, "point_map: capacity too small");
    for (size_t k = 0; k < keys.size(); ++k) {
        pairs[2 * k] = int32_t(keys[k] / P.nvy);
        pairs[2 * k + 1] = int32_t(keys[k] % P.nvy);
    }
    return DISCO_OK;
}

int disco_candidates_coarse_to_fine(const int32_t* pairs, int64_t npairs, const int32_t* c2f_x, int32_t ncx,
                                    const int32_t* c2f_y, int32_t ncy, int32_t rings, const disco_mesh* Xf,
                                    const disco_mesh* Yf, uint8_t* allowed) {
    if (!Xf || !Yf || !Xf->T || !Yf->T || !allowed || !c2f_x || !c2f_y || rings < 0 || npairs < 0 ||
        (npairs > 0 && !pairs))
        return fail(DISCO_ERR_INVALID_ARG, "coarse_to_fine: bad arguments");
    const int nx = Xf->nv, ny = Yf->nv;
    for (int32_t i = 0; i < ncx; ++i)
        if (c2f_x[i] < 0 || c2f_x[i] >= nx) return fail(DISCO_ERR_INVALID_ARG, "coarse_to_fine: c2f_x out of range");
    for (int32_t i = 0; i < ncy; ++i)
        if (c2f_y[i] < 0 || c2f_y[i] >= ny) return fail(DISCO_ERR_INVALID_ARG, "coarse_to_fine: c2f_y out of range");
    // vertices within `rings` edges of every seed vertex, by breadth-first search on each mesh
    auto adjacency = [](const disco_mesh* M, std::vector<std::vector<int32_t>>* adj) {
        adj->assign(size_t(M->nv), {});
        for (int t = 0; t < M->nt; ++t)
            for (int v = 0; v < 3; ++v) {
                const int32_t a = M->T[3 * t + v], b = M->T[3 * t + (v + 1) % 3];
                if (a < 0 || a >= M->nv || b < 0 || b >= M->nv) return false;
                (*adj)[a].push_back(b);
                (*adj)[b].push_back(a);
            }
        return true;
    };
    std::vector<std::vector<int32_t>> ax, ay;
    if (!adjacency(Xf, &ax) || !adjacency(Yf, &ay)) return fail(DISCO_ERR_INVALID_ARG, "coarse_to_fine: bad mesh");
    auto ball = [rings](const std::vector<std::vector<int32_t>>& adj, int32_t src, std::vector<int32_t>* out,
                        std::vector<int32_t>* dist) {
        out->assign(1, src);
        (*dist)[src] = 0;
        for (size_t q = 0; q < out->size(); ++q) {
            const int32_t u = (*out)[q];
            if ((*dist)[u] == rings) continue;
            for (int32_t w : adj[u])
                if ((*dist)[w] < 0) {
                    (*dist)[w] = (*dist)[u] + 1;
                    out->push_back(w);
                }
        }
        for (int32_t u : *out) (*dist)[u] = -1;
    };
    std::vector<uint8_t> mask(size_t(nx) * ny, 0);
    std::vector<int32_t> dx(size_t(nx), -1), dy(size_t(ny), -1), bx, by;
    for (int64_t k = 0; k < npairs; ++k) {
        const int32_t m = pairs[2 * k], n = pairs[2 * k + 1];
        if (m < 0 || m >= ncx || n < 0 || n >= ncy) return fail(DISCO_ERR_INVALID_ARG, "coarse_to_fine: pair out of range");
        ball(ax, c2f_x[m], &bx, &dx);
        ball(ay, c2f_y[n], &by, &dy);
        for (int32_t a : bx)
            for (int32_t b : by) mask[size_t(a) * ny + b] = 1;
    }
    if (is_device_ptr(allowed)) {
        CK(cudaMemcpy(allowed, mask.data(), mask.size(), cudaMemcpyHostToDevice));
    } else {
        std::memcpy(allowed, mask.data(), mask.size());
    }
    return DISCO_OK;
}

int disco_compile_host(const disco_mesh* X, const disco_mesh* Y, const float* d, const uint8_t* allowed,
                       int32_t split_chunk, int32_t split_max_segments, disco_info_t* info, int32_t* slot_var,
                       int32_t* slot_width, int64_t nslots, int8_t* fixed, int64_t nvars) {
    if (!X || !Y || !d || !info || !X->T || !Y->T || split_chunk < 0 || split_max_segments < 0)
        return fail(DISCO_ERR_INVALID_ARG, "compile_host: bad arguments");
    Plan P;
    std::string err;
    int rc = build_plan(MeshIn{X->nv, X->nt, X->T, X->V}, MeshIn{Y->nv, Y->nt, Y->T, Y->V}, d, allowed, split_chunk,
                        split_max_segments, 0, &P, &err);
    if (rc) return fail(rc, "compile_host: " + err);
    std::memset(info, 0, sizeof(*info));
    info->nvars = P.nvars;
    info->nrows = P.nrows;
    info->nvars_free = P.n_free;
    info->nvars_aux = P.n_aux;
    info->nbdds = int64_t(P.segs.size());
    info->nslots = int64_t(P.slot_var.size());
    info->nnodes = P.n_nodes;
    info->max_layers = P.max_layers;
    info->max_width = P.max_width;
    info->constant = P.constant;
    info->build_ms = P.build_ms;
    info->bytes_per_iter = 2 * (8 * P.n_nodes + 20 * info->nslots + 8 * (P.n_free + P.n_aux));
    if (nslots >= info->nslots) {
        for (int64_t i = 0; i < info->nslots; ++i) {
            const int32_t v = P.slot_var[i];
            if (slot_var) slot_var[i] = v < P.n_free ? P.free_orig[v] : int32_t(P.nvars + (v - P.n_free));
            if (slot_width) slot_width[i] = int32_t(P.slot_desc[i] & 63u) + 1;
        }
    }
    if (fixed && nvars >= P.nvars) std::memcpy(fixed, P.fixed.data(), size_t(P.nvars));
    return DISCO_OK;
}

int disco_dual(disco_handle* h, int32_t iters) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (iters < 0) return fail(DISCO_ERR_INVALID_ARG, "dual: iters < 0");
    return run_iterations(h, iters);
}

int disco_dual_qn(disco_handle* h, int32_t calls, int32_t mma_iters) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (calls < 0 || mma_iters < 0) return fail(DISCO_ERR_INVALID_ARG, "dual_qn: calls < 0 or mma_iters < 0");
    for (int c = 0; c < calls; ++c)
        if ((rc = qn_call(h, mma_iters))) return rc;
    return DISCO_OK;
}

int disco_lower_bound(disco_handle* h, double* lb) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!lb) return fail(DISCO_ERR_INVALID_ARG, "lower_bound: null output");
    return lower_bound(h, lb);
}

int disco_converge(disco_handle* h, int32_t max_iters, int32_t* iters_done, double* lb_out) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (max_iters < 0) return fail(DISCO_ERR_INVALID_ARG, "converge: max_iters < 0");
    double prev = 0.0, lb = 0.0;
    if ((rc = lower_bound(h, &prev))) return rc;
    int done = 0;
    bool converged = false;
    while (done < max_iters) {
        const int n = std::min(h->opts.lb_every, max_iters - done);
        if ((rc = h->opts.qn_memory > 0 ? qn_call(h, n) : run_iterations(h, n))) return rc;
        done += n;
        if ((rc = lower_bound(h, &lb))) return rc;
        if (std::fabs(lb - prev) < h->opts.conv_rel_tol * std::max(std::fabs(lb), 1e-300)) {
            converged = true;
            break;
        }
        prev = lb;
    }
    if (done == 0) lb = prev;
    if (iters_done) *iters_done = done;
    if (lb_out) *lb_out = lb;
    return converged || max_iters == 0 ? DISCO_OK : fail(DISCO_ERR_TIMEOUT, "converge: max_iters reached");
}

int disco_min_marginals(disco_handle* h, float* out, int64_t n) {
    int rc = check_handle(h);
    if (rc) return rc;
    const int64_t ns = h->nslots();
    if (!out || n < ns) return fail(DISCO_ERR_INVALID_ARG, "min_marginals: output too small");
    if ((rc = h->pass(Pass::FwdMM))) return rc;
    if ((rc = h->pass(Pass::BwdMM))) return rc;
    CK(launch_gather_f32(h->mm_slot, h->canon_pos, ns, h->tmp, h->stream));
    if ((rc = h->fetch_status())) return rc;
    if ((rc = write_out(out, h->tmp, size_t(ns) * 4, h->stream))) return rc;
    return h->check_status();
}

int disco_get_state(disco_handle* h, float* lam, int64_t n, float* pend, int64_t n_pend) {
    int rc = check_handle(h);
    if (rc) return rc;
    const int64_t ns = h->nslots();
    if (!lam || n < ns || (pend && n_pend < h->nint)) return fail(DISCO_ERR_INVALID_ARG, "get_state: output too small");
    CK(launch_gather_f32(h->lam, h->canon_pos, ns, h->tmp, h->stream));
    if ((rc = write_out(lam, h->tmp, size_t(ns) * 4, h->stream))) return rc;
    if (pend) {
        CK(launch_pend(h->msum_rd(), h->deg, h->nint, h->fx.inv, h->tmp, h->stream));
        if ((rc = write_out(pend, h->tmp, size_t(h->nint) * 4, h->stream))) return rc;
    }
    return DISCO_OK;
}

int disco_set_state(disco_handle* h, const float* lam, int64_t n, const float* pend, int64_t n_pend) {
    int rc = check_handle(h);
    if (rc) return rc;
    const int64_t ns = h->nslots();
    if (!lam || n < ns || (pend && n_pend < h->nint)) return fail(DISCO_ERR_INVALID_ARG, "set_state: input too small");
    CK(cudaMemcpyAsync(h->tmp, lam, size_t(ns) * 4, cudaMemcpyDefault, h->stream));
    CK(launch_scatter_f32(h->tmp, h->canon_pos, ns, h->lam, h->stream));
    CK(cudaMemsetAsync(h->lam_lo, 0, size_t(h->nslots_tile) * 4, h->stream));
    if (pend) {
        CK(cudaMemcpyAsync(h->tmp, pend, size_t(h->nint) * 4, cudaMemcpyDefault, h->stream));
        CK(launch_set_pend(h->tmp, h->deg, h->nint, h->fx.scale, h->msum_rd(), h->status, h->stream));
    } else {
        CK(cudaMemsetAsync(h->msum_rd(), 0, size_t(h->nint) * sizeof(long long), h->stream));
    }
    CK(cudaMemsetAsync(h->msum[h->phase], 0, size_t(h->nint) * sizeof(long long), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->has_b = false;
    return DISCO_OK;
}

}  // extern "C"

namespace {

// x of one instance from its presolve values and the rounded internal variables; exact check
// of A x = b and the cost (a fixed-order sum of per-chunk sums). Returns feasibility.
bool assemble_instance(const Plan& P, const uint8_t* st, int nth, uint8_t* x, double* cost) {
    parallel_chunks(P.nvars, nth, [&](int, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) x[i] = P.fixed[i] == 1 ? 1 : 0;
    });
    std::vector<uint8_t> undecided(static_cast<size_t>(nth), 0);
    parallel_chunks(P.n_free, nth, [&](int c, int64_t lo, int64_t hi) {
        for (int64_t v = lo; v < hi; ++v) {
            x[P.free_orig[v]] = st[v] == kFix1 ? 1 : 0;
            if (st[v] == kFree) undecided[c] = 1;
        }
    });
    const bool all = std::find(undecided.begin(), undecided.end(), uint8_t(1)) == undecided.end();
    // every row's residual, over row ranges of about equal entry counts (projection rows are
    // long), taken dynamically; the cost in fixed element blocks (a thread-count-independent sum)
    const int nck = 64;
    std::vector<int64_t> cut(size_t(nck) + 1, P.nrows);
    cut[0] = 0;
    const int64_t ntot = P.row_ptr[size_t(P.nrows)];
    for (int c = 1; c < nck; ++c)
        cut[size_t(c)] = std::max<int64_t>(
            cut[size_t(c) - 1],
            int64_t(std::lower_bound(P.row_ptr.begin(), P.row_ptr.begin() + P.nrows, ntot * c / nck) - P.row_ptr.begin()));
    std::vector<uint8_t> violated(nck, 0);
    std::vector<double> part(nck, 0.0);
    parallel_tasks(nck, nth, [&](int64_t c) {
        uint8_t bad = 0;
        for (int64_t r = cut[size_t(c)]; r < cut[size_t(c) + 1]; ++r) {
            int64_t sum = 0;
            for (int64_t e = P.row_ptr[r]; e < P.row_ptr[r + 1]; ++e) sum += int64_t(P.row_coef[e]) * x[P.row_var[e]];
            bad |= uint8_t(sum != P.rhs[r]);
        }
        violated[size_t(c)] = bad;
        double s = 0.0;
        for (int64_t i = P.nvars * c / nck; i < P.nvars * (c + 1) / nck; ++i) s += x[i] ? P.cost[i] : 0.0;
        part[size_t(c)] = s;
    });
    double c = 0.0;
    for (double q : part) c += q;
    *cost = c;
    return all && std::find(violated.begin(), violated.end(), uint8_t(1)) == violated.end();
}

// Rounding of every instance of the handle at once (the fixings of one instance never touch
// another's BDDs); x_out holds the instances' elements one after another.
int primal_all(disco_handle* h, uint8_t* x_out, double* costs, int32_t* status) {
    const disco_opts& o = h->opts;
    cudaStream_t s = h->stream;
    const int64_t nint = h->nint;
    int rc;
    CK(cudaMemsetAsync(h->state, 0, size_t(nint), s));
    Trace tr;
    tr.scope = "primal";
    auto mark = [&](const char* what) {
        if (tr.on) cudaStreamSynchronize(s);
        tr.mark(what);
    };
    float delta = o.perturb_delta0;
    bool done = nint == 0;
    for (int r = 0; r < o.primal_rounds && !done; ++r) {
        // 1. lambda <- lambda + pend; min-marginals under the fixings
        CK(launch_flush(h->var, h->desc, h->nslots_tile, h->msum_rd(), h->fx.inv, h->lam, h->lam_lo, s));
        if ((rc = h->clear_sums())) return rc;
        if ((rc = h->pass(Pass::FwdMM))) return rc;
        if ((rc = h->pass(Pass::BwdMM))) return rc;
        // 2. agreement: every slot strictly positive -> 0, strictly negative -> 1
        CK(launch_decide(h->mm_var, h->deg, h->state, nint, o.tie_tau, h->trial, s));
        mark("min-marginals, decide");
        // 3. propagate the trial fixings to a fixpoint; an instance whose trial runs into a
        //    conflict keeps its fixings of the previous round (other instances go on)
        const int64_t ni = h->n_inst();
        std::vector<uint8_t> reverted(static_cast<size_t>(ni), 0);
        int sweeps = 0;
        for (;;) {
            CK(cudaMemsetAsync(h->counters, 0, size_t(4 * ni) * sizeof(int), s));
            uint8_t* keep = h->state;
            h->state = h->trial;  // the support pass reads the trial fixings
            rc = h->pass(Pass::Supports);
            h->state = keep;
            if (rc) return rc;
            CK(launch_apply(h->sup, h->deg, h->var_inst, nint, h->trial, h->counters, s));
            CK(cudaMemcpyAsync(h->h_counters, h->counters, size_t(4 * ni) * sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            bool changed = false;
            for (int64_t i = 0; i < ni; ++i) {
                if (reverted[i]) continue;
                if (h->h_counters[4 * i + 1] > 0) {
                    reverted[i] = 1;
                    const int64_t v0 = h->var_base[i], v1 = h->var_base[i + 1];
                    CK(cudaMemcpyAsync(h->trial + v0, h->state + v0, size_t(v1 - v0), cudaMemcpyDeviceToDevice, s));
                } else if (h->h_counters[4 * i] > 0) {
                    changed = true;
                }
            }
            if (!changed) break;
            if (++sweeps > o.propagate_limit) return fail(DISCO_ERR_TIMEOUT, "primal: propagation did not settle");
        }
        mark("propagation");
        CK(cudaMemcpyAsync(h->state, h->trial, size_t(nint), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(h->counters, 0, size_t(4 * ni) * sizeof(int), s));
        CK(launch_count_free(h->state, h->deg, h->var_inst, nint, h->counters, s));
        CK(cudaMemcpyAsync(h->h_counters, h->counters, size_t(4 * ni) * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        int64_t left = 0;
        for (int64_t i = 0; i < ni; ++i) left += h->h_counters[4 * i + 2];
        if (left == 0) { done = true; break; }
        // 4. push undecided variables towards their majority, then continue the dual
        CK(launch_perturb(h->var, h->desc, h->nslots_tile, h->mm_var, h->state, delta, h->lam, h->lam_lo, s));
        delta *= o.perturb_growth;
        if ((rc = h->pass(Pass::BwdReset))) return rc;
        for (int t = 0; t < o.primal_inner_iters; ++t) {
            if ((rc = h->pass(Pass::FwdMMARound))) return rc;
            if ((rc = h->pass(Pass::BwdMMARound))) return rc;
        }
        mark("perturb, dual");
    }
    // read the fixings back
    std::vector<uint8_t> st(static_cast<size_t>(nint), uint8_t(0));
    if (nint) CK(cudaMemcpyAsync(st.data(), h->state, size_t(nint), cudaMemcpyDeviceToHost, s));
    if ((rc = h->fetch_status())) return rc;
    CK(cudaStreamSynchronize(s));
    if ((rc = h->check_status())) return rc;
    // the dual continues from an unrestricted state
    CK(cudaMemsetAsync(h->state, 0, size_t(nint), s));
    h->has_b = false;
    const int64_t ni = h->n_inst();
    const int hw = host_threads(o);
    const int outer = std::max(1, std::min<int>(int(ni), hw));
    mark("read back");
    pod_vector<uint8_t> x(static_cast<size_t>(h->nelems()));  // every element is written by its instance
    std::vector<uint8_t> ok(static_cast<size_t>(ni), 0);
    std::vector<double> cs(static_cast<size_t>(ni), 0.0);
    parallel_chunks(ni, outer, [&](int, int64_t i0, int64_t i1) {
        for (int64_t i = i0; i < i1; ++i)
            ok[i] = assemble_instance(h->plans[i], st.data() + h->var_base[i], std::max(1, hw / outer),
                                      x.data() + h->elem_base[i], &cs[i]);
    });
    bool all = true;
    for (int64_t i = 0; i < ni; ++i) {
        if (costs) costs[i] = cs[i];
        if (status) status[i] = ok[i] ? DISCO_OK : DISCO_ERR_PRIMAL_FAILED;
        all = all && ok[i];
    }
    mark("assemble, check");
    if ((rc = write_out(x_out, x.data(), x.size(), s))) return rc;
    mark("write");
    return all ? DISCO_OK : fail(DISCO_ERR_PRIMAL_FAILED, "primal: no feasible assignment within the round limit");
}

}  // namespace

extern "C" {

int disco_primal(disco_handle* h, uint8_t* x_out, int64_t nvars, double* cost) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!x_out || nvars < h->nelems()) return fail(DISCO_ERR_INVALID_ARG, "primal: output too small");
    std::vector<double> cs(static_cast<size_t>(h->n_inst()), 0.0);
    rc = primal_all(h, x_out, cs.data(), nullptr);
    if (cost) {
        double c = 0.0;
        for (double q : cs) c += q;
        *cost = c;
    }
    return rc;
}

int disco_primal_batch(disco_handle* h, uint8_t* x_out, int64_t nvars, double* costs, int32_t* status, int32_t n) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!x_out || nvars < h->nelems() || n < h->n_inst())
        return fail(DISCO_ERR_INVALID_ARG, "primal_batch: output too small");
    return primal_all(h, x_out, costs, status);
}

int disco_info(disco_handle* h, disco_info_t* info) {
    if (!h || !info) return fail(DISCO_ERR_INVALID_ARG, "info: null argument");
    std::memset(info, 0, sizeof(*info));
    for (const Plan& P : h->plans) fill_info(P, info);
    info->ntiles = h->ntiles;
    info->device_bytes = h->device_bytes;
    info->iterations = h->iterations;
    info->upload_ms = h->upload_ms;
    info->launch_geometry = h->geometry;
    // per iteration: 8 B per node and 20 B per slot per half-pass, 8 B per variable for the averaging
    info->bytes_per_iter = 2 * (8 * info->nnodes + 20 * info->nslots + 8 * (info->nvars_free + info->nvars_aux));
    return DISCO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Differentiation: the bound after T iterations from lambda^0 = c / |J| as a function of the
// pair costs. disco_record runs the iterations keeping a checkpoint every few iterations;
// disco_grad replays each block from its checkpoint, recording every half-pass's inputs and
// the node costs it stores, then walks the passes backwards, reversing each by its adjoint
// kernel (adjoint.cu) on the recorded values (bit-identical mins).
namespace {

using Snap = disco_handle::Snap;

// A checkpoint holds lambda, the averaging sectors and the other direction's node costs; a
// tape entry holds lambda, the per-variable deferred means and the pass's own node costs.
int alloc_snap(disco_handle* h, Snap* s, bool tape = false) {
    if (s->lam) return DISCO_OK;
    int rc;
    if ((rc = h->alloc(&s->lam, h->nslots_tile))) return rc;
    if ((rc = h->alloc(&s->lam_lo, h->nslots_tile))) return rc;
    if (tape) {
        if ((rc = h->alloc(&s->pend, h->nint))) return rc;
    } else if ((rc = h->alloc(&s->msum, h->nint))) {
        return rc;
    }
    if ((rc = h->alloc(&s->nodes, h->nnodes_tile))) return rc;
    return DISCO_OK;
}

int d2d(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
    return DISCO_OK;
}

// Saves lambda, the averaging sums the next pass reads and the given node costs (none when
// nodes is null).
int save_snap(disco_handle* h, Snap* s, const float* nodes) {
    int rc;
    const size_t ns = size_t(h->nslots_tile) * 4, na = size_t(h->nint) * sizeof(long long),
                 nn = size_t(h->nnodes_tile) * 4;
    if ((rc = d2d(s->lam, h->lam, ns, h->stream)) || (rc = d2d(s->lam_lo, h->lam_lo, ns, h->stream)) ||
        (rc = d2d(s->msum, h->msum_rd(), na, h->stream)) || (nodes && (rc = d2d(s->nodes, nodes, nn, h->stream))))
        return rc;
    s->phase = h->phase;
    return DISCO_OK;
}

// Restores a saved state at its averaging phase (the buffer the next update pass writes is
// cleared, as it is between passes).
int load_snap(disco_handle* h, const Snap& s, float* nodes) {
    int rc;
    const size_t ns = size_t(h->nslots_tile) * 4, na = size_t(h->nint) * sizeof(long long),
                 nn = size_t(h->nnodes_tile) * 4;
    h->phase = s.phase;
    if ((rc = d2d(h->lam, s.lam, ns, h->stream)) || (rc = d2d(h->lam_lo, s.lam_lo, ns, h->stream)) ||
        (rc = d2d(h->msum_rd(), s.msum, na, h->stream)) || (rc = d2d(nodes, s.nodes, nn, h->stream)))
        return rc;
    CK(cudaMemsetAsync(h->msum[h->phase], 0, na, h->stream));
    return DISCO_OK;
}

AdjArgs adj_args(disco_handle* h) {
    AdjArgs a{};
    a.tiles = h->tiles;
    a.var = h->var;
    a.desc = h->desc;
    a.lbar = h->lbar;
    a.omega = h->opts.omega;
    a.fx = h->fx;
    return a;
}

// One adjoint launch per width group, in tile order (tiles are independent).
cudaError_t launch_adjoint_all(disco_handle* h, Adj kind, AdjArgs a) {
    for (const WidthClass& c : h->classes) {
        a.tile0 = c.tile0;
        a.tile_end = c.tile_end;
        const cudaError_t e = launch_adjoint(kind, c.W, a, h->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int64_t pair_cost_count(const disco_handle* h) {
    int64_t n = 0;
    for (const Plan& P : h->plans) n += int64_t(P.nvx) * P.nvy;
    return n;
}

}  // namespace

extern "C" {

int disco_record(disco_handle* h, int32_t iters, int32_t checkpoint_every) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (iters < 0 || checkpoint_every < 1) return fail(DISCO_ERR_INVALID_ARG, "record: iters < 0 or checkpoint_every < 1");
    const int nck = std::max(1, (iters + checkpoint_every - 1) / checkpoint_every);
    h->checkpoints.resize(size_t(std::max<size_t>(h->checkpoints.size(), size_t(nck))));
    for (int k = 0; k < nck; ++k)
        if ((rc = alloc_snap(h, &h->checkpoints[k]))) return rc;
    cudaStream_t s = h->stream;
    const size_t ns = size_t(h->nslots_tile) * 4;
    if ((rc = d2d(h->lam, h->lam0, ns, s)) || (rc = d2d(h->lam_lo, h->lam0_lo, ns, s))) return rc;
    if ((rc = h->clear_sums())) return rc;
    CK(cudaMemsetAsync(h->state, 0, size_t(h->nint), s));
    h->phase = 0;
    h->iterations = 0;
    if ((rc = reset_b(h))) return rc;
    for (int k = 0; k < nck; ++k) {
        if ((rc = save_snap(h, &h->checkpoints[k], h->B))) return rc;
        const int n = std::min(checkpoint_every, iters - k * checkpoint_every);
        if (n > 0 && (rc = run_iterations(h, n))) return rc;
    }
    h->rec_iters = iters;
    h->rec_every = checkpoint_every;
    CK(cudaStreamSynchronize(s));
    return DISCO_OK;
}

int disco_grad(disco_handle* h, float* dlb_dpair_costs, int64_t n) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (h->rec_iters < 0) return fail(DISCO_ERR_INVALID_ARG, "grad: call disco_record first");
    const int64_t need = pair_cost_count(h);
    if (!dlb_dpair_costs || n < need) return fail(DISCO_ERR_INVALID_ARG, "grad: output too small");
    const int T = h->rec_iters, G = h->rec_every;
    const int nck = std::max(1, (T + G - 1) / G);
    if (h->tape.size() < size_t(2 * G)) h->tape.resize(size_t(2 * G));
    for (int e = 0; e < std::min(2 * G, 2 * T); ++e)
        if ((rc = alloc_snap(h, &h->tape[e], true))) return rc;
    if ((rc = alloc_snap(h, &h->final_state))) return rc;
    if (!h->lbar) {
        if ((rc = h->alloc(&h->lbar, h->nslots_tile)) || (rc = h->alloc(&h->mub[0], h->nint * kAccStride)) ||
            (rc = h->alloc(&h->mub[1], h->nint * kAccStride)) || (rc = h->alloc(&h->Fbar, h->nnodes_tile)) ||
            (rc = h->alloc(&h->Bbar, h->nnodes_tile)) || (rc = h->alloc(&h->cbar, h->nint)) ||
            (rc = h->alloc(&h->rbar, h->nint)) || (rc = h->alloc(&h->pend_tmp, h->nint)))
            return rc;
    }
    cudaStream_t s = h->stream;
    Trace tr;
    tr.scope = "grad";
    auto mark = [&](const char* what) {
        if (tr.on) cudaStreamSynchronize(s);
        tr.mark(what);
    };
    mark("setup");
    if ((rc = save_snap(h, &h->final_state, h->B))) return rc;
    CK(cudaMemsetAsync(h->lbar, 0, size_t(h->nslots_tile) * 4, s));
    CK(cudaMemsetAsync(h->Fbar, 0, size_t(h->nnodes_tile) * 4, s));
    CK(cudaMemsetAsync(h->Bbar, 0, size_t(h->nnodes_tile) * 4, s));
    // the bound: forward min-sum on lambda + pend (recompute its node costs, then reverse)
    if ((rc = h->pass(Pass::FwdMM))) return rc;
    {
        CK(launch_pend_table(h->msum_rd(), h->deg, h->nint, h->fx.inv, h->pend_tmp, s));
        AdjArgs a = adj_args(h);
        a.lam_in = h->lam;
        a.lam_in_lo = h->lam_lo;
        a.pend_in = h->pend_tmp;
        a.own = h->F;
        a.mubar_out = h->mub[0];
        CK(launch_adjoint_all(h, Adj::Bound, a));
    }
    mark("bound adjoint");
    int nx = 0;  // mub[nx]: adjoint of the deferred means the pass being reversed produced
    for (int k = nck - 1; k >= 0; --k) {
        if ((rc = load_snap(h, h->checkpoints[k], h->B))) return rc;
        const int nit = std::min(G, T - k * G);
        // replay: each half-pass's inputs (lambda, and the deferred means it adds as a
        // per-variable table) go to the tape, and the pass stores its node costs straight into
        // the tape (the node arrays are pointed there); the node costs it reads are the
        // previous pass's (or the checkpoint's) stored ones
        float* const F0 = h->F;
        float* const B0 = h->B;
        const size_t ns = size_t(h->nslots_tile) * 4;
        for (int t = 0; t < nit && !rc; ++t)
            for (int dir = 0; dir < 2 && !rc; ++dir) {
                Snap& tp = h->tape[2 * t + dir];
                if ((rc = d2d(tp.lam, h->lam, ns, s)) || (rc = d2d(tp.lam_lo, h->lam_lo, ns, s))) break;
                const cudaError_t e = launch_pend_table(h->msum_rd(), h->deg, h->nint, h->fx.inv, tp.pend, s);
                if (e != cudaSuccess) {
                    rc = fail(DISCO_ERR_CUDA, std::string("grad: pend table: ") + cudaGetErrorString(e));
                    break;
                }
                (dir == 0 ? h->F : h->B) = tp.nodes;
                rc = h->pass(dir == 0 ? Pass::FwdMMA : Pass::BwdMMA);
            }
        h->F = F0;
        h->B = B0;
        if (rc) return rc;
        mark("block replay");
        for (int e = 2 * nit - 1; e >= 0; --e) {
            const Snap& tp = h->tape[e];
            const bool fwd = (e % 2) == 0;
            CK(launch_rbar_table(h->mub[nx], h->deg, h->nint, h->rbar, s));
            AdjArgs a = adj_args(h);
            a.lam_in = tp.lam;
            a.lam_in_lo = tp.lam_lo;
            a.pend_in = tp.pend;
            a.other = e == 0 ? h->checkpoints[k].nodes : h->tape[e - 1].nodes;
            a.own = tp.nodes;
            a.own_bar = fwd ? h->Fbar : h->Bbar;
            a.other_bar = fwd ? h->Bbar : h->Fbar;
            a.rbar = h->rbar;
            a.mubar_out = h->mub[nx ^ 1];
            CK(launch_adjoint_all(h, fwd ? Adj::Fwd : Adj::Bwd, a));
            nx ^= 1;
        }
        mark("block reverse");
    }
    // the initial backward min-sum on lambda^0
    {
        const Snap& c0 = h->checkpoints[0];
        if ((rc = load_snap(h, c0, h->B))) return rc;
        if ((rc = h->pass(Pass::BwdReset))) return rc;
        CK(launch_pend_table(c0.msum, h->deg, h->nint, h->fx.inv, h->pend_tmp, s));
        AdjArgs a = adj_args(h);
        a.lam_in = c0.lam;
        a.lam_in_lo = c0.lam_lo;
        a.pend_in = h->pend_tmp;
        a.own = h->B;
        a.own_bar = h->Bbar;
        CK(launch_adjoint_all(h, Adj::Reset, a));
    }
    CK(launch_adj_cost(h->var, h->desc, h->nslots_tile, h->lbar, h->deg, h->nint, h->mub[nx ^ 1], h->cbar, s));
    if ((rc = load_snap(h, h->final_state, h->B))) return rc;
    h->has_b = true;
    std::vector<float> cb(static_cast<size_t>(h->nint));
    CK(cudaMemcpyAsync(cb.data(), h->cbar, cb.size() * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    mark("reset adjoint, costs");
    // chain rule to the pair costs: c_e = (mean of e's three pair costs) / scale, or with
    // cost model 1 (Eq. 2) c_e = sum over the corners of (A_X(m) + A_Y(n)) d(m, n) / scale
    std::vector<float> g(static_cast<size_t>(need), 0.0f);
    std::vector<int64_t> offs(h->plans.size() + 1, 0);
    for (size_t i = 0; i < h->plans.size(); ++i) offs[i + 1] = offs[i] + int64_t(h->plans[i].nvx) * h->plans[i].nvy;
    parallel_chunks(int64_t(h->plans.size()), std::min<int>(host_threads(h->opts), int(h->plans.size())),
                    [&](int, int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i) {
        const Plan& P = h->plans[i];
        const int64_t off = offs[i];
        std::vector<double> ge(static_cast<size_t>(P.nvars), 0.0);
        for (int64_t u = 0; u < P.n_free; ++u) ge[size_t(P.free_orig[u])] = cb[size_t(h->var_base[i] + u)];
        double cc = 0.0;
        for (int64_t e = 0; e < P.nvars; ++e) {
            if (P.fixed[e] == 1) ge[e] = 1.0;
            cc += ge[e] * P.cost[e];
        }
        std::vector<double> gp(static_cast<size_t>(P.nvx) * P.nvy, 0.0);
        for (int64_t e = 0; e < P.nvars; ++e) {
            double gr = ge[e] / P.cost_scale;
            if (e == P.cost_scale_elem) gr -= cc / P.cost_scale;
            if (gr == 0.0) continue;
            if (P.area_x.empty()) {
                for (int v = 0; v < 3; ++v) gp[size_t(P.vm[3 * e + v]) * P.nvy + P.vn[3 * e + v]] += gr / 3.0;
            } else {
                for (int v = 0; v < 3; ++v) {
                    const int m = P.vm[3 * e + v], nn = P.vn[3 * e + v];
                    gp[size_t(m) * P.nvy + nn] += gr * (P.area_x[size_t(m)] + P.area_y[size_t(nn)]);
                }
            }
        }
        for (size_t q = 0; q < gp.size(); ++q) g[size_t(off) + q] = float(gp[q]);
    }
    });
    mark("chain to pair costs");
    rc = write_out(dlb_dpair_costs, g.data(), g.size() * 4, s);
    mark("output");
    return rc;
}

void disco_free(disco_handle* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    delete h;
}

}  // extern "C"
