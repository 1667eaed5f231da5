// sm_103a kernels of the dual / primal hot path.
//
// One warp per tile of 32 BDD segments, one lane per segment (tile layout in kernels.h): at
// every step the 32 lanes touch the same layer index of their own segment, so each field
// of a layer (variable, descriptor, lambda, the node costs of one state s) is one coalesced
// 128-byte line. The node costs of the current layer live in registers (W per lane); only
// the costs that the other direction needs are stored (F forward, B backward: 8 bytes per
// node per iteration).
//
// Passages: shortest paths through BDDs (Sec. 3.2), min-marginal differences (App. A.5),
// deferred, parallel-across-BDDs min-marginal averaging (Alg. 1 "MMA"), dual bound (Eq. D),
// rounding by min-marginal agreement and propagation (App. A.5, Sec. 3 pipeline).
//
// Averaging in the same launch, without waiting: a slot of variable i reads i's sum of the
// masses the previous update pass removed (8 bytes; its mean is the deferred mean), and adds
// the mass it removes itself, rounded to the fixed-point grid, into i's sum of this pass with
// a fire-and-forget red.add (device_util.cuh). Integer sums do not depend on the order of the
// additions, so every result is deterministic and the same for every launch geometry.
#include <atomic>
#include <cfloat>

#include "device_util.cuh"
#include "kernels.h"

namespace disco {

std::atomic<int64_t> g_launches{0};

namespace {

constexpr int kWarpsPerBlock = 2;
// Resident warps per SM the fused half-pass kernels are compiled for (caps their registers).
constexpr int kFusedWarpsPerSM = 24;

using namespace dev;

// Index checks of the bounds-checking build (DISCO_BOUNDS_CHECK): an index outside its array
// sets kStatusBounds in the status word and the access is skipped; the host turns the bit into
// an error at its next synchronisation. The normal build compiles the checks away.
#ifdef DISCO_BOUNDS_CHECK
__device__ __forceinline__ bool in_bounds(int64_t i, int64_t n, uint32_t* status) {
    if (i >= 0 && i < n) return true;
    atomicOr(status, kStatusBounds);
    return false;
}
#define DISCO_IN(i, n) in_bounds((i), (n), a.status)
#else
#define DISCO_IN(i, n) true
#endif

// ---------------------------------------------------------------------------------------
// Inputs of one layer of one lane are staged in shared memory ahead of their use. A lane's
// layers form a sequential recurrence only through the node costs it keeps in registers;
// every load (lambda, its low part, the variable's averaging sum, the other direction's
// node costs) is independent of it. Each lane therefore keeps kRing layers in flight with
// asynchronous copies (cp.async, one commit group per layer) into its own slots of a
// per-warp ring; descriptors and variable ids are fetched kRing layers before the copies
// that need them. Lanes only ever read their own slots, so no warp synchronisation is needed.
constexpr int kRing = 3;

// Stage layout (floats, per warp): lam[32] lo[32] sum[32][2] nodes[W][32].
template <int W>
__host__ __device__ constexpr int stage_floats() { return (4 + W) * 32; }
template <int W>
__host__ __device__ constexpr int ring_floats() { return kRing * stage_floats<W>(); }

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(float* dst, const void* src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// red.add of a signed fixed-point mass into a variable's sum (two's complement: the unsigned
// 64-bit add is the signed one); the result is not read, so no round trip is waited for.
__device__ __forceinline__ void red_add(long long* p, long long q) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(q));
}

__device__ __forceinline__ void load_head(const KArgs& a, int64_t si, bool ok, uint32_t& v, uint32_t& d) {
    ok = ok && DISCO_IN(si, a.nslots);
    v = ok ? __ldg(a.var + si) : kNoVar;
    d = ok ? __ldg(a.desc + si) : 0u;
#ifdef DISCO_BOUNDS_CHECK
    if (v != kNoVar && !DISCO_IN(int64_t(v), a.nvars)) v = kNoVar;
#endif
}

// Copies of one layer's inputs into stage `st` (this lane's slots), then one commit.
// NODES: 0 none, 1 = B of layer l + 1 (count wn), 2 = F of layer l (count w); `nodes` is that
// array and `ni` the index of the row's first node (state 0) of this lane.
template <int W, int NODES>
__device__ __forceinline__ void stage_issue(const KArgs& a, float* st, int lane, int64_t si, const float* nodes,
                                            int64_t ni, uint32_t v, uint32_t dsc) {
    if (v != kNoVar) {
        cp_async4(st + lane, a.lam + si);
        cp_async4(st + 32 + lane, a.lam_lo + si);
        cp_async8(st + 64 + 2 * lane, a.msum_rd + v);
        if (NODES) {
            const int n = NODES == 1 ? int((dsc >> 6) & 63u) + 1 : int(dsc & 63u) + 1;
#pragma unroll
            for (int s = 0; s < W; ++s)
                if (s < n && DISCO_IN(ni + s * 32, a.nnodes)) cp_async4(st + (4 + s) * 32 + lane, nodes + ni + s * 32);
        }
    }
    cp_commit();
}

// The staged inputs of one layer, read back into registers.
template <int W>
struct Staged {
    float lam, lo;
    long long sum;
    float nb[W];
};

template <int W, int NODES>
__device__ __forceinline__ void stage_read(const float* st, int lane, const Desc& d, Staged<W>& x) {
    x.lam = st[lane];
    x.lo = st[32 + lane];
    x.sum = *reinterpret_cast<const long long*>(st + 64 + 2 * lane);
    if (NODES) {
        const int n = NODES == 1 ? d.wn : d.w;
#pragma unroll
        for (int s = 0; s < W; ++s) x.nb[s] = s < n ? st[(4 + s) * 32 + lane] : BIG;
    }
}

// The averaging step of an update pass for a free variable: round the removed mass to the
// grid, add it to the variable's sum of this pass, flag a mass outside the grid's range.
// Returns the mass as rounded (what lambda loses).
__device__ __forceinline__ float deposit(const KArgs& a, uint32_t v, float removed) {
    long long q;
    const float r = fx_round(removed, a.fx, q);
    if (!(fabsf(removed) < a.fx.lim)) atomicOr(a.status, kStatusRange);
    red_add(a.msum_wr + v, q);
    return r;
}

// ---------------------------------------------------------------------------------------
// Forward half-pass with min-marginal averaging (and the plain forward min-sum variants).
//   MODE 0: MMA update, store F.       MODE 1: MMA update under fixings, store F.
//   MODE 2: lower bound (no store).    MODE 3: plain min-sum under fixings, store F.
template <int W, int MODE>
__device__ __forceinline__ void forward_tile(const KArgs& a, const int tile, const TileInfo& ti, float* ring) {
    constexpr bool kUpdate = MODE <= 1;
    constexpr bool kRound = MODE == 1 || MODE == 3;
    constexpr bool kStoreF = MODE != 2;
    constexpr int NODES = kUpdate ? 1 : 0;
    constexpr int P = kRing;
    constexpr int SF = stage_floats<W>();
    const int lane = threadIdx.x & 31;
    const int64_t sb = ti.slot_base + lane;
    const int64_t nb = ti.node_base + lane;  // node (l, s) of this lane at nb + (l * W + s) * 32
    const int L = ti.L;
    float f[W];
#pragma unroll
    for (int s = 0; s < W; ++s) f[s] = s == 0 ? 0.0f : BIG;
    uint32_t cv[P], cd[P], hv[P], hd[P];  // descriptors of layers l (staged) and l + P (next to stage)
#pragma unroll
    for (int k = 0; k < P; ++k) {
        load_head(a, sb + int64_t(k) * 32, k < L, cv[k], cd[k]);
        stage_issue<W, NODES>(a, ring + k * SF, lane, sb + int64_t(k) * 32, a.B, nb + int64_t(k + 1) * W * 32, cv[k],
                              cd[k]);
        load_head(a, sb + int64_t(k + P) * 32, k + P < L, hv[k], hd[k]);
    }
    for (int l0 = 0; l0 < L; l0 += P) {
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const int l = l0 + k;
            const uint32_t v = cv[k];
            if (v == kNoVar) goto done;
            cp_wait<P - 1>();
            const Desc d = decode(cd[k]);
            Staged<W> c;
            stage_read<W, NODES>(ring + k * SF, lane, d, c);
            uint32_t nv, nd;
            load_head(a, sb + int64_t(l + 2 * P) * 32, l + 2 * P < L, nv, nd);
            const int64_t si = sb + int64_t(l) * 32;
            const df p = fx_mean(c.sum, d.deg, a.fx.inv);
            df Lm{c.lam, c.lo};
            const uint8_t st = kRound ? __ldg(a.state + v) : kFree;
            const bool al0 = st != kFix1, al1 = st != kFix0;
            float lm = Lm.hi;
            if (kStoreF) {
                const int64_t fr = nb + int64_t(l) * W * 32;
#pragma unroll
                for (int s = 0; s < W; ++s)
                    if (s < d.w && DISCO_IN(fr + s * 32, a.nnodes)) a.F[fr + s * 32] = f[s];
            }
            if (kUpdate) {
                if (st == kFree) {
                    Lm = df_add(Lm, p);
                    // hx[s + 1] = b of node s's 0-child, hx[s + 1 + a] = b of its arithmetic 1-child
                    float hx[W + 2];
                    shift_ext(c.nb, d.d0, hx);
                    const bool up = d.d1 > d.d0;
                    float m0 = BIG, m1 = BIG;
#pragma unroll
                    for (int s = 0; s < W; ++s) m0 = fminf(m0, f[s] + hx[s + 1]);
                    if (d.one) {
                        m1 = f[0] + at_dyn(c.nb, d.d1);
                    } else {
#pragma unroll
                        for (int s = 0; s < W; ++s) m1 = fminf(m1, f[s] + (up ? hx[s + 2] : hx[s]));
                    }
                    const float M = (m1 + Lm.hi) - m0;
                    Lm = df_add_f(Lm, -deposit(a, v, a.omega * M));
                    a.lam[si] = Lm.hi;
                    a.lam_lo[si] = Lm.lo;
                    lm = Lm.hi;
                }
                if (d.rank == 0) a.msum_zero[v] = 0;  // the next update pass's sums start at zero
            } else {
                lm = df_add(Lm, p).hi;
            }
            // gx[s + 1] = f of node s's 0-parent, gx[s + 1 - a] = f of its arithmetic 1-parent
            float gx[W + 2];
            shift_ext(f, -d.d0, gx);
            const bool upf = d.d1 > d.d0;
            const float f0 = f[0];  // a one-hot 1-arc leaves node 0 (read before f is overwritten)
#pragma unroll
            for (int s = 0; s < W; ++s) {
                const float v0 = al0 ? gx[s + 1] : BIG;
                float v1 = BIG;
                if (al1) v1 = (d.one ? (s == d.d1 ? f0 : BIG) : (upf ? gx[s] : gx[s + 2])) + lm;
                f[s] = s < d.wn ? fminf(v0, v1) : BIG;
            }
            // stage layer l + P into the slot just consumed
            stage_issue<W, NODES>(a, ring + k * SF, lane, sb + int64_t(l + P) * 32, a.B, nb + int64_t(l + P + 1) * W * 32,
                                  hv[k], hd[k]);
            cv[k] = hv[k];
            cd[k] = hd[k];
            hv[k] = nv;
            hd[k] = nd;
        }
    }
done:
    cp_wait<0>();
    if (MODE == 2) {
        double x = double(f[0]);  // cost of the cheapest root -> TOP path (0 for an empty lane)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) a.tile_sum[tile] = x;
    }
}

// One width class per launch; dynamic shared memory: kWarpsPerBlock rings of width W.
template <int W, int MODE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_forward(KArgs a) {
    extern __shared__ float smem[];
    const int tile = a.tile0 + int(blockIdx.x) * kWarpsPerBlock + int(threadIdx.x >> 5);
    if (tile >= a.tile_end) return;
    const TileInfo ti = a.tiles[tile];
    forward_tile<W, MODE>(a, tile, ti, smem + (threadIdx.x >> 5) * ring_floats<W>());
}

// Width classes 2, 4 and 6 in one launch (tiles ordered longest first), so that short tiles
// fill the SMs around the long ones; every warp's ring is sized for width kFusedMaxW.
// WPB warps (tiles) per block; every geometry computes the same results.
template <int MODE, int WPB>
__global__ void __launch_bounds__(WPB * 32, kFusedWarpsPerSM / WPB) k_forward_fused(KArgs a) {
    static_assert(kFusedMaxW == 6, "fused dispatch covers widths 2, 4, 6");
    extern __shared__ float smem[];
    const int tile = a.tile0 + int(blockIdx.x) * WPB + int(threadIdx.x >> 5);
    if (tile >= a.tile_end) return;
    const TileInfo ti = a.tiles[tile];
    float* ring = smem + (threadIdx.x >> 5) * ring_floats<kFusedMaxW>();
    if (ti.W == 2) forward_tile<2, MODE>(a, tile, ti, ring);
    else if (ti.W == 4) forward_tile<4, MODE>(a, tile, ti, ring);
    else forward_tile<6, MODE>(a, tile, ti, ring);
}

// ---------------------------------------------------------------------------------------
// Backward half-pass with min-marginal averaging (and plain backward variants).
//   MODE 0: MMA update, store B.                 MODE 1: MMA update under fixings, store B.
//   MODE 2: min-marginals under fixings (out).   MODE 3: plain min-sum under fixings, store B.
template <int W, int MODE>
__device__ __forceinline__ void backward_tile(const KArgs& a, const TileInfo& ti, float* ring) {
    constexpr bool kUpdate = MODE <= 1;
    constexpr bool kRound = MODE >= 1;
    constexpr bool kStoreB = MODE != 2;
    constexpr bool kNeedF = MODE != 3;
    constexpr int NODES = kNeedF ? 2 : 0;
    constexpr int P = kRing;
    constexpr int SF = stage_floats<W>();
    const int lane = threadIdx.x & 31;
    const int64_t sb = ti.slot_base + lane;
    const int64_t nb = ti.node_base + lane;  // node (l, s) of this lane at nb + (l * W + s) * 32
    const int L = ti.L;
    float bn[W];
#pragma unroll
    for (int s = 0; s < W; ++s) bn[s] = s == 0 ? 0.0f : BIG;
    uint32_t cv[P], cd[P], hv[P], hd[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const int l = L - 1 - k;
        load_head(a, sb + int64_t(l) * 32, l >= 0, cv[k], cd[k]);
        stage_issue<W, NODES>(a, ring + k * SF, lane, sb + int64_t(l) * 32, a.F, nb + int64_t(l) * W * 32, cv[k], cd[k]);
        load_head(a, sb + int64_t(l - P) * 32, l - P >= 0, hv[k], hd[k]);
    }
    for (int l0 = L - 1; l0 >= 0; l0 -= P) {
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const int l = l0 - k;
            if (l < 0) goto done;
            uint32_t nv, nd;
            load_head(a, sb + int64_t(l - 2 * P) * 32, l - 2 * P >= 0, nv, nd);
            const uint32_t v = cv[k];
            if (v != kNoVar) {
                cp_wait<P - 1>();
                const Desc d = decode(cd[k]);
                Staged<W> c;
                stage_read<W, NODES>(ring + k * SF, lane, d, c);
                const int64_t si = sb + int64_t(l) * 32;
                const df p = fx_mean(c.sum, d.deg, a.fx.inv);
                df Lm{c.lam, c.lo};
                const uint8_t st = kRound ? __ldg(a.state + v) : kFree;
                const bool al0 = st != kFix1, al1 = st != kFix0;
                float lm = Lm.hi;
                const float b1 = d.one ? at_dyn(bn, d.d1) : BIG;  // target of node 0's 1-arc (one-hot chains)
                // hx[s + 1] = b of node s's 0-child, hx[s + 1 + a] = b of its arithmetic 1-child
                float hx[W + 2];
                shift_ext(bn, d.d0, hx);
                const bool up = d.d1 > d.d0;
                if (kNeedF) {
                    float m0 = BIG, m1 = BIG;
#pragma unroll
                    for (int s = 0; s < W; ++s) m0 = fminf(m0, c.nb[s] + (al0 ? hx[s + 1] : BIG));
                    if (al1) {
                        if (d.one) {
                            m1 = c.nb[0] + b1;
                        } else {
#pragma unroll
                            for (int s = 0; s < W; ++s) m1 = fminf(m1, c.nb[s] + (up ? hx[s + 2] : hx[s]));
                        }
                    }
                    if (kUpdate) {
                        if (st == kFree) {
                            Lm = df_add(Lm, p);
                            const float M = (m1 + Lm.hi) - m0;
                            Lm = df_add_f(Lm, -deposit(a, v, a.omega * M));
                            a.lam[si] = Lm.hi;
                            a.lam_lo[si] = Lm.lo;
                            lm = Lm.hi;
                        }
                        if (d.rank == 0) a.msum_zero[v] = 0;  // the next update pass's sums start at zero
                    } else {
                        lm = df_add(Lm, p).hi;
                        const float M = (m1 + lm) - m0;
                        a.mm_slot[si] = M;
                        a.mm_var[size_t(v) * kAccStride + d.rank] = M;
                    }
                } else {
                    lm = df_add(Lm, p).hi;
                }
                const int64_t br = nb + int64_t(l) * W * 32;
#pragma unroll
                for (int s = 0; s < W; ++s) {
                    const float v0 = al0 ? hx[s + 1] : BIG;
                    float v1 = BIG;
                    if (al1) v1 = (d.one ? (s == 0 ? b1 : BIG) : (up ? hx[s + 2] : hx[s])) + lm;
                    bn[s] = s < d.w ? fminf(v0, v1) : BIG;
                    if (kStoreB && s < d.w && DISCO_IN(br + s * 32, a.nnodes)) a.B[br + s * 32] = bn[s];
                }
            }
            stage_issue<W, NODES>(a, ring + k * SF, lane, sb + int64_t(l - P) * 32, a.F, nb + int64_t(l - P) * W * 32,
                                  hv[k], hd[k]);
            cv[k] = hv[k];
            cd[k] = hd[k];
            hv[k] = nv;
            hd[k] = nd;
        }
    }
done:
    cp_wait<0>();
}

template <int W, int MODE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_backward(KArgs a) {
    extern __shared__ float smem[];
    const int tile = a.tile0 + int(blockIdx.x) * kWarpsPerBlock + int(threadIdx.x >> 5);
    if (tile >= a.tile_end) return;
    const TileInfo ti = a.tiles[tile];
    backward_tile<W, MODE>(a, ti, smem + (threadIdx.x >> 5) * ring_floats<W>());
}

template <int MODE, int WPB>
__global__ void __launch_bounds__(WPB * 32, kFusedWarpsPerSM / WPB) k_backward_fused(KArgs a) {
    extern __shared__ float smem[];
    const int tile = a.tile0 + int(blockIdx.x) * WPB + int(threadIdx.x >> 5);
    if (tile >= a.tile_end) return;
    const TileInfo ti = a.tiles[tile];
    float* ring = smem + (threadIdx.x >> 5) * ring_floats<kFusedMaxW>();
    if (ti.W == 2) backward_tile<2, MODE>(a, ti, ring);
    else if (ti.W == 4) backward_tile<4, MODE>(a, ti, ring);
    else backward_tile<6, MODE>(a, ti, ring);
}

// ---------------------------------------------------------------------------------------
// Value supports under fixings: which values of each slot's variable lie on some
// root -> TOP path of its segment that respects the fixings (bit-parallel over nodes).
template <int W>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_supports(KArgs a) {
    const int lane = threadIdx.x & 31;
    const int tile = a.tile0 + int(blockIdx.x) * kWarpsPerBlock + int(threadIdx.x >> 5);
    if (tile >= a.tile_end) return;
    const TileInfo ti = a.tiles[tile];
    const int64_t sb = ti.slot_base + lane;
    uint64_t rf = 1;  // nodes of the current layer reachable from the root
    int Ll = 0;
    for (int l = 0; l < ti.L; ++l) {
        const int64_t si = sb + int64_t(l) * 32;
        const uint32_t v = __ldg(a.var + si);
        if (v == kNoVar) break;
        const Desc d = decode(__ldg(a.desc + si));
        const uint8_t st = __ldg(a.state + v);
        a.reach[si] = uint32_t(rf);
        uint64_t n0 = st != kFix1 ? shl(rf, d.d0) : 0;
        uint64_t n1 = 0;
        if (st != kFix0) n1 = d.one ? ((rf & 1ull) << d.d1) : shl(rf, d.d1);
        rf = (n0 | n1) & low_mask(d.wn);
        Ll = l + 1;
    }
    uint64_t rb = 1;  // nodes of the next layer that reach TOP
    for (int l = Ll - 1; l >= 0; --l) {
        const int64_t si = sb + int64_t(l) * 32;
        const uint32_t v = __ldg(a.var + si);
        const Desc d = decode(__ldg(a.desc + si));
        const uint8_t st = __ldg(a.state + v);
        const uint64_t rfl = a.reach[si];
        const uint64_t ok0 = st != kFix1 ? (shl(rb, -d.d0) & low_mask(d.w)) : 0;
        uint64_t ok1 = 0;
        if (st != kFix0) ok1 = d.one ? ((rb >> d.d1) & 1ull) : (shl(rb, -d.d1) & low_mask(d.w));
        const uint8_t sup = uint8_t(((rfl & ok0) ? 1 : 0) | ((rfl & ok1) ? 2 : 0));
        a.sup_var[size_t(v) * kAccStride + d.rank] = sup;
        rb = ok0 | ok1;
    }
}

template <int WPB>
cudaError_t launch_fused_g(Pass pass, const KArgs& a, cudaStream_t s) {
    const int n = a.tile_end - a.tile0;
    if (n <= 0) return cudaSuccess;
    const dim3 grid((n + WPB - 1) / WPB), block(WPB * 32);
    const size_t sm = size_t(WPB) * ring_floats<kFusedMaxW>() * sizeof(float);
    switch (pass) {
        case Pass::FwdMMA: k_forward_fused<0, WPB><<<grid, block, sm, s>>>(a); break;
        case Pass::BwdMMA: k_backward_fused<0, WPB><<<grid, block, sm, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_fused(Pass pass, const KArgs& a, cudaStream_t s, int geometry) {
    const int n = a.tile_end - a.tile0;
    if (n <= 0) return cudaSuccess;
    if (pass == Pass::FwdMMA || pass == Pass::BwdMMA) {
        switch (geometry) {
            case 1: return launch_fused_g<1>(pass, a, s);
            case 4: return launch_fused_g<4>(pass, a, s);
            default: return launch_fused_g<2>(pass, a, s);
        }
    }
    constexpr int WPB = kWarpsPerBlock;
    const dim3 grid((n + WPB - 1) / WPB), block(WPB * 32);
    const size_t sm = size_t(WPB) * ring_floats<kFusedMaxW>() * sizeof(float);
    switch (pass) {
        case Pass::FwdMMARound: k_forward_fused<1, WPB><<<grid, block, sm, s>>>(a); break;
        case Pass::Lb: k_forward_fused<2, WPB><<<grid, block, sm, s>>>(a); break;
        case Pass::FwdMM: k_forward_fused<3, WPB><<<grid, block, sm, s>>>(a); break;
        case Pass::BwdMMARound: k_backward_fused<1, WPB><<<grid, block, sm, s>>>(a); break;
        case Pass::BwdMM: k_backward_fused<2, WPB><<<grid, block, sm, s>>>(a); break;
        case Pass::BwdReset: k_backward_fused<3, WPB><<<grid, block, sm, s>>>(a); break;
        case Pass::Supports: k_supports<kFusedMaxW><<<grid, block, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <int W>
cudaError_t launch_w(Pass pass, const KArgs& a, cudaStream_t s) {
    const int n = a.tile_end - a.tile0;
    if (n <= 0) return cudaSuccess;
    const dim3 grid((n + kWarpsPerBlock - 1) / kWarpsPerBlock), block(kWarpsPerBlock * 32);
    const size_t sm = size_t(kWarpsPerBlock) * ring_floats<W>() * sizeof(float);
    switch (pass) {
        case Pass::FwdMMA: k_forward<W, 0><<<grid, block, sm, s>>>(a); g_launches.fetch_add(1, std::memory_order_relaxed); break;
        case Pass::FwdMMARound: k_forward<W, 1><<<grid, block, sm, s>>>(a); g_launches.fetch_add(1, std::memory_order_relaxed); break;
        case Pass::Lb: k_forward<W, 2><<<grid, block, sm, s>>>(a); g_launches.fetch_add(1, std::memory_order_relaxed); break;
        case Pass::FwdMM: k_forward<W, 3><<<grid, block, sm, s>>>(a); g_launches.fetch_add(1, std::memory_order_relaxed); break;
        case Pass::BwdMMA: k_backward<W, 0><<<grid, block, sm, s>>>(a); g_launches.fetch_add(1, std::memory_order_relaxed); break;
        case Pass::BwdMMARound: k_backward<W, 1><<<grid, block, sm, s>>>(a); g_launches.fetch_add(1, std::memory_order_relaxed); break;
        case Pass::BwdMM: k_backward<W, 2><<<grid, block, sm, s>>>(a); g_launches.fetch_add(1, std::memory_order_relaxed); break;
        case Pass::BwdReset: k_backward<W, 3><<<grid, block, sm, s>>>(a); g_launches.fetch_add(1, std::memory_order_relaxed); break;
        case Pass::Supports: k_supports<W><<<grid, block, 0, s>>>(a); g_launches.fetch_add(1, std::memory_order_relaxed); break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Per instance: its tiles' sums in its fixed tile order plus its constant (one block each).
__global__ void k_sum_instances(const double* __restrict__ x, const int32_t* __restrict__ ptr,
                                const int32_t* __restrict__ tiles, const double* __restrict__ add, double* out) {
    __shared__ double sh[256];
    const int i = blockIdx.x;
    double s = 0.0;
    for (int k = ptr[i] + threadIdx.x; k < ptr[i + 1]; k += blockDim.x) s += x[tiles[k]];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (int(threadIdx.x) < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = sh[0] + add[i];
}

__global__ void k_sum_tiles(const double* __restrict__ x, int64_t n, double add, double* out) {
    __shared__ double sh[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (int(threadIdx.x) < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] + add;
}

__global__ void k_gather(const float* __restrict__ src, const int64_t* __restrict__ pos, int64_t n, float* dst) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = src[pos[i]];
}

__global__ void k_scatter(const float* __restrict__ src, const int64_t* __restrict__ pos, int64_t n, float* dst) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        dst[pos[i]] = src[i];
}

__global__ void k_pend(const long long* __restrict__ msum, const uint8_t* __restrict__ deg, int64_t n, float inv,
                       float* pend) {
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x)
        pend[v] = deg[v] ? fx_mean(msum[v], deg[v], inv).hi : 0.0f;
}

// The sum whose deferred mean is pend[v]: pend[v] deg[v] on the grid (a one-off import, so
// FP64 is fine here); a value outside the sums' range is clamped and flagged.
__global__ void k_set_pend(const float* __restrict__ pend, const uint8_t* __restrict__ deg, int64_t n, float scale,
                           long long* msum, uint32_t* status) {
    const double lim = double(1ll << (kFxSumBits - 1));
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        double x = double(pend[v]) * double(deg[v]) * double(scale);
        if (!(fabs(x) < lim)) {
            atomicOr(status, kStatusRange);
            x = x > 0.0 ? lim : -lim;
        }
        msum[v] = __double2ll_rn(x);
    }
}

__global__ void k_flush(const uint32_t* __restrict__ var, const uint32_t* __restrict__ desc, int64_t n,
                        const long long* __restrict__ msum, float inv, float* lam, float* lam_lo) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t v = var[i];
        if (v == kNoVar) continue;
        const df L = df_add(df{lam[i], lam_lo[i]}, fx_mean(msum[v], decode(desc[i]).deg, inv));
        lam[i] = L.hi;
        lam_lo[i] = L.lo;
    }
}

__global__ void k_decide(const float* __restrict__ mm_var, const uint8_t* __restrict__ deg,
                         const uint8_t* __restrict__ state, int64_t n, float tau, uint8_t* trial) {
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        uint8_t st = state[v];
        if (st == kFree && deg[v] > 0) {
            bool pos = true, neg = true;
            for (int r = 0; r < deg[v]; ++r) {
                const float M = mm_var[v * kAccStride + r];
                pos = pos && (M > tau);
                neg = neg && (M < -tau);
            }
            st = pos ? kFix0 : (neg ? kFix1 : kFree);
        }
        trial[v] = st;
    }
}

// Per instance (4 counters each, instance of variable v = inst[v]): [0] newly forced
// variables, [1] conflicts, [2] free variables left.
__global__ void k_apply(const uint8_t* __restrict__ sup, const uint8_t* __restrict__ deg,
                        const int32_t* __restrict__ inst, int64_t n, uint8_t* state, int* counters) {
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        const int dg = deg[v];
        if (dg == 0) continue;
        int* c = counters + 4 * inst[v];
        bool can0 = true, can1 = true;
        for (int r = 0; r < dg; ++r) {
            const uint8_t s = sup[v * kAccStride + r];
            can0 = can0 && (s & 1);
            can1 = can1 && (s & 2);
        }
        const uint8_t st = state[v];
        if ((st == kFix0 && !can0) || (st == kFix1 && !can1) || (st == kFree && !can0 && !can1)) {
            atomicAdd(c + 1, 1);
        } else if (st == kFree) {
            if (!can0) { state[v] = kFix1; atomicAdd(c, 1); }
            else if (!can1) { state[v] = kFix0; atomicAdd(c, 1); }
            else atomicAdd(c + 2, 1);
        }
    }
}

// Free variables per instance into counters[4 * i + 2].
__global__ void k_count_free(const uint8_t* __restrict__ state, const uint8_t* __restrict__ deg,
                             const int32_t* __restrict__ inst, int64_t n, int* counters) {
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x)
        if (deg[v] && state[v] == kFree) atomicAdd(counters + 4 * inst[v] + 2, 1);
}

__global__ void k_perturb(const uint32_t* __restrict__ var, const uint32_t* __restrict__ desc, int64_t n,
                          const float* __restrict__ mm_var, const uint8_t* __restrict__ state, float delta, float* lam,
                          float* lam_lo) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t v = var[i];
        if (v == kNoVar || state[v] != kFree) continue;
        const int dg = decode(desc[i]).deg;
        float s = 0.0f;
        for (int r = 0; r < dg; ++r) s += mm_var[size_t(v) * kAccStride + r];
        const df L = df_add_f(df{lam[i], lam_lo[i]}, s >= 0.0f ? delta : -delta);
        lam[i] = L.hi;
        lam_lo[i] = L.lo;
    }
}

// ---- feature distances: d[m, n] = mean_k (FX[m,k] - FY[n,k])^2, 64 x 64 tiles, 4 x 4 per thread
constexpr int kPT = 64, kPK = 32;
// NORM = false: mean squared difference; NORM = true: Euclidean distance (Eq. 2).
template <bool NORM>
__global__ void __launch_bounds__(256) k_pair_costs(const float* __restrict__ FX, const float* __restrict__ FY, int nvx,
                                                    int nvy, int dim, float* __restrict__ d) {
    __shared__ float sx[kPK][kPT + 1];
    __shared__ float sy[kPK][kPT + 1];
    const int m0 = blockIdx.y * kPT, n0 = blockIdx.x * kPT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < dim; k0 += kPK) {
        for (int i = threadIdx.x; i < kPT * kPK; i += 256) {
            const int r = i / kPK, c = i % kPK;
            const int m = m0 + r, n = n0 + r, k = k0 + c;
            sx[c][r] = (m < nvx && k < dim) ? FX[size_t(m) * dim + k] : 0.0f;
            sy[c][r] = (n < nvy && k < dim) ? FY[size_t(n) * dim + k] : 0.0f;
        }
        __syncthreads();
        const int kk = min(kPK, dim - k0);
        for (int c = 0; c < kk; ++c) {
            float xv[4], yv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { xv[i] = sx[c][ty * 4 + i]; yv[i] = sy[c][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float t = xv[i] - yv[j];
                    acc[i][j] = fmaf(t, t, acc[i][j]);
                }
        }
        __syncthreads();
    }
    const float inv = 1.0f / float(dim);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < nvx && n < nvy) d[size_t(m) * nvy + n] = NORM ? sqrtf(acc[i][j]) : acc[i][j] * inv;
        }
}

__global__ void k_transpose(const float* __restrict__ src, int rows, int cols, float* __restrict__ dst) {
    __shared__ float t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[i][threadIdx.x] = src[size_t(r) * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[size_t(c) * rows + r] = t[threadIdx.x][i];
    }
}

// k smallest entries of every row (ties to the lower column), one warp per row: k rounds of
// a warp-wide arg-min over the entries ordered after the previous pick. Entries that are not
// below FLT_MAX (+inf, NaN) are never picked; the missing picks are written as -1.
__global__ void k_topk_rows(const float* __restrict__ d, int rows, int cols, int k, int32_t* __restrict__ idx) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const float* r = d + size_t(row) * cols;
    float pv = -FLT_MAX;
    int pi = -1;
    for (int t = 0; t < k && t < cols; ++t) {
        float bv = FLT_MAX;
        int bi = INT32_MAX;
        for (int c = lane; c < cols; c += 32) {
            const float x = r[c];
            const bool after = (x > pv) || (x == pv && c > pi);
            if (after && ((x < bv) || (x == bv && c < bi))) { bv = x; bi = c; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if ((ov < bv) || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        // no entry left below the sentinel (the rest are +inf or NaN): no pick
        if (lane == 0) idx[size_t(row) * k + t] = bi == INT32_MAX ? -1 : bi;
        pv = bv;
        pi = bi;
    }
}

// allowed[m, n] = 1 for every n in the closed 1-ring of a pick of row m (transposed: the
// rows are Y vertices n and the ring is on X).
__global__ void k_dilate(const int32_t* __restrict__ topk, int rows, int k, const int32_t* __restrict__ ring_ptr,
                         const int32_t* __restrict__ ring, int nvy, bool transposed, uint8_t* allowed) {
    const int row = blockIdx.x;
    if (row >= rows) return;
    for (int t = threadIdx.y; t < k; t += blockDim.y) {
        const int c = topk[size_t(row) * k + t];
        if (c < 0) continue;  // fewer than k finite entries in the row
        for (int j = ring_ptr[c] + threadIdx.x; j < ring_ptr[c + 1]; j += blockDim.x) {
            const int o = ring[j];
            if (!transposed) allowed[size_t(row) * nvy + o] = 1;
            else allowed[size_t(o) * nvy + row] = 1;
        }
    }
}

inline int grid_for(int64_t n, int block) {
    const int64_t g = (n + block - 1) / block;
    return int(g < 1 ? 1 : (g > 152 * 64 ? 152 * 64 : g));
}

}  // namespace

cudaError_t launch_pass(Pass pass, int W, const KArgs& a, cudaStream_t s, int geometry) {
    switch (W) {
        case 0: return launch_fused(pass, a, s, geometry);
        case 8: return launch_w<8>(pass, a, s);
        case 16: return launch_w<16>(pass, a, s);
        case 32: return launch_w<32>(pass, a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sum_instances(const double* tile_sum, const int32_t* ptr, const int32_t* tiles, const double* add,
                                 int64_t n, double* out, cudaStream_t s) {
    if (n > 0) k_sum_instances<<<unsigned(n), 256, 0, s>>>(tile_sum, ptr, tiles, add, out);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}
cudaError_t launch_sum_tiles(const double* tile_sum, int64_t n, double add, double* out, cudaStream_t s) {
    k_sum_tiles<<<1, 1024, 0, s>>>(tile_sum, n, add, out);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}
cudaError_t launch_gather_f32(const float* src, const int64_t* pos, int64_t n, float* dst, cudaStream_t s) {
    if (n > 0) k_gather<<<grid_for(n, 256), 256, 0, s>>>(src, pos, n, dst);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}
cudaError_t launch_scatter_f32(const float* src, const int64_t* pos, int64_t n, float* dst, cudaStream_t s) {
    if (n > 0) k_scatter<<<grid_for(n, 256), 256, 0, s>>>(src, pos, n, dst);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}
cudaError_t launch_pend(const long long* msum, const uint8_t* deg, int64_t n, float inv, float* pend, cudaStream_t s) {
    if (n > 0) k_pend<<<grid_for(n, 256), 256, 0, s>>>(msum, deg, n, inv, pend);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}
cudaError_t launch_set_pend(const float* pend, const uint8_t* deg, int64_t n, float scale, long long* msum,
                            uint32_t* status, cudaStream_t s) {
    if (n > 0) k_set_pend<<<grid_for(n, 256), 256, 0, s>>>(pend, deg, n, scale, msum, status);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}
cudaError_t launch_flush(const uint32_t* var, const uint32_t* desc, int64_t n, const long long* msum, float inv,
                         float* lam, float* lam_lo, cudaStream_t s) {
    if (n > 0) k_flush<<<grid_for(n, 256), 256, 0, s>>>(var, desc, n, msum, inv, lam, lam_lo);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}
cudaError_t launch_decide(const float* mm_var, const uint8_t* deg, const uint8_t* state, int64_t n, float tau,
                          uint8_t* trial, cudaStream_t s) {
    if (n > 0) k_decide<<<grid_for(n, 256), 256, 0, s>>>(mm_var, deg, state, n, tau, trial);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}
cudaError_t launch_apply(const uint8_t* sup_var, const uint8_t* deg, const int32_t* inst, int64_t n, uint8_t* state,
                         int* counters, cudaStream_t s) {
    if (n > 0) k_apply<<<grid_for(n, 256), 256, 0, s>>>(sup_var, deg, inst, n, state, counters);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}
cudaError_t launch_count_free(const uint8_t* state, const uint8_t* deg, const int32_t* inst, int64_t n, int* counters,
                              cudaStream_t s) {
    if (n > 0) k_count_free<<<grid_for(n, 256), 256, 0, s>>>(state, deg, inst, n, counters);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}
cudaError_t launch_perturb(const uint32_t* var, const uint32_t* desc, int64_t n, const float* mm_var,
                           const uint8_t* state, float delta, float* lam, float* lam_lo, cudaStream_t s) {
    if (n > 0) k_perturb<<<grid_for(n, 256), 256, 0, s>>>(var, desc, n, mm_var, state, delta, lam, lam_lo);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}
cudaError_t launch_pair_costs(const float* FX, const float* FY, int nvx, int nvy, int dim, float* d, cudaStream_t s,
                              bool norm) {
    const dim3 grid((nvy + kPT - 1) / kPT, (nvx + kPT - 1) / kPT);
    if (norm) k_pair_costs<true><<<grid, 256, 0, s>>>(FX, FY, nvx, nvy, dim, d);
    else k_pair_costs<false><<<grid, 256, 0, s>>>(FX, FY, nvx, nvy, dim, d);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}
cudaError_t launch_transpose(const float* src, int rows, int cols, float* dst, cudaStream_t s) {
    const dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    k_transpose<<<grid, block, 0, s>>>(src, rows, cols, dst);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}
cudaError_t launch_topk_rows(const float* d, int rows, int cols, int k, int32_t* idx, cudaStream_t s) {
    k_topk_rows<<<(rows + 7) / 8, 256, 0, s>>>(d, rows, cols, k, idx);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}
cudaError_t launch_dilate(const int32_t* topk, int rows, int k, const int32_t* ring_ptr, const int32_t* ring, int nvy,
                          bool transposed, uint8_t* allowed, cudaStream_t s) {
    k_dilate<<<rows, dim3(8, 8), 0, s>>>(topk, rows, k, ring_ptr, ring, nvy, transposed, allowed);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace disco
