// Adjoint (reverse mode) of the deferred-MMA dual iterations: d(bound) / d(lambda^0).
//
// The bound after T iterations (Eq. D objective at lambda + pend) is a piecewise linear
// function of the costs: every operation of a half-pass (Alg. 1 "MMA": min-marginals from
// shortest paths, Sec. 3.2 / App. A.5, the damped update, the deferred mean) is a min, a
// sum or a scaling. Its gradient pushes adjoints back through each min to the argument that
// attained it. Each kernel here reverses one pass of one lane's BDD segment (same tile
// layout as the forward kernels, one lane per segment, no atomics). It reads the pass's
// inputs and the own-direction node costs the pass stored, both recorded when the pass was
// replayed by the normal kernel, so every min is decided on bit-identical values; the lane
// sweeps its layers in the opposite order carrying the adjoints of the current layer's node
// costs in registers.
//
// Per layer of a forward MMA half-pass (backward is the mirror image):
//   mu = lambda_in + pend_in;  m0 = min_s f[s] + b[c0(s)];  m1 = min_s f[s] + b[c1(s)]
//   r = omega (m1 + mu - m0);  lambda_out = mu - r;  removed mass (for the next mean) = r
//   f'[s'] = min(f[0-parent(s')], f[1-parent(s')] + lambda_out)
// so with L = adjoint of lambda_out (from later passes plus the 1-arcs that won in f'),
// R = adjoint of the removed mass (the next mean's adjoint / |J|):
//   rbar = R - L;  mubar = L + omega rbar;  m1bar = omega rbar;  m0bar = -omega rbar,
// and mubar is both the adjoint of lambda_in and this slot's share of the adjoint of pend_in.
#include "device_util.cuh"
#include "kernels.h"

namespace disco {
namespace {

using namespace dev;

constexpr int kAdjWarps = 4;

// x[i] += v for a runtime i (nothing outside [0, W)).
template <int W>
__device__ __forceinline__ void add_dyn(float (&x)[W], int i, float v) {
#pragma unroll
    for (int j = 0; j < W; ++j) x[j] += (i == j) ? v : 0.0f;
}

// x[j + 1] = a[j + k] for j in [-1, W] and a runtime k in {-1, 0, 1}, 0 outside [0, W): the
// adjoint counterpart of shift_ext (arc offsets d0 are in {-1, 0, 1} and an arithmetic
// 1-arc is d0 +- 1, so every arc's adjoint lands by one shift and one fixed offset).
template <int W>
__device__ __forceinline__ void shift_zero(const float (&a)[W], int k, float (&x)[W + 2]) {
#pragma unroll
    for (int j = -1; j <= W; ++j) {
        const float lo = (j - 1 >= 0 && j - 1 < W) ? a[(j - 1 >= 0 && j - 1 < W) ? j - 1 : 0] : 0.0f;
        const float mid = (j >= 0 && j < W) ? a[(j >= 0 && j < W) ? j : 0] : 0.0f;
        const float hi = (j + 1 >= 0 && j + 1 < W) ? a[(j + 1 >= 0 && j + 1 < W) ? j + 1 : 0] : 0.0f;
        x[j + 1] = k < 0 ? lo : (k > 0 ? hi : mid);
    }
}

// Layers of a lane's segment: those before the first padding slot (kNoVar). Segments start
// at layer 0 and are padded at the end, so a binary search over the tile's L layers finds
// the count in log2(L) loads.
__device__ __forceinline__ int lane_length(const AdjArgs& a, const TileInfo& ti, int64_t sb) {
    int lo = 0, hi = ti.L;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(a.var + sb + int64_t(mid) * 32) != kNoVar) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Adjoint of the removed mass: the next mean's adjoint (sum over ranks) divided by |J_v|.
__device__ __forceinline__ float removed_bar(const float4& a, const float4& b, int deg) {
    const float q[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    float s = 0.0f;
#pragma unroll
    for (int r = 0; r < 8; ++r)
        if (r < deg) s += q[r];
    return s / float(deg);
}

// The inputs of one layer of one lane. They are loaded one layer before they are used (two
// register sets alternate), and the layer's variable id and descriptor one layer before
// that, so a lane keeps its next layer's loads in flight while it computes.
//   own  : forward: F of layer l;       backward: B of layer l + 1 (the terminal layer: 0 / BIG)
//   ownb : the adjoint of own's layer-l node costs from the following pass (0 if none)
//   oth  : forward: B of layer l + 1;   backward: F of layer l
template <int W>
struct LayerIn {
    uint32_t v, dsc;
    float lam, lo, lb;
    float2 pend;  // the deferred mean the pass added (double-float, from the pend table)
    float rb;     // adjoint of the mass the pass removed (from the rbar table)
    float own[W], ownb[W], oth[W];
};

template <int W>
__device__ __forceinline__ void load_head(const AdjArgs& a, int64_t sb, int l, uint32_t& v, uint32_t& dsc) {
    v = __ldg(a.var + sb + int64_t(l) * 32);
    dsc = __ldg(a.desc + sb + int64_t(l) * 32);
}

template <int W, Adj KIND>
__device__ __forceinline__ void load_layer(const AdjArgs& a, int64_t sb, int64_t nb, int l, int n, uint32_t v,
                                           uint32_t dsc, LayerIn<W>& x) {
    constexpr bool kFwd = KIND == Adj::Fwd || KIND == Adj::Bound;
    constexpr bool kMMA = KIND == Adj::Fwd || KIND == Adj::Bwd;
    const Desc d = decode(dsc);
    const int64_t si = sb + int64_t(l) * 32;
    x.v = v;
    x.dsc = dsc;
    x.lam = __ldg(a.lam_in + si);
    x.lo = __ldg(a.lam_in_lo + si);
    x.lb = (kMMA || KIND == Adj::Reset) ? a.lbar[si] : 0.0f;
    x.pend = __ldg(a.pend_in + v);
    if (kMMA) x.rb = __ldg(a.rbar + v);
    const float* Lr = a.own + nb + int64_t(l) * W * 32;  // own-direction row of layer l
    const float* Nr = Lr + W * 32;                       // and of layer l + 1
#pragma unroll
    for (int s = 0; s < W; ++s) {
        if (kFwd) x.own[s] = s < d.w ? __ldg(Lr + s * 32) : BIG;
        else if (l == n - 1) x.own[s] = s == 0 ? 0.0f : BIG;
        else x.own[s] = s < d.wn ? __ldg(Nr + s * 32) : BIG;
        x.ownb[s] = (KIND != Adj::Bound && a.own_bar && s < d.w) ? __ldg(a.own_bar + nb + (int64_t(l) * W + s) * 32)
                                                                 : 0.0f;
        if (KIND == Adj::Fwd) x.oth[s] = s < d.wn ? __ldg(a.other + nb + (int64_t(l + 1) * W + s) * 32) : BIG;
        else if (KIND == Adj::Bwd) x.oth[s] = s < d.w ? __ldg(a.other + nb + (int64_t(l) * W + s) * 32) : BIG;
    }
}

// Reverse of layer l of a forward MMA half-pass (Fwd) or of the final bound pass (Bound:
// forward min-sum on lambda + pend; the lane's bound term f_n[0] has adjoint 1). fbar holds
// the adjoint of layer l + 1's node costs on entry and of layer l's on return.
template <int W, bool BOUND>
__device__ __forceinline__ void adj_forward_layer(const AdjArgs& a, const LayerIn<W>& x, int64_t si, int64_t nb, int l,
                                                  float (&fbar)[W]) {
    const Desc d = decode(x.dsc);
    float fl_bar[W];
#pragma unroll
    for (int s = 0; s < W; ++s) fl_bar[s] = x.ownb[s];
    df Lm{x.lam, x.lo};
    const df p{x.pend.x, x.pend.y};
    float lm;
    int s0 = -1, s1 = -1, c0 = -1, c1 = -1;
    if (!BOUND) {
        Lm = df_add(Lm, p);
        float hx[W + 2];
        shift_ext(x.oth, d.d0, hx);
        const bool up = d.d1 > d.d0;
        float m0 = BIG, m1 = BIG;
#pragma unroll
        for (int s = 0; s < W; ++s) {
            const float t = x.own[s] + hx[s + 1];
            if (t < m0) { m0 = t; s0 = s; }
        }
        if (d.one) {
            m1 = x.own[0] + at_dyn(x.oth, d.d1);
            s1 = 0;
            c1 = d.d1;
        } else {
#pragma unroll
            for (int s = 0; s < W; ++s) {
                const float t = x.own[s] + (up ? hx[s + 2] : hx[s]);
                if (t < m1) { m1 = t; s1 = s; }
            }
            c1 = s1 + d.d1;
        }
        c0 = s0 + d.d0;
        const float M = (m1 + Lm.hi) - m0;
        long long q;
        lm = df_add_f(Lm, -fx_round(a.omega * M, a.fx, q)).hi;  // the mass as the pass removed it
    } else {
        lm = df_add(Lm, p).hi;
    }
    // arcs into layer l + 1: the winning parent of each node takes its adjoint
    float gx[W + 2];
    shift_ext(x.own, -d.d0, gx);
    const bool upf = d.d1 > d.d0;
    const float f0 = x.own[0];
    float arcs = 0.0f;  // adjoint reaching lambda_out through winning 1-arcs
    float g0[W], g1[W];  // node sp's adjoint, split by the arc that won its min
#pragma unroll
    for (int sp = 0; sp < W; ++sp) {
        const float v0 = gx[sp + 1];
        const float v1 = (d.one ? (sp == d.d1 ? f0 : BIG) : (upf ? gx[sp] : gx[sp + 2])) + lm;
        const bool win0 = v0 <= v1;
        const float g = sp < d.wn ? fbar[sp] : 0.0f;
        g0[sp] = win0 ? g : 0.0f;
        g1[sp] = win0 ? 0.0f : g;
        arcs += g1[sp];
    }
    // parent s of node sp: sp - d0 on the 0-arc, sp - d1 on an arithmetic 1-arc, 0 on a one-hot one
    float e0[W + 2], e1[W + 2];
    shift_zero(g0, d.d0, e0);
    shift_zero(g1, d.d0, e1);
#pragma unroll
    for (int s = 0; s < W; ++s) fl_bar[s] += e0[s + 1] + (d.one ? (s == 0 ? arcs : 0.0f) : (upf ? e1[s + 2] : e1[s]));
    float mubar;
    if (!BOUND) {
        const float L = x.lb + arcs;
        const float rbar = x.rb - L;
        mubar = L + a.omega * rbar;
        const float m0bar = -a.omega * rbar, m1bar = a.omega * rbar;
        add_dyn(fl_bar, s0, m0bar);
        add_dyn(fl_bar, s1, m1bar);
        float* Bb = a.other_bar + nb + int64_t(l + 1) * W * 32;
#pragma unroll
        for (int s = 0; s < W; ++s)
            if (s < d.wn) Bb[s * 32] = (s == c0 ? m0bar : 0.0f) + (s == c1 ? m1bar : 0.0f);
        if (l == 0) {
#pragma unroll
            for (int s = 0; s < W; ++s)
                if (s < d.w) a.other_bar[nb + s * 32] = 0.0f;  // the root layer's b is never read
        }
    } else {
        mubar = arcs;
    }
    a.lbar[si] = mubar;
    a.mubar_out[size_t(x.v) * kAccStride + d.rank] = mubar;
#pragma unroll
    for (int s = 0; s < W; ++s) fbar[s] = fl_bar[s];
}

// Reverse of layer l of a backward MMA half-pass (RESET = false) or of the initial backward
// min-sum on lambda^0 (RESET = true: no update; its adjoint is added to lbar). carry holds
// the adjoint reaching layer l's node costs from layer l - 1 on entry, and layer l + 1's on
// return.
template <int W, bool RESET>
__device__ __forceinline__ void adj_backward_layer(const AdjArgs& a, const LayerIn<W>& x, int64_t si, int64_t nb,
                                                   int l, float (&carry)[W]) {
    const Desc d = decode(x.dsc);
    float bl_bar[W];
#pragma unroll
    for (int s = 0; s < W; ++s) bl_bar[s] = carry[s] + x.ownb[s];
    df Lm{x.lam, x.lo};
    const df p{x.pend.x, x.pend.y};
    float hx[W + 2];
    shift_ext(x.own, d.d0, hx);
    const bool up = d.d1 > d.d0;
    const float b1 = d.one ? at_dyn(x.own, d.d1) : BIG;
    float lm;
    int s0 = -1, s1 = -1, c0 = -1, c1 = -1;
    if (!RESET) {
        float m0 = BIG, m1 = BIG;
#pragma unroll
        for (int s = 0; s < W; ++s) {
            const float t = x.oth[s] + hx[s + 1];
            if (t < m0) { m0 = t; s0 = s; }
        }
        if (d.one) {
            m1 = x.oth[0] + b1;
            s1 = 0;
            c1 = d.d1;
        } else {
#pragma unroll
            for (int s = 0; s < W; ++s) {
                const float t = x.oth[s] + (up ? hx[s + 2] : hx[s]);
                if (t < m1) { m1 = t; s1 = s; }
            }
            c1 = s1 + d.d1;
        }
        c0 = s0 + d.d0;
        Lm = df_add(Lm, p);
        const float M = (m1 + Lm.hi) - m0;
        long long q;
        lm = df_add_f(Lm, -fx_round(a.omega * M, a.fx, q)).hi;  // the mass as the pass removed it
    } else {
        lm = df_add(Lm, p).hi;
    }
    // b[s] = min(b'[s + d0], b'[1-child(s)] + lambda_out): the winning child takes the adjoint
    float arcs = 0.0f;
    float g0[W], g1[W];  // node s's adjoint, split by the arc that won its min
#pragma unroll
    for (int s = 0; s < W; ++s) {
        const float v0 = hx[s + 1];
        const float v1 = (d.one ? (s == 0 ? b1 : BIG) : (up ? hx[s + 2] : hx[s])) + lm;
        const bool win0 = v0 <= v1;
        const float g = s < d.w ? bl_bar[s] : 0.0f;
        g0[s] = win0 ? g : 0.0f;
        g1[s] = win0 ? 0.0f : g;
        arcs += g1[s];
    }
    // child t of node s: s + d0 on the 0-arc, s + d1 on an arithmetic 1-arc, d1 on a one-hot one
    float e0[W + 2], e1[W + 2];
    shift_zero(g0, -d.d0, e0);
    shift_zero(g1, -d.d0, e1);
    float nxt[W];
#pragma unroll
    for (int t = 0; t < W; ++t) nxt[t] = e0[t + 1] + (d.one ? 0.0f : (up ? e1[t] : e1[t + 2]));
    if (d.one) add_dyn(nxt, d.d1, arcs);
    if (!RESET) {
        const float L = x.lb + arcs;
        const float rbar = x.rb - L;
        const float mubar = L + a.omega * rbar;
        const float m0bar = -a.omega * rbar, m1bar = a.omega * rbar;
        add_dyn(nxt, c0, m0bar);
        add_dyn(nxt, c1, m1bar);
        float* Fb = a.other_bar + nb + int64_t(l) * W * 32;
#pragma unroll
        for (int s = 0; s < W; ++s)
            if (s < d.w) Fb[s * 32] = (s == s0 ? m0bar : 0.0f) + (s == s1 ? m1bar : 0.0f);
        a.lbar[si] = mubar;
        a.mubar_out[size_t(x.v) * kAccStride + d.rank] = mubar;
    } else {
        a.lbar[si] = x.lb + arcs;
    }
#pragma unroll
    for (int s = 0; s < W; ++s) carry[s] = nxt[s];
}

template <Adj KIND, int W>
__device__ __forceinline__ void adj_layer(const AdjArgs& a, const LayerIn<W>& x, int64_t sb, int64_t nb, int l,
                                          float (&g)[W]) {
    const int64_t si = sb + int64_t(l) * 32;
    if (KIND == Adj::Fwd) adj_forward_layer<W, false>(a, x, si, nb, l, g);
    else if (KIND == Adj::Bound) adj_forward_layer<W, true>(a, x, si, nb, l, g);
    else if (KIND == Adj::Bwd) adj_backward_layer<W, false>(a, x, si, nb, l, g);
    else adj_backward_layer<W, true>(a, x, si, nb, l, g);
}

// One lane's segment: forward-pass adjoints sweep the layers last to first, backward-pass
// adjoints first to last (the reverse of the pass they undo). Register sets A and B take
// alternate layers: while one layer is computed, the next one's inputs are in flight.
template <Adj KIND, int W>
__device__ void adj_tile(const AdjArgs& a, const TileInfo& ti, int lane) {
    constexpr bool kFwd = KIND == Adj::Fwd || KIND == Adj::Bound;
    constexpr int kStep = kFwd ? -1 : 1;
    const int64_t sb = ti.slot_base + lane;
    const int64_t nb = ti.node_base + lane;
    const int n = lane_length(a, ti, sb);
    if (n == 0) return;
    float g[W];  // forward: adjoint of layer l + 1's costs; backward: what reaches layer l
#pragma unroll
    for (int s = 0; s < W; ++s) g[s] = (KIND == Adj::Bound && s == 0) ? 1.0f : 0.0f;
    const int first = kFwd ? n - 1 : 0;
    auto inside = [n](int l) { return l >= 0 && l < n; };
    LayerIn<W> A, B;
    uint32_t hv, hd;
    load_head<W>(a, sb, first, hv, hd);
    load_layer<W, KIND>(a, sb, nb, first, n, hv, hd, A);
    if (inside(first + kStep)) load_head<W>(a, sb, first + kStep, hv, hd);
    for (int l = first;; l += 2 * kStep) {
        const int l1 = l + kStep, l2 = l + 2 * kStep, l3 = l + 3 * kStep;
        if (inside(l1)) load_layer<W, KIND>(a, sb, nb, l1, n, hv, hd, B);
        if (inside(l2)) load_head<W>(a, sb, l2, hv, hd);
        adj_layer<KIND, W>(a, A, sb, nb, l, g);
        if (!inside(l1)) break;
        if (inside(l2)) load_layer<W, KIND>(a, sb, nb, l2, n, hv, hd, A);
        if (inside(l3)) load_head<W>(a, sb, l3, hv, hd);
        adj_layer<KIND, W>(a, B, sb, nb, l1, g);
        if (!inside(l2)) break;
    }
}

// One launch per width group (tiles [tile0, tile_end)): group 0 holds widths 2, 4 and 6,
// the others one width each, so every kernel's register budget fits its widest layer.
template <Adj KIND, int WG>
__global__ void __launch_bounds__(kAdjWarps * 32, WG == 0 ? 4 : (WG == 8 ? 3 : 1)) k_adjoint(AdjArgs a) {
    const int tile = a.tile0 + int(blockIdx.x) * kAdjWarps + int(threadIdx.x >> 5);
    if (tile >= a.tile_end) return;
    const TileInfo ti = a.tiles[tile];
    const int lane = threadIdx.x & 31;
    if (WG == 0) {
        if (ti.W == 2) adj_tile<KIND, 2>(a, ti, lane);
        else if (ti.W == 4) adj_tile<KIND, 4>(a, ti, lane);
        else adj_tile<KIND, 6>(a, ti, lane);
    } else {
        adj_tile<KIND, WG == 0 ? 2 : WG>(a, ti, lane);
    }
}

// pend[v]: the deferred mean of variable v from its averaging sum, exactly as the passes add it.
__global__ void k_pend_table(const long long* __restrict__ msum, const uint8_t* __restrict__ deg, int64_t n, float inv,
                             float2* __restrict__ out) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        const int dg = deg[v];
        const df m = dg > 0 ? fx_mean(msum[v], dg, inv) : df{0.0f, 0.0f};
        out[v] = make_float2(m.hi, m.lo);
    }
}

// rbar[v]: the adjoint of each removed mass of v, the sum of its sector / deg.
__global__ void k_rbar_table(const float* __restrict__ mub, const uint8_t* __restrict__ deg, int64_t n,
                             float* __restrict__ out) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        const int dg = deg[v];
        const float4* p = reinterpret_cast<const float4*>(mub + size_t(v) * kAccStride);
        out[v] = dg > 0 ? removed_bar(p[0], dg > 4 ? p[1] : make_float4(0.0f, 0.0f, 0.0f, 0.0f), dg) : 0.0f;
    }
}

__global__ void k_slot_table(const uint32_t* __restrict__ var, const uint32_t* __restrict__ desc, int64_t n,
                             const float* __restrict__ x, float* __restrict__ tab) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t v = var[i];
        if (v != kNoVar) tab[size_t(v) * kAccStride + ((desc[i] >> 22) & 7u)] = x[i];
    }
}

__global__ void k_table_mean(const float* __restrict__ tab, const uint8_t* __restrict__ deg, int64_t n,
                             float* __restrict__ out) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        const int dg = deg[v];
        float s = 0.0f;
        for (int r = 0; r < dg; ++r) s += tab[size_t(v) * kAccStride + r];
        out[v] = dg > 0 ? s / float(dg) : 0.0f;
    }
}

inline unsigned grid_of(int64_t n, int block) {
    const int64_t g = (n + block - 1) / block;
    return unsigned(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

template <Adj KIND>
void launch_kind(int group, const dim3& grid, const dim3& block, const AdjArgs& a, cudaStream_t s) {
    switch (group) {
        case 0: k_adjoint<KIND, 0><<<grid, block, 0, s>>>(a); break;
        case 8: k_adjoint<KIND, 8><<<grid, block, 0, s>>>(a); break;
        case 16: k_adjoint<KIND, 16><<<grid, block, 0, s>>>(a); break;
        default: k_adjoint<KIND, 32><<<grid, block, 0, s>>>(a); break;
    }
}

}  // namespace

cudaError_t launch_adjoint(Adj kind, int group, const AdjArgs& a, cudaStream_t s) {
    if (group != 0 && group != 8 && group != 16 && group != 32) return cudaErrorInvalidValue;
    const int ntiles = a.tile_end - a.tile0;
    if (ntiles <= 0) return cudaSuccess;
    const dim3 grid((ntiles + kAdjWarps - 1) / kAdjWarps), block(kAdjWarps * 32);
    switch (kind) {
        case Adj::Fwd: launch_kind<Adj::Fwd>(group, grid, block, a, s); break;
        case Adj::Bwd: launch_kind<Adj::Bwd>(group, grid, block, a, s); break;
        case Adj::Bound: launch_kind<Adj::Bound>(group, grid, block, a, s); break;
        case Adj::Reset: launch_kind<Adj::Reset>(group, grid, block, a, s); break;
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_pend_table(const long long* msum, const uint8_t* deg, int64_t n, float inv, float2* out,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_pend_table<<<grid_of(n, 256), 256, 0, s>>>(msum, deg, n, inv, out);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_rbar_table(const float* mub, const uint8_t* deg, int64_t n, float* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_rbar_table<<<grid_of(n, 256), 256, 0, s>>>(mub, deg, n, out);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_adj_cost(const uint32_t* var, const uint32_t* desc, int64_t nslots, const float* lbar,
                            const uint8_t* deg, int64_t nint, float* tab, float* cbar, cudaStream_t s) {
    if (nslots > 0) k_slot_table<<<grid_of(nslots, 256), 256, 0, s>>>(var, desc, nslots, lbar, tab);
    if (nint > 0) k_table_mean<<<grid_of(nint, 256), 256, 0, s>>>(tab, deg, nint, cbar);
    g_launches.fetch_add(2, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace disco
