// Adjoint (reverse mode) of the deferred-MMA dual iterations: d(bound) / d(lambda^0).
//
// The bound after T iterations (Eq. D objective at lambda + pend) is a piecewise linear
// function of the costs: every operation of a half-pass (Alg. 1 "MMA": min-marginals from
// shortest paths, Sec. 3.2 / App. A.5, the damped update, the deferred mean) is a min, a
// sum or a scaling. Its gradient pushes adjoints back through each min to the argument that
// attained it. Each kernel here reverses one pass of one lane's BDD segment (same tile
// layout as the forward kernels, one lane per segment, no atomics): the pass's own-direction
// node costs are first recomputed by the normal kernel from the pass's recorded inputs, so
// every min is decided on bit-identical values, then the lane sweeps its layers in the
// opposite order carrying the adjoints of the current layer's node costs in registers.
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

__device__ __forceinline__ int lane_length(const AdjArgs& a, const TileInfo& ti, int64_t sb) {
    int n = 0;
    while (n < ti.L && __ldg(a.var + sb + int64_t(n) * 32) != kNoVar) ++n;
    return n;
}

// Adjoint of the removed mass of variable v: the next mean's adjoint divided by |J_v|.
__device__ __forceinline__ float removed_bar(const AdjArgs& a, uint32_t v, int deg) {
    const float* q = a.mubar_next + size_t(v) * kAccStride;
    float s = 0.0f;
    for (int r = 0; r < deg; ++r) s += q[r];
    return s / float(deg);
}

// Reverse of a forward MMA half-pass (BOUND = false) or of the final bound pass (BOUND =
// true: forward min-sum on lambda + pend, the lane's bound term f_n[0] has adjoint 1).
template <int W, bool BOUND>
__device__ void adj_forward(const AdjArgs& a, const TileInfo& ti, int lane) {
    const int64_t sb = ti.slot_base + lane;
    const int64_t nb = ti.node_base + lane;
    const int n = lane_length(a, ti, sb);
    float fbar[W];  // adjoint of the node costs of layer l + 1
#pragma unroll
    for (int s = 0; s < W; ++s) fbar[s] = (BOUND && s == 0 && n > 0) ? 1.0f : 0.0f;
    for (int l = n - 1; l >= 0; --l) {
        const int64_t si = sb + int64_t(l) * 32;
        const uint32_t v = __ldg(a.var + si);
        const Desc d = decode(__ldg(a.desc + si));
        const float* Fr = a.own + nb + int64_t(l) * W * 32;
        float f[W], fl_bar[W];
#pragma unroll
        for (int s = 0; s < W; ++s) {
            f[s] = s < d.w ? Fr[s * 32] : BIG;
            fl_bar[s] = (!BOUND && a.own_bar && s < d.w) ? a.own_bar[nb + (int64_t(l) * W + s) * 32] : 0.0f;
        }
        df Lm{a.lam_in[si], a.lam_in_lo[si]};
        const df p = pend_of(a.acc_in, v, d.deg);
        float lm;
        int s0 = -1, s1 = -1, c0 = -1, c1 = -1;
        if (!BOUND) {
            const float* Br = a.other + nb + int64_t(l + 1) * W * 32;
            float bn[W];
#pragma unroll
            for (int s = 0; s < W; ++s) bn[s] = s < d.wn ? Br[s * 32] : BIG;
            Lm = df_add(Lm, p);
            float hx[W + 2];
            shift_ext(bn, d.d0, hx);
            const bool up = d.d1 > d.d0;
            float m0 = BIG, m1 = BIG;
#pragma unroll
            for (int s = 0; s < W; ++s) {
                const float x = f[s] + hx[s + 1];
                if (x < m0) { m0 = x; s0 = s; }
            }
            if (d.one) {
                m1 = f[0] + at_dyn(bn, d.d1);
                s1 = 0;
                c1 = d.d1;
            } else {
#pragma unroll
                for (int s = 0; s < W; ++s) {
                    const float x = f[s] + (up ? hx[s + 2] : hx[s]);
                    if (x < m1) { m1 = x; s1 = s; }
                }
                c1 = s1 + d.d1;
            }
            c0 = s0 + d.d0;
            const float M = (m1 + Lm.hi) - m0;
            const float removed = a.omega * M;
            lm = df_add_f(Lm, -removed).hi;
        } else {
            lm = df_add(Lm, p).hi;
        }
        // arcs into layer l + 1: the winning parent of each node takes its adjoint
        float gx[W + 2];
        shift_ext(f, -d.d0, gx);
        const bool upf = d.d1 > d.d0;
        const float f0 = f[0];
        float arcs = 0.0f;  // adjoint reaching lambda_out through winning 1-arcs
#pragma unroll
        for (int sp = 0; sp < W; ++sp) {
            if (sp < d.wn) {
                const float g = fbar[sp];
                const float v0 = gx[sp + 1];
                const float v1 = (d.one ? (sp == d.d1 ? f0 : BIG) : (upf ? gx[sp] : gx[sp + 2])) + lm;
                if (v0 <= v1) {
                    add_dyn(fl_bar, sp - d.d0, g);
                } else {
                    add_dyn(fl_bar, d.one ? 0 : sp - d.d1, g);
                    arcs += g;
                }
            }
        }
        float mubar;
        if (!BOUND) {
            const float L = a.lbar[si] + arcs;
            const float rbar = removed_bar(a, v, d.deg) - L;
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
        a.mubar_out[size_t(v) * kAccStride + d.rank] = mubar;
#pragma unroll
        for (int s = 0; s < W; ++s) fbar[s] = fl_bar[s];
    }
}

// Reverse of a backward MMA half-pass (RESET = false) or of the initial backward min-sum
// on lambda^0 (RESET = true: no update; its adjoint is added to lbar).
template <int W, bool RESET>
__device__ void adj_backward(const AdjArgs& a, const TileInfo& ti, int lane) {
    const int64_t sb = ti.slot_base + lane;
    const int64_t nb = ti.node_base + lane;
    const int n = lane_length(a, ti, sb);
    float carry[W];  // adjoint reaching the node costs of layer l from layer l - 1
#pragma unroll
    for (int s = 0; s < W; ++s) carry[s] = 0.0f;
    for (int l = 0; l < n; ++l) {
        const int64_t si = sb + int64_t(l) * 32;
        const uint32_t v = __ldg(a.var + si);
        const Desc d = decode(__ldg(a.desc + si));
        float bl_bar[W], bn[W];
#pragma unroll
        for (int s = 0; s < W; ++s) {
            bl_bar[s] = carry[s] + ((a.own_bar && s < d.w) ? a.own_bar[nb + (int64_t(l) * W + s) * 32] : 0.0f);
            if (l == n - 1) bn[s] = s == 0 ? 0.0f : BIG;  // terminal layer
            else bn[s] = s < d.wn ? a.own[nb + (int64_t(l + 1) * W + s) * 32] : BIG;
        }
        df Lm{a.lam_in[si], a.lam_in_lo[si]};
        const df p = pend_of(a.acc_in, v, d.deg);
        float hx[W + 2];
        shift_ext(bn, d.d0, hx);
        const bool up = d.d1 > d.d0;
        const float b1 = d.one ? at_dyn(bn, d.d1) : BIG;
        float lm;
        int s0 = -1, s1 = -1, c0 = -1, c1 = -1;
        if (!RESET) {
            const float* Fr = a.other + nb + int64_t(l) * W * 32;
            float F[W];
#pragma unroll
            for (int s = 0; s < W; ++s) F[s] = s < d.w ? Fr[s * 32] : BIG;
            float m0 = BIG, m1 = BIG;
#pragma unroll
            for (int s = 0; s < W; ++s) {
                const float x = F[s] + hx[s + 1];
                if (x < m0) { m0 = x; s0 = s; }
            }
            if (d.one) {
                m1 = F[0] + b1;
                s1 = 0;
                c1 = d.d1;
            } else {
#pragma unroll
                for (int s = 0; s < W; ++s) {
                    const float x = F[s] + (up ? hx[s + 2] : hx[s]);
                    if (x < m1) { m1 = x; s1 = s; }
                }
                c1 = s1 + d.d1;
            }
            c0 = s0 + d.d0;
            Lm = df_add(Lm, p);
            const float M = (m1 + Lm.hi) - m0;
            const float removed = a.omega * M;
            lm = df_add_f(Lm, -removed).hi;
        } else {
            lm = df_add(Lm, p).hi;
        }
        // b[s] = min(b'[s + d0], b'[1-child(s)] + lambda_out): the winning child takes the adjoint
        float nxt[W];
#pragma unroll
        for (int s = 0; s < W; ++s) nxt[s] = 0.0f;
        float arcs = 0.0f;
#pragma unroll
        for (int s = 0; s < W; ++s) {
            if (s < d.w) {
                const float g = bl_bar[s];
                const float v0 = hx[s + 1];
                const float v1 = (d.one ? (s == 0 ? b1 : BIG) : (up ? hx[s + 2] : hx[s])) + lm;
                if (v0 <= v1) {
                    add_dyn(nxt, s + d.d0, g);
                } else {
                    add_dyn(nxt, d.one ? d.d1 : s + d.d1, g);
                    arcs += g;
                }
            }
        }
        if (!RESET) {
            const float L = a.lbar[si] + arcs;
            const float rbar = removed_bar(a, v, d.deg) - L;
            const float mubar = L + a.omega * rbar;
            const float m0bar = -a.omega * rbar, m1bar = a.omega * rbar;
            add_dyn(nxt, c0, m0bar);
            add_dyn(nxt, c1, m1bar);
            float* Fb = a.other_bar + nb + int64_t(l) * W * 32;
#pragma unroll
            for (int s = 0; s < W; ++s)
                if (s < d.w) Fb[s * 32] = (s == s0 ? m0bar : 0.0f) + (s == s1 ? m1bar : 0.0f);
            a.lbar[si] = mubar;
            a.mubar_out[size_t(v) * kAccStride + d.rank] = mubar;
        } else {
            a.lbar[si] += arcs;
        }
#pragma unroll
        for (int s = 0; s < W; ++s) carry[s] = nxt[s];
    }
}

template <Adj KIND, int W>
__device__ __forceinline__ void adj_tile(const AdjArgs& a, const TileInfo& ti, int lane) {
    if (KIND == Adj::Fwd) adj_forward<W, false>(a, ti, lane);
    else if (KIND == Adj::Bound) adj_forward<W, true>(a, ti, lane);
    else if (KIND == Adj::Bwd) adj_backward<W, false>(a, ti, lane);
    else adj_backward<W, true>(a, ti, lane);
}

template <Adj KIND>
__global__ void __launch_bounds__(kAdjWarps * 32) k_adjoint(AdjArgs a) {
    const int tile = int(blockIdx.x) * kAdjWarps + int(threadIdx.x >> 5);
    if (tile >= a.ntiles) return;
    const TileInfo ti = a.tiles[tile];
    const int lane = threadIdx.x & 31;
    switch (ti.W) {
        case 2: adj_tile<KIND, 2>(a, ti, lane); break;
        case 4: adj_tile<KIND, 4>(a, ti, lane); break;
        case 6: adj_tile<KIND, 6>(a, ti, lane); break;
        case 8: adj_tile<KIND, 8>(a, ti, lane); break;
        case 16: adj_tile<KIND, 16>(a, ti, lane); break;
        default: adj_tile<KIND, 32>(a, ti, lane); break;
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

}  // namespace

cudaError_t launch_adjoint(Adj kind, const AdjArgs& a, cudaStream_t s) {
    if (a.ntiles <= 0) return cudaSuccess;
    const dim3 grid((a.ntiles + kAdjWarps - 1) / kAdjWarps), block(kAdjWarps * 32);
    switch (kind) {
        case Adj::Fwd: k_adjoint<Adj::Fwd><<<grid, block, 0, s>>>(a); break;
        case Adj::Bwd: k_adjoint<Adj::Bwd><<<grid, block, 0, s>>>(a); break;
        case Adj::Bound: k_adjoint<Adj::Bound><<<grid, block, 0, s>>>(a); break;
        case Adj::Reset: k_adjoint<Adj::Reset><<<grid, block, 0, s>>>(a); break;
    }
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
