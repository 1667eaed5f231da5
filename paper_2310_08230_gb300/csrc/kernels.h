// Device store layout and kernel launchers of the dual / primal hot path.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include <atomic>

namespace disco {

// Kernel launches issued by this library so far (all devices, all handles).
extern std::atomic<int64_t> g_launches;

// A warp tile: 32 BDD segments (one per lane) of one width class.
//   slot (layer l, lane)      at slot_base + l * 32 + lane              (var, desc, lambda)
//   node (layer l, s, lane)   at node_base + (l * W + s) * 32 + lane    (F, B)
// Layers 0..L-1 hold variables; layer L is the terminal (B = 0 at s = 0). Lanes with fewer
// layers, or no segment, carry var = kNoVar from their end on.
struct TileInfo {
    int64_t slot_base;
    int64_t node_base;
    int32_t L;
    int32_t W;
};

constexpr uint32_t kNoVar = 0xFFFFFFFFu;
constexpr int kAccStride = 8;  // entries per variable in the per-rank tables (min-marginals, supports, adjoints)

// Fixed-point grid of the averaging sums (device_util.cuh): scale = 2^F, inv = 2^-F, lim =
// the largest mass one slot may remove (2^(42 - F)).
struct FxScale {
    float scale, inv, lim;
};

// Bits of the per-handle device status word, set by kernels and read by the host at its
// synchronisation points.
enum : uint32_t {
    kStatusRange = 1u,   // a removed mass reached FxScale::lim (or was not finite)
    kStatusBounds = 2u,  // bounds-checking build: an index fell outside its array (access skipped)
};
// Width classes up to kFusedMaxW share one launch (launch_pass with W = 0); wider classes
// launch on their own.
constexpr int kFusedMaxW = 6;
enum : uint8_t { kFree = 0, kFix0 = 1, kFix1 = 2 };

struct KArgs {
    const TileInfo* tiles;
    int32_t tile0, tile_end;         // tiles of one width class
    const uint32_t* var;
    const uint32_t* desc;
    float* lam;                      // dual variables, high part (the FP32 value used by the passes)
    float* lam_lo;                   // low part: lambda = lam + lam_lo (double-float)
    float* F;
    float* B;
    // Averaging state (three rotating buffers of one signed 64-bit sum per variable): msum_rd
    // holds the masses removed by the last update pass (its mean is each variable's deferred
    // mean, read by every pass); an update pass adds its removed masses into msum_wr (zero on
    // entry) and clears msum_zero, the buffer the next update pass writes (rank-0 slots).
    const long long* msum_rd;
    long long* msum_wr;
    long long* msum_zero;
    FxScale fx;
    uint32_t* status;                // device status word (kStatus* bits)
    const uint8_t* state;            // per variable, rounding only
    float omega;
    float* mm_slot;                  // per slot (tile layout)
    float* mm_var;                   // kAccStride per variable
    double* tile_sum;                // per tile
    uint32_t* reach;                 // per slot (tile layout)
    uint8_t* sup_var;                // kAccStride per variable
    // array sizes, checked by the bounds-checking build only
    int64_t nslots, nnodes, nvars;
};

// Arguments of the adjoint kernels (adjoint.cu). A pass's inputs come from the tape (the
// values the pass read when it ran, its deferred means as a per-variable table), its
// own-direction node costs too (as the pass stored them when it was replayed). Adjoints:
// lbar per slot (in: of lambda after the pass; out: of lambda before it); rbar per variable
// (the adjoint of each mass the pass removed, from the following pass's sectors); mubar_out
// per variable and rank (sectors like the averaging tables: of the deferred means the pass
// read); node-array adjoints own_bar (of the costs this pass stored, read) and other_bar (of
// the costs it read from the previous pass, written).
struct AdjArgs {
    const TileInfo* tiles;
    int32_t tile0, tile_end;  // the launch's tiles (one width group)
    const uint32_t* var;
    const uint32_t* desc;
    const float* lam_in;
    const float* lam_in_lo;
    const float2* pend_in;  // per variable: the deferred mean the pass added (launch_pend_table)
    const float* other;     // node costs the pass read (B forward, F backward)
    const float* own;       // node costs the pass stored (recorded)
    const float* own_bar;   // adjoint of `own` (from the following pass); may be null = 0
    float* other_bar;       // adjoint of `other` (for the preceding pass)
    float* lbar;
    const float* rbar;      // per variable: adjoint of each mass the pass removed (launch_rbar_table)
    float* mubar_out;
    float omega;
    FxScale fx;             // the forward passes' rounding of the removed masses
};

enum class Adj {
    Fwd,    // forward MMA half-pass
    Bwd,    // backward MMA half-pass
    Bound,  // final bound: forward min-sum on lambda + pend (lbar, mubar_out written)
    Reset,  // initial backward min-sum on lambda (lbar accumulated)
};

// group: 0 = the fused widths 2, 4, 6; else 8, 16 or 32 (a.tile0 .. a.tile_end must hold
// only tiles of that group).
cudaError_t launch_adjoint(Adj kind, int group, const AdjArgs& a, cudaStream_t s);
// cbar[v] = (sum over v's slots of lbar) / deg[v], via a rank-sector table (tab).
// pend[v] = the deferred mean of v's averaging sum (double-float, exactly as the passes add it);
// rbar[v] = (sum of v's adjoint sector) / deg[v].
cudaError_t launch_pend_table(const long long* msum, const uint8_t* deg, int64_t n, float inv, float2* out,
                              cudaStream_t s);
cudaError_t launch_rbar_table(const float* mub, const uint8_t* deg, int64_t n, float* out, cudaStream_t s);
cudaError_t launch_adj_cost(const uint32_t* var, const uint32_t* desc, int64_t nslots, const float* lbar,
                            const uint8_t* deg, int64_t nint, float* tab, float* cbar, cudaStream_t s);

// Store construction (store.cu). launch_layout: segment k (in tile order) has seg_len[k]
// layers at canonical slots seg_canon[k] + l, placed at tile slot seg_pos[k] + 32 l; its
// variable ids are offset by seg_vb[k] (the instance's first variable). canon_pos[c] = the
// tile slot of canonical slot c. launch_instance_of: out[v] = i with base[i] <= v < base[i + 1].
cudaError_t launch_layout(const int64_t* seg_canon, const int32_t* seg_len, const int64_t* seg_pos,
                          const uint32_t* seg_vb, int64_t nseg, const int32_t* cvar, const uint32_t* cdesc,
                          const float* clam, const float* clam_lo, uint32_t* var, uint32_t* desc, float* lam,
                          float* lam_lo, int64_t* canon_pos, cudaStream_t s);
cudaError_t launch_instance_of(const int64_t* base, int32_t ni, int64_t n, int32_t* out, cudaStream_t s);

// Quasi-Newton vector kernels (qn.cu); n = slots in tile layout.
cudaError_t launch_qn_sign(const float* mm, const uint32_t* var, int64_t n, float* g, cudaStream_t s);
int qn_dot_blocks();
cudaError_t launch_qn_dot(const float* a, const float* b, int64_t n, double* partial, cudaStream_t s);
cudaError_t launch_qn_axpy(float* y, float a, const float* x, int64_t n, cudaStream_t s);
cudaError_t launch_qn_scale(float* x, float a, int64_t n, cudaStream_t s);
cudaError_t launch_qn_sub(const float* a, const float* b, int64_t n, float* out, cudaStream_t s);
cudaError_t launch_qn_project(float* x, const uint32_t* var, const uint32_t* desc, int64_t n, float* tab,
                              cudaStream_t s);
cudaError_t launch_qn_step(const float* lam, const float* lam_lo, const float* d, float gamma, const uint32_t* var,
                           int64_t n, float* out, float* out_lo, cudaStream_t s);
cudaError_t launch_qn_delta(const float* lam, const float* lam_lo, const long long* msum, float inv, const float* old,
                            const float* old_lo, const uint32_t* var, const uint32_t* desc, int64_t n, float* s_out,
                            cudaStream_t s);

enum class Pass {
    FwdMMA,      // forward half-pass with updates, stores F
    BwdMMA,      // backward half-pass with updates, stores B
    FwdMMARound, // same, fixed variables masked and not updated
    BwdMMARound,
    Lb,          // forward min-sum on lambda + pend, per-tile sum of BDD minima
    FwdMM,       // forward min-sum on lambda + pend (fixings masked), stores F
    BwdMM,       // backward min-sum, writes min-marginals
    BwdReset,    // backward min-sum on lambda + pend (fixings masked), stores B
    Supports     // reachability under fixings, writes per-slot value supports
};

// Launches `pass` over the tiles [a.tile0, a.tile_end) of width class W (8, 16, 32);
// W = 0: tiles of classes 2, 4 and 6 mixed in one launch (each tile carries its class).
// `geometry` (1, 2 or 4 warps per block) applies to the fused MMA half-passes; all
// geometries give identical results.
cudaError_t launch_pass(Pass pass, int W, const KArgs& a, cudaStream_t s, int geometry = 2);

cudaError_t launch_sum_tiles(const double* tile_sum, int64_t n, double add, double* out, cudaStream_t s);
cudaError_t launch_sum_instances(const double* tile_sum, const int32_t* ptr, const int32_t* tiles, const double* add,
                                 int64_t n, double* out, cudaStream_t s);
cudaError_t launch_gather_f32(const float* src, const int64_t* pos, int64_t n, float* dst, cudaStream_t s);
cudaError_t launch_scatter_f32(const float* src, const int64_t* pos, int64_t n, float* dst, cudaStream_t s);
// pend[v] = the deferred mean of v (FP32); launch_set_pend: the sums whose means are pend
// (pend[v] deg[v] on the grid); launch_flush: lambda += the deferred mean of its variable.
cudaError_t launch_pend(const long long* msum, const uint8_t* deg, int64_t n, float inv, float* pend, cudaStream_t s);
cudaError_t launch_set_pend(const float* pend, const uint8_t* deg, int64_t n, float scale, long long* msum,
                            uint32_t* status, cudaStream_t s);
cudaError_t launch_flush(const uint32_t* var, const uint32_t* desc, int64_t nslots, const long long* msum, float inv,
                         float* lam, float* lam_lo, cudaStream_t s);
cudaError_t launch_decide(const float* mm_var, const uint8_t* deg, const uint8_t* state, int64_t n, float tau,
                          uint8_t* trial, cudaStream_t s);
cudaError_t launch_apply(const uint8_t* sup_var, const uint8_t* deg, const int32_t* inst, int64_t n, uint8_t* state,
                         int* counters, cudaStream_t s);
cudaError_t launch_count_free(const uint8_t* state, const uint8_t* deg, const int32_t* inst, int64_t n, int* counters,
                              cudaStream_t s);
cudaError_t launch_perturb(const uint32_t* var, const uint32_t* desc, int64_t nslots, const float* mm_var,
                           const uint8_t* state, float delta, float* lam, float* lam_lo, cudaStream_t s);
cudaError_t launch_pair_costs(const float* FX, const float* FY, int nvx, int nvy, int dim, float* d, cudaStream_t s,
                              bool norm = false);
cudaError_t launch_transpose(const float* src, int rows, int cols, float* dst, cudaStream_t s);
cudaError_t launch_topk_rows(const float* d, int rows, int cols, int k, int32_t* idx, cudaStream_t s);
cudaError_t launch_dilate(const int32_t* topk, int rows, int k, const int32_t* ring_ptr, const int32_t* ring,
                          int nvy, bool transposed, uint8_t* allowed, cudaStream_t s);

}  // namespace disco
