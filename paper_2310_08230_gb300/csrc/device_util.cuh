// Device helpers shared by the half-pass kernels (kernels.cu) and their adjoints
// (adjoint.cu): layer descriptors, shifts of a layer's node costs by an arc offset, and
// double-float arithmetic for the dual variables.
#pragma once

#include <cstdint>

#include "kernels.h"

namespace disco {
namespace dev {

constexpr float BIG = 1e30f;

struct Desc {
    int w, wn, d0, d1, one, rank, deg;
};

__device__ __forceinline__ Desc decode(uint32_t x) {
    Desc d;
    d.w = int(x & 63u) + 1;
    d.wn = int((x >> 6) & 63u) + 1;
    d.d0 = int((x >> 12) & 7u) - 2;
    d.d1 = int((x >> 15) & 63u) - 2;
    d.one = int((x >> 21) & 1u);
    d.rank = int((x >> 22) & 7u);
    d.deg = int((x >> 25) & 7u);
    return d;
}

// x[j + 1] = a[j + k] for every j in [-1, W] and a runtime k in {-1, 0, 1} (BIG outside
// [0, W)). With x = the other layer's costs shifted by the 0-arc offset d0, an arithmetic
// 1-arc (d1 = d0 +- 1) is x shifted by one more place, which stays inside [-1, W].
template <int W>
__device__ __forceinline__ void shift_ext(const float (&a)[W], int k, float (&x)[W + 2]) {
#pragma unroll
    for (int j = -1; j <= W; ++j) {
        const float lo = (j - 1 >= 0 && j - 1 < W) ? a[(j - 1 >= 0 && j - 1 < W) ? j - 1 : 0] : BIG;
        const float mid = (j >= 0 && j < W) ? a[(j >= 0 && j < W) ? j : 0] : BIG;
        const float hi = (j + 1 >= 0 && j + 1 < W) ? a[(j + 1 >= 0 && j + 1 < W) ? j + 1 : 0] : BIG;
        x[j + 1] = k < 0 ? lo : (k == 0 ? mid : hi);
    }
}

// a[i] for a runtime i; BIG outside [0, W).
template <int W>
__device__ __forceinline__ float at_dyn(const float (&a)[W], int i) {
    float r = BIG;
#pragma unroll
    for (int j = 0; j < W; ++j) r = (i == j) ? a[j] : r;
    return r;
}

// Double-float ("df") arithmetic for the dual variables: a value is hi + lo with |lo| <=
// ulp(hi) / 2. TwoSum (Knuth, TAOCP vol. 2, 4.2.2) gives the exact rounding error of a float
// sum; Fast2Sum (Dekker 1971) renormalises. Keeping lambda and the deferred mean in df keeps
// sum_j lambda^j_i + |J_i| pend_i = c_i (Eq. D) exact to about 2^-48 while node costs stay FP32.
struct df {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ df fast2sum(float s, float e) {
    const float h = s + e;
    return df{h, e - (h - s)};
}
__device__ __forceinline__ df df_add(df a, df b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return fast2sum(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ df df_add_f(df a, float b) {
    float s, e;
    two_sum(a.hi, b, s, e);
    return fast2sum(s, e + a.lo);
}
// a / n for a small positive integer n. q = a.hi * (1/n) is within an ulp of a.hi / n, so the
// remainder a.hi - q n is exact with an FMA (the classic division-by-reciprocal argument);
// the low part needs only single precision.
__device__ __forceinline__ df df_div_i(df a, int n) {
    const float fn = float(n);
    const float rcp = n == 2 ? 0.5f : (n == 3 ? 0.333333343f : (n == 4 ? 0.25f : (n == 5 ? 0.2f : 1.0f / fn)));
    const float q = a.hi * rcp;
    const float r = fmaf(-q, fn, a.hi) + a.lo;
    return fast2sum(q, r * rcp);
}

// Deferred means from fixed-point sums (the averaging step of Alg. 1 "MMA"). Every update
// pass adds the mass each slot removes, on the grid 2^-F, into one signed 64-bit integer per
// variable: integer addition is exact and order-free, so the sum, and everything built on it,
// is the same for every schedule of the lanes and needs no second pass over the slots. The
// slot subtracts exactly the rounded mass from its lambda, so sum_j lambda^j_i + |J_i| pend_i
// = c_i (Eq. D) holds as exactly as before. F is chosen per handle from the largest cost;
// lim = 2^(59 - F) bounds one mass, so sums of up to 7 stay inside the 64-bit range.
//
// m on the grid: q = round(m 2^F) and the return value q 2^-F, both exact (m 2^F has 24
// significant bits, so rounding it to an integer leaves at most 24, which FP32 holds).
__device__ __forceinline__ float fx_round(float m, const FxScale& fx, long long& q) {
    const float t = rintf(m * fx.scale);
    q = __float2ll_rn(t);
    return t * fx.inv;
}
// A sum S (units of 2^-F) as double-float: hi = S rounded to FP32, lo = the exact integer
// remainder S - hi rounded to FP32 (|lo| <= ulp(hi) / 2, so the pair is normalised); the
// scaling by 2^-F is exact. Relative error about 2^-48.
__device__ __forceinline__ df fx_to_df(long long S, float inv) {
    const float hi = __ll2float_rn(S);
    const float lo = __ll2float_rn(S - __float2ll_rn(hi));
    return df{hi * inv, lo * inv};
}
// The deferred mean of a variable: its sum / deg, in double-float.
__device__ __forceinline__ df fx_mean(long long S, int deg, float inv) { return df_div_i(fx_to_df(S, inv), deg); }

__device__ __forceinline__ uint64_t shl(uint64_t x, int k) { return k >= 0 ? (x << k) : (x >> (-k)); }
__device__ __forceinline__ uint64_t low_mask(int n) { return n >= 64 ? ~0ull : ((1ull << n) - 1ull); }


}  // namespace dev
}  // namespace disco
