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

// Deferred mean of variable v: sum of its deg removed masses (rank order) / deg, in df.
__device__ __forceinline__ df pend_of(const float* __restrict__ acc, uint32_t v, int deg) {
    const float4* p = reinterpret_cast<const float4*>(acc + size_t(v) * kAccStride);
    const float4 a = __ldg(p);
    df s = df_add_f(df{a.x, 0.0f}, a.y);
    if (deg > 2) s = df_add_f(s, a.z);
    if (deg > 3) s = df_add_f(s, a.w);
    if (deg > 4) {
        const float4 b = __ldg(p + 1);
        s = df_add_f(s, b.x);
        if (deg > 5) s = df_add_f(s, b.y);
        if (deg > 6) s = df_add_f(s, b.z);
    }
    return df_div_i(s, deg);
}

__device__ __forceinline__ uint64_t shl(uint64_t x, int k) { return k >= 0 ? (x << k) : (x >> (-k)); }
__device__ __forceinline__ uint64_t low_mask(int n) { return n >= 64 ? ~0ull : ((1ull << n) - 1ull); }


}  // namespace dev
}  // namespace disco
