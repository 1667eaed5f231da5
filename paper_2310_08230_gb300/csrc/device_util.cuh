// Device helpers shared by the half-pass kernels (kernels.cu) and their adjoints
// (adjoint.cu): layer descriptors, shifts of a layer's node costs by an arc offset, and
// double-float arithmetic for the dual variables.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#include "kernels.h"

// Functions marked DH are also compiled for the host: the averaging arithmetic is checked on
// the CPU against exact integer arithmetic.
#define DH __host__ __device__ __forceinline__

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

DH uint32_t bits_of(float x) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return u;
#endif
}
DH float float_of(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float x;
    std::memcpy(&x, &u, 4);
    return x;
#endif
}

DH void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
DH df fast2sum(float s, float e) {
    const float h = s + e;
    return df{h, e - (h - s)};
}
DH df df_add(df a, df b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return fast2sum(s, e + (a.lo + b.lo));
}
DH df df_add_f(df a, float b) {
    float s, e;
    two_sum(a.hi, b, s, e);
    return fast2sum(s, e + a.lo);
}
// a / n for a small positive integer n. q = a.hi * (1/n) is within an ulp of a.hi / n, so the
// remainder a.hi - q n is exact with an FMA (the classic division-by-reciprocal argument);
// the low part needs only single precision.
// 1/n correctly rounded to FP32 for the possible degrees n = 2 .. 7 (entries 0 and 1 unused).
static __constant__ float kRcpDeg[8] = {1.0f, 1.0f, 0.5f, 0.333333343f, 0.25f, 0.200000003f, 0.166666672f,
                                        0.142857149f};
DH float rcp_deg(int n) {
#ifdef __CUDA_ARCH__
    return kRcpDeg[n & 7];
#else
    static const float t[8] = {1.0f, 1.0f, 0.5f, 0.333333343f, 0.25f, 0.200000003f, 0.166666672f, 0.142857149f};
    return t[n & 7];
#endif
}

DH df df_div_i(df a, int n) {
    const float fn = float_of(0x4B000000u | uint32_t(n)) - 8388608.0f;  // exact for 0 <= n < 2^23
    const float rcp = rcp_deg(n);
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
// one rounded mass is at most 2^42 grid units (lim = 2^(42 - F); the kernels flag a larger
// one), so a sum of up to 7 stays below 2^45.
//
// No conversion instruction touches a 64-bit integer: those run on the FP64 pipe, which is a
// small fraction of the FP32 rate on this GPU. Integers of fewer than 24 bits move between
// the integer and FP32 registers by the 2^23 significand trick: for 0 <= n < 2^23 the float
// with bits 0x4B000000 + n is exactly 2^23 + n (and 0x4B400000 + n is 1.5 * 2^23 + n for
// -2^22 <= n < 2^22).
constexpr float kTwo23 = 8388608.0f;        // 2^23
constexpr float kOneHalf23 = 12582912.0f;   // 1.5 * 2^23
constexpr float kTwo42 = 4398046511104.0f;  // 2^42
constexpr int kFxSumBits = 45;              // |sum| < 2^45 grid units

// m on the grid: q = m 2^F rounded to an integer (ties to even), and the return value q 2^-F,
// both exact. With t = m 2^F clamped to |t| <= 2^42 (a clamped mass is flagged by the caller
// as out of range): h = rint(t 2^-23) and l = rint(t - h 2^23) by the significand trick
// (|t 2^-23| <= 2^19 and |t - h 2^23| <= 2^22), so q = h 2^23 + l = rint(t), with h and l read
// from the significands as integers; q 2^-F has at most 24 significant bits, so FP32 holds it.
DH float fx_round(float m, const FxScale& fx, long long& q) {
    const float t = fminf(fmaxf(m * fx.scale, -kTwo42), kTwo42);
    const float hs = fmaf(t, 1.0f / kTwo23, kOneHalf23);  // 1.5 2^23 + rint(t 2^-23), exact
    const float h = hs - kOneHalf23;
    const float ls = (fmaf(-h, kTwo23, t)) + kOneHalf23;  // 1.5 2^23 + rint(remainder)
    const float l = ls - kOneHalf23;
    const int32_t hi = int32_t(bits_of(hs) - 0x4B400000u);
    const int32_t lo = int32_t(bits_of(ls) - 0x4B400000u);
    q = (long long)hi * (1 << 23) + lo;
    return fmaf(h, kTwo23, l) * fx.inv;
}

// A sum S (units of 2^-F, |S| < 2^45) as double-float, exactly: S = A 2^23 + C with
// 0 <= C < 2^23 and |A| < 2^22, both parts exact in FP32, added without error (the pair holds
// 48 bits); the scaling by 2^-F is exact.
DH df fx_to_df(long long S, float inv) {
    const uint32_t c = uint32_t(S) & 0x7FFFFFu;
    const int32_t a = int32_t(S >> 23);
    const float cf = float_of(0x4B000000u + c) - kTwo23;
    const float af = (float_of(uint32_t(0x4B400000 + a)) - kOneHalf23) * kTwo23;
    // |af| >= |cf| whenever A != 0 (C < 2^23 <= |A| 2^23), and A = 0 gives (cf, 0): Fast2Sum
    // is exact here
    const df r = fast2sum(af, cf);
    return df{r.hi * inv, r.lo * inv};
}
// The deferred mean of a variable: its sum / deg, in double-float.
DH df fx_mean(long long S, int deg, float inv) { return df_div_i(fx_to_df(S, inv), deg); }

__device__ __forceinline__ uint64_t shl(uint64_t x, int k) { return k >= 0 ? (x << k) : (x >> (-k)); }
__device__ __forceinline__ uint64_t low_mask(int n) { return n >= 64 ? ~0ull : ((1ull << n) - 1ull); }


}  // namespace dev
}  // namespace disco
