// Host-side check of the averaging arithmetic of the half-pass kernels (device_util.cuh):
// the rounding of a removed mass to the fixed-point grid (with its integer value), the split
// of a 64-bit sum into a double-float and the deferred mean. Every result is
// compared with exact integer or extended-precision arithmetic. Prints "ok <cases>" or the
// first failure and exits non-zero.
#include <cfenv>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>

#include "../../paper_2310_08230_gb300/csrc/device_util.cuh"

using namespace disco;
using namespace disco::dev;

static int fails = 0;
static long cases = 0;

#define EXPECT(cond, ...)                              \
    do {                                               \
        ++cases;                                       \
        if (!(cond)) {                                 \
            if (fails++ < 10) std::printf(__VA_ARGS__); \
        }                                              \
    } while (0)

static float ulp_of(float x) {
    const float a = std::fabs(x);
    return std::nextafter(a, INFINITY) - a;
}

int main() {
    std::mt19937_64 rng(12345);
    // 2. fx_round: q = round-half-even(m 2^F), the returned mass = q 2^-F, for F = 2 .. 52 (the
    //    grids a handle can choose), masses below the range limit 2^(42 - F); beyond it the
    //    rounded value is clamped to 2^42 grid units
    std::fesetround(FE_TONEAREST);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    for (int F = 2; F <= 52; F += 5) {
        const FxScale fx{std::ldexp(1.0f, F), std::ldexp(1.0f, -F), std::ldexp(1.0f, 42 - F)};
        for (int k = 0; k < 40000; ++k) {
            const double mag = std::ldexp(1.0, -int(rng() % 40) + (42 - F));
            const float m = float(U(rng) * mag);
            long long q;
            const float r = fx_round(m, fx, q);
            const long long want = std::llrint(std::ldexp(double(m), F));  // exact product, ties to even
            EXPECT(q == want, "fx_round F=%d m=%.9g: q=%lld want %lld\n", F, m, q, want);
            EXPECT(double(r) == std::ldexp(double(want), -F), "fx_round F=%d m=%.9g: r=%.17g\n", F, m, double(r));
        }
        for (double t : {0.5, 1.5, 2.5, -0.5, -2.5, 8388607.5, 8388608.0, -8388607.5, 4194303.5, 0.0, -0.0}) {
            const float m = float(std::ldexp(t, -F));
            long long q;
            fx_round(m, fx, q);
            EXPECT(q == std::llrint(t), "fx_round tie F=%d t=%g: q=%lld\n", F, t, q);
        }
        // remainders at the +-2^22 edge of the low half, and halves of either sign
        for (double t : {5.0 * 8388608.0 + 4194304.0, -5.0 * 8388608.0 - 4194304.0, 3.0 * 8388608.0 - 4194304.0,
                         std::ldexp(1.0, 42), -std::ldexp(1.0, 42), std::ldexp(1.0, 42) - std::ldexp(1.0, 18),
                         -std::ldexp(3.0, 40) + 0.0, 8388608.0 * 1000.0 + 1.0}) {
            const float m = float(std::ldexp(t, -F));
            long long q;
            const float r = fx_round(m, fx, q);
            const long long want = std::llrint(std::ldexp(double(m), F));
            EXPECT(q == want, "fx_round edge F=%d t=%.17g: q=%lld want %lld\n", F, t, q, want);
            EXPECT(double(r) == std::ldexp(double(want), -F), "fx_round edge F=%d t=%.17g\n", F, t);
        }
        for (double t : {std::ldexp(1.0, 43), -std::ldexp(3.0, 50), 1e30}) {
            long long q;
            fx_round(float(std::ldexp(t, -F)), fx, q);
            EXPECT(std::llabs(q) == (1ll << 42), "fx_round clamp F=%d: q=%lld\n", F, q);
        }
        {
            long long q;
            fx_round(std::nanf(""), fx, q);
            EXPECT(std::llabs(q) == (1ll << 42), "fx_round NaN F=%d: q=%lld\n", F, q);
        }
    }
    // 3. fx_to_df is exact: hi + lo == S 2^-F for |S| < 2^45, and |lo| <= ulp(hi) / 2
    auto draw_sum = [&]() {
        const int bitsz = int(rng() % kFxSumBits);
        int64_t S = int64_t(rng() >> (64 - bitsz - 1)) >> 1;  // |S| < 2^bitsz
        return (rng() & 1) ? -S : S;
    };
    for (int k = 0; k < 400000; ++k) {
        const int64_t S = draw_sum();
        const int F = 2 + int(rng() % 51);
        const df d = fx_to_df(S, std::ldexp(1.0f, -F));
        const long double want = std::ldexp((long double)S, -F);
        EXPECT((long double)d.hi + (long double)d.lo == want, "fx_to_df S=%lld F=%d not exact\n", (long long)S, F);
        EXPECT(d.hi == 0.0f ? d.lo == 0.0f : std::fabs(d.lo) <= 0.5f * ulp_of(d.hi),
               "fx_to_df S=%lld: not normalised (%.9g, %.9g)\n", (long long)S, d.hi, d.lo);
    }
    for (int64_t S : {int64_t(0), int64_t(1), int64_t(-1), (int64_t(1) << 45) - 1, -(int64_t(1) << 45) + 1,
                      int64_t(7) << 42, -(int64_t(7) << 42), int64_t(0x7FFFFF), int64_t(0x800000)}) {
        const df d = fx_to_df(S, 1.0f);
        EXPECT((long double)d.hi + (long double)d.lo == (long double)S, "fx_to_df edge S=%lld\n", (long long)S);
    }
    // 4. fx_mean: the deferred mean S / deg, deg = 2 .. 7, to 2^-45 relative (the split is
    //    exact; the double-float division adds up to 2^-45.6, the worst at deg 7)
    for (int k = 0; k < 200000; ++k) {
        const int64_t S = draw_sum();
        const int deg = 2 + int(rng() % 6);
        const int F = 32;
        const df d = fx_mean(S, deg, std::ldexp(1.0f, -F));
        const long double want = std::ldexp((long double)S, -F) / deg;
        const long double got = (long double)d.hi + (long double)d.lo;
        EXPECT(std::fabs(got - want) <= std::ldexp(std::fabs(want), -45), "fx_mean S=%lld deg=%d\n", (long long)S, deg);
    }
    // 5. a sum of rounded masses (what red.add accumulates) converts back to their exact total
    for (int k = 0; k < 100000; ++k) {
        const int F = 32;
        const FxScale fx{std::ldexp(1.0f, F), std::ldexp(1.0f, -F), std::ldexp(1.0f, 42 - F)};
        const int deg = 2 + int(rng() % 6);
        long long S = 0;
        long double tot = 0;
        for (int r = 0; r < deg; ++r) {
            long long q;
            const float mr = fx_round(float(U(rng) * std::ldexp(1.0, 9 - int(rng() % 30))), fx, q);
            S += q;
            tot += (long double)mr;
        }
        const df d = fx_to_df(S, fx.inv);
        EXPECT((long double)d.hi + (long double)d.lo == tot, "sum of masses: S=%lld\n", S);
    }
    if (fails) {
        std::printf("FAILED %d of %ld\n", fails, cases);
        return 1;
    }
    std::printf("ok %ld\n", cases);
    return 0;
}
