// Host-side check of the library's FP64/FP32 conversions and compares on IEEE
// bit patterns (md_internal.cuh) against the hardware's own conversions:
// f64_of_f32 on every float; f32_of_f64 on random bit patterns of every
// exponent, on random values of the ranges the kernels meet, on exact
// rounding ties and on edge cases; f32_of_pos / f64_of_pos / lt_nonneg on
// their stated domains.  Prints one line and exits non-zero on a mismatch.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <limits>
#include <random>

#include "../paper_2009_07400_gb300/csrc/md_internal.cuh"

using namespace mdk;

static bool same(float a, float b) { return bits_of(a) == bits_of(b) || (std::isnan(a) && std::isnan(b)); }
static bool same(double a, double b) { return bits_of(a) == bits_of(b) || (std::isnan(a) && std::isnan(b)); }

int main(int argc, char **argv)
{
    const long nrand = argc > 1 ? std::atol(argv[1]) : 4000000;
    long bad = 0, checked = 0;
    auto f32 = [&](double a) {
        checked++;
        if (!same(f32_of_f64(a), (float)a)) {
            if (bad++ < 5) std::printf("f32_of_f64(%a) = %a, expected %a\n", a, f32_of_f64(a), (float)a);
        }
    };
    // every float through f64_of_f32 (exact widening)
    for (uint64_t u = 0; u <= 0xffffffffULL; u++) {
        const float f = float_of((unsigned int)u);
        checked++;
        if (!same(f64_of_f32(f), (double)f)) {
            if (bad++ < 5) std::printf("f64_of_f32(%a) = %a\n", f, f64_of_f32(f));
        }
    }
    std::mt19937_64 g(20091);
    for (long k = 0; k < nrand; k++) {
        f32(double_of((long long)g()));                                  // any exponent
        const double v = std::ldexp((double)(g() >> 11), -53) * 3.0 - 1.5;
        f32(v);                                                           // |p| <= s/2 range
        f32(double_of((bits_of(v) & ~((1LL << 29) - 1)) | (1LL << 28)));   // exact tie
        f32(double_of((bits_of(v) & ~((1LL << 29) - 1)) | (1LL << 28) | (1LL << 29)));
        // positive-domain helpers: values of r^2 the force and contact kernels meet
        const double r2 = 0.01 + std::ldexp((double)(g() >> 11), -53) * 1e4;
        checked += 2;
        const float p = f32_of_pos(r2);
        if (std::fabs((double)p - r2) > std::ldexp(r2, -24)) { if (bad++ < 5) std::printf("f32_of_pos(%a)\n", r2); }
        if (!same(f64_of_pos(p), (double)p)) { if (bad++ < 5) std::printf("f64_of_pos(%a)\n", p); }
        const double q = std::ldexp((double)(g() >> 11), -53) * 1e4;
        checked++;
        if (lt_nonneg(r2, q) != (r2 < q)) { if (bad++ < 5) std::printf("lt_nonneg(%a, %a)\n", r2, q); }
    }
    const double inf = std::numeric_limits<double>::infinity();
    const double edge[] = {0.0, -0.0, 1.0, -1.0, 1e-40, -1e-40, 1.1754943508222875e-38, 1.1754942e-38,
                           -1.1754943508222875e-38, 3.4028234663852886e38, 3.4028235677973366e38,
                           3.5e38, -3.5e38, inf, -inf, std::nan(""), 5e-324, 2.2250738585072014e-308};
    for (double e : edge) f32(e);
    checked++;
    if (lt_nonneg(std::nan(""), 1.0)) bad++;                             // NaN compares false
    std::printf("%s: %ld checks, %ld mismatches\n", bad ? "FAIL" : "ok", checked, bad);
    return bad ? 1 : 0;
}
