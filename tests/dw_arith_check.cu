// Host-side check of the double-word building blocks (dw_arith.cuh) and of
// the position split (dw_split, md_internal.cuh) that the MD_DW kernels use,
// against exact or long-double references:
//   two_sum, fast_two_sum, two_prod   exact (s + e == a + b, p + e == a b);
//   dw_mul                            within 2^-43 of the product (low parts
//                                     up to 2 ulps of the high ones);
//   dw_add                            within 2^-44 (|x| + |y|) of the sum;
//   r^2 from dw_sq_of and dw_add      within 2^-42 of the exact r^2 of a
//                                     displacement 0.8 .. 2.8 long (the low
//                                     part carries the cross terms 2 h l,
//                                     ~2^-20, rounded in FP32);
//   dw_recip, dw_rsqrt                within 2^-44 of 1/a and 1/sqrt(a) from
//                                     seeds 2^-21 away (the hardware
//                                     approximations are within 2^-22);
//   dw_split                          h on the grid, |h| below 2^24 g, h + l
//                                     within 2^-24 g of p, differences of
//                                     high parts exact in FP32;
//   LJ force factor chain             within 4e-13 of its terms' scale
//                                     (seeds 2^-22 away).
// Built with floating-point contraction off (nvcc -Xcompiler
// -ffp-contract=off); prints one line and exits non-zero on a failure.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>

#include "../paper_2009_07400_gb300/csrc/md_internal.cuh"
#include "../paper_2009_07400_gb300/csrc/dw_arith.cuh"

using namespace mdk;
using namespace mdk::dwa;
typedef long double LD;

static long bad = 0, checked = 0;
static double worst[8] = {0};

static void expect(bool ok, int k, double err, const char *what, double a, double b)
{
    checked++;
    if (err > worst[k]) worst[k] = err;
    if (!ok && bad++ < 8) std::printf("%s failed for %a %a (err %.3g)\n", what, a, b, err);
}

static LD val(dw x) { return (LD)x.h + (LD)x.l; }

int main(int argc, char **argv)
{
    const long n = argc > 1 ? std::atol(argv[1]) : 200000;
    std::mt19937_64 g(2009);
    std::uniform_real_distribution<double> u(-1.0, 1.0), pos(0.5, 2.0);
    auto rf = [&](int emin, int emax) {
        std::uniform_int_distribution<int> e(emin, emax);
        return (float)std::ldexp(u(g), e(g));
    };
    // a double word with |l| up to 2 ulps of h (the kernels' low parts are
    // not always renormalised)
    auto rdw = [&](int emin, int emax) {
        const float h = rf(emin, emax);
        const float l = (float)(u(g) * 2.0 * std::ldexp(1.0, std::ilogb(h) - 23));
        return dw{h, l};
    };
    for (long k = 0; k < n; k++) {
        // error-free transformations (operands within 2^28 of each other,
        // so the exact results fit a double)
        const float a = rf(-20, 20), b = (float)(a * std::ldexp(u(g), -(int)(g() % 28)));
        const dw s = two_sum(a, b);
        expect((double)s.h + (double)s.l == (double)a + (double)b, 0, 0, "two_sum", a, b);
        const float big = std::fabs(a) >= std::fabs(b) ? a : b, small = big == a ? b : a;
        const dw f = fast_two_sum(big, small);
        expect((double)f.h + (double)f.l == (double)big + (double)small, 0, 0, "fast_two_sum", big, small);
        const float c = rf(-20, 20);
        const dw p = two_prod(a, c);
        expect((double)p.h + (double)p.l == (double)a * (double)c, 0, 0, "two_prod", a, c);

        // products and sums of double words
        const dw x = rdw(-10, 10), y = rdw(-10, 10);
        const LD xy = val(x) * val(y);
        const double em = (double)(std::fabs(val(dw_mul(x, y)) - xy) / std::fabs(xy));
        expect(em <= std::ldexp(1.0, -43), 1, em, "dw_mul", x.h, y.h);
        const double sc = std::ldexp(1.0, (int)(g() % 8) - 4);
        const dw y2 = {(float)(y.h * sc), (float)(y.l * sc)};
        const LD sum = val(x) + val(y2);
        const double ea = (double)(std::fabs(val(dw_add(x, y2)) - sum) /
                                   (std::fabs(val(x)) + std::fabs(val(y2))));
        expect(ea <= std::ldexp(1.0, -44), 2, ea, "dw_add", x.h, y2.h);

        // r^2 of a pair displacement as the kernels form it: components with
        // exact high parts on the position grid (2^-21) and low parts below
        // 2^-22, |d| from 0.8 to 2.8, three dw_sq_of and two dw_add
        {
            double dir[3], nn = 0;
            for (double &c : dir) { c = u(g); nn += c * c; }
            const double len = (0.8 + 2.0 * (0.5 + 0.5 * u(g))) / std::sqrt(nn);
            float dh[3], dl[3];
            LD r2x = 0;
            for (int q = 0; q < 3; q++) {
                dh[q] = (float)std::ldexp(std::nearbyint(std::ldexp(dir[q] * len, 21)), -21);
                dl[q] = (float)(u(g) * std::ldexp(1.0, -22));
                r2x += ((LD)dh[q] + dl[q]) * ((LD)dh[q] + dl[q]);
            }
            const dw r2 = dw_add(dw_add(dw_sq_of(dh[0], dl[0]), dw_sq_of(dh[1], dl[1])),
                                 dw_sq_of(dh[2], dl[2]));
            const double es = (double)(std::fabs(val(r2) - r2x) / r2x);
            expect(es <= std::ldexp(1.0, -42), 3, es, "r^2 from dw_sq_of", dh[0], dl[0]);
        }

        // reciprocal and reciprocal square root from perturbed seeds
        const dw r2 = {(float)(pos(g) * std::ldexp(1.0, (int)(g() % 6) - 2)), 0.f};
        const dw r2l = {r2.h, (float)(u(g) * std::ldexp(1.0, std::ilogb(r2.h) - 23))};
        const float af = add_rn(r2l.h, r2l.l);
        const float seed = (float)((1.0 / af) * (1.0 + u(g) * std::ldexp(1.0, -21)));
        const LD inv = 1.0L / val(r2l);
        const double er = (double)(std::fabs(val(dw_recip(r2l, af, seed)) - inv) / inv);
        expect(er <= std::ldexp(1.0, -44), 4, er, "dw_recip", r2l.h, seed);
        const float rseed = (float)((1.0 / std::sqrt((double)af)) * (1.0 + u(g) * std::ldexp(1.0, -21)));
        const LD rs = 1.0L / std::sqrt(val(r2l));
        const double eq = (double)(std::fabs(val(dw_rsqrt(r2l, af, rseed)) - rs) / rs);
        expect(eq <= std::ldexp(1.0, -44), 5, eq, "dw_rsqrt", r2l.h, rseed);
    }

    // the position split on the grid of a replica with cells of side 2.83
    {
        Rep R{};
        const double s = 2.8288, gs = std::ldexp(1.0, -21);   // 2^24 g = 8 >= 2.5 s
        R.dw_magic = 1.5 * std::ldexp(gs, 52);
        R.dw_lim = (float)(std::ldexp(gs, 24) - s - gs);
        const double sh = std::nearbyint(s / gs) * gs;
        for (long k = 0; k < n; k++) {
            const double p = u(g) * 1.5 * s, q = u(g) * 1.5 * s;
            float h, l, hq, lq;
            const bool ok = dw_split(R, p, h, l) && dw_split(R, q, hq, lq);
            const double onj = std::fmod((double)h / gs, 1.0);
            const double e = std::fabs(p - ((double)h + (double)l));
            expect(ok && onj == 0.0 && e <= std::ldexp(gs, -24), 6, e / gs, "dw_split", p, h);
            // p_i -+ s_h: exact in FP32 within the guarded range; the
            // difference with p_j too wherever it is below 2^24 g (every
            // pair within the list radius)
            for (int o = -1; o <= 1; o++) {
                const float qh = (float)((double)h - o * sh);
                const double dx = (double)qh - (double)hq;
                const float d = qh - hq;
                expect((double)qh == (double)h - o * sh &&
                       (std::fabs(dx) >= std::ldexp(gs, 24) || (double)d == dx), 6, 0,
                       "split difference", p, q);
            }
        }
    }

    // the LJ force factor f = sr2 sr6 (48 sr6 - 24) in double word against
    // long double, for pair distances 0.85 .. 2.5 (sigma = eps = 1)
    {
        const dw a12 = {48.f, 0.f}, a6n = {-24.f, 0.f};
        for (long k = 0; k < n; k++) {
            const double r = 0.85 + 1.65 * (0.5 + 0.5 * u(g));
            const dw r2 = {(float)(r * r), (float)(r * r - (double)(float)(r * r))};
            const float af = add_rn(r2.h, r2.l);
            const float seed = (float)((1.0 / af) * (1.0 + u(g) * std::ldexp(1.0, -22)));
            const dw sr2 = dw_recip(r2, af, seed);
            const dw sr6 = dw_mul(dw_mul(sr2, sr2), sr2);
            const dw f = dw_mul(dw_mul(sr2, sr6), dw_add(dw_mul(a12, sr6), a6n));
            const LD R2 = val(r2), S2 = 1.0L / R2, S6 = S2 * S2 * S2;
            const LD fe = S2 * S6 * (48.0L * S6 - 24.0L);
            const double scale = (double)(S2 * S6 * (48.0L * S6 + 24.0L));
            const double ef = (double)std::fabs(val(f) - fe) / scale;
            expect(ef <= 4e-13, 7, ef, "LJ factor", r, 0.0);
        }
    }
    if (bad) {
        std::printf("FAILED: %ld of %ld checks\n", bad, checked);
        return 1;
    }
    std::printf("ok: %ld checks; worst dw_mul %.3g, dw_add %.3g, r^2 %.3g, dw_recip %.3g, "
                "dw_rsqrt %.3g, split %.3g g, LJ factor %.3g\n", checked, worst[1], worst[2], worst[3],
                worst[4], worst[5], worst[6], worst[7]);
    return 0;
}
