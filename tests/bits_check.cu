// Host-side check of the bit-level FP64/FP32 helpers of md_device.cuh
// against the hardware conversions and their stated error bounds, on random
// bit patterns and edge values.  Built and run by test_bit_helpers.py (no GPU
// needed: the helpers are __host__ __device__).  Prints one line per helper
// and exits non-zero on any mismatch.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "md_device.cuh"

using namespace pasta;

static double ulp_of(double h) { return std::ldexp(1.0, std::ilogb(h) - 23); }   // FP32 ulp of h

int main(int argc, char** argv) {
    const long n = argc > 1 ? std::atol(argv[1]) : 2000000;
    std::mt19937_64 g(12345);
    long bad_w = 0, bad_n = 0, bad_s = 0, bad_x = 0, cnt_n = 0, cnt_s = 0;
    double worst_s = 0.0;
    // widen: exact (double)f, bit for bit, for every non-NaN float pattern drawn
    const float fedge[] = {0.0f, -0.0f, 1e-45f, -1e-45f, 1.17549435e-38f, 3.4e38f, INFINITY, -INFINITY, 1.0f, -2.5f};
    for (float f : fedge) {
        const double w = widen(f), r = (double)f;
        if (std::memcmp(&w, &r, 8) != 0) ++bad_w;
    }
    for (long i = 0; i < n; ++i) {
        const unsigned b = (unsigned)g();
        const float f = f_from(b);
        if (std::isnan(f)) continue;
        const double w = widen(f), r = (double)f;
        if (std::memcmp(&w, &r, 8) != 0) ++bad_w;
    }
    std::uniform_real_distribution<double> U(-1500.0, 1500.0);
    for (long i = 0; i < n; ++i) {
        const int kind = i % 4;
        const double x = kind == 0 ? U(g) : kind == 1 ? U(g) * 1e-9 : kind == 2 ? std::ldexp(U(g), -60) : d_from(g());
        if (std::isnan(x) || std::isinf(x)) continue;
        const double ax = std::fabs(x);
        // narrow_trunc: |t| <= |x|, relative gap below 2^-23, same sign (normal FP32 range)
        const float t = narrow_trunc(x);
        if (ax >= 1.2e-38 && ax < 3.0e38) {
            ++cnt_n;
            const double at = std::fabs((double)t);
            if (!(at <= ax && ax - at <= ax * std::ldexp(1.0, -23) && (t == 0.0f || std::signbit(t) == std::signbit(x))))
                ++bad_n;
        } else if (x == 0.0) {
            if (t != 0.0f || std::signbit(t) != std::signbit(x)) ++bad_n;
        }
        // split_hilo: hi nearest to x within half an FP32 ulp, |x - hi - lo| <= 2^-49 |x|
        float hi, lo;
        split_hilo(x, hi, lo);
        if (ax >= 6e-23 && ax < 8.0e37) {
            ++cnt_s;
            const double err = std::fabs(((double)hi + (double)lo) - x);
            worst_s = std::fmax(worst_s, err / ax);
            if (!(err <= ax * std::ldexp(1.0, -49)) || !(std::fabs((double)hi - x) <= 0.5 * ulp_of((double)hi)))
                ++bad_s;
        } else if (x == 0.0 && (hi != 0.0f || lo != 0.0f)) {
            ++bad_s;
        }
    }
    // wrap_box_bits == wrap_box over [-L, 2L) and the edges
    const double L = 172.35468;
    const double xedge[] = {0.0, -0.0, L, std::nextafter(L, 0.0), -1e-300, -L, 2.0 * L - 1e-9, 1e-320};
    for (double x : xedge)
        if (wrap_box_bits(x, L) != wrap_box(x, L) || std::signbit(wrap_box_bits(x, L)) != std::signbit(wrap_box(x, L)))
            ++bad_x;
    std::uniform_real_distribution<double> W(-L, 2.0 * L);
    for (long i = 0; i < n; ++i) {
        const double x = W(g);
        if (wrap_box_bits(x, L) != wrap_box(x, L)) ++bad_x;
    }
    std::printf("widen: %ld mismatches\n", bad_w);
    std::printf("narrow_trunc: %ld of %ld outside the bound\n", bad_n, cnt_n);
    std::printf("split_hilo: %ld of %ld outside the bound, worst |x-hi-lo|/|x| = %.3g (2^-49 = %.3g)\n", bad_s,
                cnt_s, worst_s, std::ldexp(1.0, -49));
    std::printf("wrap_box_bits: %ld mismatches\n", bad_x);
    return (bad_w || bad_n || bad_s || bad_x) ? 1 : 0;
}
