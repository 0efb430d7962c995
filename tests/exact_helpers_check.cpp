// Host build of the projection kernels' exact-arithmetic helpers
// (paper_1207_1114_gb300/csrc/exact.cuh) against plain FP64 arithmetic:
//   quant64_of_f32(v, q) == rint((double)v / q) * q   for quanta q = 2^e
//   f64_to_f32_rn(d)     == (float)d
//   AbsDiffMax           == the FP64 maximum of fabs((double)v - (double)x)
//   d < float_at_least(t) (FP32) == d < t (FP64), for floats d
// on random bit patterns, scaled values, exact ties and the edges of each
// helper's range.  Prints the counts and exits non-zero on any mismatch.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <random>

#include "exact.cuh"

using fpfp::f32_bits;
using fpfp::f32_from_bits;
using fpfp::f64_bits;
using fpfp::f64_from_bits;

static bool same64(double a, double b) { return f64_bits(a) == f64_bits(b) || (isnan(a) && isnan(b)); }
static bool same32(float a, float b) { return f32_bits(a) == f32_bits(b) || (isnan(a) && isnan(b)); }

int main(int argc, char** argv) {
    const long n = argc > 1 ? atol(argv[1]) : 2000000;
    std::mt19937_64 g(20240611);
    std::uniform_real_distribution<double> u01(0.0, 1.0);
    long bad_q = 0, bad_c = 0, bad_m = 0;

    // quant64_of_f32 against the FP64 definition (the quantum's scales are
    // plain powers of two here, not the helper's)
    for (long i = 0; i < n; ++i) {
        const int E = (int)(g() % 400) - 150;   // bound exponents, inside and outside the FP32 route
        const fpfp::Quant64 q = fpfp::quant64_from_exp(E);
        const int Ec = E > 900 ? 900 : (E < -900 ? -900 : E);
        const double dn = ldexp(1.0, 52 - Ec), up = ldexp(1.0, Ec - 52);
        float v;
        switch (i % 6) {
            case 0: v = f32_from_bits((unsigned)g()); break;                            // any float
            case 1: v = (float)ldexp(2.0 * u01(g) - 1.0, E + 1); break;               // |v| up to the bound
            case 2: v = (float)ldexp(2.0 * u01(g) - 1.0, E - 52 + (int)(g() % 30)); break;  // near the quantum
            case 3: v = (float)ldexp((double)(g() % (1u << 20)) + 0.5, E - 52); break;  // exact ties
            case 4: v = (g() & 1) ? 0.f : -0.f; break;
            default: v = (float)ldexp(u01(g), (int)(g() % 300) - 150); break;
        }
        const double want = rint((double)v * dn) * up;
        const double got = fpfp::quant64_of_f32(v, q);
        if (!same64(want, got)) {
            if (bad_q < 5) printf("quant64_of_f32(%a, 2^%d): %a, FP64 %a\n", v, Ec - 52, got, want);
            ++bad_q;
        }
    }

    // f64_to_f32_rn against the conversion
    for (long i = 0; i < n; ++i) {
        double d;
        switch (i % 5) {
            case 0: d = f64_from_bits(g()); break;
            case 1: d = ldexp(2.0 * u01(g) - 1.0, (int)(g() % 320) - 160); break;
            case 2: {   // exact midpoints between neighbouring floats, and one ulp of FP64 off them
                const float f = f32_from_bits((unsigned)g() & 0x7f7fffffu);
                const double h = ldexp(1.0, ilogb((double)f) - 24);
                d = (double)f + h + (double)((int)(g() % 3) - 1) * ldexp(h, -29);
                break;
            }
            case 3: d = ldexp(1.0 + u01(g), (g() & 1) ? 127 : -126) * ((g() & 1) ? 1 : -1); break;
            default: d = (g() & 1) ? 0.0 : -0.0; break;
        }
        const float want = (float)d, got = fpfp::f64_to_f32_rn(d);
        if (!same32(want, got)) {
            if (bad_c < 5) printf("f64_to_f32_rn(%a): %a, conversion %a\n", d, got, want);
            ++bad_c;
        }
        if (fpfp::f64_is_finite(d) != (bool)isfinite(d)) ++bad_c;
    }

    // float_at_least: d < t in FP64 exactly when d < float_at_least(t) in FP32
    long bad_t = 0;
    for (long i = 0; i < n; ++i) {
        double t;
        switch (i % 5) {
            case 0: t = (double)f32_from_bits((unsigned)g()); break;                  // t a float
            case 1: t = ldexp(u01(g), (int)(g() % 300) - 150); break;                 // between floats
            case 2: t = f64_from_bits(g()); break;                                    // any double
            case 3: t = ldexp(1.0 + u01(g), 127 + (int)(g() % 3)); break;             // the top of the range
            default: t = ldexp(u01(g), -149 - (int)(g() % 4)); break;                 // below the subnormals
        }
        const float th = fpfp::float_at_least(t);
        for (int k = 0; k < 4; ++k) {
            float d;
            if (k == 0) d = th;
            else if (k == 1) d = nextafterf(th, -INFINITY);
            else if (k == 2) d = (float)t;
            else d = f32_from_bits((unsigned)g());
            if (((double)d < t) != (d < th)) {
                if (bad_t < 5) printf("float_at_least(%a) = %a: d = %a\n", t, th, d);
                ++bad_t;
            }
        }
    }
    bad_c += bad_t;

    // AbsDiffMax against the FP64 maximum, on runs of 1 to 256 elements
    for (long i = 0; i < n / 16; ++i) {
        fpfp::AbsDiffMax m;
        double want = 0.0;
        const int len = 1 + (int)(g() % 256);
        const int kind = (int)(i % 5);
        for (int k = 0; k < len; ++k) {
            float v, x;
            if (kind == 0) {          // an iterate ~1/N against a start 2^-40 below it
                v = (float)(u01(g) * 1e-3);
                x = (float)(ldexp(1.0 + u01(g), -40));
            } else if (kind == 1) {   // close values: cancellation
                x = (float)u01(g);
                v = f32_from_bits(f32_bits(x) + (unsigned)(g() % 5) - 2u);
            } else if (kind == 2) {   // any floats (NaN, infinities, overflowing differences)
                v = f32_from_bits((unsigned)g());
                x = f32_from_bits((unsigned)g());
            } else if (kind == 3) {   // opposite signs near the top of the range
                v = (float)ldexp(1.0 + u01(g), 127);
                x = -(float)ldexp(1.0 + u01(g), 127);
            } else {                  // mixed magnitudes and equal pairs
                x = (float)ldexp(u01(g), (int)(g() % 60) - 40);
                v = (g() % 4) ? (float)ldexp(u01(g), (int)(g() % 60) - 40) : x;
            }
            m.add(v, x);
            want = fmax(want, fabs((double)v - (double)x));
        }
        if (!same64(want, m.value())) {
            if (bad_m < 5) printf("AbsDiffMax run %ld (kind %d): %a, FP64 %a\n", i, kind, m.value(), want);
            ++bad_m;
        }
    }

    printf("quant64_of_f32 mismatches %ld of %ld\n", bad_q, n);
    printf("f64_to_f32_rn / f64_is_finite / float_at_least mismatches %ld of %ld\n", bad_c, n);
    printf("AbsDiffMax mismatches %ld of %ld runs\n", bad_m, n / 16);
    return (bad_q || bad_c || bad_m) ? 1 : 0;
}
