// exact.cuh -- exact-arithmetic helpers of the projection kernels: the FP64
// quanta of the order-free sums, FP64 results formed with FP32 and integer
// operations (the FP64 unit of this part is slow), and the exact max|v - x|
// of the outer stop.  Written for the device and the host alike, so that a
// host build can check every helper against plain FP64 arithmetic.
#pragma once

#include <math.h>
#include <string.h>

#if defined(__CUDACC__)
#define FPFP_HD __host__ __device__ __forceinline__
#else
#define FPFP_HD inline
#endif

namespace fpfp {

// ------------------------------------------------------------- bit views
FPFP_HD unsigned f32_bits(float f) {
#if defined(__CUDA_ARCH__)
    return __float_as_uint(f);
#else
    unsigned u;
    memcpy(&u, &f, sizeof u);
    return u;
#endif
}
FPFP_HD float f32_from_bits(unsigned u) {
#if defined(__CUDA_ARCH__)
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
#endif
}
FPFP_HD unsigned long long f64_bits(double d) {
#if defined(__CUDA_ARCH__)
    return (unsigned long long)__double_as_longlong(d);
#else
    unsigned long long u;
    memcpy(&u, &d, sizeof u);
    return u;
#endif
}
FPFP_HD double f64_from_bits(unsigned long long u) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)u);
#else
    double d;
    memcpy(&d, &u, sizeof d);
    return d;
#endif
}

// ------------------------------------------------ FP64 quanta of the sums
// Order-free FP64 sums (totals s, the input's column sums): every
// contribution is rounded to a multiple of a power-of-two quantum q before
// its atomic add; with every partial sum below 2^53 q each addition is exact,
// so the sum does not depend on the order of the adds.  For a bound b the
// quantum is q = 2^(E-52), E = floor(log2 b), so b < 2^(E+1) = 2^53 q; b <= 0
// (only zeros to add) takes q = 1.  The scales are built from exponent bits.
struct Quant64 {
    double dn, up;
};
FPFP_HD Quant64 quant64_from_exp(int E) {
    E = E > 900 ? 900 : (E < -900 ? -900 : E);
    return Quant64{f64_from_bits((unsigned long long)(1023 + 52 - E) << 52),
                   f64_from_bits((unsigned long long)(1023 - 52 + E) << 52)};
}
FPFP_HD Quant64 quant64_for(double bound) {
    if (!(bound > 0.0)) return Quant64{1.0, 1.0};
    return quant64_from_exp((int)((f64_bits(bound) >> 52) & 0x7ff) - 1023);
}
// The same from a float bound (positive, finite).
FPFP_HD Quant64 quant64_for_f(float bound) {
    if (!(bound > 0.f)) return Quant64{1.0, 1.0};
    return quant64_from_exp((int)((f32_bits(bound) >> 23) & 0xff) - 127);
}
FPFP_HD double quant64(double v, Quant64 q) { return rint(v * q.dn) * q.up; }

// quant64 of an FP32 value without FP64 arithmetic, the same bits.  For a
// quantum 2^e with -126 <= e <= 104 and |v| < 2^(e+23), |v| + 2^(e+23) lies
// in [2^(e+23), 2^(e+24)], where floats are 2^e apart, so the addition
// rounds |v| to the nearest multiple of 2^e (ties to an even multiple, as
// rint does) and the subtraction is exact; a float |v| >= 2^(e+23) already
// is a multiple of 2^e.  The result is 0 or a normal float, widened to FP64
// by its bits.  Other quanta, and infinite or NaN v, take the FP64 route.
FPFP_HD double quant64_of_f32(float v, Quant64 q) {
    const int e = (int)((f64_bits(q.up) >> 52) & 0x7ff) - 1023;
    const float a = f32_from_bits(f32_bits(v) & 0x7fffffffu);
    if (e < -126 || e > 104 || !(a <= 3.402823466e38f)) return quant64((double)v, q);
    const float C = f32_from_bits((unsigned)(127 + 23 + e) << 23);
    const unsigned b = f32_bits(a < C ? (a + C) - C : a) | (f32_bits(v) & 0x80000000u);
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    if ((b & 0x7fffffffu) == 0u) return f64_from_bits(sign);
    return f64_from_bits(sign | ((unsigned long long)(((b >> 23) & 0xffu) + 896u) << 52) |
                         ((unsigned long long)(b & 0x7fffffu) << 29));
}

// ------------------------------------------------- FP64 -> FP32, finiteness
// (float)d by integer operations (round to nearest, ties to even), for
// results in the normal float range; zero, results below it, overflow,
// infinities and NaN take the conversion instruction.  A carry out of the
// fraction moves into the exponent, as rounding does (to infinity from the
// top binade).
FPFP_HD float f64_to_f32_rn(double d) {
    const unsigned long long b = f64_bits(d);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex < 1023 - 126 || ex > 1023 + 127) return (float)d;
    const unsigned long long rest = b & 0x1fffffffull;   // the 29 fraction bits dropped
    unsigned bits = ((unsigned)(ex - 1023 + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffull);
    if (rest > 0x10000000ull || (rest == 0x10000000ull && (bits & 1u))) bits += 1u;
    return f32_from_bits(bits | ((unsigned)(b >> 63) << 31));
}
FPFP_HD bool f64_is_finite(double d) { return ((f64_bits(d) >> 52) & 0x7ff) != 0x7ff; }

// The least float >= t (t itself when it is a float; +inf above the float
// range; NaN stays NaN): a float d is below it exactly when d < t in FP64, so
// a stop test of an FP32 quantity against an FP64 tolerance compares in FP32.
// Host only (the threshold is formed once per launch).
inline float float_at_least(double t) {
    float f = (float)t;
    if ((double)f < t) f = nextafterf(f, INFINITY);
    return f;
}

// --------------------------------------------------- exact max |v - x|
// The maximum over elements of |v - x| rounded once to FP64 (what
// fabs((double)v - (double)x) gives), with FP32 arithmetic per element: the
// FP64 units of this part run at a small fraction of the FP32 rate.  Knuth's
// TwoSum splits v - x exactly into s + t (s = fl(v - x), |t| <= ulp(s)/2);
// then |v - x| = |s| + sign(s) t, and the pairs (|s|, sign(s) t) order like
// the exact differences under lexicographic comparison (rounding is
// monotone), so the running maximum is kept as a pair and rounded to FP64
// once.  A difference that overflows FP32 (s or t not finite) takes the
// FP64 path; NaN differences are ignored, as fmax ignores them.
struct AbsDiffMax {
    float hi = 0.f, lo = 0.f;   // the largest |v - x| so far, exactly hi + lo
    double big = 0.0;           // the FP64 maximum of the differences FP32 cannot hold
    FPFP_HD static bool finite32(float f) { return (f32_bits(f) & 0x7f800000u) != 0x7f800000u; }
    FPFP_HD void add(float v, float x) {
        const float s = v - x;
        const float vr = s + x;            // TwoSum of v and -x
        const float xr = s - vr;
        const float t = (v - vr) - (x + xr);
        const float as = f32_from_bits(f32_bits(s) & 0x7fffffffu), at = s < 0.f ? -t : t;
        if (as > hi || (as == hi && at > lo)) {
            if (finite32(as) && finite32(at)) {
                hi = as;
                lo = at;
            } else {
                big = fmax(big, fabs((double)v - (double)x));
            }
        }
    }
#if defined(__CUDACC__)
    FPFP_HD void add4(float4 v, float4 x) {
        add(v.x, x.x);
        add(v.y, x.y);
        add(v.z, x.z);
        add(v.w, x.w);
    }
#endif
    FPFP_HD double value() const { return fmax(big, (double)hi + (double)lo); }
};

}  // namespace fpfp
