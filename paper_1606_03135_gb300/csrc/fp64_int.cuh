// fp64_int.cuh -- FP64 helpers that keep work off GB300's narrow FP64 pipe: reciprocals and
// square roots refined on the integer pipe, exact small-integer constants, and magnitude
// keys / FP32 approximations built from FP64 bit patterns with integer instructions.  Every
// function here is written from the Newton-Raphson iteration and the IEEE-754 binary64
// layout; the test-suite checks them against the FP64 division and square root.
#pragma once
#include <cuda_runtime.h>

namespace rbffd {

// The double equal to the integer v (0 <= v < 2^31), assembled from its bits with integer
// instructions (an int-to-FP64 conversion would occupy the narrow FP64 pipe).
__device__ __forceinline__ double exact_double(int v) {
    if (v == 0) return 0.0;
    const int e = 31 - __clz(v);  // v = 1.f * 2^e
    const unsigned long long mant = ((unsigned long long)v << (52 - e)) & 0xFFFFFFFFFFFFFull;
    return __longlong_as_double((long long)(((unsigned long long)(1023 + e) << 52) | mant));
}

// Reciprocal of an FP64 value on the integer pipe (GB300's FP64 pipe is ~1/64 of its FP32
// rate, and a scalar division issued by one warp occupies it as a full warp instruction).
// rcp_core covers normal x whose reciprocal is normal (biased exponent in [1, 0x7fc]) and
// sets *slow for every other input; it has no branches, so the compiler can interleave it
// with independent work.  A 24-bit FP32 seed t0 of 1/m for the mantissa m is refined by one
// cubic Newton-Raphson step t1 = t0 (1 + e + e^2), e = 1 - m t0, in 64-bit fixed point
// (error about e^3, below 2^-62), then rounded to 53 bits: within 1 ulp of 1/x.  Powers of
// two are exact.
__device__ __forceinline__ double rcp_core(double x, bool* slow) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long sign = b >> 63;
    const int e = (int)((b >> 52) & 0x7ff);
    const unsigned long long f = b & 0xFFFFFFFFFFFFFull;
    *slow = (e == 0) | (e >= 0x7fd);
    const unsigned long long M = f | (1ull << 52);  // m = M / 2^52 in [1, 2)
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__int_as_float(0x3F800000 | (int)(f >> 29))));
    const unsigned rb = __float_as_uint(rf);
    unsigned long long Y =  // Y = t0 2^64, t0 in (1/2, 1]
        rb >= 0x3F800000u ? ~0ull : (unsigned long long)((rb & 0x7FFFFFu) | 0x800000u) << 40;
    const unsigned long long lo = M * Y, hi = __umul64hi(M, Y);    // P = M Y = m t0 2^116
    const unsigned long long H = (1ull << 52) - hi - (lo != 0ull);  // 2^116 - P, high part
    const long long Dv = (long long)((H << 12) | ((0ull - lo) >> 52));  // 2^64 e
    const unsigned long long aD = Dv >= 0 ? (unsigned long long)Dv : 0ull - (unsigned long long)Dv;
    const long long S = Dv + (long long)__umul64hi(aD, aD);        // 2^64 (e + e^2)
    const unsigned long long aS = S >= 0 ? (unsigned long long)S : 0ull - (unsigned long long)S;
    const unsigned long long C = __umul64hi(Y, aS);
    Y = S >= 0 ? Y + C : Y - C;
    unsigned long long m53 = (Y + (1ull << 10)) >> 11;
    const int ov = (int)(m53 >> 53);
    m53 >>= ov;
    const unsigned long long ex = (unsigned long long)(1022 - (e - 1023) + ov);
    const unsigned long long nb = (sign << 63) | (ex << 52) | (m53 & 0xFFFFFFFFFFFFFull);
    const unsigned long long pb = (sign << 63) | ((unsigned long long)(2046 - e) << 52);
    return __longlong_as_double((long long)(f == 0ull ? pb : nb));
}

__device__ __forceinline__ double rcp_fixed(double x) {
    bool slow;
    const double r = rcp_core(x, &slow);
    return slow ? 1.0 / x : r;
}

// Square root of an FP64 value with three FP64 instructions.  A 24-bit seed y0 of 1/sqrt(m)
// for the mantissa m (times 2 for an odd exponent) comes from the FP32 unit; one
// Newton-Raphson step for the inverse square root, y1 = y0 (3 - m y0^2) / 2, runs in 64-bit
// fixed point on the integer pipe (about 44 correct bits); then h = x y1 and one Newton step
// for the square root, h + (x - h^2) y1 / 2, in FP64.  Within about 1 ulp for normal x > 0;
// zero, subnormal, negative, infinite and NaN inputs use the FP64 square root.
__device__ __forceinline__ double sqrt_fast(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)(b >> 52);  // the sign bit is included: negative x takes the slow path
    if (e == 0 || e >= 0x7ff) return sqrt(x);
    const int k = e - 1023;  // x = m 2^k, m in [1, 2)
    const int odd = k & 1;
    const int h2 = (k - odd) >> 1;  // x = m' 4^h2 with m' = m or 2m in [1, 4)
    const unsigned long long frac = b & 0xFFFFFFFFFFFFFull;
    if (frac == 0ull && !odd)  // a power of 4: exact
        return __longlong_as_double((long long)((unsigned long long)(1023 + h2) << 52));
    const unsigned long long Mq = (frac | (1ull << 52)) << (10 + odd);  // m' 2^62
    const float mf = __int_as_float(((127 + odd) << 23) | (int)(frac >> 29));
    const unsigned yb = __float_as_uint(rsqrtf(mf));  // y0 in (1/2, 1)
    const int ye = (int)(yb >> 23);
    unsigned long long Y = ye >= 127 ? ~0ull
                                     : (unsigned long long)((yb & 0x7FFFFFu) | 0x800000u) << (40 - (126 - ye));
    const unsigned long long Y2 = __umul64hi(Y, Y);              // y0^2 2^64
    const unsigned long long P = __umul64hi(Mq, Y2);             // m' y0^2 2^62
    const unsigned long long Tq = (3ull << 62) - P;              // (3 - m' y0^2) 2^62
    Y = __umul64hi(Y, Tq) << 1;                                  // y1 2^64, y1 in (1/2, 1)
    const unsigned long long f52 = (Y >> 11) & 0xFFFFFFFFFFFFFull;
    const double y = __longlong_as_double((long long)(((unsigned long long)(1022 - h2) << 52) | f52));
    const double yh = __longlong_as_double((long long)(((unsigned long long)(1021 - h2) << 52) | f52));
    const double h = x * y;
    return fma(fma(-h, h, x), yh, h);
}

// A float close to the non-negative double with IEEE bits `b` (top 23 mantissa bits,
// exponent clamped to the float range), built with integer operations only.
__device__ __forceinline__ float approx_f32(unsigned long long b) {
    const int e = (int)(b >> 52) - 1023;
    if (b == 0ull) return 0.0f;
    const int ef = e < -126 ? -126 : (e > 127 ? 127 : e);
    const unsigned mant = (unsigned)((b >> 29) & 0x7fffffu);
    return __int_as_float((int)(((unsigned)(ef + 127) << 23) | mant));
}

__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

// Sign-free top 32 bits of an FP64 value (exponent and 20 mantissa bits): ordering these keys
// orders the magnitudes up to a relative 2^-20, with no FP64 instruction.
__device__ __forceinline__ unsigned mag_key(double v) {
    return (unsigned)__double2hiint(v) & 0x7fffffffu;
}

}  // namespace rbffd
