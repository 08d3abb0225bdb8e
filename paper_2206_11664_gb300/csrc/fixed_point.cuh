// Fixed-point arithmetic of the complex128 tile passes: conversions between
// doubles and 64-bit integers on a tile's common exponent, Q1.62 rotations.
// Device code in the library and in the kernels compiled at run time; it
// also compiles as host C++ given host versions of the few CUDA intrinsics
// it uses (__mul64hi, __umul64hi, __clzll, __double_as_longlong,
// __longlong_as_double) and of longlong2, which the host tests provide.
#pragma once

#include "dev_types.h"

#if defined(__CUDACC__) || defined(__CUDACC_RTC__)
#define SD_FX __device__ __forceinline__
#else
#define SD_FX inline
#endif

namespace sd {

// ------------------------------------------------------------ complex128 in fixed point
// Complex128 passes compiled at run time compute in 64-bit fixed point, since
// this GPU's FP64 rate is a small fraction of its integer rate.  The
// amplitudes of a tile share one unit 2^U, set by the tile's largest
// component; the one-qubit butterflies are exact integer adds; rotations
// multiply by unit complex numbers in Q1.62 (1.0 = 2^62).

// Biased binary exponent of |d| (0 for zero and subnormal values).
SD_FX uint32_t fx_exp(double d) {
    return (uint32_t)((unsigned long long)__double_as_longlong(d) >> 52) & 0x7ffu;
}

// d in units of 2^(S - 1085 + hr), S = largest biased exponent of the tile:
// the 53-bit significand m (value m 2^(e - 1075)) shifted right by
// S - e - 10 + hr, so that |v| < 2^(63 - hr).  Truncates toward zero;
// subnormal inputs give 0.
SD_FX long long fx_from(double d, uint32_t S, int hr) {
    const long long b = __double_as_longlong(d);
    const uint32_t e = (uint32_t)((unsigned long long)b >> 52) & 0x7ffu;
    const unsigned long long m = ((unsigned long long)b & 0xfffffffffffffull) | 0x10000000000000ull;
    const int sh = (int)S - (int)e - 10 + hr;
    unsigned long long v = sh >= 0 ? (sh < 64 ? (m >> sh) : 0ull) : (m << (-sh));
    if (e == 0) v = 0ull;
    return b < 0 ? -(long long)v : (long long)v;
}

// v * 2^U as a double, rounded to nearest (halfway cases away from zero);
// results below the normal range give zero.
SD_FX double fx_to(long long v, int U) {
    const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ull;
    unsigned long long m = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    if (m == 0ull) return 0.0;
    const int lz = __clzll((long long)m);
    m <<= lz;                                   // leading bit at 63
    int ex = U + 63 - lz + 1023;                // biased exponent of the leading bit
    const unsigned long long r = m + 0x400ull;  // round at bit 10
    unsigned long long frac;
    if (r < m) {                                // carried out of bit 63: 2^(leading + 1)
        ex += 1;
        frac = 0ull;
    } else {
        frac = (r >> 11) & 0xfffffffffffffull;
    }
    if (ex <= 0) return __longlong_as_double((long long)sgn);
    return __longlong_as_double((long long)(sgn | ((unsigned long long)ex << 52) | frac));
}

// 2 pi 2^61 (= pi 2^62) and 2^63 / sqrt(2) (= sqrt(2) 2^62), rounded to integers.
constexpr unsigned long long kTwoPiQ61 = 0xC90FDAA22168C235ull;
constexpr long long kRsqrt2Q63 = 0x5A827999FCEF3242ll;

// a * b / 2^62 for Q1.62 b (the 2 lowest bits dropped).
SD_FX long long fx_mulq(long long a, long long b) { return __mul64hi(a, b) << 2; }

// (Er, Ei) = e^{2 pi i t} in Q1.62 for Q0.64 turns t: t = k1 2^56 + k2 2^48 + r;
// e^{2 pi i t} = T1[k1] T2[k2] e^{i phi}, phi = 2 pi r / 2^64 < 2 pi / 65536, with
// cos phi = 1 - phi^2/2 and sin phi = phi - phi^3/6 (next terms below 2^-57).
// T1 may carry a scale factor.
SD_FX void fx_cis(uint64_t t, const longlong2 *__restrict__ T1, const longlong2 *__restrict__ T2,
                  long long &Er, long long &Ei) {
    const longlong2 e1 = T1[t >> 56], e2 = T2[(t >> 48) & 255u];
    const unsigned long long r = t & 0xffffffffffffull;
    const unsigned long long p = __umul64hi(r << 16, kTwoPiQ61);  // phi 2^77
    const unsigned long long p2 = __umul64hi(p, p);              // phi^2 2^90
    const unsigned long long p3 = __umul64hi(p2, p);             // phi^3 2^103
    const long long c = (1ll << 62) - (long long)(p2 >> 29);     // Q1.62
    const long long sn = (long long)(p >> 15) - (long long)__umul64hi(p3 >> 41, 0x2AAAAAAAAAAAAAABull);
    const long long xr = fx_mulq(e1.x, e2.x) - fx_mulq(e1.y, e2.y);
    const long long xi = fx_mulq(e1.x, e2.y) + fx_mulq(e1.y, e2.x);
    Er = fx_mulq(xr, c) - fx_mulq(xi, sn);
    Ei = fx_mulq(xr, sn) + fx_mulq(xi, c);
}

// (re, im) <- (re, im) * e^{-2 pi i t} for Q0.64 turns t (fx_cis).
SD_FX void fx_rotate(long long &re, long long &im, uint64_t t,
                     const longlong2 *__restrict__ T1, const longlong2 *__restrict__ T2) {
    long long Er, Ei;
    fx_cis(t, T1, T2, Er, Ei);
    const long long nr = fx_mulq(re, Er) + fx_mulq(im, Ei);
    const long long ni = fx_mulq(im, Er) - fx_mulq(re, Ei);
    re = nr;
    im = ni;
}

// (re, im) <- (re, im) * i^k.
SD_FX void fx_mul_ipow(long long &re, long long &im, int k) {
    const long long r = re, i = im;
    switch (k & 3) {
    case 1: re = -i; im = r; break;
    case 2: re = -r; im = -i; break;
    case 3: re = i; im = -r; break;
    default: break;
    }
}

}  // namespace sd
