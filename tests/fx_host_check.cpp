// Host check of the fixed-point arithmetic of the complex128 passes
// (fixed_point.cuh), built by tests/test_fixed_point_host.py with host
// versions of the CUDA intrinsics it uses.  Exit status 0 = every check held.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include <vector_types.h>

static long long __double_as_longlong(double d) { long long b; std::memcpy(&b, &d, 8); return b; }
static double __longlong_as_double(long long b) { double d; std::memcpy(&d, &b, 8); return d; }
static int __clzll(long long v) { return v == 0 ? 64 : __builtin_clzll((unsigned long long)v); }
static long long __mul64hi(long long a, long long b) { return (long long)(((__int128)a * b) >> 64); }
static unsigned long long __umul64hi(unsigned long long a, unsigned long long b) {
    return (unsigned long long)(((unsigned __int128)a * b) >> 64);
}

#include "fixed_point.cuh"

using namespace sd;

int main() {
    int bad = 0;
    std::mt19937_64 g(7);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    // conversions: round trip within one unit of the tile's last place
    for (int k = 0; k < 200000 && bad < 10; k++) {
        const double d = U(g) * std::ldexp(1.0, (int)(g() % 60) - 30);
        const uint32_t S = fx_exp(d) + (uint32_t)(g() % 4);
        const int hr = 10 + (int)(g() % 8);
        const long long v = fx_from(d, S, hr);
        const double back = fx_to(v, (int)S - 1085 + hr);
        const double unit = std::ldexp(1.0, (int)S - 1085 + hr);
        if (std::fabs(back - d) > unit * 1.0000001) {
            std::printf("round trip: d %.17g back %.17g unit %g\n", d, back, unit);
            bad++;
        }
        if (std::llabs(v) >= (1ll << (63 - hr))) {
            std::printf("headroom: |v| %lld >= 2^%d\n", v, 63 - hr);
            bad++;
        }
    }
    // exact integers and signed zero / tiny values
    const long long ints[] = {1, -1, 3, -3, 1ll << 62, -(1ll << 62), 123456789012345ll, (1ll << 53) + 2};
    for (long long v : ints) {
        const double want = (double)v;   // correctly rounded
        if (fx_to(v, 0) != want) { std::printf("fx_to(%lld)\n", v); bad++; }
    }
    if (fx_to(0, 0) != 0.0 || fx_to(1, -2000) != 0.0) { std::printf("zero / underflow\n"); bad++; }
    // rounding to nearest, halfway cases away from zero: 2^53 + 1 and 2^53 + 3 (ties)
    if (fx_to((1ll << 53) + 1, 0) != 9007199254740994.0) { std::printf("tie +1\n"); bad++; }
    if (fx_to((1ll << 53) + 3, 0) != 9007199254740996.0) { std::printf("tie +3\n"); bad++; }
    if (fx_to(-((1ll << 53) + 1), 0) != -9007199254740994.0) { std::printf("tie -1\n"); bad++; }
    // not a tie: 2^54 + 1 rounds down to 2^54, 2^54 + 3 up to 2^54 + 4
    if (fx_to((1ll << 54) + 1, 0) != 18014398509481984.0) { std::printf("below half\n"); bad++; }
    if (fx_to((1ll << 54) + 3, 0) != 18014398509481988.0) { std::printf("above half\n"); bad++; }
    // rotation: e^{-2 pi i t} against long double trigonometry
    longlong2 T1[256], T2[256];
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int k = 0; k < 256; k++) {
        const long double a = 2 * pi * k / 256, b = 2 * pi * k / 65536;
        T1[k] = longlong2{llroundl(ldexpl(cosl(a), 62)), llroundl(ldexpl(sinl(a), 62))};
        T2[k] = longlong2{llroundl(ldexpl(cosl(b), 62)), llroundl(ldexpl(sinl(b), 62))};
    }
    double worst = 0;
    for (int k = 0; k < 200000; k++) {
        const uint64_t t = g();
        const long long re = (long long)(U(g) * std::ldexp(1.0, 60)), im = (long long)(U(g) * std::ldexp(1.0, 60));
        const long double th = 2 * pi * (long double)t / 18446744073709551616.0L;
        const long double er = re * cosl(th) + im * sinl(th), ei = im * cosl(th) - re * sinl(th);
        long long r2 = re, i2 = im;
        fx_rotate(r2, i2, t, T1, T2);
        const double e = (double)((fabsl(r2 - er) + fabsl(i2 - ei)) / ldexpl(1.0L, 60));
        if (e > worst) worst = e;
    }
    if (worst > 1e-15) { std::printf("rotation error %g\n", worst); bad++; }
    // cos and sin of 2 pi t in Q1.62, then as doubles (the adjoint kernel's rotation factor)
    double worst_cs = 0;
    for (int k = 0; k < 200000; k++) {
        const uint64_t t = k < 4 ? (uint64_t)k << 62 : g();
        const long double th = 2 * pi * (long double)t / 18446744073709551616.0L;
        long long er, ei;
        fx_cis(t, T1, T2, er, ei);
        const double c = fx_to(er, -62), s = fx_to(ei, -62);
        const double e = (double)(fabsl(c - cosl(th)) + fabsl(s - sinl(th)));
        if (e > worst_cs) worst_cs = e;
    }
    if (worst_cs > 2e-16) { std::printf("cis error %g\n", worst_cs); bad++; }
    // quarter turns
    long long a = 5, b = 7;
    fx_mul_ipow(a, b, 1);
    if (a != -7 || b != 5) { std::printf("i^1\n"); bad++; }
    fx_mul_ipow(a, b, 3);
    if (a != 5 || b != 7) { std::printf("i^3\n"); bad++; }
    std::printf("fixed point: %s (rotation error %.3g, cis error %.3g)\n", bad ? "FAILED" : "ok", worst, worst_cs);
    return bad ? 1 : 0;
}
