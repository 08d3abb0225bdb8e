// Device helpers of the tile passes, shared by the precompiled interpreter
// kernel and the kernels generated per pass at run time (NVRTC).
#pragma once

#include "dev_types.h"

namespace sd {

template <typename T> struct VT;
template <> struct VT<float> { using A = float2; };
template <> struct VT<double> { using A = double2; };

__device__ __forceinline__ int popc64(uint64_t v) { return __popcll(v); }

// (cos 2 pi t, sin 2 pi t) of Q0.64 turns t, in the state precision.
__device__ __forceinline__ void turns_sc(uint64_t t, float &s, float &c) {
    int32_t hi = (int32_t)((t + 0x80000000ull) >> 32);   // nearest 2^-32 turn
    float tf = (float)hi * 2.3283064365386963e-10f;
    sincospif(2.0f * tf, &s, &c);
}
__device__ __forceinline__ void turns_sc(uint64_t t, double &s, double &c) {
    double tf = (double)(int64_t)t * 5.421010862427522170e-20;   // 2^-64
    sincospi(2.0 * tf, &s, &c);
}

// a <- a * i^k
template <typename A>
__device__ __forceinline__ A mul_ipow(A a, int k) {
    A r = a;
    switch (k & 3) {
    case 1: r.x = -a.y; r.y = a.x; break;
    case 2: r.x = -a.x; r.y = -a.y; break;
    case 3: r.x = a.y; r.y = -a.x; break;
    default: break;
    }
    return r;
}

// a <- a * exp(-2 pi i t) * sc
template <typename T, typename A>
__device__ __forceinline__ A rotate(A a, uint64_t t, T sc) {
    T s, c;
    turns_sc(t, s, c);
    c *= sc;
    s *= sc;
    A r;
    r.x = a.x * c + a.y * s;
    r.y = a.y * c - a.x * s;
    return r;
}

// v * i^P with P known at compile time (a register permutation with negations).
template <int P, typename A>
__device__ __forceinline__ A ipow_c(A v) {
    A r;
    if (P == 0) { r = v; }
    else if (P == 1) { r.x = -v.y; r.y = v.x; }
    else if (P == 2) { r.x = -v.x; r.y = -v.y; }
    else { r.x = v.y; r.y = -v.x; }
    return r;
}

// Canonical Clifford S^B H S^PA on register slot I (unnormalised H):
// (u, v) -> (u + i^PA v, i^B (u - i^PA v)), the difference formed as
// (u + w) - 2 w so that both outputs are written in place.
template <int I, int PA, int B, typename A>
__device__ __forceinline__ void had_fixed(A *a) {
#pragma unroll
    for (int s = 0; s < 16; s++)
        if (!((s >> I) & 1)) {
            const A w = ipow_c<PA>(a[s | (1 << I)]);
            A u = a[s];
            u.x = u.x + w.x;
            u.y = u.y + w.y;
            A d;
            d.x = fma(decltype(w.x)(-2), w.x, u.x);
            d.y = fma(decltype(w.y)(-2), w.y, u.y);
            a[s] = u;
            a[s | (1 << I)] = ipow_c<B>(d);
        }
}

// Canonical Clifford X^XX S^PA on register slot I.
template <int I, int PA, int XX, typename A>
__device__ __forceinline__ void mono_fixed(A *a) {
#pragma unroll
    for (int s = 0; s < 16; s++)
        if (!((s >> I) & 1)) {
            const A w = ipow_c<PA>(a[s | (1 << I)]);
            if (XX) {
                a[s | (1 << I)] = a[s];
                a[s] = w;
            } else {
                a[s | (1 << I)] = w;
            }
        }
}

// In-place Walsh-Hadamard transform of 16 register values.
__device__ __forceinline__ void wht16(uint64_t *G) {
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int s = 0; s < 16; s++)
            if (!((s >> i) & 1)) {
                uint64_t u = G[s], v = G[s | (1 << i)];
                G[s] = u + v;
                G[s | (1 << i)] = u - v;
            }
}
__device__ __forceinline__ void wht16(double *G) {
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int s = 0; s < 16; s++)
            if (!((s >> i) & 1)) {
                double u = G[s], v = G[s | (1 << i)];
                G[s] = u + v;
                G[s | (1 << i)] = u - v;
            }
}

// e^{-2 pi i t} of Q0.64 turns t (times sc) applied to a: the top 8 bits of t
// index a table of e^{2 pi i k/256}; the remaining angle phi < 2 pi/256 goes
// through the Taylor series of cos and sin (truncation error below 1e-10 in
// single precision and 1e-18 in double precision).
__device__ __forceinline__ float2 rotate_tw(float2 a, uint64_t t, const float2 *__restrict__ tw, float sc) {
    const float2 e = tw[t >> 56];
    const uint32_t r = (uint32_t)((t << 8) >> 32);
    const float phi = (float)r * (float)(6.283185307179586 / 256.0 / 4294967296.0);
    const float p2 = phi * phi;
    const float cp = fmaf(p2, fmaf(p2, 1.0f / 24.0f, -0.5f), 1.0f);
    const float sp = phi * fmaf(p2, -1.0f / 6.0f, 1.0f);
    const float C = (e.x * cp - e.y * sp) * sc;
    const float S = (e.y * cp + e.x * sp) * sc;
    float2 o;
    o.x = a.x * C + a.y * S;
    o.y = a.y * C - a.x * S;
    return o;
}
__device__ __forceinline__ double2 rotate_tw(double2 a, uint64_t t, const double2 *__restrict__ tw, double sc) {
    const double2 e = tw[t >> 56];
    const uint64_t r = (t << 8) >> 12;             // 52 bits below the table index
    const double phi = (double)r * (6.283185307179586 / 256.0 / 4503599627370496.0);
    const double p2 = phi * phi;
    const double cp = fma(p2, fma(p2, fma(p2, -1.0 / 720.0, 1.0 / 24.0), -0.5), 1.0);
    const double sp = phi * fma(p2, fma(p2, fma(p2, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0), 1.0);
    const double C = (e.x * cp - e.y * sp) * sc;
    const double S = (e.y * cp + e.x * sp) * sc;
    double2 o;
    o.x = a.x * C + a.y * S;
    o.y = a.y * C - a.x * S;
    return o;
}



// Group exponential on the thread's 16 amplitudes: T(s) = sum_j q_j
// (-1)^{|x & m_j|} with x = (tile, fixed positions lf, register bits s).
// Terms are sorted by their register projection u (class u); per class the
// sum over the fixed positions gives G[u], and a 4-level Walsh-Hadamard
// transform over the register bits turns G into T.
template <typename A, typename T>
__device__ __forceinline__ void diag_apply(A *a, uint32_t lf, const DevDiag &d,
                                           const StagedTerm *__restrict__ st,
                                           const A *__restrict__ tw, T sc, uint64_t g0) {
    uint64_t G[16];
#pragma unroll
    for (int s = 0; s < 16; s++) {
        uint64_t acc0 = 0, acc1 = 0;
        int j = d.off[s];
        const int e = d.off[s + 1];
        for (; j + 1 < e; j += 2) {
            const StagedTerm t0 = st[j], t1 = st[j + 1];
            acc0 += (__popc(lf & t0.ml) & 1) ? (0 - t0.q) : t0.q;
            acc1 += (__popc(lf & t1.ml) & 1) ? (0 - t1.q) : t1.q;
        }
        if (j < e) {
            const StagedTerm t0 = st[j];
            acc0 += (__popc(lf & t0.ml) & 1) ? (0 - t0.q) : t0.q;
        }
        G[s] = acc0 + acc1;
    }
    G[0] += g0;
    wht16(G);
#pragma unroll
    for (int s = 0; s < 16; s++) a[s] = rotate_tw(a[s], G[s], tw, sc);
}

// S/CZ layer: a(x) *= i^{k(x)}, k = |x&sp| - |x&sm| + 2 sum_CZ x_c x_t.
template <typename A>
__device__ __forceinline__ void phase_apply(A *a, uint64_t xf, const int *gq, const DevPhase &ph,
                                            const uint64_t *__restrict__ pool) {
    int kb = popc64(xf & ph.sp) - popc64(xf & ph.sm);
    int Q = 0;
    uint64_t rest = xf;
    while (rest) {
        int c = __ffsll((long long)rest) - 1;
        rest &= rest - 1;
        Q ^= popc64(xf & __ldg(pool + ph.up_base + c)) & 1;
    }
    kb += 2 * Q;
    int lin[4];
#pragma unroll
    for (int i = 0; i < 4; i++)
        lin[i] = ph.lin_s[i] + 2 * (popc64(xf & __ldg(pool + ph.adj_base + gq[i])) & 1);
#pragma unroll
    for (int s = 0; s < 16; s++) {
        int k = kb;
#pragma unroll
        for (int i = 0; i < 4; i++)
            if ((s >> i) & 1) k += lin[i];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = i + 1; j < 4; j++)
                if (((s >> i) & 1) && ((s >> j) & 1) && ((ph.quad >> (i * 4 + j)) & 1)) k += 2;
        a[s] = mul_ipow(a[s], k);
    }
}



// Signed sum over a warp's strided share of `count` tile-constant terms,
// reduced across the warp (every lane returns the total).
__device__ __forceinline__ uint64_t warp_const_sum(uint64_t xo, const uint64_t *__restrict__ mo,
                                                   const int64_t *__restrict__ q, int begin, int count,
                                                   int lane) {
    uint64_t acc = 0;
    for (int j = lane; j < count; j += 32) {
        const uint64_t v = (uint64_t)__ldg(q + begin + j);
        acc += (__popcll(xo & __ldg(mo + begin + j)) & 1) ? (0 - v) : v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    return acc;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Dynamic shared memory available to a tile pass (227 KB per block minus the
// static tables of the kernel).
__host__ __device__ constexpr size_t tile_smem_limit() { return 227 * 1024 - 28 * 1024; }

// Shared-memory size of a tile pass: exchange + prefetch buffers, staged terms.
template <typename A, int K>
__host__ __device__ constexpr size_t tile_smem_bytes(int max_stage) {
    return 2 * (sizeof(A) << K) + sizeof(StagedTerm) * (size_t)(max_stage > 0 ? max_stage : 1);
}


}  // namespace sd
