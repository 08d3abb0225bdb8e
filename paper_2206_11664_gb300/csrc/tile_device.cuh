// Device helpers of the tile passes, shared by the precompiled interpreter
// kernel and the kernels generated per pass at run time (NVRTC).
#pragma once

#include "dev_types.h"
#include "fixed_point.cuh"

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
__device__ __forceinline__ void wht16(uint32_t *G) {
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int s = 0; s < 16; s++)
            if (!((s >> i) & 1)) {
                uint32_t u = G[s], v = G[s | (1 << i)];
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

// e^{-2 pi i t} (times sc) applied to a, for turns t: the top 8 bits of t
// index a table of e^{2 pi i k/256}; the remaining angle phi < 2 pi/256 goes
// through the Taylor series of cos and sin (truncation error below 1e-10 in
// single precision and 1e-18 in double precision).  Single precision takes
// Q0.32 turns (the low 24 bits, exact in a float, are the remaining angle);
// double precision takes Q0.64 turns.
__device__ __forceinline__ float2 rotate_tw32(float2 a, uint32_t t, const float2 *__restrict__ tw, float sc) {
    const float2 e = tw[t >> 24];
    const float phi = (float)(t & 0xffffffu) * (float)(6.283185307179586 / 4294967296.0);
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
// rotate_tw32 for an amplitude held in one of the representations of the
// complex64 passes' butterflies: the stored pair p has re = SRI p[SWI] and
// im = SII p[1 - SWI] (signs +-1), and the result is stored the same way
// with SWO, SRO, SIO.  The signs and the order fold into the arithmetic.
template <int SWI, int SRI, int SII, int SWO, int SRO, int SIO>
__device__ __forceinline__ float2 rotate_tw32_rep(float2 p, uint32_t t, const float2 *__restrict__ tw, float sc) {
    const float2 v = make_float2((float)SRI * (SWI ? p.y : p.x), (float)SII * (SWI ? p.x : p.y));
    const float2 r = rotate_tw32(v, t, tw, sc);
    float2 q;
    if (SWO) {
        q.y = (float)SRO * r.x;
        q.x = (float)SIO * r.y;
    } else {
        q.x = (float)SRO * r.x;
        q.y = (float)SIO * r.y;
    }
    return q;
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


// e^{-2 pi i t} (times sc) applied to the two amplitudes of a packed pair
// (R = their real parts, I = their imaginary parts), for Q0.32 turns t0 and
// t1: the top 9 bits index tables of cos and sin of 2 pi k/512 (TC, TS); the
// low 23 bits, exact as the mantissa of a float in [1, 2), give the remaining
// angle phi < 2 pi/512, whose cosine and sine come from their Taylor series
// (truncation below 1e-9 relative).  Every step but the table index and the
// mantissa works on both amplitudes with one packed f32x2 instruction.
__device__ __forceinline__ void rotate_pair32(float2 &R, float2 &I, uint32_t t0, uint32_t t1,
                                              const float *__restrict__ TC, const float *__restrict__ TS, float sc) {
    const uint32_t i0 = t0 >> 23, i1 = t1 >> 23;
    const float2 ec = make_float2(TC[i0], TC[i1]);
    const float2 es = make_float2(TS[i0], TS[i1]);
    const float k = (float)(6.283185307179586 / 512.0);
    const float2 f = make_float2(__uint_as_float(0x3f800000u | (t0 & 0x7fffffu)),
                                 __uint_as_float(0x3f800000u | (t1 & 0x7fffffu)));
    const float2 phi = __ffma2_rn(f, make_float2(k, k), make_float2(-k, -k));   // (f - 1) 2 pi/512
    const float2 p2 = __fmul2_rn(phi, phi);
    const float2 cp = __ffma2_rn(p2, __ffma2_rn(p2, make_float2(1.0f / 24.0f, 1.0f / 24.0f), make_float2(-0.5f, -0.5f)),
                                 make_float2(1.0f, 1.0f));
    const float2 sp = __fmul2_rn(phi, __ffma2_rn(p2, make_float2(-1.0f / 6.0f, -1.0f / 6.0f), make_float2(1.0f, 1.0f)));
    const float2 m1 = make_float2(-1.0f, -1.0f);
    // C + iS = e^{2 pi i k/512} (cp + i sp) = e^{2 pi i t}
    float2 C = __ffma2_rn(es, __fmul2_rn(sp, m1), __fmul2_rn(ec, cp));
    float2 S = __ffma2_rn(ec, sp, __fmul2_rn(es, cp));
    if (sc != 1.0f) {
        C = __fmul2_rn(C, make_float2(sc, sc));
        S = __fmul2_rn(S, make_float2(sc, sc));
    }
    const float2 nS = __fmul2_rn(S, m1);
    const float2 r = __ffma2_rn(I, S, __fmul2_rn(R, C));    // re C + im S
    I = __ffma2_rn(R, nS, __fmul2_rn(I, C));                // im C - re S
    R = r;
}

// Rounding bias of the class totals: complex64 passes finish the angle in
// Q0.32 (the high word of G + 2^31 is G rounded to 2^-32 turns, the float
// rotation's own resolution); complex128 passes keep Q0.64.
template <typename A> struct TotalBias;
template <> struct TotalBias<float2> { static constexpr uint64_t value = 1ull << 31; };
template <> struct TotalBias<double2> { static constexpr uint64_t value = 0ull; };

// Angles T from the class sums G by the 4-level Walsh-Hadamard transform over
// the register bits, then the rotation of the thread's 16 amplitudes.
__device__ __forceinline__ void diag_rotate(float2 *a, const uint64_t *G, const float2 *__restrict__ tw,
                                            float sc) {
    uint32_t g[16];
#pragma unroll
    for (int s = 0; s < 16; s++) g[s] = (uint32_t)(G[s] >> 32);
    wht16(g);
#pragma unroll
    for (int s = 0; s < 16; s++) a[s] = rotate_tw32(a[s], g[s], tw, sc);
}
__device__ __forceinline__ void diag_rotate(double2 *a, uint64_t *G, const double2 *__restrict__ tw,
                                            double sc) {
    wht16(G);
#pragma unroll
    for (int s = 0; s < 16; s++) a[s] = rotate_tw(a[s], G[s], tw, sc);
}

// Group exponential on the thread's 16 amplitudes (layout of DevDiag): per
// class u, G[u] = TQ[tot + u] - 2 (sum of the slots with odd |lf & ml|).
template <typename A, typename T>
__device__ __forceinline__ void diag_apply(A *a, uint32_t lf, const DevDiag &d,
                                           const StagedTerm *__restrict__ st,
                                           const uint64_t *__restrict__ TQ,
                                           const A *__restrict__ tw, T sc) {
    uint64_t G[16];
#pragma unroll
    for (int s = 0; s < 16; s++) {
        uint64_t o0 = 0, o1 = 0;
        int j = d.off[s];
        const int e = d.off[s + 1];
        for (; j + 1 < e; j += 2) {
            const StagedTerm t0 = st[j], t1 = st[j + 1];
            if (__popc(lf & t0.ml) & 1) o0 += t0.q;
            if (__popc(lf & t1.ml) & 1) o1 += t1.q;
        }
        if (j < e) {
            const StagedTerm t0 = st[j];
            if (__popc(lf & t0.ml) & 1) o0 += t0.q;
        }
        G[s] = TQ[d.tot + s] - 2ull * (o0 + o1);
    }
    diag_rotate(a, G, tw, sc);
}

// Term slots of a round staged for the tile with outer bits xo: ST[j] holds
// the slot's signed angle sum sum_t q_t (-1)^{|xo & mo_t|} and its mask ml.
// Term t is read at mo[t - toff], q[t - toff] (the pass's cached copy in
// shared memory, or the global arrays with toff = 0).
__device__ __forceinline__ void stage_slots(uint64_t xo, const DevSlot *__restrict__ slots, int slot_begin,
                                            int slot_count, const uint64_t *mo, const int64_t *q, int toff,
                                            StagedTerm *ST, int tid, int nt) {
    for (int j = tid; j < slot_count; j += nt) {
        const DevSlot sl = slots[slot_begin + j];
        uint64_t acc = 0;
        for (int t = sl.tb - toff; t < sl.tb - toff + sl.tn; t++) {
            const uint64_t v = (uint64_t)q[t];
            acc += (__popcll(xo & mo[t]) & 1) ? (0 - v) : v;
        }
        StagedTerm st;
        st.q = acc;
        st.ml = sl.ml;
        st.pad = 0;
        ST[j] = st;
    }
}

// Copy of the pass's terms into shared memory (TCM: outer masks, TCQ: angles).
__device__ __forceinline__ void cache_terms(const KParams &kp, int term_begin, int term_count, uint64_t *TCM,
                                            int64_t *TCQ, int tid, int nt) {
    for (int i = tid; i < term_count; i += nt) {
        TCM[i] = __ldg(kp.term_mo + term_begin + i);
        TCQ[i] = __ldg(kp.term_q + term_begin + i);
    }
}

// Class totals of the round's group exponentials (after stage_slots and the
// tile-constant sums CST): TQ[16 k + u] = bias + sum of class u's slots of
// the k-th exponential, plus its tile constant in class 0.
__device__ __forceinline__ void stage_totals(const KParams &kp, int diag_begin, int n_diag,
                                             const StagedTerm *ST, const uint64_t *CST, uint64_t bias,
                                             uint64_t *TQ, int tid, int nt) {
    for (int i = tid; i < 16 * n_diag; i += nt) {
        const DevDiag &d = kp.diags[diag_begin + (i >> 4)];
        const int u = i & 15;
        uint64_t t = bias;
        if (d.zs[u] >= 0) t += ST[d.zs[u]].q;
        for (int j = d.off[u]; j < d.off[u + 1]; j++) t += ST[j].q;
        if (u == 0 && d.cst >= 0) t += CST[d.cst];
        TQ[i] = t;
    }
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

// S/CZ layer on fixed-point amplitudes (as phase_apply).
__device__ __forceinline__ void fx_phase_apply(long long *ar, long long *ai, uint64_t xf, const int *gq,
                                               const DevPhase &ph, const uint64_t *__restrict__ pool) {
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
        fx_mul_ipow(ar[s], ai[s], k);
    }
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// all but the most recent group of this thread's copies
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

}  // namespace sd
