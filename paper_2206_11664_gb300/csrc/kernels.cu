// State-vector kernels for sm_103a.
//
//  tile_pass_kernel   one HBM pass of the grouped Trotter step: a tile of 2^K
//                     amplitudes per CTA, 16 per thread in registers; one-
//                     qubit Clifford gates (H, S, S^dag) on register bits,
//                     the S/CZ quarter-turn layer and the group exponential
//                     (Sec. 3.4 items 1-3) as diagonal ops, CNOT runs as
//                     tile permutations on the shared-memory exchange.
//  onchip_kernel      whole small state in one CTA's shared memory, every
//                     step in one launch.
//  pauli_rot_kernel   baseline: one exp(-i a P) per pass (Eq. trotter_decomp).
//  expect / grad      FP64 reductions for <O> and the adjoint gradient.
//
// Phases are carried as Q0.64 fixed-point turns: exp(-2 pi i T) with T the
// exact (wrap-around) sum of the per-term quantised angles.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace sd {
namespace {

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

template <int I, typename A>
__device__ __forceinline__ void h_fixed(A *a) {
#pragma unroll
    for (int s = 0; s < 16; s++)
        if (!((s >> I) & 1)) {
            A u = a[s], v = a[s | (1 << I)];
            a[s].x = u.x + v.x;
            a[s].y = u.y + v.y;
            a[s | (1 << I)].x = u.x - v.x;
            a[s | (1 << I)].y = u.y - v.y;
        }
}

template <int I, typename A>
__device__ __forceinline__ void s_fixed(A *a, int k) {
#pragma unroll
    for (int s = 0; s < 16; s++)
        if ((s >> I) & 1) a[s] = mul_ipow(a[s], k);
}

template <typename A>
__device__ __forceinline__ void h_slot(A *a, int slot) {
    switch (slot) {
    case 0: h_fixed<0>(a); break;
    case 1: h_fixed<1>(a); break;
    case 2: h_fixed<2>(a); break;
    default: h_fixed<3>(a); break;
    }
}

template <typename A>
__device__ __forceinline__ void s_slot(A *a, int slot, int k) {
    switch (slot) {
    case 0: s_fixed<0>(a, k); break;
    case 1: s_fixed<1>(a, k); break;
    case 2: s_fixed<2>(a, k); break;
    default: s_fixed<3>(a, k); break;
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

// Group exponential on the thread's 16 amplitudes: T(s) = sum_j q_j
// (-1)^{|x & m_j|} with x = xf | (register bits of s).  Terms arrive sorted
// by their register projection u (class u); per class the sum over the
// fixed bits gives G[u], and a 4-level WHT over the register bits gives T.
template <typename T, typename A>
__device__ __forceinline__ void diag_apply(A *a, uint64_t xf, const DevDiag &d,
                                           const uint64_t *__restrict__ tm,
                                           const int64_t *__restrict__ tq, T sc) {
    uint64_t G[16];
#pragma unroll
    for (int s = 0; s < 16; s++) {
        uint64_t acc = 0;
        const int64_t b = d.base;
        for (int j = d.off[s]; j < d.off[s + 1]; j++) {
            uint64_t m = __ldg(tm + b + j);
            uint64_t q = (uint64_t)__ldg(tq + b + j);
            acc += (popc64(xf & m) & 1) ? (0 - q) : q;
        }
        G[s] = acc;
    }
    wht16(G);
#pragma unroll
    for (int s = 0; s < 16; s++) a[s] = rotate<T>(a[s], G[s], sc);
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

struct KParams {
    const DevPass *passes;
    const DevRound *rounds;
    const DevOp *ops;
    const DevPerm *perms;
    const DevDiag *diags;
    const DevPhase *phases;
    const uint64_t *term_masks;
    const int64_t *term_q;
    const uint64_t *mask_pool;
    int c;
};

template <typename T, int K>
__global__ void __launch_bounds__(1 << (K - 4))
tile_pass_kernel(typename VT<T>::A *__restrict__ psi, int n, int pass_idx, KParams kp) {
    using A = typename VT<T>::A;
    extern __shared__ __align__(16) unsigned char smraw[];
    A *sm = reinterpret_cast<A *>(smraw);
    __shared__ DevPass P;
    __shared__ DevRound RR[12];
    __shared__ uint32_t swzc[16];
    const int tid = threadIdx.x;
    if (tid == 0) P = kp.passes[pass_idx];
    __syncthreads();
    if (tid < P.n_rounds) RR[tid] = kp.rounds[P.round_begin + tid];
    if (tid < K) {
        uint32_t col = 1u << tid;
        if (tid >= kp.c) {
            uint32_t span = (1u << kp.c) - 1u;
            col |= 1u + (uint32_t)((tid - kp.c) % (int)span);
        }
        swzc[tid] = col;
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    const int64_t ntiles = (int64_t)1 << (n - K);
    const int nr = P.n_rounds;
    const T pass_scale = P.scale_in_diag ? (T)1 : (T)P.scale;
    const T diag_scale = (T)P.scale;

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        uint64_t xo = 0;
        for (int k = 0; k < P.n_outer; k++)
            xo |= (uint64_t)((tile >> k) & 1) << P.outer_bits[k];
        A a[16];
        for (int r = 0; r < nr; r++) {
            const DevRound &R = RR[r];
            uint32_t lf = 0;
#pragma unroll
            for (int i = 0; i < 5; i++) lf |= (uint32_t)((lane >> i) & 1) << R.lane_pos[i];
#pragma unroll
            for (int i = 0; i < K - 9; i++) lf |= (uint32_t)((warp >> i) & 1) << R.warp_pos[i];
            uint64_t xf = xo;
            uint32_t sw = 0;
#pragma unroll
            for (int p = 0; p < K; p++)
                if ((lf >> p) & 1) {
                    xf |= (uint64_t)1 << P.tile_bits[p];
                    sw ^= swzc[p];
                }
            int gq[4];
#pragma unroll
            for (int i = 0; i < 4; i++) gq[i] = P.tile_bits[R.reg_pos[i]];
            if (r == 0) {
#pragma unroll
                for (int s = 0; s < 16; s++) {
                    uint64_t x = xf;
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        if ((s >> i) & 1) x |= (uint64_t)1 << gq[i];
                    a[s] = psi[x];
                }
            } else {
                uint32_t cs[4];
#pragma unroll
                for (int i = 0; i < 4; i++) cs[i] = swzc[R.reg_pos[i]];
#pragma unroll
                for (int s = 0; s < 16; s++) {
                    uint32_t ad = sw;
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        if ((s >> i) & 1) ad ^= cs[i];
                    a[s] = sm[ad];
                }
            }
            for (int o = R.op_begin; o < R.op_end; o++) {
                const DevOp op = kp.ops[o];
                switch (op.kind) {
                case D_H: h_slot(a, op.slot); break;
                case D_S: s_slot(a, op.slot, 1); break;
                case D_SDG: s_slot(a, op.slot, 3); break;
                case D_PHASE: phase_apply(a, xf, gq, kp.phases[op.arg], kp.mask_pool); break;
                default:
                    diag_apply<T>(a, xf, kp.diags[op.arg], kp.term_masks, kp.term_q,
                                  op.pad ? diag_scale : (T)1);
                    break;
                }
            }
            if (R.flags & 2) {
#pragma unroll
                for (int s = 0; s < 16; s++) {
                    uint64_t x = xf;
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        if ((s >> i) & 1) x |= (uint64_t)1 << gq[i];
                    A v = a[s];
                    v.x *= pass_scale;
                    v.y *= pass_scale;
                    psi[x] = v;
                }
            } else {
                __syncthreads();
                uint32_t base, cs[4];
                if (R.perm >= 0) {
                    const DevPerm &pm = kp.perms[R.perm];
                    uint32_t l = 0;
#pragma unroll
                    for (int p = 0; p < K; p++)
                        if ((lf >> p) & 1) l ^= pm.col[p];
                    for (int k = 0; k < P.n_outer; k++)
                        if ((tile >> k) & 1) l ^= pm.ocol[k];
                    base = 0;
#pragma unroll
                    for (int p = 0; p < K; p++)
                        if ((l >> p) & 1) base ^= swzc[p];
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        uint32_t v = pm.col[R.reg_pos[i]], w = 0;
#pragma unroll
                        for (int p = 0; p < K; p++)
                            if ((v >> p) & 1) w ^= swzc[p];
                        cs[i] = w;
                    }
                } else {
                    base = sw;
#pragma unroll
                    for (int i = 0; i < 4; i++) cs[i] = swzc[R.reg_pos[i]];
                }
#pragma unroll
                for (int s = 0; s < 16; s++) {
                    uint32_t ad = base;
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        if ((s >> i) & 1) ad ^= cs[i];
                    sm[ad] = a[s];
                }
                __syncthreads();
            }
        }
    }
}

struct OccCache {
    int blocks[2][14];
    bool init[2][14];
};
OccCache g_occ{};

template <typename T, int K>
cudaError_t run_tile(void *psi, int n, const DevSchedule &S, int pass, int num_sms, cudaStream_t st) {
    using A = typename VT<T>::A;
    const int threads = 1 << (K - 4);
    const size_t smem = sizeof(A) << K;
    const int d = sizeof(T) == 8;
    if (!g_occ.init[d][K]) {
        cudaError_t e = cudaFuncSetAttribute(tile_pass_kernel<T, K>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tile_pass_kernel<T, K>, threads, smem);
        if (e != cudaSuccess) return e;
        g_occ.blocks[d][K] = b > 0 ? b : 1;
        g_occ.init[d][K] = true;
    }
    KParams kp{S.passes, S.rounds, S.ops, S.perms, S.diags, S.phases,
               S.term_masks, S.term_q, S.mask_pool, S.c};
    int64_t ntiles = (int64_t)1 << (n - K);
    int64_t grid = (int64_t)num_sms * g_occ.blocks[d][K];
    if (grid > ntiles) grid = ntiles;
    tile_pass_kernel<T, K><<<(unsigned)grid, threads, smem, st>>>(reinterpret_cast<A *>(psi), n, pass, kp);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_tile_t(void *psi, int n, const DevSchedule &S, int pass, int num_sms, cudaStream_t st) {
    switch (S.K) {
    case 9: return run_tile<T, 9>(psi, n, S, pass, num_sms, st);
    case 10: return run_tile<T, 10>(psi, n, S, pass, num_sms, st);
    case 11: return run_tile<T, 11>(psi, n, S, pass, num_sms, st);
    case 12: return run_tile<T, 12>(psi, n, S, pass, num_sms, st);
    case 13: return run_tile<T, 13>(psi, n, S, pass, num_sms, st);
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------ on-chip path

struct KFlat {
    const DevFlatOp *ops;
    int64_t n_ops;
    const DevDiagFlat *diags;
    const uint64_t *dmasks;
    const int64_t *dq;
    const uint64_t *sp, *sm, *up;
};

template <typename T>
__global__ void __launch_bounds__(1024)
onchip_kernel(typename VT<T>::A *__restrict__ psi, int n, KFlat kf, int64_t reps,
              const uint64_t *__restrict__ oz, const double *__restrict__ oc, int nobs,
              double *__restrict__ trace) {
    using A = typename VT<T>::A;
    extern __shared__ __align__(16) unsigned char smraw[];
    A *st = reinterpret_cast<A *>(smraw);
    __shared__ double red[32];
    const int64_t N = (int64_t)1 << n;
    const int tid = threadIdx.x, nt = blockDim.x;
    const T r2 = (T)0.70710678118654752440;
    for (int64_t i = tid; i < N; i += nt) st[i] = psi[i];
    __syncthreads();
    for (int64_t rep = 0; rep < reps; rep++) {
        for (int64_t o = 0; o < kf.n_ops; o++) {
            const DevFlatOp op = kf.ops[o];
            if (op.kind == OK_H || op.kind == OK_S || op.kind == OK_SDG) {
                const int64_t bq = (int64_t)1 << op.q;
                for (int64_t i = tid; i < N / 2; i += nt) {
                    int64_t lo = i & (bq - 1);
                    int64_t y = ((i - lo) << 1) | lo;
                    if (op.kind == OK_H) {
                        A u = st[y], v = st[y | bq];
                        st[y].x = (u.x + v.x) * r2;
                        st[y].y = (u.y + v.y) * r2;
                        st[y | bq].x = (u.x - v.x) * r2;
                        st[y | bq].y = (u.y - v.y) * r2;
                    } else {
                        st[y | bq] = mul_ipow(st[y | bq], op.kind == OK_S ? 1 : 3);
                    }
                }
            } else if (op.kind == OK_CNOT) {
                const int c = op.q, t = op.q2;
                const int lo = c < t ? c : t, hi = c < t ? t : c;
                for (int64_t i = tid; i < N / 4; i += nt) {
                    int64_t y = i;
                    y = ((y >> lo) << (lo + 1)) | (y & (((int64_t)1 << lo) - 1));
                    y = ((y >> hi) << (hi + 1)) | (y & (((int64_t)1 << hi) - 1));
                    y |= (int64_t)1 << c;
                    int64_t w = y | ((int64_t)1 << t);
                    A u = st[y];
                    st[y] = st[w];
                    st[w] = u;
                }
            } else if (op.kind == OK_PHASE) {
                const uint64_t sp = kf.sp[op.idx], smk = kf.sm[op.idx];
                const uint64_t *up = kf.up + (int64_t)op.idx * n;
                for (int64_t x = tid; x < N; x += nt) {
                    int k = popc64(x & sp) - popc64(x & smk);
                    int Q = 0;
                    for (int c = 0; c < n; c++)
                        if ((x >> c) & 1) Q ^= popc64(x & up[c]) & 1;
                    st[x] = mul_ipow(st[x], k + 2 * Q);
                }
            } else {  // OK_DIAG
                const DevDiagFlat d = kf.diags[op.idx];
                for (int64_t x = tid; x < N; x += nt) {
                    uint64_t Tt = 0;
                    for (int64_t j = 0; j < d.count; j++) {
                        uint64_t m = kf.dmasks[d.begin + j];
                        uint64_t q = (uint64_t)kf.dq[d.begin + j];
                        Tt += (popc64((uint64_t)x & m) & 1) ? (0 - q) : q;
                    }
                    st[x] = rotate<T>(st[x], Tt, (T)1);
                }
            }
            __syncthreads();
        }
        if (nobs > 0) {
            double acc = 0.0;
            for (int64_t x = tid; x < N; x += nt) {
                double p = (double)st[x].x * st[x].x + (double)st[x].y * st[x].y;
                double f = 0.0;
                for (int k = 0; k < nobs; k++) f += (popc64((uint64_t)x & oz[k]) & 1) ? -oc[k] : oc[k];
                acc += p * f;
            }
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if ((tid & 31) == 0) red[tid >> 5] = acc;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                for (int w = 0; w < (nt + 31) / 32; w++) s += red[w];
                trace[rep] = s;
            }
            __syncthreads();
        }
    }
    for (int64_t i = tid; i < N; i += nt) psi[i] = st[i];
}

// ------------------------------------------------------------ per-Pauli baseline

template <typename T>
__global__ void pauli_rot_kernel(typename VT<T>::A *__restrict__ psi, int n, uint64_t x, uint64_t z,
                                 T c, T s) {
    using A = typename VT<T>::A;
    const int64_t N = (int64_t)1 << n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x == 0) {
        for (; i < N; i += stride) {
            A a = psi[i];
            T ss = (popc64((uint64_t)i & z) & 1) ? -s : s;
            A r;
            r.x = c * a.x + ss * a.y;
            r.y = c * a.y - ss * a.x;
            psi[i] = r;
        }
        return;
    }
    const int p = __ffsll((long long)x) - 1;
    const int64_t lowm = ((int64_t)1 << p) - 1;
    const int kxz = popc64(x & z);
    for (; i < N / 2; i += stride) {
        int64_t y = ((i & ~lowm) << 1) | (i & lowm);
        int64_t w = y ^ (int64_t)x;
        A a = psi[y], b = psi[w];
        A py = mul_ipow(b, kxz + 2 * (popc64((uint64_t)w & z) & 1));
        A pw = mul_ipow(a, kxz + 2 * (popc64((uint64_t)y & z) & 1));
        A ry, rw;
        ry.x = c * a.x + s * py.y;
        ry.y = c * a.y - s * py.x;
        rw.x = c * b.x + s * pw.y;
        rw.y = c * b.y - s * pw.x;
        psi[y] = ry;
        psi[w] = rw;
    }
}

// ------------------------------------------------------------ reductions

__device__ __forceinline__ void block_sum_store(double acc, double *out) {
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; w++) s += red[w];
        *out = s;
    }
}

template <typename T>
__global__ void expect_diag_kernel(const typename VT<T>::A *__restrict__ psi, int n,
                                   const uint64_t *__restrict__ oz, const double *__restrict__ oc,
                                   int terms, double *__restrict__ partial) {
    const int64_t N = (int64_t)1 << n;
    double acc = 0.0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N;
         x += (int64_t)gridDim.x * blockDim.x) {
        double p = (double)psi[x].x * psi[x].x + (double)psi[x].y * psi[x].y;
        double f = 0.0;
        for (int k = 0; k < terms; k++) f += (popc64((uint64_t)x & oz[k]) & 1) ? -oc[k] : oc[k];
        acc += p * f;
    }
    block_sum_store(acc, partial + blockIdx.x);
}

template <typename T>
__global__ void expect_pauli_kernel(const typename VT<T>::A *__restrict__ psi, int n, uint64_t x,
                                    uint64_t z, double coef, double *__restrict__ partial) {
    using A = typename VT<T>::A;
    const int64_t N = (int64_t)1 << n;
    const int kxz = popc64(x & z);
    double acc = 0.0;
    for (int64_t y = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; y < N;
         y += (int64_t)gridDim.x * blockDim.x) {
        int64_t w = y ^ (int64_t)x;
        A b = mul_ipow(psi[w], kxz + 2 * (popc64((uint64_t)w & z) & 1));
        A a = psi[y];
        acc += (double)a.x * b.x + (double)a.y * b.y;
    }
    block_sum_store(acc * coef, partial + blockIdx.x);
}

__global__ void reduce_kernel(const double *__restrict__ partial, int64_t count, double *out,
                              int accumulate) {
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) acc += partial[i];
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; w++) s += red[w];
        out[0] = accumulate ? out[0] + s : s;
    }
}

template <typename T>
__global__ void apply_observable_kernel(const typename VT<T>::A *__restrict__ phi,
                                        typename VT<T>::A *__restrict__ lam, int n,
                                        const uint64_t *__restrict__ ox, const uint64_t *__restrict__ oz,
                                        const double *__restrict__ oc, int terms) {
    using A = typename VT<T>::A;
    const int64_t N = (int64_t)1 << n;
    for (int64_t y = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; y < N;
         y += (int64_t)gridDim.x * blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int k = 0; k < terms; k++) {
            int64_t w = y ^ (int64_t)ox[k];
            A b = mul_ipow(phi[w], popc64(ox[k] & oz[k]) + 2 * (popc64((uint64_t)w & oz[k]) & 1));
            re += oc[k] * (double)b.x;
            im += oc[k] * (double)b.y;
        }
        A r;
        r.x = (T)re;
        r.y = (T)im;
        lam[y] = r;
    }
}

// Gradient contribution at a group's diagonal point; 16 consecutive
// amplitudes per thread (register bits = index bits 0..3).
template <typename T>
__global__ void __launch_bounds__(256)
grad_diag_kernel(typename VT<T>::A *__restrict__ chi, typename VT<T>::A *__restrict__ mu, int n,
                 DevGrad g, const uint64_t *__restrict__ masks_f, const int64_t *__restrict__ qinv,
                 double *__restrict__ partial) {
    using A = typename VT<T>::A;
    extern __shared__ double acc[];
    for (int j = threadIdx.x; j < g.m; j += blockDim.x) acc[j] = 0.0;
    __syncthreads();
    const int64_t nchunks = ((int64_t)1 << n) >> 4;
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (int64_t wb = wid * 32; wb < nchunks; wb += warps_total * 32) {
        const int64_t chunk = wb + lane;
        const bool live = chunk < nchunks;
        const uint64_t xf = (uint64_t)chunk << 4;
        A cv[16], mv[16];
        double w[16];
#pragma unroll
        for (int s = 0; s < 16; s++) {
            if (live) {
                cv[s] = chi[xf + s];
                mv[s] = mu[xf + s];
            } else {
                cv[s].x = cv[s].y = mv[s].x = mv[s].y = (T)0;
            }
            w[s] = (double)mv[s].x * cv[s].y - (double)mv[s].y * cv[s].x;
        }
        wht16(w);
        const int64_t b = g.base;
#pragma unroll
        for (int s = 0; s < 16; s++) {
            for (int j = g.off[s]; j < g.off[s + 1]; j++) {
                double v = (popc64(xf & __ldg(masks_f + b + j)) & 1) ? -w[s] : w[s];
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if (lane == 0) atomicAdd(&acc[j], v);
            }
        }
        uint64_t G[16];
#pragma unroll
        for (int s = 0; s < 16; s++) {
            uint64_t a = 0;
            for (int j = g.off[s]; j < g.off[s + 1]; j++) {
                uint64_t q = (uint64_t)__ldg(qinv + b + j);
                a += (popc64(xf & __ldg(masks_f + b + j)) & 1) ? (0 - q) : q;
            }
            G[s] = a;
        }
        wht16(G);
        if (live) {
#pragma unroll
            for (int s = 0; s < 16; s++) {
                chi[xf + s] = rotate<T>(cv[s], G[s], (T)1);
                mu[xf + s] = rotate<T>(mv[s], G[s], (T)1);
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < g.m; j += blockDim.x) partial[(int64_t)blockIdx.x * g.m + j] = acc[j];
}


}  // namespace

cudaError_t launch_tile_pass(bool dbl, void *psi, int n, const DevSchedule &S, int pass, int num_sms,
                             cudaStream_t st) {
    return dbl ? run_tile_t<double>(psi, n, S, pass, num_sms, st)
               : run_tile_t<float>(psi, n, S, pass, num_sms, st);
}

int onchip_max_qubits(bool dbl) { return dbl ? 12 : 13; }

cudaError_t launch_onchip(bool dbl, void *psi, int n, const DevCircuit &C, int64_t reps,
                          const uint64_t *d_oz, const double *d_oc, int obs_terms, double *d_trace,
                          cudaStream_t st) {
    KFlat kf{C.ops, C.n_ops, C.diags, C.dmasks, C.dq, C.phase_sp, C.phase_sm, C.phase_up};
    size_t smem = (size_t)(dbl ? 16 : 8) << n;
    if (dbl) {
        cudaError_t e = cudaFuncSetAttribute(onchip_kernel<double>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        onchip_kernel<double><<<1, 1024, smem, st>>>(reinterpret_cast<double2 *>(psi), n, kf, reps,
                                                      d_oz, d_oc, obs_terms, d_trace);
    } else {
        cudaError_t e = cudaFuncSetAttribute(onchip_kernel<float>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        onchip_kernel<float><<<1, 1024, smem, st>>>(reinterpret_cast<float2 *>(psi), n, kf, reps,
                                                     d_oz, d_oc, obs_terms, d_trace);
    }
    return cudaGetLastError();
}

static unsigned grid_for(int64_t work, int num_sms) {
    int64_t g = (work + 255) / 256;
    int64_t cap = (int64_t)num_sms * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

cudaError_t launch_pauli_rotation(bool dbl, void *psi, int n, uint64_t x, uint64_t z, double c,
                                  double s, int num_sms, cudaStream_t st) {
    int64_t work = x ? ((int64_t)1 << (n - 1)) : ((int64_t)1 << n);
    unsigned g = grid_for(work, num_sms);
    if (dbl)
        pauli_rot_kernel<double><<<g, 256, 0, st>>>(reinterpret_cast<double2 *>(psi), n, x, z, c, s);
    else
        pauli_rot_kernel<float><<<g, 256, 0, st>>>(reinterpret_cast<float2 *>(psi), n, x, z,
                                                    (float)c, (float)s);
    return cudaGetLastError();
}

cudaError_t launch_expect_diag(bool dbl, const void *psi, int n, const uint64_t *d_oz,
                               const double *d_oc, int terms, double *partial, int blocks,
                               cudaStream_t st) {
    if (dbl)
        expect_diag_kernel<double><<<blocks, 256, 0, st>>>(reinterpret_cast<const double2 *>(psi), n,
                                                           d_oz, d_oc, terms, partial);
    else
        expect_diag_kernel<float><<<blocks, 256, 0, st>>>(reinterpret_cast<const float2 *>(psi), n,
                                                          d_oz, d_oc, terms, partial);
    return cudaGetLastError();
}

cudaError_t launch_expect_pauli(bool dbl, const void *psi, int n, uint64_t x, uint64_t z, double coef,
                                double *partial, int blocks, cudaStream_t st) {
    if (dbl)
        expect_pauli_kernel<double><<<blocks, 256, 0, st>>>(reinterpret_cast<const double2 *>(psi), n,
                                                            x, z, coef, partial);
    else
        expect_pauli_kernel<float><<<blocks, 256, 0, st>>>(reinterpret_cast<const float2 *>(psi), n,
                                                           x, z, coef, partial);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double *partial, int64_t count, double *out, int accumulate,
                          cudaStream_t st) {
    reduce_kernel<<<1, 1024, 0, st>>>(partial, count, out, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_apply_observable(bool dbl, const void *phi, void *lam, int n, const uint64_t *d_ox,
                                    const uint64_t *d_oz, const double *d_oc, int terms,
                                    cudaStream_t st) {
    unsigned g = grid_for((int64_t)1 << n, 148);
    if (dbl)
        apply_observable_kernel<double><<<g, 256, 0, st>>>(reinterpret_cast<const double2 *>(phi),
                                                           reinterpret_cast<double2 *>(lam), n, d_ox,
                                                           d_oz, d_oc, terms);
    else
        apply_observable_kernel<float><<<g, 256, 0, st>>>(reinterpret_cast<const float2 *>(phi),
                                                          reinterpret_cast<float2 *>(lam), n, d_ox,
                                                          d_oz, d_oc, terms);
    return cudaGetLastError();
}

int grad_blocks(int n, int num_sms) {
    int64_t warps = (((int64_t)1 << n) >> 4) / 32;   // one 32-chunk slab per warp at least
    int64_t b = (warps + 7) / 8;
    int64_t cap = (int64_t)num_sms * 4;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_grad_diag(bool dbl, void *chi, void *mu, int n, const DevGrad &g,
                             const uint64_t *masks_f, const int64_t *qinv, const int32_t *,
                             double *partial, int blocks, cudaStream_t st) {
    size_t smem = sizeof(double) * (size_t)(g.m > 0 ? g.m : 1);
    if (smem > 48 * 1024) {
        cudaError_t e = dbl ? cudaFuncSetAttribute(grad_diag_kernel<double>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                            : cudaFuncSetAttribute(grad_diag_kernel<float>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (dbl)
        grad_diag_kernel<double><<<blocks, 256, smem, st>>>(reinterpret_cast<double2 *>(chi),
                                                            reinterpret_cast<double2 *>(mu), n, g,
                                                            masks_f, qinv, partial);
    else
        grad_diag_kernel<float><<<blocks, 256, smem, st>>>(reinterpret_cast<float2 *>(chi),
                                                           reinterpret_cast<float2 *>(mu), n, g,
                                                           masks_f, qinv, partial);
    return cudaGetLastError();
}

cudaError_t launch_copy(void *dst, const void *src, size_t bytes, cudaStream_t st) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
}

}  // namespace sd

namespace sd {
namespace {
__global__ void grad_finalize_kernel(const double *__restrict__ partial, int blocks, int m,
                                     const int32_t *__restrict__ term_id,
                                     const double *__restrict__ factor, double *__restrict__ gacc) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double s = 0.0;
    for (int b = 0; b < blocks; b++) s += partial[(int64_t)b * m + j];
    gacc[term_id[j]] += factor[j] * s;
}
}  // namespace

cudaError_t launch_grad_finalize(const double *partial, int blocks, int m, const int32_t *term_id,
                                 const double *factor, double *gacc, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    grad_finalize_kernel<<<(m + 127) / 128, 128, 0, st>>>(partial, blocks, m, term_id, factor, gacc);
    return cudaGetLastError();
}
}  // namespace sd
