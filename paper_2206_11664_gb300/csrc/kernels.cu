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
#include "tile_device.cuh"

namespace sd {
namespace {

constexpr int kMaxRounds = 12;

// Packed op word: kind (3 bits) | slot (2) | p1 (2) | p2 (2) | arg (23).
// D_HAD: p1 = a, p2 = b; D_MONO: p1 = a, p2 = x; D_DIAG: p1 = scale flag.
__host__ __device__ __forceinline__ int32_t pack_op(const DevOp &o) {
    int p1 = 0, p2 = 0, arg = 0;
    if (o.kind == D_HAD) { p1 = c1_a(o.arg); p2 = c1_b(o.arg); }
    else if (o.kind == D_MONO) { p1 = c1_a(o.arg); p2 = c1_x(o.arg); }
    else { p1 = o.pad; arg = o.arg; }
    return o.kind | (o.slot << 3) | (p1 << 5) | (p2 << 7) | (arg << 9);
}

// One pass over the state vector.  Per tile: the prefetch buffer (filled by
// cp.async while the previous tile was processed) is read in the load
// layout; the next tile's prefetch is issued; the rounds run on registers
// with exchanges through the swizzled buffer; the last round stores.
// Per-round thread layouts (tile index, swizzled index, global offset of the
// fixed bits) come from tables built once per block.
template <typename T, int K>
__device__ __forceinline__ void tile_pass_body(typename VT<T>::A *__restrict__ psi, int n, int pass_idx,
                                               const KParams &kp, int64_t first_tile, int64_t tile_stride) {
    using A = typename VT<T>::A;
    constexpr int NT = 1 << (K - 4);
    constexpr int NW = NT / 32;
    constexpr int E = 16 / (int)sizeof(A);            // amplitudes per 16-byte copy
    constexpr int NCOPY = (1 << K) / E / NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    A *X = reinterpret_cast<A *>(smraw);                // exchange buffer (swizzled)
    A *Pf = X + (1 << K);                               // prefetch buffer (tile order)
    StagedTerm *ST = reinterpret_cast<StagedTerm *>(Pf + (1 << K));   // P.max_stage slots
    uint64_t *TQ = nullptr;                             // P.max_tot class totals, after ST
    __shared__ DevPass P;
    __shared__ DevRound RR[kMaxRounds];
    __shared__ uint32_t swzc[16];
    __shared__ A TW[256];
    __shared__ uint64_t SPLO[256], SPHI[32];           // spread of tile index bits 0-7, 8-12
    __shared__ uint64_t OUTT[4][256];                  // deposit of tile number bytes
    __shared__ uint32_t LTL[kMaxRounds][32], LTW[kMaxRounds][NW];   // lf | swz(lf) << 16
    __shared__ uint64_t XL[kMaxRounds][32], XW[kMaxRounds][NW];     // spread(lf) parts
    __shared__ uint32_t RCS[kMaxRounds][4];            // register column | swizzled << 16
    __shared__ uint64_t RG[kMaxRounds][4];             // global offset of register slot
    __shared__ int32_t OPS[kMaxPassOps];
    __shared__ uint64_t CST[4];
    const int tid = threadIdx.x;
    if (tid == 0) P = kp.passes[pass_idx];
    __syncthreads();
    const int nr = P.n_rounds;
    TQ = reinterpret_cast<uint64_t *>(ST + (P.max_stage > 0 ? P.max_stage : 1));
    const uint64_t *tmo = kp.term_mo;
    const int64_t *tqv = kp.term_q;
    int toff = 0;
    if (P.term_cache) {
        uint64_t *TCM = TQ + P.max_tot;
        int64_t *TCQ = reinterpret_cast<int64_t *>(TCM + P.term_count);
        cache_terms(kp, P.term_begin, P.term_count, TCM, TCQ, tid, NT);
        tmo = TCM;
        tqv = TCQ;
        toff = P.term_begin;
    }
    if (tid < nr) RR[tid] = kp.rounds[P.round_begin + tid];
    if (tid < K) {
        uint32_t col = 1u << tid;
        if (tid >= kp.c) {
            const uint32_t span = (1u << kp.c) - 1u;
            col |= 1u + (uint32_t)((tid - kp.c) % (int)span);
        }
        swzc[tid] = col;
    }
    for (int i = tid; i < 256; i += NT) {
        const double2 e = kp.tw[i];
        TW[i].x = (T)e.x;
        TW[i].y = (T)e.y;
        uint64_t v = 0;
        for (int b = 0; b < 8 && b < K; b++)
            if ((i >> b) & 1) v |= (uint64_t)1 << P.tile_bits[b];
        SPLO[i] = v;
        if (i < 32) {
            uint64_t w = 0;
            for (int b = 0; b < 5 && 8 + b < K; b++)
                if ((i >> b) & 1) w |= (uint64_t)1 << P.tile_bits[8 + b];
            SPHI[i] = w;
        }
#pragma unroll
        for (int byte = 0; byte < 4; byte++) {
            uint64_t o = 0;
            for (int b = 0; b < 8; b++) {
                const int k = byte * 8 + b;
                if (k < P.n_outer && ((i >> b) & 1)) o |= (uint64_t)1 << P.outer_bits[k];
            }
            OUTT[byte][i] = o;
        }
    }
    __syncthreads();
    {
        const int op0 = RR[0].op_begin, nops = RR[nr - 1].op_end - op0;
        for (int i = tid; i < nops; i += NT) OPS[i] = pack_op(kp.ops[op0 + i]);
        for (int i = tid; i < nr * (32 + NW); i += NT) {
            const int r = i / (32 + NW), k = i % (32 + NW);
            const DevRound &R = RR[r];
            uint32_t lfp = 0;
            if (k < 32) {
                for (int b = 0; b < 5; b++)
                    if ((k >> b) & 1) lfp |= 1u << R.lane_pos[b];
            } else {
                for (int b = 0; b < K - 9; b++)
                    if (((k - 32) >> b) & 1) lfp |= 1u << R.warp_pos[b];
            }
            uint32_t sw = 0;
            for (int p = 0; p < K; p++)
                if ((lfp >> p) & 1) sw ^= swzc[p];
            const uint64_t xp = SPLO[lfp & 255] | SPHI[lfp >> 8];
            if (k < 32) {
                LTL[r][k] = lfp | (sw << 16);
                XL[r][k] = xp;
            } else {
                LTW[r][k - 32] = lfp | (sw << 16);
                XW[r][k - 32] = xp;
            }
        }
        for (int i = tid; i < nr * 4; i += NT) {
            const int r = i >> 2, s = i & 3, p = RR[r].reg_pos[s];
            RCS[r][s] = (1u << p) | (swzc[p] << 16);
            RG[r][s] = (uint64_t)1 << P.tile_bits[p];
        }
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    const int64_t ntiles = (int64_t)1 << (n - K);
    const int op0 = RR[0].op_begin;
    const T pass_scale = P.scale_in_diag ? (T)1 : (T)P.scale;
    const T diag_scale = (T)P.scale;
    auto deposit = [&](int64_t t) -> uint64_t {
        return OUTT[0][t & 255] | OUTT[1][(t >> 8) & 255] | OUTT[2][(t >> 16) & 255] |
               OUTT[3][(t >> 24) & 255];
    };
    auto prefetch = [&](int64_t t) {
        const uint64_t xo = deposit(t);
#pragma unroll
        for (int k = 0; k < NCOPY; k++) {
            const uint32_t l = (uint32_t)(tid + k * NT) * E;
            cp_async16(Pf + l, psi + (xo | SPLO[l & 255] | SPHI[l >> 8]));
        }
        cp_async_commit();
    };

    int64_t tile = first_tile;
    if (tile < ntiles) prefetch(tile);
    for (; tile < ntiles; tile += tile_stride) {
        const uint64_t xo = deposit(tile);
        A a[16];
        for (int r = 0; r < nr; r++) {
            const DevRound &R = RR[r];
            if (r == 0) cp_async_wait_all();
            __syncthreads();
            if (R.n_diag > 0) {
                stage_slots(xo, kp.slots, R.slot_begin, R.slot_count, tmo, tqv, toff, ST, tid, NT);
                for (int c = warp; c < 4; c += NW)
                    if (R.cst_count[c] > 0) {
                        const uint64_t v = warp_const_sum(xo, kp.cst_mo, kp.cst_q, R.cst_begin[c],
                                                          R.cst_count[c], lane);
                        if (lane == 0) CST[c] = v;
                    }
                __syncthreads();
                stage_totals(kp, R.diag_begin, R.n_diag, ST, CST, TotalBias<A>::value, TQ, tid, NT);
                __syncthreads();
            }
            const uint32_t v = LTL[r][lane] ^ LTW[r][warp];
            const uint32_t lf = v & 0xffffu, sw = v >> 16;
            uint32_t lreg[4], cs[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const uint32_t c2 = RCS[r][i];
                lreg[i] = c2 & 0xffffu;
                cs[i] = c2 >> 16;
            }
            if (r == 0) {
#pragma unroll
                for (int s = 0; s < 16; s++) {
                    uint32_t l = lf;
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        if ((s >> i) & 1) l |= lreg[i];
                    a[s] = Pf[l];
                }
                __syncthreads();
                if (tile + tile_stride < ntiles) prefetch(tile + tile_stride);
            } else {
#pragma unroll
                for (int s = 0; s < 16; s++) {
                    uint32_t ad = sw;
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        if ((s >> i) & 1) ad ^= cs[i];
                    a[s] = X[ad];
                }
            }
            const uint64_t xf = xo | XL[r][lane] | XW[r][warp];
            for (int o = R.op_begin; o < R.op_end; o++) {
                const int32_t code = OPS[o - op0];
                switch (code & 511) {
                case D_HAD | (0 << 3) | (0 << 5) | (0 << 7): had_fixed<0, 0, 0>(a); break;
                case D_HAD | (0 << 3) | (0 << 5) | (1 << 7): had_fixed<0, 0, 1>(a); break;
                case D_HAD | (0 << 3) | (0 << 5) | (2 << 7): had_fixed<0, 0, 2>(a); break;
                case D_HAD | (0 << 3) | (0 << 5) | (3 << 7): had_fixed<0, 0, 3>(a); break;
                case D_HAD | (0 << 3) | (1 << 5) | (0 << 7): had_fixed<0, 1, 0>(a); break;
                case D_HAD | (0 << 3) | (1 << 5) | (1 << 7): had_fixed<0, 1, 1>(a); break;
                case D_HAD | (0 << 3) | (1 << 5) | (2 << 7): had_fixed<0, 1, 2>(a); break;
                case D_HAD | (0 << 3) | (1 << 5) | (3 << 7): had_fixed<0, 1, 3>(a); break;
                case D_HAD | (0 << 3) | (2 << 5) | (0 << 7): had_fixed<0, 2, 0>(a); break;
                case D_HAD | (0 << 3) | (2 << 5) | (1 << 7): had_fixed<0, 2, 1>(a); break;
                case D_HAD | (0 << 3) | (2 << 5) | (2 << 7): had_fixed<0, 2, 2>(a); break;
                case D_HAD | (0 << 3) | (2 << 5) | (3 << 7): had_fixed<0, 2, 3>(a); break;
                case D_HAD | (0 << 3) | (3 << 5) | (0 << 7): had_fixed<0, 3, 0>(a); break;
                case D_HAD | (0 << 3) | (3 << 5) | (1 << 7): had_fixed<0, 3, 1>(a); break;
                case D_HAD | (0 << 3) | (3 << 5) | (2 << 7): had_fixed<0, 3, 2>(a); break;
                case D_HAD | (0 << 3) | (3 << 5) | (3 << 7): had_fixed<0, 3, 3>(a); break;
                case D_HAD | (1 << 3) | (0 << 5) | (0 << 7): had_fixed<1, 0, 0>(a); break;
                case D_HAD | (1 << 3) | (0 << 5) | (1 << 7): had_fixed<1, 0, 1>(a); break;
                case D_HAD | (1 << 3) | (0 << 5) | (2 << 7): had_fixed<1, 0, 2>(a); break;
                case D_HAD | (1 << 3) | (0 << 5) | (3 << 7): had_fixed<1, 0, 3>(a); break;
                case D_HAD | (1 << 3) | (1 << 5) | (0 << 7): had_fixed<1, 1, 0>(a); break;
                case D_HAD | (1 << 3) | (1 << 5) | (1 << 7): had_fixed<1, 1, 1>(a); break;
                case D_HAD | (1 << 3) | (1 << 5) | (2 << 7): had_fixed<1, 1, 2>(a); break;
                case D_HAD | (1 << 3) | (1 << 5) | (3 << 7): had_fixed<1, 1, 3>(a); break;
                case D_HAD | (1 << 3) | (2 << 5) | (0 << 7): had_fixed<1, 2, 0>(a); break;
                case D_HAD | (1 << 3) | (2 << 5) | (1 << 7): had_fixed<1, 2, 1>(a); break;
                case D_HAD | (1 << 3) | (2 << 5) | (2 << 7): had_fixed<1, 2, 2>(a); break;
                case D_HAD | (1 << 3) | (2 << 5) | (3 << 7): had_fixed<1, 2, 3>(a); break;
                case D_HAD | (1 << 3) | (3 << 5) | (0 << 7): had_fixed<1, 3, 0>(a); break;
                case D_HAD | (1 << 3) | (3 << 5) | (1 << 7): had_fixed<1, 3, 1>(a); break;
                case D_HAD | (1 << 3) | (3 << 5) | (2 << 7): had_fixed<1, 3, 2>(a); break;
                case D_HAD | (1 << 3) | (3 << 5) | (3 << 7): had_fixed<1, 3, 3>(a); break;
                case D_HAD | (2 << 3) | (0 << 5) | (0 << 7): had_fixed<2, 0, 0>(a); break;
                case D_HAD | (2 << 3) | (0 << 5) | (1 << 7): had_fixed<2, 0, 1>(a); break;
                case D_HAD | (2 << 3) | (0 << 5) | (2 << 7): had_fixed<2, 0, 2>(a); break;
                case D_HAD | (2 << 3) | (0 << 5) | (3 << 7): had_fixed<2, 0, 3>(a); break;
                case D_HAD | (2 << 3) | (1 << 5) | (0 << 7): had_fixed<2, 1, 0>(a); break;
                case D_HAD | (2 << 3) | (1 << 5) | (1 << 7): had_fixed<2, 1, 1>(a); break;
                case D_HAD | (2 << 3) | (1 << 5) | (2 << 7): had_fixed<2, 1, 2>(a); break;
                case D_HAD | (2 << 3) | (1 << 5) | (3 << 7): had_fixed<2, 1, 3>(a); break;
                case D_HAD | (2 << 3) | (2 << 5) | (0 << 7): had_fixed<2, 2, 0>(a); break;
                case D_HAD | (2 << 3) | (2 << 5) | (1 << 7): had_fixed<2, 2, 1>(a); break;
                case D_HAD | (2 << 3) | (2 << 5) | (2 << 7): had_fixed<2, 2, 2>(a); break;
                case D_HAD | (2 << 3) | (2 << 5) | (3 << 7): had_fixed<2, 2, 3>(a); break;
                case D_HAD | (2 << 3) | (3 << 5) | (0 << 7): had_fixed<2, 3, 0>(a); break;
                case D_HAD | (2 << 3) | (3 << 5) | (1 << 7): had_fixed<2, 3, 1>(a); break;
                case D_HAD | (2 << 3) | (3 << 5) | (2 << 7): had_fixed<2, 3, 2>(a); break;
                case D_HAD | (2 << 3) | (3 << 5) | (3 << 7): had_fixed<2, 3, 3>(a); break;
                case D_HAD | (3 << 3) | (0 << 5) | (0 << 7): had_fixed<3, 0, 0>(a); break;
                case D_HAD | (3 << 3) | (0 << 5) | (1 << 7): had_fixed<3, 0, 1>(a); break;
                case D_HAD | (3 << 3) | (0 << 5) | (2 << 7): had_fixed<3, 0, 2>(a); break;
                case D_HAD | (3 << 3) | (0 << 5) | (3 << 7): had_fixed<3, 0, 3>(a); break;
                case D_HAD | (3 << 3) | (1 << 5) | (0 << 7): had_fixed<3, 1, 0>(a); break;
                case D_HAD | (3 << 3) | (1 << 5) | (1 << 7): had_fixed<3, 1, 1>(a); break;
                case D_HAD | (3 << 3) | (1 << 5) | (2 << 7): had_fixed<3, 1, 2>(a); break;
                case D_HAD | (3 << 3) | (1 << 5) | (3 << 7): had_fixed<3, 1, 3>(a); break;
                case D_HAD | (3 << 3) | (2 << 5) | (0 << 7): had_fixed<3, 2, 0>(a); break;
                case D_HAD | (3 << 3) | (2 << 5) | (1 << 7): had_fixed<3, 2, 1>(a); break;
                case D_HAD | (3 << 3) | (2 << 5) | (2 << 7): had_fixed<3, 2, 2>(a); break;
                case D_HAD | (3 << 3) | (2 << 5) | (3 << 7): had_fixed<3, 2, 3>(a); break;
                case D_HAD | (3 << 3) | (3 << 5) | (0 << 7): had_fixed<3, 3, 0>(a); break;
                case D_HAD | (3 << 3) | (3 << 5) | (1 << 7): had_fixed<3, 3, 1>(a); break;
                case D_HAD | (3 << 3) | (3 << 5) | (2 << 7): had_fixed<3, 3, 2>(a); break;
                case D_HAD | (3 << 3) | (3 << 5) | (3 << 7): had_fixed<3, 3, 3>(a); break;
                case D_MONO | (0 << 3) | (0 << 5) | (1 << 7): mono_fixed<0, 0, 1>(a); break;
                case D_MONO | (0 << 3) | (1 << 5) | (0 << 7): mono_fixed<0, 1, 0>(a); break;
                case D_MONO | (0 << 3) | (1 << 5) | (1 << 7): mono_fixed<0, 1, 1>(a); break;
                case D_MONO | (0 << 3) | (2 << 5) | (0 << 7): mono_fixed<0, 2, 0>(a); break;
                case D_MONO | (0 << 3) | (2 << 5) | (1 << 7): mono_fixed<0, 2, 1>(a); break;
                case D_MONO | (0 << 3) | (3 << 5) | (0 << 7): mono_fixed<0, 3, 0>(a); break;
                case D_MONO | (0 << 3) | (3 << 5) | (1 << 7): mono_fixed<0, 3, 1>(a); break;
                case D_MONO | (1 << 3) | (0 << 5) | (1 << 7): mono_fixed<1, 0, 1>(a); break;
                case D_MONO | (1 << 3) | (1 << 5) | (0 << 7): mono_fixed<1, 1, 0>(a); break;
                case D_MONO | (1 << 3) | (1 << 5) | (1 << 7): mono_fixed<1, 1, 1>(a); break;
                case D_MONO | (1 << 3) | (2 << 5) | (0 << 7): mono_fixed<1, 2, 0>(a); break;
                case D_MONO | (1 << 3) | (2 << 5) | (1 << 7): mono_fixed<1, 2, 1>(a); break;
                case D_MONO | (1 << 3) | (3 << 5) | (0 << 7): mono_fixed<1, 3, 0>(a); break;
                case D_MONO | (1 << 3) | (3 << 5) | (1 << 7): mono_fixed<1, 3, 1>(a); break;
                case D_MONO | (2 << 3) | (0 << 5) | (1 << 7): mono_fixed<2, 0, 1>(a); break;
                case D_MONO | (2 << 3) | (1 << 5) | (0 << 7): mono_fixed<2, 1, 0>(a); break;
                case D_MONO | (2 << 3) | (1 << 5) | (1 << 7): mono_fixed<2, 1, 1>(a); break;
                case D_MONO | (2 << 3) | (2 << 5) | (0 << 7): mono_fixed<2, 2, 0>(a); break;
                case D_MONO | (2 << 3) | (2 << 5) | (1 << 7): mono_fixed<2, 2, 1>(a); break;
                case D_MONO | (2 << 3) | (3 << 5) | (0 << 7): mono_fixed<2, 3, 0>(a); break;
                case D_MONO | (2 << 3) | (3 << 5) | (1 << 7): mono_fixed<2, 3, 1>(a); break;
                case D_MONO | (3 << 3) | (0 << 5) | (1 << 7): mono_fixed<3, 0, 1>(a); break;
                case D_MONO | (3 << 3) | (1 << 5) | (0 << 7): mono_fixed<3, 1, 0>(a); break;
                case D_MONO | (3 << 3) | (1 << 5) | (1 << 7): mono_fixed<3, 1, 1>(a); break;
                case D_MONO | (3 << 3) | (2 << 5) | (0 << 7): mono_fixed<3, 2, 0>(a); break;
                case D_MONO | (3 << 3) | (2 << 5) | (1 << 7): mono_fixed<3, 2, 1>(a); break;
                case D_MONO | (3 << 3) | (3 << 5) | (0 << 7): mono_fixed<3, 3, 0>(a); break;
                case D_MONO | (3 << 3) | (3 << 5) | (1 << 7): mono_fixed<3, 3, 1>(a); break;
                case D_PHASE: {
                    int gq[4];
#pragma unroll
                    for (int i = 0; i < 4; i++) gq[i] = P.tile_bits[R.reg_pos[i]];
                    phase_apply(a, xf, gq, kp.phases[code >> 9], kp.mask_pool);
                    break;
                }
                default:
                    if ((code & 7) == D_DIAG) {
                        const DevDiag &dg = kp.diags[code >> 9];
                        diag_apply(a, lf, dg, ST, TQ, TW, ((code >> 5) & 1) ? diag_scale : (T)1);
                    }
                    break;
                }
            }
            if (R.flags & 2) {
                uint64_t goff[4];
#pragma unroll
                for (int i = 0; i < 4; i++) goff[i] = RG[r][i];
#pragma unroll
                for (int s = 0; s < 16; s++) {
                    uint64_t x = xf;
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        if ((s >> i) & 1) x |= goff[i];
                    A w = a[s];
                    w.x *= pass_scale;
                    w.y *= pass_scale;
                    psi[x] = w;
                }
            } else {
                uint32_t base = sw;
                if (R.perm >= 0) {
                    if (r > 0) __syncthreads();   // others may still read what this thread overwrites
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
                        const uint32_t cv = pm.col[R.reg_pos[i]];
                        uint32_t w = 0;
#pragma unroll
                        for (int p = 0; p < K; p++)
                            if ((cv >> p) & 1) w ^= swzc[p];
                        cs[i] = w;
                    }
                }
#pragma unroll
                for (int s = 0; s < 16; s++) {
                    uint32_t ad = base;
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        if ((s >> i) & 1) ad ^= cs[i];
                    X[ad] = a[s];
                }
            }
        }
    }
}

template <typename T, int K>
__global__ void __launch_bounds__(1 << (K - 4))
tile_pass_kernel(typename VT<T>::A *__restrict__ psi, int n, int pass_idx, KParams kp) {
    tile_pass_body<T, K>(psi, n, pass_idx, kp, blockIdx.x, gridDim.x);
}

// Level-synchronous batch: block b serves instance cta_inst[b]; at `level`
// that instance runs pass f(level) of its head / core / tail programs.
template <typename T, int K>
__global__ void __launch_bounds__(1 << (K - 4))
tile_pass_batch_kernel(const BatchInstance *__restrict__ inst, const uint16_t *__restrict__ cta_inst,
                       int64_t level) {
    const BatchInstance &I = inst[cta_inst[blockIdx.x]];
    if (level >= I.levels) return;
    int prog, pass;
    if (level < I.npass[0]) {
        prog = 0;
        pass = (int)level;
    } else if (level - I.npass[0] < (int64_t)I.npass[1] * I.reps_core) {
        prog = 1;
        pass = (int)((level - I.npass[0]) % I.npass[1]);
    } else {
        prog = 2;
        pass = (int)(level - I.npass[0] - (int64_t)I.npass[1] * I.reps_core);
    }
    tile_pass_body<T, K>(reinterpret_cast<typename VT<T>::A *>(I.psi), I.n, pass, I.kp[prog],
                         (int64_t)blockIdx.x - I.cta_begin, I.cta_count);
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
    const int d = sizeof(T) == 8;
    const size_t smem = pass_smem_bytes(S.host_passes[pass], sizeof(A), K);
    const size_t smem_max = kTileSmemLimit;
    if (smem > smem_max) return cudaErrorInvalidConfiguration;
    if (!g_occ.init[d][K]) {
        cudaError_t e = cudaFuncSetAttribute(tile_pass_kernel<T, K>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
        if (e != cudaSuccess) return e;
        g_occ.init[d][K] = true;
    }
    int b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tile_pass_kernel<T, K>, threads, smem);
    if (e != cudaSuccess) return e;
    if (b < 1) b = 1;
    KParams kp{S.passes, S.rounds, S.ops, S.perms, S.diags, S.phases,
               S.term_mo, S.slots, S.term_q, S.mask_pool, S.cst_mo, S.cst_q, S.c, S.tw, S.fxt};
    int64_t ntiles = (int64_t)1 << (n - K);
    int64_t grid = (int64_t)num_sms * b;
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
            if (op.kind == OK_C1) {
                const int64_t bq = (int64_t)1 << op.q;
                const int had = c1_had(op.q2), pa = c1_a(op.q2), pb = c1_b(op.q2), xx = c1_x(op.q2);
                for (int64_t i = tid; i < N / 2; i += nt) {
                    int64_t lo = i & (bq - 1);
                    int64_t y = ((i - lo) << 1) | lo;
                    A u = st[y], w = mul_ipow(st[y | bq], pa);
                    if (had) {
                        A o0, o1;
                        o0.x = (u.x + w.x) * r2;
                        o0.y = (u.y + w.y) * r2;
                        o1.x = (u.x - w.x) * r2;
                        o1.y = (u.y - w.y) * r2;
                        st[y] = o0;
                        st[y | bq] = mul_ipow(o1, pb);
                    } else if (xx) {
                        st[y] = w;
                        st[y | bq] = u;
                    } else {
                        st[y | bq] = w;
                    }
                }
            } else if (is_1q(op.kind)) {
                const int64_t bq = (int64_t)1 << op.q;
                const int k = op.kind == OK_S ? 1 : (op.kind == OK_Z ? 2 : 3);
                for (int64_t i = tid; i < N / 2; i += nt) {
                    int64_t lo = i & (bq - 1);
                    int64_t y = ((i - lo) << 1) | lo;
                    if (op.kind == OK_H) {
                        A u = st[y], v = st[y | bq];
                        st[y].x = (u.x + v.x) * r2;
                        st[y].y = (u.y + v.y) * r2;
                        st[y | bq].x = (u.x - v.x) * r2;
                        st[y | bq].y = (u.y - v.y) * r2;
                    } else if (op.kind == OK_X) {
                        A u = st[y];
                        st[y] = st[y | bq];
                        st[y | bq] = u;
                    } else {
                        st[y | bq] = mul_ipow(st[y | bq], k);
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
template <typename A> __device__ __forceinline__ A make_cplx(decltype(A::x) re, decltype(A::x) im) {
    A a;
    a.x = re;
    a.y = im;
    return a;
}

template <typename T>
__global__ void __launch_bounds__(256)
grad_diag_kernel(typename VT<T>::A *__restrict__ chi, typename VT<T>::A *__restrict__ mu, int n,
                 DevGrad g, const uint64_t *__restrict__ masks_f, const int64_t *__restrict__ qinv,
                 const longlong2 *__restrict__ fxt, double *__restrict__ partial, int per_thread) {
    using A = typename VT<T>::A;
    // per_thread: acc[j * blockDim.x + tid] is thread tid's own sum for term
    // j (one add per term and chunk, reduced once at the end); otherwise
    // acc[j] takes each warp's shuffle-reduced sum
    extern __shared__ double acc[];
    const int nacc = per_thread ? g.m * (int)blockDim.x : g.m;
    for (int j = threadIdx.x; j < nacc; j += blockDim.x) acc[j] = 0.0;
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
                if (per_thread) {
                    acc[j * (int)blockDim.x + (int)threadIdx.x] += v;
                } else {
                    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                    if (lane == 0) atomicAdd(&acc[j], v);
                }
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
                // one rotation factor e^{-2 pi i G} for both vectors; in double
                // precision its cosine and sine come from the Q1.62 tables and
                // series in integer arithmetic, which leaves the FP64 pipe (the
                // kernel's bound on this GPU) to the products with chi and mu
                T sn, cs;
                if constexpr (sizeof(T) == 8) {
                    long long er, ei;
                    fx_cis(G[s], fxt, fxt + 256, er, ei);
                    cs = fx_to(er, -62);
                    sn = fx_to(ei, -62);
                } else {
                    turns_sc(G[s], sn, cs);
                }
                A a = cv[s], b = mv[s];
                chi[xf + s] = make_cplx<A>(a.x * cs + a.y * sn, a.y * cs - a.x * sn);
                mu[xf + s] = make_cplx<A>(b.x * cs + b.y * sn, b.y * cs - b.x * sn);
            }
        }
    }
    __syncthreads();
    if (per_thread) {
        const int nw = (int)blockDim.x >> 5, wp = (int)threadIdx.x >> 5;
        for (int j = wp; j < g.m; j += nw) {
            double v = 0.0;
            for (int t = lane; t < (int)blockDim.x; t += 32) v += acc[j * (int)blockDim.x + t];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) partial[(int64_t)blockIdx.x * g.m + j] = v;
        }
    } else {
        for (int j = threadIdx.x; j < g.m; j += blockDim.x) partial[(int64_t)blockIdx.x * g.m + j] = acc[j];
    }
}


}  // namespace

template <typename T, int K>
cudaError_t run_batch(const BatchInstance *d_inst, const uint16_t *d_cta, int blocks, size_t smem,
                      int64_t level, cudaStream_t st) {
    static bool init = false;
    if (!init) {
        cudaError_t e = cudaFuncSetAttribute(tile_pass_batch_kernel<T, K>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kTileSmemLimit);
        if (e != cudaSuccess) return e;
        init = true;
    }
    tile_pass_batch_kernel<T, K><<<blocks, 1 << (K - 4), smem, st>>>(d_inst, d_cta, level);
    return cudaGetLastError();
}

int tile_pass_batch_occupancy(bool dbl, int K, size_t smem) {
    int b = 0;
    const int threads = 1 << (K - 4);
#define SD_OCC_CASE(KK)                                                                            \
    case KK:                                                                                       \
        if (dbl) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tile_pass_batch_kernel<double, KK>, threads, smem); \
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tile_pass_batch_kernel<float, KK>, threads, smem);     \
        break;
    switch (K) {
        SD_OCC_CASE(9)
        SD_OCC_CASE(10)
        SD_OCC_CASE(11)
        SD_OCC_CASE(12)
        SD_OCC_CASE(13)
    default: break;
    }
#undef SD_OCC_CASE
    cudaGetLastError();
    return b > 0 ? b : 1;
}

cudaError_t launch_tile_pass_batch(bool dbl, int K, const BatchInstance *d_inst, const uint16_t *d_cta_inst,
                                   int blocks, size_t smem, int64_t level, cudaStream_t st) {
#define SD_BATCH_CASE(KK)                                                                         \
    case KK:                                                                                      \
        return dbl ? run_batch<double, KK>(d_inst, d_cta_inst, blocks, smem, level, st)          \
                   : run_batch<float, KK>(d_inst, d_cta_inst, blocks, smem, level, st);
    switch (K) {
        SD_BATCH_CASE(9)
        SD_BATCH_CASE(10)
        SD_BATCH_CASE(11)
        SD_BATCH_CASE(12)
        SD_BATCH_CASE(13)
    default: return cudaErrorInvalidValue;
    }
#undef SD_BATCH_CASE
}


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

// 16-byte grid-stride copy; either side may be page-locked host memory
// addressed through its mapped (unified) address, so that the SMs move the
// state over the host link.
__global__ void copy16_kernel(const int4 *__restrict__ src, int4 *__restrict__ dst, int64_t n16) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += stride) dst[i] = src[i];
}

cudaError_t launch_copy16(const void *src, void *dst, size_t bytes, int num_sms, cudaStream_t st) {
    const int64_t n16 = (int64_t)(bytes / 16);
    if (n16 == 0) return cudaSuccess;
    int64_t grid = (int64_t)num_sms * 4;
    if (grid > (n16 + 511) / 512) grid = (n16 + 511) / 512;
    copy16_kernel<<<(unsigned)grid, 512, 0, st>>>((const int4 *)src, (int4 *)dst, n16);
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
                             const uint64_t *masks_f, const int64_t *qinv, const longlong2 *fxt,
                             double *partial, int blocks, cudaStream_t st) {
    // per-thread term sums while they fit beside nothing else in shared memory
    constexpr int kThreads = 256;
    const int per_thread = (size_t)g.m * kThreads * sizeof(double) <= 160 * 1024 ? 1 : 0;
    size_t smem = sizeof(double) * (size_t)(g.m > 0 ? g.m : 1) * (per_thread ? kThreads : 1);
    if (smem > 48 * 1024) {
        cudaError_t e = dbl ? cudaFuncSetAttribute(grad_diag_kernel<double>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                            : cudaFuncSetAttribute(grad_diag_kernel<float>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (dbl)
        grad_diag_kernel<double><<<blocks, kThreads, smem, st>>>(reinterpret_cast<double2 *>(chi),
                                                                 reinterpret_cast<double2 *>(mu), n, g,
                                                                 masks_f, qinv, fxt, partial, per_thread);
    else
        grad_diag_kernel<float><<<blocks, kThreads, smem, st>>>(reinterpret_cast<float2 *>(chi),
                                                                reinterpret_cast<float2 *>(mu), n, g,
                                                                masks_f, qinv, fxt, partial, per_thread);
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
