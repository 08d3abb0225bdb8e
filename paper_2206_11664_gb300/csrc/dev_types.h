// Types shared by host code, the precompiled kernels and the kernels
// generated at run time (NVRTC): kept free of standard-library headers.
#pragma once

#if defined(__CUDACC_RTC__)
typedef unsigned long long uint64_t;
typedef long long int64_t;
typedef unsigned int uint32_t;
typedef int int32_t;
typedef unsigned char uint8_t;
typedef decltype(sizeof(0)) size_t;
#else
#include <vector_types.h>
#include <cstdint>
#endif

#if defined(__CUDACC__) || defined(__CUDACC_RTC__)
#define SD_HD __host__ __device__
#else
#define SD_HD
#endif

namespace sd {

constexpr int kRegBits = 4;   // amplitudes per thread = 16
constexpr int kLaneBits = 5;

// OK_C1 parameters: had = 1: S^b H S^a (apply S^a, then H, then S^b);
// had = 0: X^x S^a (apply S^a, then X if x).  H is the unnormalised
// butterfly; its 1/sqrt(2) is part of the pass's deferred scale.
inline SD_HD int32_t c1_pack(int had, int a, int b, int x) { return had | (a << 1) | (b << 3) | (x << 5); }
inline SD_HD int c1_had(int32_t v) { return v & 1; }
inline SD_HD int c1_a(int32_t v) { return (v >> 1) & 3; }
inline SD_HD int c1_b(int32_t v) { return (v >> 3) & 3; }
inline SD_HD int c1_x(int32_t v) { return (v >> 5) & 1; }

// Device ops of a round: one-qubit Cliffords on register slot `slot` with
// the OK_C1 parameters in `arg` (D_HAD: S^b H S^a, D_MONO: X^x S^a), or
// diagonal ops with table index `arg`.  pad = 1 on the D_DIAG op that also
// applies the pass's scale.
enum DevOpKind : int32_t { D_HAD = 0, D_MONO = 1, D_PHASE = 3, D_DIAG = 4 };

struct DevOp {
    int32_t kind, slot, arg, pad;
};
constexpr int kMaxPassOps = 1024;

struct DevRound {
    uint8_t reg_pos[4];
    uint8_t lane_pos[5];  // lane bit i <-> tile position lane_pos[i]
    uint8_t warp_pos[7];
    int32_t op_begin, op_end;
    int32_t perm;       // -1 or index of an in-tile permutation applied on the round's smem write
    int32_t flags;      // 1: load from global, 2: store to global
    int32_t slot_begin; // term slots of the round's group exponentials: kp.slots[slot_begin, +slot_count)
    int32_t slot_count;
    int32_t diag_begin; // the round's group exponentials: kp.diags[diag_begin, +n_diag)
    int32_t n_diag;
    // Terms whose masks meet no tile qubit of the round take one value on the
    // whole tile: their signed sum is formed once per tile into slot c
    // (pool range [cst_begin[c], cst_begin[c] + cst_count[c]) of cst_mo/cst_q).
    int32_t cst_begin[4];
    int32_t cst_count[4];
};

struct DevPass {
    int32_t round_begin, n_rounds;
    int32_t n_outer;
    int32_t scale_in_diag;   // 1 if the deferred scale is folded into a D_DIAG op
    int32_t max_stage;       // most term slots staged by one round
    int32_t max_tot;         // most class totals staged by one round (16 per group exponential)
    int32_t term_begin;      // the pass's group-exponential terms: term_mo/term_q[term_begin, +term_count)
    int32_t term_count;
    int32_t term_cache;      // 1: the pass copies its terms to shared memory once per block
    int32_t pad;
    double scale;            // 2^(-h/2) for h Hadamards in the pass
    uint8_t tile_bits[16];
    uint8_t outer_bits[48];
};

// In-tile linear permutation (a run of CNOTs whose targets are tile qubits):
// the amplitude at tile index l of the tile with outer bits h moves to
// (xor of col[p] over set bits p of l) ^ (xor of ocol[k] over set outer bits k).
struct DevPerm {
    uint32_t col[16];
    uint32_t ocol[48];
};

// Per-round diagonal descriptor.  The angle of amplitude x is
//   T(x) = sum_j q_j (-1)^{|x & m_j|},
// with x = (outer bits of the tile, fixed tile positions lf of the thread,
// the 4 register bits s).  Terms are sorted by their register projection
// (class u = the bits of m_j on the round's register positions), and within
// a class by their mask ml on the fixed positions: the terms of one
// (class, ml) pair form a slot, whose signed sum over the outer bits is one
// number per tile.  Per class, G[u] = (sum of all its slots) - 2 (sum of the
// slots whose ml has odd parity with lf); a 4-level Walsh-Hadamard
// transform over the register bits turns G into T.
//   off[u]..off[u+1]: the class's slots with ml != 0 (indices relative to
//                     the round's slot_begin);
//   zs[u]:            its slot with ml == 0, or -1;
//   tot:              class totals live at TQ[tot + u] (tot = 16 k for the
//                     round's k-th group exponential);
//   cst:              tile-constant slot of the round folded into class 0, or -1.
struct DevDiag {
    int32_t off[17];
    int32_t zs[16];
    int32_t tot;
    int32_t cst;
};

// A slot: terms [tb, tb + tn) of term_mo/term_q sharing a class and the mask
// ml on the round's fixed tile positions.
struct DevSlot {
    int32_t tb, tn;
    uint32_t ml;
    int32_t pad;
};

// Per-round phase descriptor (S/CZ layer).
struct DevPhase {
    uint64_t sp, sm;      // global masks
    int64_t adj_base;     // index of n adjacency masks (symmetric) in the mask pool
    int64_t up_base;      // index of n upper adjacency masks
    int32_t lin_s[4];     // +1 / -1 / 0: S or S^dag on the qubit of register slot i
    int32_t quad;         // bit (i*4+j) set: CZ between register slots i<j
    int32_t n;
};


// A slot staged in shared memory for one tile: its Q0.64 angle sum with the
// signs of the tile's outer bits folded in, and its mask ml.
struct StagedTerm {
    uint64_t q;
    uint32_t ml;
    uint32_t pad;
};

// Dynamic shared memory a tile pass may use: 227 KB per block less the
// kernels' static tables.
constexpr size_t kTileSmemLimit = 227 * 1024 - 28 * 1024;
// Passes with at most this many group-exponential terms keep them in shared
// memory (16 bytes each), so that staging a tile reads no global memory.
constexpr int kTermCache = 2048;

// Dynamic shared memory of a tile pass with 2^K amplitudes of `amp` bytes per
// tile: exchange and prefetch buffers, staged slots, class totals, and the
// cached terms (outer masks, then angles).
inline SD_HD size_t pass_smem_bytes(const DevPass &P, size_t amp, int K) {
    return 2 * (amp << K) + sizeof(StagedTerm) * (size_t)(P.max_stage > 0 ? P.max_stage : 1) +
           sizeof(uint64_t) * (size_t)P.max_tot + (P.term_cache ? 16 * (size_t)P.term_count : 0);
}

// Pointers a tile-pass kernel reads besides the state.
struct KParams {
    const DevPass *passes;
    const DevRound *rounds;
    const DevOp *ops;
    const DevPerm *perms;
    const DevDiag *diags;
    const DevPhase *phases;
    const uint64_t *term_mo;
    const DevSlot *slots;
    const int64_t *term_q;
    const uint64_t *mask_pool;
    const uint64_t *cst_mo;
    const int64_t *cst_q;
    int c;
    // per-device constant tables: e^{2 pi i k/256} (FP64, entries 0..255)
    // and e^{2 pi i k/512} (FP64, entries 256..767); in Q1.62
    // e^{2 pi i k/256} (entries 0..255) and e^{2 pi i k/65536} (256..511)
    const double2 *tw;
    const longlong2 *fxt;
};

}  // namespace sd
