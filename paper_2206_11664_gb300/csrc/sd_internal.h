// Internal host-side types shared by the planner, the pass scheduler, the
// kernels' launchers and the C ABI.  Not part of the public interface.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace sd {

// ------------------------------------------------------------ planner

enum GateKind : int32_t { G_H = 0, G_S = 1, G_CNOT = 2, G_CZ = 3 };

struct Gate {
    int32_t kind, a, b;  // b = -1 for one-qubit gates
};

// Stages of the synthesis, used to cut the circuit into kernel layers
// (Fig. clifford_block: H layer, CNOT layer, S/CZ layer, H layer).
enum Stage : int32_t { ST_PRE = 0, ST_ALG2 = 1, ST_ALG3 = 2, ST_ALG4 = 3, ST_ALG5 = 4 };

struct GroupPlan {
    std::vector<int64_t> terms;     // input indices, input order
    std::vector<Gate> gates;        // application order
    std::vector<int32_t> stage;     // stage of each gate
    std::vector<uint64_t> masks;    // per term: Z mask after C_g
    std::vector<uint8_t> signs;     // per term: sign bit
    std::vector<uint64_t> cnot_cols, cnot_inv_cols;  // n each
};

struct Plan {
    int n = 0;
    int skip_rule = 2;
    std::vector<GroupPlan> groups;
};

// Returns an empty string on success, else the reason of failure.
std::string make_plan(int n, int64_t m, const uint64_t *x, const uint64_t *z,
                      int skip_rule, Plan &out);

// ------------------------------------------------------------ flat ops

// One Trotter step (or any circuit) as a flat list of state-vector ops.
enum OpKind : int32_t {
    OK_H = 0,      // Hadamard on qubit q (unnormalised butterfly; 1/sqrt2 deferred)
    OK_S = 1,      // S on qubit q
    OK_SDG = 2,    // S^dag on qubit q
    OK_CNOT = 3,   // CNOT(c = q, t = q2)
    OK_PHASE = 4,  // diagonal quarter-turn layer: index into phase table
    OK_DIAG = 5    // group exponential: index into diag table
};

struct FlatOp {
    int32_t kind;
    int32_t q, q2;   // qubits (1q gates, CNOT)
    int32_t idx;     // PHASE / DIAG table index
    uint64_t support;  // qubits a diagonal op depends on
};

// S/CZ layer as a diagonal: multiplies |x> by i^{k(x)} with
// k(x) = |x & sp| - |x & sm| + 2 * sum_{(c,t) in CZ} x_c x_t  (mod 4).
struct PhaseLayer {
    uint64_t sp = 0, sm = 0;
    std::vector<uint64_t> adj;  // n symmetric CZ adjacency masks (duplicates cancel)
    std::vector<uint64_t> up;   // n upper adjacency masks: bit t of up[c] for CZ(c,t), c<t
};

// Group exponential: |x> -> exp(-2 pi i * T(x)) with
// T(x) = sum_j t_j (-1)^{|x & mask_j|}, t_j = f dt c_j (-1)^{r_j} / (2 pi).
struct DiagLayer {
    int32_t group;
    double frac;  // f: 1 for a full step, 0.5 for a half step, -1/-0.5 inverse
    std::vector<uint64_t> masks;
    std::vector<int64_t> q;  // Q0.64 turns of each term
};

struct Circuit {
    std::vector<FlatOp> ops;
    std::vector<PhaseLayer> phases;
    std::vector<DiagLayer> diags;
};

// Q0.64 fixed-point turns of angle_turns (reduced mod 1 in FP64).
int64_t turns_q64(double angle_turns);

// Append C_g, the group exponential (fraction f of dt) and C_g^dag.
void append_group_step(const Plan &plan, int g, double f, double dt,
                       const std::vector<double> &coeffs, Circuit &c);
// Append only C_g (forward=true) or C_g^dag.
void append_clifford(const Plan &plan, int g, bool forward, Circuit &c);

// ------------------------------------------------------------ pass schedule

constexpr int kRegBits = 4;   // amplitudes per thread = 16
constexpr int kLaneBits = 5;

enum DevOpKind : int32_t { D_H = 0, D_S = 1, D_SDG = 2, D_PHASE = 3, D_DIAG = 4 };

struct DevOp {
    int32_t kind, slot, arg, pad;
};

struct DevRound {
    uint8_t reg_pos[4];
    uint8_t lane_pos[5];
    uint8_t warp_pos[7];
    int32_t op_begin, op_end;
    int32_t perm;       // -1 or index of an in-tile permutation applied on the round's smem write
    int32_t flags;      // 1: load from global, 2: store to global
};

struct DevPass {
    int32_t round_begin, n_rounds;
    int32_t n_outer;
    int32_t scale_in_diag;   // 1 if the deferred scale is folded into a D_DIAG op
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

// Per-round diagonal descriptor: terms sorted by their register projection.
struct DevDiag {
    int32_t off[17];      // class s occupies [off[s], off[s+1]) of the term arrays
    int32_t pad;
    int64_t base;         // first term in the term arrays
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

struct Schedule {
    int K = 0;
    int c = 0;            // low qubits that must be lanes for coalesced loads/stores
    std::vector<DevPass> passes;
    std::vector<DevRound> rounds;
    std::vector<DevOp> ops;
    std::vector<DevPerm> perms;
    std::vector<DevDiag> diags;
    std::vector<DevPhase> phases;
    std::vector<uint64_t> term_masks;   // diag term pool: register-free mask part
    std::vector<int64_t> term_q;        // diag term pool: Q0.64 turns
    std::vector<uint64_t> mask_pool;    // phase adjacency pool
    int64_t diag_passes = 0;
};

// Schedule a circuit on n qubits into tile passes of 2^K amplitudes;
// c = log2(128 bytes / amplitude size).  Returns "" or an error.
std::string schedule_circuit(const Circuit &circ, int n, int K, int c, Schedule &out);

// Swizzle column of tile position p (identity on the low c bits).
uint32_t swizzle_col(int p, int c);

}  // namespace sd
