// Internal host-side types shared by the planner, the pass scheduler, the
// kernels' launchers and the C ABI.  Not part of the public interface.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "dev_types.h"

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

// Message returned by sd_last_error(NULL) on this thread.
void set_last_error(const std::string &msg);

// Commuting partition of the terms (Sec. 2.3: greedy).  grouping: 0 = first
// fit in input order; 1 = first fit in order of decreasing anticommutation
// degree (largest first); 2 = DSATUR; 3 = first fit in order of decreasing
// |c_j|.  Groups in order of creation, terms inside a group in input order.
std::vector<std::vector<int64_t>> partition_terms(int64_t m, const uint64_t *x, const uint64_t *z,
                                                  const double *c, int grouping);

// Returns an empty string on success, else the reason of failure.
std::string make_plan(int n, int64_t m, const uint64_t *x, const uint64_t *z,
                      int skip_rule, Plan &out, int grouping = 0, const double *c = nullptr);

// ------------------------------------------------------------ flat ops

// One Trotter step (or any circuit) as a flat list of state-vector ops.
enum OpKind : int32_t {
    OK_H = 0,      // Hadamard on qubit q (unnormalised butterfly; 1/sqrt2 deferred)
    OK_S = 1,      // S on qubit q
    OK_SDG = 2,    // S^dag on qubit q
    OK_CNOT = 3,   // CNOT(c = q, t = q2)
    OK_PHASE = 4,  // diagonal quarter-turn layer: index into phase table
    OK_DIAG = 5,   // group exponential: index into diag table
    OK_Z = 6,      // Pauli Z (= S S) on qubit q
    OK_X = 7,      // Pauli X on qubit q
    OK_C1 = 8      // canonical one-qubit Clifford on qubit q, parameters in q2 (c1_* below)
};

inline SD_HD bool is_1q(int32_t kind) {
    return kind == OK_H || kind == OK_S || kind == OK_SDG || kind == OK_Z || kind == OK_X ||
           kind == OK_C1;
}



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

// Merge every run of one-qubit gates on a qubit (no other op on that qubit
// in between) into the canonical form S^a, X S^a or S^b H S^a of its
// product (at most one Hadamard), and carry the dropped global phase
// (a multiple of pi/4) exactly as a mask-0 term of the first group
// exponential, or of an appended one if the circuit has none.
void canonicalize_1q(Circuit &c, int n);

// ------------------------------------------------------------ pass schedule


struct Schedule {
    int K = 0;
    int c = 0;            // low qubits that must be lanes for coalesced loads/stores
    // 1: tile position 0 (qubit 0) is register slot 0 in every round, so that
    // a thread's amplitudes pair up along it (packed two-amplitude layout).
    int pin0 = 0;
    // Prefetch buffers of the passes compiled at run time (1 or 2; 2 only
    // where the shared memory allows it).
    int prefetch = 1;
    std::vector<DevPass> passes;
    std::vector<DevRound> rounds;
    std::vector<DevOp> ops;
    std::vector<DevPerm> perms;
    std::vector<DevDiag> diags;
    std::vector<DevPhase> phases;
    std::vector<uint64_t> term_mo;      // diag term pool: mask on the outer qubits
    std::vector<DevSlot> slots;         // diag term slots (class, mask on the round's fixed positions)
    std::vector<int64_t> term_q;        // diag term pool: Q0.64 turns
    std::vector<uint64_t> cst_mo;       // tile-constant terms: outer mask
    std::vector<int64_t> cst_q;         // tile-constant terms: Q0.64 turns
    std::vector<uint64_t> mask_pool;    // phase adjacency pool
    int64_t diag_passes = 0;
};

// Schedule a circuit on n qubits into tile passes of 2^K amplitudes;
// c = log2(128 bytes / amplitude size).  pin0: keep tile position 0 in
// register slot 0 of every round (see Schedule::pin0).  Returns "" or an
// error.
std::string schedule_circuit(const Circuit &circ, int n, int K, int c, Schedule &out, bool pin0 = false,
                             bool tail_deferral = false);

// Swizzle column of tile position p (identity on the low c bits).
uint32_t swizzle_col(int p, int c);

// Bank bits of the paired exchange layout: 16-byte units of two amplitudes
// that differ in tile position 0, 8 units per 128-byte row.
constexpr int kPairBankBits = 3;

// Swizzle column, in units, of tile position p >= 1 in the paired layout
// (identity on positions 1..kPairBankBits).
uint32_t pair_swizzle_col(int p);

}  // namespace sd
