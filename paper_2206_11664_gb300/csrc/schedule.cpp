// Circuit building (Eq. trotter_simul_diag: C_g, exp(-i Lambda_g dt), C_g^dag
// per group, with the layer structure of Fig. clifford_block) and the pass
// scheduler that packs the resulting op stream into tile passes over the
// state vector.
//
// A pass streams the state once through HBM in tiles of 2^K amplitudes.  A
// tile is the set of indices that agree on every bit outside K "tile
// qubits"; the lowest c qubits are always tile qubits so that loads and
// stores move whole 128-byte lines.  Inside a pass, a thread block holds a
// tile with 16 amplitudes per thread; a "round" assigns 4 tile positions to
// the thread's registers, 5 to the warp lanes and the rest to the warps.
// One-qubit gates are applied in registers on register positions; diagonal
// ops (S/CZ layers, group exponentials) apply in any round; a run of CNOTs
// whose targets are tile qubits is a permutation of the tile applied while
// the registers are written back to shared memory between rounds.
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <set>

#include "sd_internal.h"

namespace sd {

int64_t turns_q64(double t) {
    double f = t - std::nearbyint(t);   // in [-0.5, 0.5]
    if (f >= 0.5) f -= 1.0;
    if (f < -0.5) f += 1.0;
    // f * 2^64 lies in [-2^63, 2^63): exact split into two 32-bit halves.
    double s = std::ldexp(f, 32);              // [-2^31, 2^31)
    double hi = std::floor(s);
    double lo = std::ldexp(s - hi, 32);        // [0, 2^32)
    int64_t h = (int64_t)hi;
    uint64_t l = (uint64_t)std::nearbyint(lo);
    uint64_t v = ((uint64_t)h << 32) + l;      // wraps mod 2^64
    return (int64_t)v;
}

uint32_t swizzle_col(int p, int c) {
    if (p < c) return 1u << p;
    uint32_t span = (1u << c) - 1u;
    uint32_t s = 1u + (uint32_t)((p - c) % (int)span);
    return (1u << p) | s;
}

uint32_t pair_swizzle_col(int p) {
    const int b = p - 1;   // unit index bit of position p
    if (b < kPairBankBits) return 1u << b;
    const uint32_t span = (1u << kPairBankBits) - 1u;
    return (1u << b) | (1u + (uint32_t)((b - kPairBankBits) % (int)span));
}

namespace {

void layers(const GroupPlan &gp, std::vector<Gate> &ua, std::vector<Gate> &cn,
            std::vector<Gate> &scz, std::vector<Gate> &hb) {
    for (size_t k = 0; k < gp.gates.size(); k++) {
        switch (gp.stage[k]) {
        case ST_PRE:
        case ST_ALG2: ua.push_back(gp.gates[k]); break;
        case ST_ALG3: cn.push_back(gp.gates[k]); break;
        case ST_ALG4: scz.push_back(gp.gates[k]); break;
        default: hb.push_back(gp.gates[k]); break;
        }
    }
}

int add_phase(Circuit &c, int n, const std::vector<Gate> &scz, bool inverse) {
    if (scz.empty()) return -1;
    PhaseLayer L;
    L.adj.assign(n, 0);
    L.up.assign(n, 0);
    for (auto &g : scz) {
        if (g.kind == G_S) {
            if (inverse) L.sm ^= uint64_t(1) << g.a; else L.sp ^= uint64_t(1) << g.a;
        } else {
            int a = std::min(g.a, g.b), b = std::max(g.a, g.b);
            L.adj[a] ^= uint64_t(1) << b;
            L.adj[b] ^= uint64_t(1) << a;
            L.up[a] ^= uint64_t(1) << b;
        }
    }
    uint64_t sup = L.sp | L.sm;
    for (int q = 0; q < n; q++)
        if (L.adj[q]) sup |= uint64_t(1) << q;
    if (sup == 0) return -1;
    c.phases.push_back(L);
    FlatOp op{OK_PHASE, -1, -1, (int32_t)c.phases.size() - 1, sup};
    c.ops.push_back(op);
    return (int)c.phases.size() - 1;
}

void add_1q(Circuit &c, const Gate &g, bool inverse) {
    int32_t k = g.kind == G_H ? OK_H : (inverse ? OK_SDG : OK_S);
    c.ops.push_back(FlatOp{k, g.a, -1, -1, uint64_t(1) << g.a});
}

void add_cnot(Circuit &c, const Gate &g) {
    c.ops.push_back(FlatOp{OK_CNOT, g.a, g.b, -1, (uint64_t(1) << g.a) | (uint64_t(1) << g.b)});
}

}  // namespace

void append_clifford(const Plan &plan, int g, bool forward, Circuit &c) {
    std::vector<Gate> ua, cn, scz, hb;
    layers(plan.groups[g], ua, cn, scz, hb);
    if (forward) {
        for (auto &x : ua) add_1q(c, x, false);
        for (auto &x : cn) add_cnot(c, x);
        add_phase(c, plan.n, scz, false);
        for (auto &x : hb) add_1q(c, x, false);
    } else {
        for (auto it = hb.rbegin(); it != hb.rend(); ++it) add_1q(c, *it, true);
        add_phase(c, plan.n, scz, true);
        for (auto it = cn.rbegin(); it != cn.rend(); ++it) add_cnot(c, *it);
        for (auto it = ua.rbegin(); it != ua.rend(); ++it) add_1q(c, *it, true);
    }
}

void append_group_step(const Plan &plan, int g, double f, double dt,
                       const std::vector<double> &coeffs, Circuit &c) {
    const GroupPlan &gp = plan.groups[g];
    append_clifford(plan, g, true, c);
    DiagLayer D;
    D.group = g;
    D.frac = f;
    uint64_t sup = 0;
    const double inv2pi = 1.0 / (2.0 * M_PI);
    for (size_t k = 0; k < gp.terms.size(); k++) {
        double a = f * dt * coeffs[gp.terms[k]];
        if (gp.signs[k]) a = -a;
        D.masks.push_back(gp.masks[k]);
        D.q.push_back(turns_q64(a * inv2pi));
        sup |= gp.masks[k];
    }
    c.diags.push_back(std::move(D));
    c.ops.push_back(FlatOp{OK_DIAG, -1, -1, (int32_t)c.diags.size() - 1, sup});
    append_clifford(plan, g, false, c);
}

// ------------------------------------------------------------ 1q canonical form

namespace {

using C2 = std::complex<double>;
struct M2 {
    C2 a, b, c, d;  // [[a, b], [c, d]]
};
M2 mul(const M2 &x, const M2 &y) {  // x * y
    return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c,
            x.c * y.b + x.d * y.d};
}
M2 spow(int a);
M2 gate_matrix(int32_t kind, int32_t par = 0);
M2 c1_matrix(int32_t v) {
    M2 m = spow(c1_a(v));
    if (c1_had(v)) m = mul(spow(c1_b(v)), mul(gate_matrix(OK_H), m));
    else if (c1_x(v)) m = mul(gate_matrix(OK_X), m);
    return m;
}
M2 gate_matrix(int32_t kind, int32_t par) {
    const double r = std::sqrt(0.5);
    if (kind == OK_C1) return c1_matrix(par);
    const C2 I(0, 1);
    switch (kind) {
    case OK_H: return {r, r, r, -r};
    case OK_S: return {1.0, 0.0, 0.0, I};
    case OK_SDG: return {1.0, 0.0, 0.0, -I};
    case OK_Z: return {1.0, 0.0, 0.0, -1.0};
    default: return {0.0, 1.0, 1.0, 0.0};  // OK_X
    }
}
M2 spow(int a) {
    const C2 p = std::pow(C2(0, 1), a);
    return {1.0, 0.0, 0.0, p};
}
bool close(const M2 &x, const M2 &y, C2 ph) {
    auto d = [&](C2 u, C2 v) { return std::abs(u - ph * v); };
    return d(x.a, y.a) + d(x.b, y.b) + d(x.c, y.c) + d(x.d, y.d) < 1e-9;
}
void emit_c1(std::vector<FlatOp> &out, int q, int had, int a, int b, int x) {
    if (!had && a == 0 && x == 0) return;   // identity
    out.push_back(FlatOp{OK_C1, q, c1_pack(had, a, b, x), -1, uint64_t(1) << q});
}
// Canonical op (application order) and phase (eighth turns) of M.
void canonical(const M2 &M, int q, std::vector<FlatOp> &out, int &phase8) {
    const M2 H = gate_matrix(OK_H), X = gate_matrix(OK_X);
    for (int k = 0; k < 8; k++) {
        const C2 ph = std::polar(1.0, M_PI * k / 4.0);
        for (int a = 0; a < 4; a++) {
            if (close(M, spow(a), ph)) {
                emit_c1(out, q, 0, a, 0, 0);
                phase8 += k;
                return;
            }
            if (close(M, mul(X, spow(a)), ph)) {
                emit_c1(out, q, 0, a, 0, 1);
                phase8 += k;
                return;
            }
            for (int b = 0; b < 4; b++)
                if (close(M, mul(spow(b), mul(H, spow(a))), ph)) {
                    emit_c1(out, q, 1, a, b, 0);
                    phase8 += k;
                    return;
                }
        }
    }
}

}  // namespace

void canonicalize_1q(Circuit &c, int n) {
    std::vector<std::vector<int>> run(n);   // pending op indices per qubit
    std::vector<std::vector<FlatOp>> repl(c.ops.size());
    std::vector<char> drop(c.ops.size(), 0);
    int phase8 = 0;
    auto flush = [&](int q) {
        if (run[q].empty()) return;
        M2 M = {1.0, 0.0, 0.0, 1.0};
        for (int j : run[q]) M = mul(gate_matrix(c.ops[j].kind, c.ops[j].q2), M);
        for (int j : run[q]) drop[j] = 1;
        canonical(M, q, repl[run[q].front()], phase8);
        run[q].clear();
    };
    for (size_t j = 0; j < c.ops.size(); j++) {
        const FlatOp &op = c.ops[j];
        if (is_1q(op.kind)) {
            run[op.q].push_back((int)j);
            continue;
        }
        uint64_t touched = op.kind == OK_CNOT ? ((uint64_t(1) << op.q) | (uint64_t(1) << op.q2))
                                               : op.support;
        for (int q = 0; q < n; q++)
            if ((touched >> q) & 1) flush(q);
    }
    for (int q = 0; q < n; q++) flush(q);
    std::vector<FlatOp> ops;
    for (size_t j = 0; j < c.ops.size(); j++) {
        for (auto &r : repl[j]) ops.push_back(r);
        if (!drop[j]) ops.push_back(c.ops[j]);
    }
    c.ops.swap(ops);
    phase8 &= 7;
    if (phase8 == 0) return;
    // e^{i pi k/4} = exp(-2 pi i (-k/8)): a constant term of -k/8 turn
    const int64_t q0 = (int64_t)(uint64_t(8 - phase8) << 61);
    for (auto &op : c.ops)
        if (op.kind == OK_DIAG) {
            c.diags[op.idx].masks.push_back(0);
            c.diags[op.idx].q.push_back(q0);
            return;
        }
    DiagLayer D;
    D.group = -1;
    D.frac = 0.0;
    D.masks.push_back(0);
    D.q.push_back(q0);
    c.diags.push_back(D);
    c.ops.push_back(FlatOp{OK_DIAG, -1, -1, (int32_t)c.diags.size() - 1, 0});
}

// ------------------------------------------------------------ scheduler

namespace {

struct SchedState {
    const Circuit &circ;
    int n, K, c;
    std::vector<std::vector<int>> preds;
    std::vector<int> done_round;  // -1 = not done; else global round id
    std::vector<char> is_cnot;
    explicit SchedState(const Circuit &cc) : circ(cc) {}
};

std::vector<int> wires_of(const FlatOp &op, int n) {
    std::vector<int> w;
    if (op.kind == OK_PHASE || op.kind == OK_DIAG) {
        for (int q = 0; q < n; q++)
            if ((op.support >> q) & 1) w.push_back(q);
    } else {
        w.push_back(op.q);
        if (op.kind == OK_CNOT) w.push_back(op.q2);
    }
    return w;
}

int rank_cols(const std::vector<uint32_t> &cols, int c) {
    std::vector<uint32_t> v;
    for (auto x : cols) v.push_back(x & ((1u << c) - 1u));
    int r = 0;
    for (int b = 0; b < c; b++) {
        int p = -1;
        for (int i = r; i < (int)v.size(); i++)
            if ((v[i] >> b) & 1) { p = i; break; }
        if (p < 0) continue;
        std::swap(v[r], v[p]);
        for (int i = 0; i < (int)v.size(); i++)
            if (i != r && ((v[i] >> b) & 1)) v[i] ^= v[r];
        r++;
    }
    return r;
}

// Lane/warp assignment of the non-register tile positions.  With pin0 the
// global load/store rounds put positions 1..c-1 on the low lanes (with
// position 0 in registers, 8 lanes then cover 128 contiguous bytes), and the
// other rounds choose lanes whose paired-layout columns span its bank bits.
void assign_layout(DevRound &R, int K, int c, bool global_io, bool pin0) {
    std::vector<int> rest;
    for (int p = 0; p < K; p++) {
        bool isreg = false;
        for (int i = 0; i < 4; i++) isreg |= R.reg_pos[i] == p;
        if (!isreg) rest.push_back(p);
    }
    // Lane bits 0..c-1 must span the c bank-selecting bits of the swizzled
    // address (conflict-free shared accesses; coalesced global accesses in
    // load/store rounds, where they are tile positions 0..c-1).
    std::vector<int> lanes;
    if (pin0 && global_io) {
        for (int p = 1; p < c; p++) lanes.push_back(p);
        for (int p : rest)
            if ((int)lanes.size() < kLaneBits && p >= c) lanes.push_back(p);
    } else if (pin0) {
        std::vector<uint32_t> cols;
        for (int p : rest) {
            if ((int)lanes.size() >= kPairBankBits) break;
            std::vector<uint32_t> t = cols;
            t.push_back(pair_swizzle_col(p));
            if (rank_cols(t, kPairBankBits) > rank_cols(cols, kPairBankBits)) {
                lanes.push_back(p);
                cols = t;
            }
        }
        for (int p : rest)
            if ((int)lanes.size() < kLaneBits &&
                std::find(lanes.begin(), lanes.end(), p) == lanes.end())
                lanes.push_back(p);
    } else if (global_io) {
        for (int p = 0; p < c; p++) lanes.push_back(p);
        for (int p : rest)
            if ((int)lanes.size() < kLaneBits && p >= c) lanes.push_back(p);
    } else {
        std::vector<uint32_t> cols;
        for (int p : rest) {
            if ((int)lanes.size() >= c) break;
            std::vector<uint32_t> t = cols;
            t.push_back(swizzle_col(p, c));
            if (rank_cols(t, c) > rank_cols(cols, c)) {
                lanes.push_back(p);
                cols = t;
            }
        }
        for (int p : rest)
            if ((int)lanes.size() < kLaneBits &&
                std::find(lanes.begin(), lanes.end(), p) == lanes.end())
                lanes.push_back(p);
    }
    for (int i = 0; i < kLaneBits; i++) R.lane_pos[i] = (uint8_t)lanes[i];
    int wi = 0;
    for (int p : rest)
        if (std::find(lanes.begin(), lanes.end(), p) == lanes.end()) R.warp_pos[wi++] = (uint8_t)p;
    for (; wi < 7; wi++) R.warp_pos[wi] = 0xff;
}

}  // namespace

std::string schedule_circuit(const Circuit &circ, int n, int K, int c, Schedule &S, bool pin0, bool tail_deferral) {
    S = Schedule{};
    S.K = K;
    S.c = c;
    S.pin0 = pin0 ? 1 : 0;
    if (K < kRegBits + kLaneBits || K > 13 || n < K) return "invalid tile size";
    const int N = (int)circ.ops.size();
    // Dependencies, per wire.  Diagonal ops commute with each other; CNOTs
    // that share a wire in the same role (all controls, or all targets)
    // commute too, so such a run of CNOTs may execute in any order, each after
    // what preceded the run.  Everything else keeps program order on a wire.
    std::vector<std::vector<int>> preds(N);
    {
        struct Wire {
            std::vector<int> run;      // current run: CNOTs of one role, or one other op
            int role = 0;              // 1: run of controls, 2: run of targets, 0: other
            std::vector<int> before;   // what the run follows
            std::vector<int> diags;    // diagonal ops since the run began
        };
        std::vector<Wire> W(n);
        for (int j = 0; j < N; j++) {
            const FlatOp &op = circ.ops[j];
            const bool isdiag = op.kind == OK_PHASE || op.kind == OK_DIAG;
            std::set<int> p;
            if (isdiag) {
                for (int w : wires_of(op, n)) p.insert(W[w].run.begin(), W[w].run.end());
                for (int w : wires_of(op, n)) W[w].diags.push_back(j);
            } else {
                std::vector<std::pair<int, int>> roles;   // (wire, role)
                if (op.kind == OK_CNOT) roles = {{op.q, 1}, {op.q2, 2}};
                else roles = {{op.q, 0}};
                for (auto &wr : roles) {
                    const Wire &s = W[wr.first];
                    if (wr.second != 0 && s.role == wr.second) p.insert(s.before.begin(), s.before.end());
                    else p.insert(s.run.begin(), s.run.end());
                    p.insert(s.diags.begin(), s.diags.end());
                }
                for (auto &wr : roles) {
                    Wire &s = W[wr.first];
                    if (wr.second != 0 && s.role == wr.second) {
                        s.run.push_back(j);
                    } else {
                        s.before = s.run;
                        s.before.insert(s.before.end(), s.diags.begin(), s.diags.end());
                        s.run.assign(1, j);
                        s.role = wr.second;
                        s.diags.clear();
                    }
                }
            }
            preds[j].assign(p.begin(), p.end());
        }
    }
    std::vector<int> done(N, -1);   // global round id in which the op ran
    int round_id = 0;
    int first = 0;
    std::map<std::pair<int, int>, int64_t> adj_base;  // phase idx -> pool bases
    auto ensure_phase_pool = [&](int idx) {
        auto key = std::make_pair(idx, 0);
        auto it = adj_base.find(key);
        if (it != adj_base.end()) return it->second;
        int64_t b = (int64_t)S.mask_pool.size();
        const PhaseLayer &L = circ.phases[idx];
        for (int q = 0; q < n; q++) S.mask_pool.push_back(L.adj[q]);
        for (int q = 0; q < n; q++) S.mask_pool.push_back(L.up[q]);
        adj_base[key] = b;
        return b;
    };

    int guard = 0;
    while (first < N) {
        if (++guard > 4 * N + 16) return "scheduler made no progress";
        // -------- choose the tile qubits
        std::vector<int> need(n, INT32_MAX);
        for (int j = first; j < N; j++) {
            if (done[j] >= 0) continue;
            const FlatOp &op = circ.ops[j];
            int q = -1;
            if (is_1q(op.kind)) q = op.q;
            else if (op.kind == OK_CNOT) q = op.q2;
            if (q >= 0 && need[q] == INT32_MAX) need[q] = j;
        }
        std::vector<int> cand;
        for (int q = c; q < n; q++) cand.push_back(q);
        std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) { return need[a] < need[b]; });
        std::vector<int> tq;
        for (int q = 0; q < c; q++) tq.push_back(q);
        std::vector<int> hi(cand.begin(), cand.begin() + (K - c));
        std::sort(hi.begin(), hi.end());
        for (int q : hi) tq.push_back(q);
        int pos_of[64];
        for (int q = 0; q < 64; q++) pos_of[q] = -1;
        for (int p = 0; p < K; p++) pos_of[tq[p]] = p;

        DevPass P{};
        P.round_begin = (int)S.rounds.size();
        P.term_begin = (int)S.term_q.size();
        const int pass_op_begin = (int)S.ops.size();
        for (int p = 0; p < K; p++) P.tile_bits[p] = (uint8_t)tq[p];
        int no = 0;
        for (int q = 0; q < n; q++)
            if (pos_of[q] < 0) P.outer_bits[no++] = (uint8_t)q;
        P.n_outer = no;
        int h_count = 0;
        int diag_op_index = -1;

        // Another pass follows if a pending gate acts on a qubit outside this
        // tile.  Then, once this pass has applied a group exponential, the
        // gates that follow it on the low (coalescing) qubits are left to the
        // next pass, which holds those qubits too: exponential passes are
        // bound by instruction issue, the passes between them by memory.
        bool more_passes = false;
        for (int j = first; j < N && !more_passes; j++) {
            if (done[j] >= 0) continue;
            const FlatOp &op = circ.ops[j];
            if (is_1q(op.kind)) more_passes = pos_of[op.q] < 0;
            else if (op.kind == OK_CNOT) more_passes = pos_of[op.q2] < 0 || pos_of[op.q] < 0;
        }
        auto deferred = [&](const FlatOp &op) {
            return more_passes && diag_op_index >= 0 && is_1q(op.kind) && op.q < c && !(pin0 && op.q == 0);
        };
        int nr = 0;
        for (;;) {
            bool is_load = nr == 0;
            // -------- register positions for this round
            // score: (first pending one-qubit op on the position, or INT32_MAX if
            // none is ready -- all its predecessors done -- yet)
            std::vector<std::pair<int, int>> score;
            for (int p = pin0 ? 1 : 0; p < K; p++) {
                if (is_load && p < c) continue;
                int best = INT32_MAX;
                for (int j = first; j < N; j++) {
                    if (done[j] >= 0) continue;
                    const FlatOp &op = circ.ops[j];
                    if (is_1q(op.kind) && op.q == tq[p]) {
                        bool ready = !deferred(op);
                        for (int pr : preds[j])
                            if (done[pr] < 0) { ready = false; break; }
                        if (ready) best = j;
                        break;
                    }
                }
                score.push_back({best, p});
            }
            std::stable_sort(score.begin(), score.end());
            DevRound R{};
            std::vector<int> regs;
            if (pin0) regs.push_back(0);
            // The low positions (< c) are lanes in the load and store layouts, so
            // their gates need a middle round: when one of them is due, take all
            // low positions with pending gates together, then the most urgent others.
            // Low positions are taken all together or not at all, and before the
            // last high positions so that the final round can also store.
            int lows_pending = 0, highs_pending = 0;
            for (auto &sc : score)
                if (sc.first != INT32_MAX) (sc.second < c ? lows_pending : highs_pending)++;
            const int free_slots = pin0 ? 3 : 4;
            const bool low_round = !is_load && lows_pending > 0 &&
                                   ((score[0].first != INT32_MAX && score[0].second < c) ||
                                    highs_pending <= free_slots);
            if (low_round)
                for (auto &sc : score)
                    if (sc.second < c && sc.first != INT32_MAX && (int)regs.size() < 4) regs.push_back(sc.second);
            for (auto &sc : score)
                if ((int)regs.size() < 4 && sc.second >= c &&
                    std::find(regs.begin(), regs.end(), sc.second) == regs.end())
                    regs.push_back(sc.second);
            for (auto &sc : score)   // only if fewer than 4 high positions exist
                if ((int)regs.size() < 4 && std::find(regs.begin(), regs.end(), sc.second) == regs.end())
                    regs.push_back(sc.second);
            std::sort(regs.begin(), regs.end());
            for (int i = 0; i < 4; i++) R.reg_pos[i] = (uint8_t)regs[i];
            R.perm = -1;
            R.flags = is_load ? 1 : 0;
            R.op_begin = (int)S.ops.size();
            R.slot_begin = (int)S.slots.size();
            R.diag_begin = (int)S.diags.size();
            R.n_diag = 0;
            // -------- execute what is ready
            std::vector<Gate> perm_cnots;
            int executed = 0;
            bool progress = true;
            while (progress) {
                progress = false;
                for (int j = first; j < N; j++) {
                    if (done[j] >= 0) continue;
                    if ((int)S.ops.size() - pass_op_begin >= kMaxPassOps - 1) break;
                    const FlatOp &op = circ.ops[j];
                    bool ok = true;
                    for (int p : preds[j]) {
                        if (done[p] < 0) { ok = false; break; }
                        // ops after a CNOT of this round's permutation wait for the next round
                        if (done[p] == round_id && circ.ops[p].kind == OK_CNOT && op.kind != OK_CNOT) {
                            ok = false;
                            break;
                        }
                    }
                    if (!ok) continue;
                    int slot = -1;
                    if (is_1q(op.kind)) {
                        int p = pos_of[op.q];
                        if (p < 0 || deferred(op)) continue;
                        for (int i = 0; i < 4; i++)
                            if (R.reg_pos[i] == p) slot = i;
                        if (slot < 0) continue;
                        if (!perm_cnots.empty()) {
                            // a 1q gate sharing a wire with a queued CNOT must precede it
                            bool clash = false;
                            for (auto &g : perm_cnots) clash |= g.a == op.q || g.b == op.q;
                            if (clash) continue;
                        }
                        int32_t par;
                        switch (op.kind) {
                        case OK_H: par = c1_pack(1, 0, 0, 0); break;
                        case OK_S: par = c1_pack(0, 1, 0, 0); break;
                        case OK_Z: par = c1_pack(0, 2, 0, 0); break;
                        case OK_SDG: par = c1_pack(0, 3, 0, 0); break;
                        case OK_X: par = c1_pack(0, 0, 0, 1); break;
                        default: par = op.q2; break;
                        }
                        DevOp d{c1_had(par) ? D_HAD : D_MONO, slot, par, 0};
                        S.ops.push_back(d);
                        if (c1_had(par)) h_count++;
                    } else if (op.kind == OK_CNOT) {
                        if (pos_of[op.q2] < 0) continue;
                        perm_cnots.push_back(Gate{G_CNOT, op.q, op.q2});
                    } else if (op.kind == OK_PHASE) {
                        if (!perm_cnots.empty()) {
                            bool clash = false;
                            for (auto &g : perm_cnots)
                                clash |= ((op.support >> g.a) & 1) || ((op.support >> g.b) & 1);
                            if (clash) continue;
                        }
                        const PhaseLayer &L = circ.phases[op.idx];
                        DevPhase ph{};
                        ph.sp = L.sp;
                        ph.sm = L.sm;
                        int64_t b = ensure_phase_pool(op.idx);
                        ph.adj_base = b;
                        ph.up_base = b + n;
                        ph.n = n;
                        for (int i = 0; i < 4; i++) {
                            int qi = tq[R.reg_pos[i]];
                            ph.lin_s[i] = ((L.sp >> qi) & 1) ? 1 : (((L.sm >> qi) & 1) ? -1 : 0);
                        }
                        ph.quad = 0;
                        for (int i = 0; i < 4; i++)
                            for (int k = i + 1; k < 4; k++) {
                                int qi = tq[R.reg_pos[i]], qk = tq[R.reg_pos[k]];
                                if ((L.adj[qi] >> qk) & 1) ph.quad |= 1 << (i * 4 + k);
                            }
                        S.phases.push_back(ph);
                        S.ops.push_back(DevOp{D_PHASE, 0, (int32_t)S.phases.size() - 1, 0});
                    } else {  // OK_DIAG
                        if (!perm_cnots.empty()) {
                            bool clash = false;
                            for (auto &g : perm_cnots)
                                clash |= ((op.support >> g.a) & 1) || ((op.support >> g.b) & 1);
                            if (clash) continue;
                        }
                        const DiagLayer &D = circ.diags[op.idx];
                        uint64_t regmask = 0;
                        int gq[4];
                        for (int i = 0; i < 4; i++) {
                            gq[i] = tq[R.reg_pos[i]];
                            regmask |= uint64_t(1) << gq[i];
                        }
                        std::vector<std::vector<int>> cls(16);
                        for (size_t t = 0; t < D.masks.size(); t++) {
                            int u = 0;
                            for (int i = 0; i < 4; i++) u |= int((D.masks[t] >> gq[i]) & 1) << i;
                            cls[u].push_back((int)t);
                        }
                        DevDiag dd{};
                        dd.cst = -1;
                        uint64_t outer_mask = 0, tile_mask = 0;
                        for (int k = 0; k < no; k++) outer_mask |= uint64_t(1) << P.outer_bits[k];
                        for (int p = 0; p < K; p++) tile_mask |= uint64_t(1) << tq[p];
                        int slot = -1;
                        for (int c2 = 0; c2 < 4; c2++)
                            if (R.cst_count[c2] == 0) { slot = c2; break; }
                        if (slot >= 0) {
                            R.cst_begin[slot] = (int)S.cst_q.size();
                            for (int t : cls[0])
                                if (!(D.masks[t] & tile_mask)) {
                                    S.cst_mo.push_back(D.masks[t]);
                                    S.cst_q.push_back(D.q[t]);
                                }
                            R.cst_count[slot] = (int)S.cst_q.size() - R.cst_begin[slot];
                            if (R.cst_count[slot] > 0) dd.cst = slot;
                        }
                        if (R.n_diag == 0) R.diag_begin = (int)S.diags.size();
                        dd.tot = 16 * R.n_diag++;
                        // per class, the terms grouped by their mask on the fixed positions
                        std::vector<std::vector<std::pair<uint32_t, int>>> byc(16);
                        for (int s = 0; s < 16; s++) {
                            for (int t : cls[s]) {
                                if (dd.cst >= 0 && s == 0 && !(D.masks[t] & tile_mask)) continue;
                                uint32_t ml = 0;
                                for (int p = 0; p < K; p++)
                                    if (!((regmask >> tq[p]) & 1) && ((D.masks[t] >> tq[p]) & 1))
                                        ml |= 1u << p;
                                byc[s].push_back({ml, t});
                            }
                            std::stable_sort(byc[s].begin(), byc[s].end(),
                                             [](const std::pair<uint32_t, int> &a,
                                                const std::pair<uint32_t, int> &b) { return a.first < b.first; });
                        }
                        auto emit = [&](int s, size_t i0, size_t i1) {
                            DevSlot sl{(int32_t)S.term_q.size(), (int32_t)(i1 - i0), byc[s][i0].first, 0};
                            for (size_t i = i0; i < i1; i++) {
                                const int t = byc[s][i].second;
                                S.term_mo.push_back(D.masks[t] & outer_mask);
                                S.term_q.push_back(D.q[t]);
                            }
                            S.slots.push_back(sl);
                        };
                        for (int s = 0; s < 16; s++) {       // slots with a fixed-position mask
                            dd.off[s] = (int)S.slots.size() - R.slot_begin;
                            size_t i = 0;
                            while (i < byc[s].size() && byc[s][i].first == 0) i++;
                            while (i < byc[s].size()) {
                                size_t e = i;
                                while (e < byc[s].size() && byc[s][e].first == byc[s][i].first) e++;
                                emit(s, i, e);
                                i = e;
                            }
                        }
                        dd.off[16] = (int)S.slots.size() - R.slot_begin;
                        for (int s = 0; s < 16; s++) {       // slots constant over the thread's fixed positions
                            dd.zs[s] = -1;
                            size_t e = 0;
                            while (e < byc[s].size() && byc[s][e].first == 0) e++;
                            if (e > 0) {
                                dd.zs[s] = (int)S.slots.size() - R.slot_begin;
                                emit(s, 0, e);
                            }
                        }
                        S.diags.push_back(dd);
                        S.ops.push_back(DevOp{D_DIAG, 0, (int32_t)S.diags.size() - 1, 0});
                        if (diag_op_index < 0) diag_op_index = (int)S.ops.size() - 1;
                    }
                    done[j] = round_id;
                    executed++;
                    progress = true;
                }
            }
            while (first < N && done[first] >= 0) first++;
            R.op_end = (int)S.ops.size();
            R.slot_count = (int)S.slots.size() - R.slot_begin;
            if (!perm_cnots.empty()) {
                DevPerm pm{};
                for (int p = 0; p < K; p++) {
                    uint64_t v = uint64_t(1) << tq[p];
                    for (auto &g : perm_cnots) v ^= ((v >> g.a) & 1) << g.b;
                    uint32_t l = 0;
                    for (int p2 = 0; p2 < K; p2++) l |= uint32_t((v >> tq[p2]) & 1) << p2;
                    pm.col[p] = l;
                }
                for (int k = 0; k < no; k++) {
                    uint64_t v = uint64_t(1) << P.outer_bits[k];
                    for (auto &g : perm_cnots) v ^= ((v >> g.a) & 1) << g.b;
                    uint32_t l = 0;
                    for (int p2 = 0; p2 < K; p2++) l |= uint32_t((v >> tq[p2]) & 1) << p2;
                    pm.ocol[k] = l;
                }
                S.perms.push_back(pm);
                R.perm = (int)S.perms.size() - 1;
            }
            bool useful = executed > 0 || is_load;
            if (!useful) break;
            // A last round that would carry a single one-qubit gate, when another
            // pass follows anyway and the previous round can store: leave that
            // gate to the next pass instead of paying a round (an exchange and
            // a block barrier per tile) for it.
            if (tail_deferral && nr >= 2 && more_passes && executed == 1 && R.n_diag == 0 && perm_cnots.empty() &&
                (int)S.ops.size() == R.op_begin + 1 &&
                (S.ops.back().kind == D_HAD || S.ops.back().kind == D_MONO)) {
                const DevRound &prev = S.rounds.back();
                bool can_store = prev.perm < 0;
                for (int i = pin0 ? 1 : 0; i < 4; i++) can_store &= prev.reg_pos[i] >= c;
                if (can_store) {
                    if (S.ops.back().kind == D_HAD) h_count--;
                    S.ops.pop_back();
                    for (int j = 0; j < N; j++)
                        if (done[j] == round_id) done[j] = -1;
                    first = 0;
                    while (first < N && done[first] >= 0) first++;
                    break;
                }
            }
            S.rounds.push_back(R);
            nr++;
            round_id++;
            if (first >= N || nr >= 8) break;
        }
        // -------- the last round stores to global memory
        DevRound &last = S.rounds.back();
        bool store_ok = last.perm < 0;
        for (int i = pin0 ? 1 : 0; i < 4; i++) store_ok &= last.reg_pos[i] >= c;
        if (!store_ok) {
            DevRound R{};
            // register positions: the 4 lowest positions >= c (with pin0:
            // position 0 and the 3 lowest positions >= c)
            for (int i = 0; i < 4; i++) R.reg_pos[i] = (uint8_t)(c + i);
            if (pin0)
                for (int i = 0; i < 4; i++) R.reg_pos[i] = (uint8_t)(i == 0 ? 0 : c + i - 1);
            R.perm = -1;
            R.op_begin = R.op_end = (int)S.ops.size();
            R.slot_begin = (int)S.slots.size();
            R.slot_count = 0;
            R.diag_begin = (int)S.diags.size();
            R.n_diag = 0;
            R.flags = 0;
            S.rounds.push_back(R);
            nr++;
            round_id++;
        }
        S.rounds.back().flags |= 2;
        for (int r = P.round_begin; r < (int)S.rounds.size(); r++)
            assign_layout(S.rounds[r], K, c, (S.rounds[r].flags & 3) != 0, pin0);
        P.n_rounds = (int)S.rounds.size() - P.round_begin;
        P.max_stage = 0;
        P.max_tot = 0;
        for (int r = P.round_begin; r < (int)S.rounds.size(); r++) {
            P.max_stage = std::max(P.max_stage, S.rounds[r].slot_count);
            P.max_tot = std::max(P.max_tot, 16 * S.rounds[r].n_diag);
        }
        P.scale = std::ldexp(1.0, -(h_count / 2)) * ((h_count & 1) ? std::sqrt(0.5) : 1.0);
        if (diag_op_index >= 0) {
            P.scale_in_diag = 1;
            S.ops[diag_op_index].pad = 1;
            S.diag_passes++;
        }
        P.term_count = (int)S.term_q.size() - P.term_begin;
        P.term_cache = 0;
        if (P.term_count > 0 && P.term_count <= kTermCache) {
            P.term_cache = 1;
            if (pass_smem_bytes(P, size_t(128) >> c, K) > kTileSmemLimit) P.term_cache = 0;
        }
        S.passes.push_back(P);
    }
    return "";
}

}  // namespace sd
