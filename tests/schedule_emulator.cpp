// Host emulation of a tile-pass schedule, for the CPU tests.
//
// It plans and schedules a Trotter step with the library's own host code
// (planner.cpp, schedule.cpp). Then it executes the schedule on a complex128
// state with plain loops, following what the device passes do:
//   - tiles of 2^K amplitudes;
//   - rounds of one-qubit Cliffords on register positions;
//   - quarter-turn layers;
//   - group exponentials assembled from the staged term slots, tile constants
//     and class structure;
//   - tile permutations on the exchange;
//   - the deferred Hadamard scale.
// The result is written out, and tests/test_schedule_emulation.py compares it
// with the oracle.
//
// This checks the scheduler's encoding of the step: op placement, slot and
// class bookkeeping, permutation columns and scale folding. It needs no GPU.
// The device kernels implement the same semantics, and the GPU parity tests
// check them.
//
// A call of several steps is split as the library splits it: first order
// runs blocks of `reps` steps scheduled as one circuit, then single steps;
// second order opens with group 1's half step, runs the cores (the
// step with the half steps of group 1 that meet between consecutive steps
// merged) in blocks of `reps` and single cores, and closes with the last
// core, whose group 1 takes a half step.
//
// It also counts, for every round, whether the warps' accesses to the
// shared-memory exchange are free of bank conflicts (see bank_stats).
//
// Usage: schedule_emulator <input> <output>, or <input> - to schedule only
// (the input then ends before the state, and nothing is executed).
// The input is binary, in this order: int32 n, int64 m, int32 skip_rule,
// int32 K, int32 c (plus 16 to pin tile position 0 to register slot 0, the
// paired complex64 schedule; plus 32 to leave single-gate last rounds to the
// next pass; plus 64 to rotate by the complex64 passes' Q0.32 angles),
// int32 order, int32 reps, int64 steps, float64 dt,
// uint64 x[m], uint64 z[m], float64 coeffs[m], complex128 psi[2^n]. The
// output is complex128 psi[2^n].
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sd_internal.h"

namespace sd {
void set_last_error(const std::string &) {}
}  // namespace sd

using namespace sd;
using cd = std::complex<double>;

namespace {

int popc(uint64_t v) { return __builtin_popcountll(v); }

cd ipow(cd v, int k) {
    switch (k & 3) {
    case 1: return cd(-v.imag(), v.real());
    case 2: return -v;
    case 3: return cd(v.imag(), -v.real());
    default: return v;
    }
}

struct Emulator {
    int n;
    const Schedule &S;
    std::vector<cd> &psi;
    // Complex64 angles: the class sums rounded to Q0.32 (bias 2^31, then the
    // high word) and the Walsh-Hadamard transform in 32 bits, as the complex64
    // passes form them; q32err is the largest distance (in turns, mod 1) from
    // the exact Q0.64 angle.
    bool q32 = false;
    double q32err = 0.0;

    void run_pass(const DevPass &P) {
        const int K = S.K;
        const int T = 1 << K;
        std::vector<cd> a(T), b(T);
        std::vector<uint64_t> spread(T);
        for (int l = 0; l < T; l++) {
            uint64_t x = 0;
            for (int p = 0; p < K; p++)
                if ((l >> p) & 1) x |= uint64_t(1) << P.tile_bits[p];
            spread[l] = x;
        }
        const double pass_scale = P.scale_in_diag ? 1.0 : P.scale;
        for (uint64_t o = 0; o < (uint64_t(1) << P.n_outer); o++) {
            uint64_t xo = 0;
            for (int k = 0; k < P.n_outer; k++)
                if ((o >> k) & 1) xo |= uint64_t(1) << P.outer_bits[k];
            for (int l = 0; l < T; l++) a[l] = psi[xo | spread[l]];
            for (int r = P.round_begin; r < P.round_begin + P.n_rounds; r++) {
                const DevRound &R = S.rounds[r];
                for (int oi = R.op_begin; oi < R.op_end; oi++) op(S.ops[oi], R, P, xo, o, spread, a);
                if (R.perm >= 0) {
                    const DevPerm &pm = S.perms[R.perm];
                    for (int l = 0; l < T; l++) {
                        uint32_t t = 0;
                        for (int p = 0; p < K; p++)
                            if ((l >> p) & 1) t ^= pm.col[p];
                        for (int k = 0; k < P.n_outer; k++)
                            if ((o >> k) & 1) t ^= pm.ocol[k];
                        b[t] = a[l];
                    }
                    a.swap(b);
                }
            }
            for (int l = 0; l < T; l++) psi[xo | spread[l]] = a[l] * pass_scale;
        }
    }

    void op(const DevOp &op, const DevRound &R, const DevPass &P, uint64_t xo, uint64_t o,
            const std::vector<uint64_t> &spread, std::vector<cd> &a) {
        const int T = (int)a.size();
        if (op.kind == D_HAD || op.kind == D_MONO) {
            const int bit = 1 << R.reg_pos[op.slot];
            for (int l = 0; l < T; l++) {
                if (l & bit) continue;
                const cd u = a[l], w = ipow(a[l | bit], c1_a(op.arg));
                if (op.kind == D_HAD) {
                    a[l] = u + w;
                    a[l | bit] = ipow(u - w, c1_b(op.arg));
                } else if (c1_x(op.arg)) {
                    a[l] = w;
                    a[l | bit] = u;
                } else {
                    a[l | bit] = w;
                }
            }
        } else if (op.kind == D_PHASE) {
            const DevPhase &ph = S.phases[op.arg];
            for (int l = 0; l < T; l++) {
                const uint64_t x = xo | spread[l];
                int k = popc(x & ph.sp) - popc(x & ph.sm);
                int q = 0;
                for (int c = 0; c < n; c++)
                    if ((x >> c) & 1) q ^= popc(x & S.mask_pool[ph.up_base + c]) & 1;
                a[l] = ipow(a[l], k + 2 * q);
            }
        } else if (op.kind == D_DIAG) {
            const DevDiag &d = S.diags[op.arg];
            auto slot_sum = [&](int j) {   // signed angle sum of slot j over the tile's outer bits
                const DevSlot &sl = S.slots[R.slot_begin + j];
                uint64_t acc = 0;
                for (int t = sl.tb; t < sl.tb + sl.tn; t++) {
                    const uint64_t q = (uint64_t)S.term_q[t];
                    acc += (popc(xo & S.term_mo[t]) & 1) ? (0 - q) : q;
                }
                return acc;
            };
            uint64_t cst = 0;
            if (d.cst >= 0)
                for (int t = R.cst_begin[d.cst]; t < R.cst_begin[d.cst] + R.cst_count[d.cst]; t++) {
                    const uint64_t q = (uint64_t)S.cst_q[t];
                    cst += (popc(xo & S.cst_mo[t]) & 1) ? (0 - q) : q;
                }
            const double sc = op.pad ? P.scale : 1.0;
            for (int l = 0; l < T; l++) {
                int s = 0;
                for (int i = 0; i < 4; i++) s |= ((l >> R.reg_pos[i]) & 1) << i;
                uint64_t angle = 0;
                uint32_t angle32 = 0;
                for (int u = 0; u < 16; u++) {
                    uint64_t G = (u == 0) ? cst : 0;
                    if (d.zs[u] >= 0) G += slot_sum(d.zs[u]);
                    for (int j = d.off[u]; j < d.off[u + 1]; j++) {
                        const uint64_t Q = slot_sum(j);
                        G += (popc((uint64_t)l & S.slots[R.slot_begin + j].ml) & 1) ? (0 - Q) : Q;
                    }
                    angle += (popc((uint64_t)(s & u)) & 1) ? (0 - G) : G;
                    const bool used = d.off[u + 1] > d.off[u] || d.zs[u] >= 0 || (u == 0 && d.cst >= 0);
                    const uint32_t g = used ? (uint32_t)((G + (uint64_t(1) << 31)) >> 32) : 0u;
                    angle32 += (popc((uint64_t)(s & u)) & 1) ? (0u - g) : g;
                }
                const double turns = (double)(int64_t)angle / 18446744073709551616.0;
                const double turns32 = (double)(int32_t)angle32 / 4294967296.0;
                double dlt = turns32 - turns;
                dlt -= std::nearbyint(dlt);
                q32err = std::max(q32err, std::fabs(dlt));
                a[l] *= std::polar(sc, -2.0 * M_PI * (q32 ? turns32 : turns));
            }
        }
    }
};

}  // namespace

// Rank over GF(2) of the low c bits (the bank-selecting bits of an
// amplitude's swizzled shared-memory index) of a set of columns.
int bank_rank(std::vector<uint32_t> cols, int c) {
    const uint32_t mask = (1u << c) - 1u;
    int r = 0;
    for (int b = c - 1; b >= 0; b--) {
        size_t i = r;
        while (i < cols.size() && !((cols[i] & mask) >> b & 1)) i++;
        if (i == cols.size()) continue;
        std::swap(cols[r], cols[i]);
        for (size_t j = 0; j < cols.size(); j++)
            if ((int)j != r && ((cols[j] & mask) >> b & 1)) cols[j] ^= cols[r];
        r++;
    }
    return r;
}

// Shared-memory bank use of a schedule's exchanges.  A warp's access to the
// exchange buffer varies the swizzled index over the XOR combinations of the
// columns of its 5 lane positions; it is free of bank conflicts when the low c
// bits of those columns have rank c.  Counted: rounds whose lane columns fall
// short, and permutation rounds whose permuted write columns fall short.
struct BankStats {
    long rounds = 0, short_lanes = 0, perm_rounds = 0, short_perm = 0;
};

// With a paired schedule the exchange moves 16-byte pairs of amplitudes
// (paired swizzle, kPairBankBits bank bits) and a quarter warp's 8 lanes must
// span those bits.
void bank_stats(const Schedule &S, BankStats &b) {
    const int c = S.c;
    for (const DevRound &R : S.rounds) {
        std::vector<uint32_t> cols;
        if (S.pin0)
            for (int i = 0; i < 3; i++) cols.push_back(pair_swizzle_col(R.lane_pos[i]));
        else
            for (int i = 0; i < 5; i++) cols.push_back(swizzle_col(R.lane_pos[i], c));
        b.rounds++;
        if (S.pin0 ? bank_rank(cols, kPairBankBits) < kPairBankBits : bank_rank(cols, c) < c) b.short_lanes++;
        if (R.perm >= 0) {
            const DevPerm &pm = S.perms[R.perm];
            std::vector<uint32_t> pc;
            for (int i = 0; i < 5; i++) {
                uint32_t t = pm.col[R.lane_pos[i]], sw = 0;
                for (int p = 0; p < S.K; p++)
                    if ((t >> p) & 1) sw ^= swizzle_col(p, c);
                pc.push_back(sw);
            }
            b.perm_rounds++;
            if (bank_rank(pc, c) < c) b.short_perm++;
        }
    }
}

// Schedules a circuit (one-qubit runs canonicalised first).  A paired
// schedule must keep tile position 0 in register slot 0 of every round.
bool schedule(Circuit circ, int n, int K, int c, bool pin0, bool tail, Schedule &S) {
    canonicalize_1q(circ, n);
    const std::string e = schedule_circuit(circ, n, K, c, S, pin0, tail);
    if (!e.empty()) std::fprintf(stderr, "schedule: %s\n", e.c_str());
    if (pin0)
        for (const DevRound &R : S.rounds)
            if (R.reg_pos[0] != 0) {
                std::fprintf(stderr, "schedule: a round without position 0 in slot 0\n");
                return false;
            }
    return e.empty();
}

int main(int argc, char **argv) {
    // "-" as the output: schedule only (no state in the input, nothing executed)
    if (argc != 3) return 2;
    const bool run = std::string(argv[2]) != "-";
    FILE *f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    int32_t n, skip, K, c, order, reps;
    int64_t m, steps;
    double dt;
    bool ok = std::fread(&n, 4, 1, f) == 1 && std::fread(&m, 8, 1, f) == 1 && std::fread(&skip, 4, 1, f) == 1 &&
              std::fread(&K, 4, 1, f) == 1 && std::fread(&c, 4, 1, f) == 1 && std::fread(&order, 4, 1, f) == 1 &&
              std::fread(&reps, 4, 1, f) == 1 && std::fread(&steps, 8, 1, f) == 1 && std::fread(&dt, 8, 1, f) == 1;
    ok = ok && reps >= 1;
    const bool pin0 = (c >> 4) & 1, tail = (c >> 5) & 1, q32 = (c >> 6) & 1;
    c &= 15;
    std::vector<uint64_t> x(m), z(m);
    std::vector<double> coef(m);
    std::vector<cd> psi(run ? (size_t)1 << n : 0);
    ok = ok && std::fread(x.data(), 8, m, f) == (size_t)m && std::fread(z.data(), 8, m, f) == (size_t)m &&
         std::fread(coef.data(), 8, m, f) == (size_t)m && std::fread(psi.data(), 16, psi.size(), f) == psi.size();
    std::fclose(f);
    if (!ok) return 2;
    Plan plan;
    std::string e = make_plan(n, m, x.data(), z.data(), skip, plan);
    if (!e.empty()) {
        std::fprintf(stderr, "plan: %s\n", e.c_str());
        return 1;
    }
    const int G = (int)plan.groups.size();
    auto add = [&](Circuit &circ, int g, double frac) { append_group_step(plan, g, frac, dt, coef, circ); };
    // one unmerged step: groups 1..G, or the Strang sequence
    Circuit step;
    if (order == 1 || G == 1) {
        for (int g = 0; g < G; g++) add(step, g, 1.0);
    } else {
        for (int g = 0; g < G - 1; g++) add(step, g, 0.5);
        add(step, G - 1, 1.0);
        for (int g = G - 2; g >= 0; g--) add(step, g, 0.5);
    }
    // the segments of the call, as (circuit, repetitions)
    std::vector<std::pair<Circuit, int64_t>> segs;
    auto repeated = [&](const Circuit &one, int64_t count) {
        if (reps > 1 && count >= reps) {
            Circuit block;
            for (int r = 0; r < reps; r++) {
                // append one copy, rebasing its table indices
                const int32_t np = (int32_t)block.phases.size(), nd = (int32_t)block.diags.size();
                for (FlatOp op : one.ops) {
                    if (op.kind == OK_PHASE) op.idx += np;
                    else if (op.kind == OK_DIAG) op.idx += nd;
                    block.ops.push_back(op);
                }
                block.phases.insert(block.phases.end(), one.phases.begin(), one.phases.end());
                block.diags.insert(block.diags.end(), one.diags.begin(), one.diags.end());
            }
            segs.push_back({block, count / reps});
            count %= reps;
        }
        if (count > 0) segs.push_back({one, count});
    };
    if (order == 1 || G == 1 || steps == 1) {
        repeated(step, steps);
    } else {
        Circuit head, core, tail;
        add(head, 0, 0.5);
        for (int g = 1; g < G - 1; g++) {
            add(core, g, 0.5);
            add(tail, g, 0.5);
        }
        add(core, G - 1, 1.0);
        add(tail, G - 1, 1.0);
        for (int g = G - 2; g >= 1; g--) {
            add(core, g, 0.5);
            add(tail, g, 0.5);
        }
        add(core, 0, 1.0);
        add(tail, 0, 0.5);
        segs.push_back({head, 1});
        repeated(core, steps - 1);
        segs.push_back({tail, 1});
    }
    size_t passes = 0;
    double q32err = 0.0;
    BankStats banks;
    std::vector<Schedule> scheds(segs.size());
    for (size_t i = 0; i < segs.size(); i++) {
        if (!schedule(segs[i].first, n, K, c, pin0, tail, scheds[i])) return 1;
        bank_stats(scheds[i], banks);
        Emulator em{n, scheds[i], psi};
        em.q32 = q32;
        if (run)
            for (int64_t r = 0; r < segs[i].second; r++)
                for (const DevPass &P : scheds[i].passes) em.run_pass(P);
        q32err = std::max(q32err, em.q32err);
        passes += scheds[i].passes.size() * (size_t)segs[i].second;
    }
    if (run) {
        f = std::fopen(argv[2], "wb");
        if (!f) return 2;
        std::fwrite(psi.data(), 16, psi.size(), f);
        std::fclose(f);
    }
    size_t rounds = 0;
    for (size_t i = 0; i < segs.size(); i++) rounds += scheds[i].rounds.size() * (size_t)segs[i].second;
    std::printf("passes %zu\n", passes);
    std::printf("rounds %zu\n", rounds);
    std::printf("q32err %.17g\n", q32err);
    std::printf("banks %ld %ld %ld %ld\n", banks.rounds, banks.short_lanes, banks.perm_rounds, banks.short_perm);
    return 0;
}
