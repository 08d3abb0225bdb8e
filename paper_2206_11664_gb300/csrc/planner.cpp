// Host planner: greedy commuting partition (Sec. 2.3), binary tableau with
// the Clifford update rules (Sec. 2.4, Table 3), independent-term search
// (Appendix, Algorithm 6), and the synthesis steps (i)-(iv) of Sec. 3.2
// (Algorithms 1-5).  Bit-packed: a Pauli row is two uint64 masks.
//
// Readings of the paper (all documented in the design notes):
//  * CNOT(c,t): x_t ^= x_c, z_c ^= z_t, r ^= x_c z_t (x_t ^ z_c ^ 1); the
//    text prints z_t ^= z_c, which contradicts Table 2 (I1 Z2 -> Z1 Z2).
//  * Algorithm 2 visits qubits from last to first; H only on a strict
//    rank increase.
//  * Algorithm 6 eliminates below the pivot row (the Appendix prose).
//  * Rank-deficient groups are completed to n_A commuting independent rows
//    (single-qubit Z, X, Y candidates, then the symplectic complement).
//  * Algorithm 3 skips a column that has no pivot at or below the diagonal.
//  * Skip rule: I/Z-only qubits untouched, I/X-only get H, and (rule 2)
//    I/Y-only get S then H; these leave steps (i)-(iv).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sd_internal.h"

namespace sd {
namespace {

inline int bit(uint64_t v, int q) { return int((v >> q) & 1u); }
inline int parity(uint64_t v) { return __builtin_popcountll(v) & 1; }

struct Row {
    uint64_t x, z;
    uint8_t r;
};

// P -> U P U^dag for one gate (Table 3 with the CNOT Z rule of Table 2).
inline void conj(const Gate &g, Row &w) {
    switch (g.kind) {
    case G_H: {
        int xt = bit(w.x, g.a), zt = bit(w.z, g.a);
        w.r ^= uint8_t(xt & zt);
        uint64_t m = uint64_t(1) << g.a;
        w.x = (w.x & ~m) | (uint64_t(zt) << g.a);
        w.z = (w.z & ~m) | (uint64_t(xt) << g.a);
        break;
    }
    case G_S: {
        int xt = bit(w.x, g.a), zt = bit(w.z, g.a);
        w.r ^= uint8_t(xt & zt);
        w.z ^= uint64_t(xt) << g.a;
        break;
    }
    case G_CNOT: {
        int c = g.a, t = g.b;
        int xc = bit(w.x, c), zc = bit(w.z, c), xt = bit(w.x, t), zt = bit(w.z, t);
        w.r ^= uint8_t(xc & zt & (xt ^ zc ^ 1));
        w.x ^= uint64_t(xc) << t;
        w.z ^= uint64_t(zt) << c;
        break;
    }
    case G_CZ: {
        int c = g.a, t = g.b;
        int xc = bit(w.x, c), zc = bit(w.z, c), xt = bit(w.x, t), zt = bit(w.z, t);
        w.r ^= uint8_t(xc & xt & (zt ^ zc));
        w.z ^= (uint64_t(xc) << t) | (uint64_t(xt) << c);
        break;
    }
    }
}

inline bool anticommute(uint64_t x1, uint64_t z1, uint64_t x2, uint64_t z2) {
    return parity((x1 & z2) ^ (z1 & x2));
}

// 2n-bit vector over GF(2): columns 0..n-1 are x, n..2n-1 are z.
struct V2 {
    uint64_t x, z;
    bool zero() const { return (x | z) == 0; }
    int get(int col, int n) const { return col < n ? bit(x, col) : bit(z, col - n); }
    void operator^=(const V2 &o) { x ^= o.x; z ^= o.z; }
};

int rank2(std::vector<V2> rows, int n) {
    int r = 0;
    for (int col = 0; col < 2 * n && r < (int)rows.size(); col++) {
        int p = -1;
        for (int i = r; i < (int)rows.size(); i++)
            if (rows[i].get(col, n)) { p = i; break; }
        if (p < 0) continue;
        std::swap(rows[r], rows[p]);
        for (int i = r + 1; i < (int)rows.size(); i++)
            if (rows[i].get(col, n)) rows[i] ^= rows[r];
        r++;
    }
    return r;
}

int rank_x(const std::vector<Row> &T) {
    std::vector<uint64_t> v;
    for (auto &w : T) v.push_back(w.x);
    int r = 0;
    for (int col = 0; col < 64 && r < (int)v.size(); col++) {
        int p = -1;
        for (int i = r; i < (int)v.size(); i++)
            if (bit(v[i], col)) { p = i; break; }
        if (p < 0) continue;
        std::swap(v[r], v[p]);
        for (int i = r + 1; i < (int)v.size(); i++)
            if (bit(v[i], col)) v[i] ^= v[r];
        r++;
    }
    return r;
}

// Appendix, Algorithm 6: indices (into `rows`) of the rows left non-zero by
// forward elimination with row swaps, in their final order.
std::vector<int> independent_rows(const std::vector<V2> &rows_in, int n) {
    std::vector<V2> rows = rows_in;
    std::vector<int> id(rows.size());
    for (size_t i = 0; i < id.size(); i++) id[i] = (int)i;
    const int N = (int)rows.size();
    int ir = 0, ic = 0;
    while (ir < N && ic < 2 * n) {
        if (!rows[ir].get(ic, n)) {
            int j = -1;
            for (int k = ir + 1; k < N; k++)
                if (rows[k].get(ic, n)) { j = k; break; }
            if (j < 0) { ic++; continue; }
            std::swap(rows[ir], rows[j]);
            std::swap(id[ir], id[j]);
        }
        for (int k = ir + 1; k < N; k++)
            if (rows[k].get(ic, n)) rows[k] ^= rows[ir];
        ir++;
        ic++;
    }
    std::vector<int> out;
    for (int i = 0; i < N; i++)
        if (!rows[i].zero()) out.push_back(id[i]);
    return out;
}

// Basis of the symplectic complement of `rows` read off the reduced row
// echelon form, one vector per free column in ascending order.
std::vector<V2> complement_basis(const std::vector<V2> &rows, int n) {
    // constraint for s = (x, z): v_x . z + v_z . x = 0 -> row (z | x)
    std::vector<V2> M;
    for (auto &s : rows) M.push_back(V2{s.z, s.x});
    std::vector<int> piv;
    int rr = 0;
    for (int col = 0; col < 2 * n; col++) {
        int p = -1;
        for (int i = rr; i < (int)M.size(); i++)
            if (M[i].get(col, n)) { p = i; break; }
        if (p < 0) continue;
        std::swap(M[rr], M[p]);
        for (int i = 0; i < (int)M.size(); i++)
            if (i != rr && M[i].get(col, n)) M[i] ^= M[rr];
        piv.push_back(col);
        rr++;
    }
    std::vector<V2> basis;
    auto setcol = [n](V2 &v, int col) {
        if (col < n) v.x |= uint64_t(1) << col; else v.z |= uint64_t(1) << (col - n);
    };
    for (int f = 0; f < 2 * n; f++) {
        if (std::find(piv.begin(), piv.end(), f) != piv.end()) continue;
        V2 v{0, 0};
        setcol(v, f);
        for (size_t i = 0; i < piv.size(); i++)
            if (M[i].get(f, n)) setcol(v, piv[i]);
        basis.push_back(v);
    }
    return basis;
}

bool complete(std::vector<V2> &rows, int n) {
    auto try_add = [&](const V2 &v) {
        for (auto &s : rows)
            if (anticommute(v.x, v.z, s.x, s.z)) return false;
        std::vector<V2> t = rows;
        t.push_back(v);
        if (rank2(t, n) == (int)rows.size()) return false;
        rows.push_back(v);
        return true;
    };
    for (int kind = 0; kind < 3; kind++) {          // Z, X, Y
        for (int q = 0; q < n && (int)rows.size() < n; q++) {
            uint64_t m = uint64_t(1) << q;
            V2 v{kind >= 1 ? m : 0, (kind == 0 || kind == 2) ? m : 0};
            try_add(v);
        }
    }
    while ((int)rows.size() < n) {
        bool added = false;
        for (auto &v : complement_basis(rows, n))
            if (try_add(v)) { added = true; break; }
        if (!added) return false;
    }
    return true;
}

// Columns of the GF(2) map that the CNOT gates (in order) apply to indices.
void cnot_map(const std::vector<Gate> &gates, int n, bool inverse, std::vector<uint64_t> &cols) {
    std::vector<Gate> cn;
    for (auto &g : gates)
        if (g.kind == G_CNOT) cn.push_back(g);
    if (inverse) std::reverse(cn.begin(), cn.end());
    cols.assign(n, 0);
    for (int q = 0; q < n; q++) {
        uint64_t v = uint64_t(1) << q;
        for (auto &g : cn) v ^= uint64_t(bit(v, g.a)) << g.b;
        cols[q] = v;
    }
}

std::string synthesize(int n, const std::vector<uint64_t> &xs, const std::vector<uint64_t> &zs,
                       int skip_rule, GroupPlan &gp) {
    std::vector<int> active;
    for (int q = 0; q < n; q++) {
        bool hx = false, hz = false, hy = false;
        for (size_t k = 0; k < xs.size(); k++) {
            int p = bit(xs[k], q) + 2 * bit(zs[k], q);
            hx |= p == 1; hz |= p == 2; hy |= p == 3;
        }
        if (skip_rule >= 1 && !hx && !hy) continue;                  // only I / Z
        if (skip_rule >= 1 && hx && !hz && !hy) {                    // only I / X
            gp.gates.push_back({G_H, q, -1});
            gp.stage.push_back(ST_PRE);
            continue;
        }
        if (skip_rule >= 2 && hy && !hx && !hz) {                    // only I / Y
            gp.gates.push_back({G_S, q, -1});
            gp.stage.push_back(ST_PRE);
            gp.gates.push_back({G_H, q, -1});
            gp.stage.push_back(ST_PRE);
            continue;
        }
        active.push_back(q);
    }
    const int nA = (int)active.size();
    if (nA > 0) {
        auto restrict_ = [&](uint64_t v) {
            uint64_t o = 0;
            for (int i = 0; i < nA; i++) o |= uint64_t(bit(v, active[i])) << i;
            return o;
        };
        std::vector<V2> rows;
        for (size_t k = 0; k < xs.size(); k++) rows.push_back(V2{restrict_(xs[k]), restrict_(zs[k])});
        std::vector<V2> gen;
        for (int i : independent_rows(rows, nA)) gen.push_back(rows[i]);
        if (!complete(gen, nA)) return "generator completion failed";
        std::vector<Row> T;
        for (auto &v : gen) T.push_back(Row{v.x, v.z, 0});
        std::vector<Gate> syn;
        std::vector<int32_t> st;
        auto apply = [&](Gate g, int stage) {
            for (auto &w : T) conj(g, w);
            syn.push_back(g);
            st.push_back(stage);
        };
        // (i) Algorithm 2
        for (int i = nA - 1; i >= 0; i--) {
            int r0 = rank_x(T);
            std::vector<Row> trial = T;
            for (auto &w : trial) conj(Gate{G_H, i, -1}, w);
            if (r0 < rank_x(trial)) apply(Gate{G_H, i, -1}, ST_ALG2);
        }
        // (ii) Algorithm 3
        for (int i = 0; i < nA; i++) {
            if (!bit(T[i].x, i)) {
                int j = -1;
                for (int k = i + 1; k < nA; k++)
                    if (bit(T[k].x, i)) { j = k; break; }
                if (j < 0) continue;
                std::swap(T[i], T[j]);
            }
            for (int j = i + 1; j < nA; j++)
                if (bit(T[i].x, j)) apply(Gate{G_CNOT, i, j}, ST_ALG3);
        }
        // (iii) Algorithm 4
        for (int i = 0; i < nA; i++) {
            for (int j = 0; j < nA; j++)
                if (j != i && bit(T[i].z, j)) apply(Gate{G_CZ, i, j}, ST_ALG4);
            if (bit(T[i].z, i)) apply(Gate{G_S, i, -1}, ST_ALG4);
        }
        // (iv) Algorithm 5
        for (int i = 0; i < nA; i++) {
            bool any = false;
            for (auto &w : T) any |= bit(w.x, i);
            if (any) apply(Gate{G_H, i, -1}, ST_ALG5);
        }
        for (auto &w : T)
            if (w.x) return "X block not cleared by steps (i)-(iv)";
        for (size_t k = 0; k < syn.size(); k++) {
            Gate g = syn[k];
            g.a = active[g.a];
            if (g.b >= 0) g.b = active[g.b];
            gp.gates.push_back(g);
            gp.stage.push_back(st[k]);
        }
    }
    for (size_t k = 0; k < xs.size(); k++) {
        Row w{xs[k], zs[k], 0};
        for (auto &g : gp.gates) conj(g, w);
        if (w.x) return "a term is not diagonal after its group's circuit";
        gp.masks.push_back(w.z);
        gp.signs.push_back(w.r);
    }
    cnot_map(gp.gates, n, false, gp.cnot_cols);
    cnot_map(gp.gates, n, true, gp.cnot_inv_cols);
    return "";
}

// First fit in the given order: each term joins the first group (in order of
// creation) all of whose members commute with it, else opens a new group.
std::vector<std::vector<int64_t>> first_fit(const std::vector<int64_t> &order, const uint64_t *x,
                                            const uint64_t *z) {
    std::vector<std::vector<int64_t>> groups;
    for (int64_t j : order) {
        size_t g = 0;
        for (; g < groups.size(); g++) {
            bool ok = true;
            for (int64_t k : groups[g])
                if (anticommute(x[j], z[j], x[k], z[k])) { ok = false; break; }
            if (ok) break;
        }
        if (g == groups.size()) groups.emplace_back();
        groups[g].push_back(j);
    }
    return groups;
}

// Number of terms each term anticommutes with (its degree in the graph whose
// colourings are the commuting partitions).
std::vector<int64_t> degrees(int64_t m, const uint64_t *x, const uint64_t *z) {
    std::vector<int64_t> d(m, 0);
    for (int64_t a = 0; a < m; a++)
        for (int64_t b = a + 1; b < m; b++)
            if (anticommute(x[a], z[a], x[b], z[b])) {
                d[a]++;
                d[b]++;
            }
    return d;
}

// DSATUR: repeatedly colour the uncoloured term with the most distinct
// colours among its coloured neighbours (ties: larger degree, then lower
// index) with the smallest colour none of them has.
std::vector<std::vector<int64_t>> dsatur(int64_t m, const uint64_t *x, const uint64_t *z) {
    const std::vector<int64_t> deg = degrees(m, x, z);
    std::vector<int64_t> colour(m, -1), sat(m, 0);
    std::vector<std::vector<char>> seen(m);   // seen[u][c]: a neighbour of u has colour c
    std::vector<std::vector<int64_t>> groups;
    for (int64_t step = 0; step < m; step++) {
        int64_t v = -1;
        for (int64_t u = 0; u < m; u++) {
            if (colour[u] >= 0) continue;
            if (v < 0 || sat[u] > sat[v] || (sat[u] == sat[v] && deg[u] > deg[v])) v = u;
        }
        int64_t c = 0;
        while (c < (int64_t)seen[v].size() && seen[v][c]) c++;
        colour[v] = c;
        if (c == (int64_t)groups.size()) groups.emplace_back();
        groups[c].push_back(v);
        for (int64_t u = 0; u < m; u++) {
            if (colour[u] >= 0 || !anticommute(x[u], z[u], x[v], z[v])) continue;
            if ((int64_t)seen[u].size() <= c) seen[u].resize(c + 1, 0);
            if (!seen[u][c]) {
                seen[u][c] = 1;
                sat[u]++;
            }
        }
    }
    return groups;
}

}  // namespace

std::vector<std::vector<int64_t>> partition_terms(int64_t m, const uint64_t *x, const uint64_t *z,
                                                  const double *c, int grouping) {
    std::vector<int64_t> order(m);
    for (int64_t j = 0; j < m; j++) order[j] = j;
    std::vector<std::vector<int64_t>> groups;
    if (grouping == 1) {
        const std::vector<int64_t> d = degrees(m, x, z);
        std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return d[a] > d[b]; });
        groups = first_fit(order, x, z);
    } else if (grouping == 2) {
        groups = dsatur(m, x, z);
    } else if (grouping == 3) {
        std::stable_sort(order.begin(), order.end(),
                         [&](int64_t a, int64_t b) { return std::fabs(c[a]) > std::fabs(c[b]); });
        groups = first_fit(order, x, z);
    } else {
        groups = first_fit(order, x, z);
    }
    for (auto &g : groups) std::sort(g.begin(), g.end());   // input order inside a group
    return groups;
}

std::string make_plan(int n, int64_t m, const uint64_t *x, const uint64_t *z, int skip_rule,
                      Plan &out, int grouping, const double *c) {
    out = Plan{};
    out.n = n;
    out.skip_rule = skip_rule;
    // Sec. 2.3: a greedy partition into mutually commuting groups (first fit
    // in input order unless another colouring order is asked for).
    const std::vector<std::vector<int64_t>> parts = partition_terms(m, x, z, c, grouping);
    for (const auto &part : parts) {
        out.groups.emplace_back();
        std::vector<uint64_t> gx, gz;
        for (int64_t j : part) {
            out.groups.back().terms.push_back(j);
            gx.push_back(x[j]);
            gz.push_back(z[j]);
        }
        std::string err = synthesize(n, gx, gz, skip_rule, out.groups.back());
        if (!err.empty()) return "group " + std::to_string(out.groups.size() - 1) + ": " + err;
    }
    return "";
}

}  // namespace sd
