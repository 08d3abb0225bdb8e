"""Pins for the oracle planner (CPU only).

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden), dense matrices (textbook Pauli and gate
matrices), or invariants that any correct planner must satisfy.
"""
import os

import numpy as np
import pytest

from oracle import planner as P
from workloads import (heisenberg_lattice, pauli_to_masks, tfim_chain,
                       random_klocal, jw_like, gradient_2local)
from tests import dense as D

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    out = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out.setdefault(key, []).append(vals)
    return out


def _parse_gate(tok):
    for k in ("CNOT", "CZ", "H", "S"):
        if tok.startswith(k):
            rest = tok[len(k):]
            if "," in rest:
                a, b = rest.split(",")
                return (k, int(a), int(b))
            return (k, int(rest), -1)
    raise ValueError(tok)


# ---------------------------------------------------------------- gate rules

def test_conjugation_tables_match_rules_and_dense():
    lines = []
    with open(os.path.join(GOLD, "conjugation_tables.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                lines.append(line.split())
    assert len(lines) == 24
    for gname, p, q in lines:
        n = len(p)
        gate = (gname, 0, -1) if n == 1 else (gname, 0, 1)
        x, z = pauli_to_masks(p)
        sign = 1 if q[0] == "-" else 0
        qx, qz = pauli_to_masks(q[1:])
        assert P.apply_gate_row(gate, x, z, 0) == (qx, qz, sign), (gname, p, q)
        U = D.gate(n, gate)
        lhs = U @ D.pauli(n, x, z) @ U.conj().T
        rhs = (-1) ** sign * D.pauli(n, qx, qz)
        assert np.allclose(lhs, rhs), (gname, p, q)


def test_gate_rules_exhaustive_dense():
    n = 3
    gates = [("H", q, -1) for q in range(n)] + [("S", q, -1) for q in range(n)]
    gates += [(k, a, b) for k in ("CNOT", "CZ") for a in range(n) for b in range(n) if a != b]
    for g in gates:
        U = D.gate(n, g)
        for x in range(8):
            for z in range(8):
                for r in (0, 1):
                    x2, z2, r2 = P.apply_gate_row(g, x, z, r)
                    lhs = (-1) ** r * U @ D.pauli(n, x, z) @ U.conj().T
                    assert np.allclose(lhs, (-1) ** r2 * D.pauli(n, x2, z2)), (g, x, z)
                # vectorised form agrees with the row form
                X, Z, R = P.apply_gates_rows([g], [x], [z], [0])
                assert (int(X[0]), int(Z[0]), int(R[0])) == P.apply_gate_row(g, x, z, 0)


def test_printed_cnot_z_rule_is_a_misprint():
    """Table 3 prints z_t ^= z_c for CNOT; Table 2 (I1Z2 -> Z1Z2) and dense
    matrices need z_c ^= z_t.  The printed rule fails the dense check."""
    n = 2
    U = D.cnot(n, 0, 1)
    x, z = pauli_to_masks("IZ")
    printed = (x, z ^ ((z & 1) << 1), 0)   # z_t ^= z_c leaves IZ unchanged
    lhs = U @ D.pauli(n, x, z) @ U.conj().T
    assert not np.allclose(lhs, D.pauli(n, printed[0], printed[1]))
    assert P.apply_gate_row(("CNOT", 0, 1), x, z, 0) == pauli_to_masks("ZZ") + (0,)


# ---------------------------------------------------------------- worked examples

def test_worked_example_gate_list_and_diagonal():
    g = _read("worked_example.txt")
    terms = g["terms"][0]
    gates_exp = [_parse_gate(t) for t in g["gates"][0]]
    diag = g["diag"][0]
    xs, zs = zip(*(pauli_to_masks(t) for t in terms))
    gates, masks, signs = P.synthesize_group(4, xs, zs, skip_rule=P.SKIP_PAPER)
    assert gates == gates_exp
    for mk, sg, d in zip(masks, signs, diag):
        assert sg == (1 if d[0] == "-" else 0)
        assert pauli_to_masks(d[1:]) == (0, mk)
    # the same result under every skip rule (no qubit of this group is skipped)
    for rule in (P.SKIP_NONE, P.SKIP_Y):
        assert P.synthesize_group(4, xs, zs, skip_rule=rule) == (gates, masks, signs)
    # dense: C H C^dag is the printed diagonal operator
    C = D.circuit(4, gates)
    H = sum(D.pauli(4, a, b) for a, b in zip(xs, zs))
    Hd = sum((-1 if d[0] == "-" else 1) * D.pauli(4, *pauli_to_masks(d[1:])) for d in diag)
    assert np.allclose(C @ H @ C.conj().T, Hd)
    assert np.allclose(Hd, np.diag(np.diag(Hd)))


def test_appendix_independent_rows():
    g = _read("appendix_independence.txt")
    terms = g["terms"][0]
    rows = [int(v) - 1 for v in g["rows"][0]]
    n = 4
    packed = [x | (z << n) for x, z in (pauli_to_masks(t) for t in terms)]
    assert P.linearly_independent_terms(packed, 2 * n) == rows


def test_independent_rows_span_the_group():
    rng = np.random.default_rng(5)
    for _ in range(50):
        n = int(rng.integers(2, 7))
        k = int(rng.integers(1, 12))
        rows = [int(v) for v in rng.integers(0, 1 << (2 * n), size=k)]
        sel = P.linearly_independent_terms(rows, 2 * n)
        assert P.gf2_rank([rows[i] for i in sel]) == len(sel) == P.gf2_rank(rows)


# ---------------------------------------------------------------- random groups

def _random_groups(rng, n, m, weights=(1, 2, 3)):
    h = random_klocal(n, m, rng, weights=tuple(w for w in weights if w <= n))
    return h, P.greedy_partition(h.x, h.z)


@pytest.mark.parametrize("rule", [P.SKIP_NONE, P.SKIP_PAPER, P.SKIP_Y])
def test_random_groups_diagonalised_dense(rule):
    rng = np.random.default_rng(11 + rule)
    count = 0
    for _ in range(25):
        n = int(rng.integers(2, 6))
        h, groups = _random_groups(rng, n, int(rng.integers(3, 14)))
        for g in groups:
            xs = [int(h.x[j]) for j in g]
            zs = [int(h.z[j]) for j in g]
            gates, masks, signs = P.synthesize_group(n, xs, zs, skip_rule=rule)
            C = D.circuit(n, gates)
            for a, b, mk, sg in zip(xs, zs, masks, signs):
                lhs = C @ D.pauli(n, a, b) @ C.conj().T
                assert np.allclose(lhs, (-1) ** sg * D.pauli(n, 0, mk))
            count += 1
    assert count > 40


def test_rank_deficient_groups_never_fail():
    """Many small groups are rank deficient; with the completion reading the
    synthesis never fails (zero padding as printed fails on about a third)."""
    rng = np.random.default_rng(3)
    deficient = 0
    for _ in range(150):
        n = int(rng.integers(3, 9))
        h, groups = _random_groups(rng, n, int(rng.integers(4, 30)), weights=(2, 3, 4))
        for g in groups:
            xs = [int(h.x[j]) for j in g]
            zs = [int(h.z[j]) for j in g]
            rank = P.gf2_rank([a | (b << n) for a, b in zip(xs, zs)])
            deficient += rank < n
            for rule in (P.SKIP_NONE, P.SKIP_Y):
                P.synthesize_group(n, xs, zs, skip_rule=rule)  # raises on failure
    assert deficient > 100


def test_large_groups_row_and_vector_rules_agree():
    rng = np.random.default_rng(8)
    h = random_klocal(32, 400, rng, weights=(2, 3, 4))
    groups = P.greedy_partition(h.x, h.z)
    for g in groups[:6]:
        xs = [int(h.x[j]) for j in g]
        zs = [int(h.z[j]) for j in g]
        gates, masks, signs = P.synthesize_group(32, xs, zs)
        for a, b, mk, sg in zip(xs, zs, masks, signs):
            r = (a, b, 0)
            for gt in gates:
                r = P.apply_gate_row(gt, *r)
            assert r == (0, mk, sg)


# ---------------------------------------------------------------- partition

def _check_partition(h, groups):
    seen = sorted(j for g in groups for j in g)
    assert seen == list(range(h.m))
    for gi, g in enumerate(groups):
        assert g == sorted(g)
        for a in g:
            for b in g:
                assert P.commutes(int(h.x[a]), int(h.z[a]), int(h.x[b]), int(h.z[b]))
        # first fit: every member conflicts with each earlier group at insertion time
        for j in g:
            for g2 in groups[:gi]:
                assert any(not P.commutes(int(h.x[j]), int(h.z[j]), int(h.x[k]), int(h.z[k]))
                           for k in g2 if k < j)


def test_partition_first_fit_invariants():
    rng = np.random.default_rng(21)
    for _ in range(10):
        h, groups = _random_groups(rng, int(rng.integers(3, 10)), int(rng.integers(5, 60)))
        _check_partition(h, groups)


def test_partition_of_model_hamiltonians():
    t = tfim_chain(10)
    g = P.greedy_partition(t.x, t.z)
    assert [len(v) for v in g] == [9, 10]
    h30 = heisenberg_lattice(5, 6)
    assert h30.m == 147 and h30.n == 30
    g = P.greedy_partition(h30.x, h30.z)
    assert [len(v) for v in g] == [49, 49, 49]
    h32 = heisenberg_lattice(6, 6, drop_corners=True)
    assert h32.n == 32 and h32.m == 156
    assert len(P.greedy_partition(h32.x, h32.z)) == 3
    _check_partition(t, P.greedy_partition(t.x, t.z))


def test_skip_rule_on_heisenberg_groups():
    h = heisenberg_lattice(2, 3)
    pl = P.plan(h.n, h.x, h.z, skip_rule=P.SKIP_Y)
    assert pl.gates[0] == [("H", q, -1) for q in range(h.n)]
    assert pl.gates[1] == [g for q in range(h.n) for g in (("S", q, -1), ("H", q, -1))]
    assert pl.gates[2] == []
    # XX -> ZZ (+), YY -> -Z -Z = +ZZ, ZZ unchanged
    for gi in range(3):
        assert all(s == 0 for s in pl.signs[gi])
    pl0 = P.plan(h.n, h.x, h.z, skip_rule=P.SKIP_NONE)
    assert any(k == "CNOT" for k, _, _ in pl0.gates[0])


def test_workload_term_counts():
    assert jw_like().m == 20000
    assert gradient_2local().m == 200


def test_cnot_layer_matrix_is_the_cnot_permutation():
    rng = np.random.default_rng(2)
    for _ in range(20):
        n = 5
        gates = []
        for _ in range(8):
            c, t = (int(v) for v in rng.choice(n, 2, replace=False))
            gates.append(("CNOT", c, t))
        A, Ainv = P.cnot_layer_matrix(gates, n)
        U = D.circuit(n, gates)
        for v in range(1 << n):
            img = 0
            for q in range(n):
                if (v >> q) & 1:
                    img ^= A[q]
            assert U[img, v] == 1
            back = 0
            for q in range(n):
                if (img >> q) & 1:
                    back ^= Ainv[q]
            assert back == v


# ---------------------------------------------------------------- grouping variants

def _valid_partition(x, z, groups):
    seen = sorted(j for g in groups for j in g)
    assert seen == list(range(len(x)))
    for g in groups:
        for a in g:
            for b in g:
                assert (bin(int(x[a]) & int(z[b])).count("1") + bin(int(z[a]) & int(x[b])).count("1")) % 2 == 0


def _crown(k):
    """u_i = Z_i and v_j = X on every qubit but j (k qubits): u_i and v_j
    anticommute exactly when i != j, the u commute, the v commute (a crown
    graph, bipartite), listed u_1, v_1, u_2, v_2, ..."""
    full = (1 << k) - 1
    x, z = [], []
    for i in range(k):
        x += [0, full ^ (1 << i)]
        z += [1 << i, 0]
    return np.array(x, dtype=np.uint64), np.array(z, dtype=np.uint64)


def test_grouping_variants_are_partitions():
    rng = np.random.default_rng(71)
    from workloads import random_klocal
    for n, m in ((6, 40), (10, 120)):
        h = random_klocal(n, m, rng, weights=(1, 2, 3))
        for g in range(4):
            _valid_partition(h.x, h.z, P.partition(h.x, h.z, g, h.c))


def test_dsatur_is_exact_on_a_crown_graph():
    """On a bipartite anticommutation graph DSATUR needs 2 groups; first fit
    in this input order needs k, and so does largest first (all degrees equal)."""
    k = 6
    x, z = _crown(k)
    assert len(P.partition(x, z, P.DSATUR)) == 2
    assert len(P.partition(x, z, P.FIRST_FIT)) == k
    assert len(P.partition(x, z, P.LARGEST_FIRST)) == k
    assert P.anticommutation_degrees(x, z).tolist() == [k - 1] * (2 * k)


def test_largest_first_and_magnitude_orders():
    # Z_0, Z_1, Z_2 commute; X_0 X_1 X_2 anticommutes with each of them
    x = np.array([0, 0, 0, 7], dtype=np.uint64)
    z = np.array([1, 2, 4, 0], dtype=np.uint64)
    assert P.anticommutation_degrees(x, z).tolist() == [1, 1, 1, 3]
    assert P.partition(x, z, P.FIRST_FIT) == [[0, 1, 2], [3]]
    assert P.partition(x, z, P.LARGEST_FIRST) == [[3], [0, 1, 2]]
    c = np.array([0.1, 0.2, 0.3, 0.05])
    assert P.partition(x, z, P.BY_MAGNITUDE, c) == [[0, 1, 2], [3]]
    c2 = np.array([0.1, 0.2, 0.3, 5.0])
    assert P.partition(x, z, P.BY_MAGNITUDE, c2) == [[3], [0, 1, 2]]


# ---------------------------------------------------------------- completion branch

def _sym(a, b, n):
    m = (1 << n) - 1
    return (((a & m) & (b >> n)) ^ ((a >> n) & (b & m))).bit_count() & 1


def _span(rows):
    out = {0}
    for r in rows:
        out |= {v ^ r for v in out}
    return out


@pytest.mark.parametrize("rows_text", [["XXXX", "ZZZZ"], ["XXXX"], ["XYZI", "ZXYI"], ["XXII", "ZZII", "IIXX"]])
def test_symplectic_complement_basis_is_the_complement(rows_text):
    """The basis returned for the symplectic complement of independent rows S
    must be a basis of {v : <v, s> = 0 for every s in S}: every vector is
    orthogonal to S, the vectors are independent, there are 2n - |S| of them,
    and (brute force over all 4^n vectors) their span is the whole set."""
    n = len(rows_text[0])
    rows = []
    for t in rows_text:
        x, z = pauli_to_masks(t)
        rows.append(x | (z << n))
    assert P.gf2_rank(rows) == len(rows)
    basis = P.symplectic_complement_basis(rows, n)
    assert len(basis) == 2 * n - len(rows)
    assert P.gf2_rank(basis) == len(basis)
    for v in basis:
        assert all(_sym(v, s, n) == 0 for s in rows)
    brute = {v for v in range(1 << (2 * n)) if all(_sym(v, s, n) == 0 for s in rows)}
    assert _span(basis) == brute


def test_completion_needs_the_complement_branch():
    """{XXXX, ZZZZ} commute (four anticommuting positions), but every qubit
    carries both X and Z, so no single-qubit Z, X or Y commutes with both:
    the completion must take its rows from the symplectic complement.  The
    completed set must hold the original rows, have n independent mutually
    commuting rows, and the synthesis must then diagonalise the group
    (dense check of C P C^dag)."""
    n = 4
    rows = []
    for t in ("XXXX", "ZZZZ"):
        x, z = pauli_to_masks(t)
        rows.append(x | (z << n))
    for q in range(n):
        for x, z in ((0, 1 << q), (1 << q, 0), (1 << q, 1 << q)):
            assert any(_sym(x | (z << n), s, n) for s in rows)
    done = P.complete_generators(rows, n)
    assert done[:2] == rows and len(done) == n
    assert P.gf2_rank(done) == n
    assert all(_sym(a, b, n) == 0 for a in done for b in done)
    # the group itself, with products in it, through the whole synthesis
    texts = ["XXXX", "ZZZZ", "YYYY"]
    xs, zs = zip(*(pauli_to_masks(t) for t in texts))
    for rule in (P.SKIP_NONE, P.SKIP_PAPER, P.SKIP_Y):
        gates, masks, signs = P.synthesize_group(n, list(xs), list(zs), skip_rule=rule)
        C = D.circuit(n, gates)
        for a, b, mk, sg in zip(xs, zs, masks, signs):
            lhs = C @ D.pauli(n, a, b) @ C.conj().T
            assert np.allclose(lhs, (-1) ** sg * D.pauli(n, 0, mk))


def test_completion_branch_on_larger_groups():
    """Groups where single-qubit candidates run out before n rows: the
    complement branch fills the rest, and every completed set is a maximal
    isotropic set containing the original generators."""
    rng = np.random.default_rng(12)
    hits = 0
    for _ in range(60):
        n = int(rng.integers(4, 8))
        # pairs of strings with X and Z on the same support commute when the support is even
        k = int(rng.integers(1, n // 2 + 1))
        rows = []
        for _ in range(k):
            supp = rng.choice(n, size=2 * int(rng.integers(1, n // 2 + 1)), replace=False)
            x = sum(1 << int(q) for q in supp)
            cand = [x, x << n]
            for v in cand:
                if all(_sym(v, s, n) == 0 for s in rows) and P.gf2_rank(rows + [v]) == len(rows) + 1:
                    rows.append(v)
        singles_left = [v for q in range(n) for v in (1 << (q + n), 1 << q, (1 << q) | (1 << (q + n)))
                        if all(_sym(v, s, n) == 0 for s in rows) and P.gf2_rank(rows + [v]) > len(rows)]
        done = P.complete_generators(rows, n)
        assert done[:len(rows)] == rows and len(done) == n
        assert P.gf2_rank(done) == n
        assert all(_sym(a, b, n) == 0 for a in done for b in done)
        hits += not singles_left
    assert hits > 0
