"""ORACLE planner -- test infrastructure only.

An independent, plain Python statement of the host-side part of the method:
greedy partition into mutually commuting groups (Sec. 2.3), the binary
tableau and its gate rules (Sec. 2.4, Table 3), the search for linearly
independent terms (Appendix, Algorithm 6), and the four synthesis steps
(i)-(iv) of Sec. 3.2 (Algorithms 1-5) that find a Clifford circuit C_g with
C_g P C_g^dag = (-1)^r Z^m for every term P of the group (Eq. hami_sim_diag).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use
this module; the simulator has its own planner and shares no code with it.

Bit conventions: qubit q (the paper's qubit q+1) is bit q of the x and z
masks; a tableau row is (x, z, r) and stands for (-1)^r times the product
over qubits of I, X, Z or Y for (x_q, z_q) = (0,0), (1,0), (0,1), (1,1).

Readings where the paper is silent or misprinted (each one is pinned by a
test against the paper's worked examples or against dense matrices):
  * CNOT(c,t) updates z_c ^= z_t (Table 2 maps I_1 Z_2 to Z_1 Z_2; the text
    and Table 3 print z_t ^= z_c), with x_t ^= x_c and
    r ^= x_c z_t (x_t ^ z_c ^ 1).
  * Algorithm 2 visits the qubits from the last to the first (the order
    that reproduces the printed H(3), H(4) of the worked example) and
    applies H(i) only on a strict rank increase.
  * Algorithm 6 eliminates the column from the rows BELOW the pivot (the
    prose of the Appendix), swapping in the first lower row with a one.
  * A rank-deficient group is completed to n_A independent, mutually
    commuting rows (single-qubit Z, then X, then Y candidates on the active
    qubits, then the first basis vector of the symplectic complement not yet
    in the span) instead of being padded with zero rows.
  * In Algorithm 3 a column with no pivot below the diagonal is skipped.
  * Skip rule of Sec. 3.2: a qubit on which every term of the group is I or
    Z is left alone, a qubit with only I or X gets H; both leave the active
    set of steps (i)-(iv).  Optional extension (skip_rule=2): a qubit with
    only I or Y gets S then H.
  * Greedy partition = first fit in input order.
"""
from __future__ import annotations

import numpy as np

SKIP_NONE, SKIP_PAPER, SKIP_Y = 0, 1, 2


def _bit(v: int, q: int) -> int:
    return (v >> q) & 1


def commutes(x1: int, z1: int, x2: int, z2: int) -> bool:
    """Pauli strings commute iff their symplectic product is even."""
    return (((x1 & z2) ^ (z1 & x2)).bit_count() & 1) == 0


# ------------------------------------------------------------ partition

FIRST_FIT, LARGEST_FIRST, DSATUR, BY_MAGNITUDE = 0, 1, 2, 3


def anticommutation_degrees(x, z):
    """deg[j] = number of terms k != j with an odd symplectic product
    |x_j & z_k| + |z_j & x_k| (the terms P_j anticommutes with)."""
    x = np.asarray(x, dtype=np.uint64)
    z = np.asarray(z, dtype=np.uint64)
    deg = np.zeros(len(x), dtype=np.int64)
    for j in range(len(x)):
        odd = (np.bitwise_count(x[j] & z) + np.bitwise_count(z[j] & x)) & 1
        deg[j] = int(odd.sum())
    return deg


def dsatur_partition(x, z):
    """DSATUR colouring of the anticommutation graph: repeatedly take the
    uncoloured term with the most distinct colours among its coloured
    anticommuting terms (ties: larger degree, then lower index) and give it
    the smallest colour none of them has.  Groups are the colour classes in
    colour order, terms in input order."""
    x = [int(v) for v in x]
    z = [int(v) for v in z]
    m = len(x)
    deg = anticommutation_degrees(np.array(x, dtype=np.uint64), np.array(z, dtype=np.uint64))

    def anti(a, b):
        return (bin(x[a] & z[b]).count("1") + bin(z[a] & x[b]).count("1")) % 2 == 1

    colour = [-1] * m
    neigh = [set() for _ in range(m)]
    groups = []
    for _ in range(m):
        v = max((u for u in range(m) if colour[u] < 0),
                key=lambda u: (len(neigh[u]), deg[u], -u))
        c = 0
        while c in neigh[v]:
            c += 1
        colour[v] = c
        if c == len(groups):
            groups.append([])
        groups[c].append(v)
        for u in range(m):
            if colour[u] < 0 and anti(u, v):
                neigh[u].add(c)
    return [sorted(g) for g in groups]


def partition(x, z, grouping=FIRST_FIT, c=None):
    """Commuting partition (Sec. 2.3 asks only for a greedy method) by
    first fit in input order, first fit in order of decreasing degree
    (largest first), DSATUR, or first fit in order of decreasing |c_j|.
    Groups in order of creation, terms inside a group in input order."""
    if grouping == FIRST_FIT:
        return greedy_partition(x, z)
    if grouping == DSATUR:
        return dsatur_partition(x, z)
    m = len(x)
    if grouping == LARGEST_FIRST:
        deg = anticommutation_degrees(x, z)
        order = sorted(range(m), key=lambda j: -deg[j])           # stable: ties by index
    elif grouping == BY_MAGNITUDE:
        order = sorted(range(m), key=lambda j: -abs(float(c[j])))
    else:
        raise ValueError("grouping must be 0, 1, 2 or 3")
    return [sorted(g) for g in greedy_partition(x, z, order)]


def greedy_partition(x, z, order=None):
    """First-fit greedy colouring: each term (in input order, or in `order`)
    joins the lowest-index group all of whose members commute with it,
    otherwise it opens a new group.  Returns a list of lists of term indices
    (in the order they joined)."""
    x = np.asarray(x, dtype=np.uint64)
    z = np.asarray(z, dtype=np.uint64)
    groups: list[list[int]] = []
    gx: list[np.ndarray] = []
    gz: list[np.ndarray] = []
    gsize: list[int] = []
    for j in (range(len(x)) if order is None else order):
        xj, zj = x[j], z[j]
        placed = False
        for g in range(len(groups)):
            k = gsize[g]
            anti = np.bitwise_count((gx[g][:k] & zj) ^ (gz[g][:k] & xj)) & np.uint8(1)
            if not anti.any():
                if k == gx[g].shape[0]:
                    gx[g] = np.concatenate([gx[g], np.zeros_like(gx[g])])
                    gz[g] = np.concatenate([gz[g], np.zeros_like(gz[g])])
                gx[g][k] = xj
                gz[g][k] = zj
                gsize[g] += 1
                groups[g].append(j)
                placed = True
                break
        if not placed:
            groups.append([j])
            gx.append(np.array([xj] + [0] * 7, dtype=np.uint64))
            gz.append(np.array([zj] + [0] * 7, dtype=np.uint64))
            gsize.append(1)
    return groups


# ------------------------------------------------------------ gate rules

def apply_gate_row(gate, x: int, z: int, r: int):
    """Conjugate one tableau row by a gate: P -> U P U^dag (Table 3, with
    the CNOT Z-propagation read as z_c ^= z_t)."""
    kind, a, b = gate
    if kind == "H":
        xt, zt = _bit(x, a), _bit(z, a)
        r ^= xt & zt
        x = (x & ~(1 << a)) | (zt << a)
        z = (z & ~(1 << a)) | (xt << a)
    elif kind == "S":
        xt, zt = _bit(x, a), _bit(z, a)
        r ^= xt & zt
        z ^= xt << a
    elif kind == "CNOT":
        c, t = a, b
        xc, zc, xt, zt = _bit(x, c), _bit(z, c), _bit(x, t), _bit(z, t)
        r ^= xc & zt & (xt ^ zc ^ 1)
        x ^= xc << t
        z ^= zt << c
    elif kind == "CZ":
        c, t = a, b
        xc, zc, xt, zt = _bit(x, c), _bit(z, c), _bit(x, t), _bit(z, t)
        r ^= xc & xt & (zt ^ zc)
        z ^= (xc << t) | (xt << c)
    else:
        raise ValueError(kind)
    return x, z, r


def apply_gates_rows(gates, x, z, r=None):
    """The same rules applied to every row of a tableau (numpy uint64)."""
    X = np.array(x, dtype=np.uint64, copy=True)
    Z = np.array(z, dtype=np.uint64, copy=True)
    R = np.zeros_like(X) if r is None else np.array(r, dtype=np.uint64, copy=True)
    one = np.uint64(1)
    for kind, a, b in gates:
        sa = np.uint64(a)
        if kind == "H":
            xt, zt = (X >> sa) & one, (Z >> sa) & one
            R ^= xt & zt
            X = (X & ~(one << sa)) | (zt << sa)
            Z = (Z & ~(one << sa)) | (xt << sa)
        elif kind == "S":
            xt, zt = (X >> sa) & one, (Z >> sa) & one
            R ^= xt & zt
            Z ^= xt << sa
        elif kind == "CNOT":
            sc, st = np.uint64(a), np.uint64(b)
            xc, zc = (X >> sc) & one, (Z >> sc) & one
            xt, zt = (X >> st) & one, (Z >> st) & one
            R ^= xc & zt & (xt ^ zc ^ one)
            X ^= xc << st
            Z ^= zt << sc
        elif kind == "CZ":
            sc, st = np.uint64(a), np.uint64(b)
            xc, zc = (X >> sc) & one, (Z >> sc) & one
            xt, zt = (X >> st) & one, (Z >> st) & one
            R ^= xc & xt & (zt ^ zc)
            Z ^= (xc << st) | (xt << sc)
        else:
            raise ValueError(kind)
    return X, Z, R


# ------------------------------------------------------------ GF(2) helpers

def gf2_rank(rows) -> int:
    """Rank of a list of bit-vectors (python ints) over GF(2)."""
    basis: list[int] = []
    for v in rows:
        for b in basis:
            v = min(v, v ^ b)
        if v:
            basis.append(v)
            basis.sort(reverse=True)
    return len(basis)


def linearly_independent_terms(rows2n, ncols):
    """Appendix / Algorithm 6: Gaussian elimination with row swaps over the
    columns x_1..x_n z_1..z_n; returns the original indices of the rows that
    remain non-zero, in their final order.  rows2n[k] is a python int whose
    bit `col` is column col (0-based)."""
    rows = list(rows2n)
    orig = list(range(len(rows)))
    N = len(rows)
    ir, ic = 0, 0
    while ir < N and ic < ncols:
        if not _bit(rows[ir], ic):
            j = next((j for j in range(ir + 1, N) if _bit(rows[j], ic)), None)
            if j is None:
                ic += 1
                continue
            rows[ir], rows[j] = rows[j], rows[ir]
            orig[ir], orig[j] = orig[j], orig[ir]
        for k in range(ir + 1, N):
            if _bit(rows[k], ic):
                rows[k] ^= rows[ir]
        ir += 1
        ic += 1
    return [orig[i] for i in range(N) if rows[i] != 0]


def _pack(x: int, z: int, n: int) -> int:
    return x | (z << n)


def symplectic_complement_basis(rows, n):
    """Basis of {v : <v, s> = 0 for every row s} where <(x,z),(x',z')> =
    x.z' + z.x' (mod 2); rows and vectors are packed x | z << n.  The basis
    is read off the reduced row-echelon form (pivot = first column with a
    one, rows reduced above and below), one vector per free column in
    ascending column order, so it is unique."""
    # constraint row for s = (x, z): coefficient of v_x is z, of v_z is x
    cons = []
    for s in rows:
        x, z = s & ((1 << n) - 1), s >> n
        cons.append(z | (x << n))
    ncols = 2 * n
    M = list(cons)
    pivots = []
    rr = 0
    for col in range(ncols):
        p = next((i for i in range(rr, len(M)) if _bit(M[i], col)), None)
        if p is None:
            continue
        M[rr], M[p] = M[p], M[rr]
        for i in range(len(M)):
            if i != rr and _bit(M[i], col):
                M[i] ^= M[rr]
        pivots.append(col)
        rr += 1
    free = [c for c in range(ncols) if c not in pivots]
    basis = []
    for f in free:
        v = 1 << f
        for i, pc in enumerate(pivots):
            if _bit(M[i], f):
                v |= 1 << pc
        basis.append(v)
    return basis


def complete_generators(rows, n):
    """Extend independent, mutually commuting rows (packed x | z << n) to n
    of them (the completion reading of a rank-deficient group)."""
    rows = list(rows)

    def sym(a, b):
        ax, az = a & ((1 << n) - 1), a >> n
        bx, bz = b & ((1 << n) - 1), b >> n
        return ((ax & bz) ^ (az & bx)).bit_count() & 1

    def try_add(v):
        if any(sym(v, s) for s in rows):
            return False
        if gf2_rank(rows + [v]) == len(rows):
            return False
        rows.append(v)
        return True

    for kind in ("Z", "X", "Y"):
        for q in range(n):
            if len(rows) == n:
                return rows
            x = (1 << q) if kind in "XY" else 0
            z = (1 << q) if kind in "ZY" else 0
            try_add(_pack(x, z, n))
    while len(rows) < n:
        for v in symplectic_complement_basis(rows, n):
            if try_add(v):
                break
        else:  # cannot happen for an isotropic set of size < n
            raise RuntimeError("completion failed")
    return rows


# ------------------------------------------------------------ synthesis

class SynthesisError(RuntimeError):
    pass


def _local_tableau_ops(n):
    """Helpers over a local tableau: list of [x, z, r] with n-bit ints."""

    def xblock_rank(T):
        return gf2_rank([row[0] for row in T])

    def apply(T, gate):
        for row in T:
            row[0], row[1], row[2] = apply_gate_row(gate, row[0], row[1], row[2])

    return xblock_rank, apply


def synthesize_group(n, xs, zs, skip_rule=SKIP_Y):
    """Clifford circuit diagonalising one group of mutually commuting terms.

    Returns (gates, masks, signs): gates in application order as tuples
    (kind, a, b) with global qubit indices (b = -1 for one-qubit gates);
    masks/signs per term with C P C^dag = (-1)^sign Z^mask."""
    xs = [int(v) for v in xs]
    zs = [int(v) for v in zs]
    pre = []
    active = []
    for q in range(n):
        has = set()
        for x, z in zip(xs, zs):
            p = _bit(x, q) + 2 * _bit(z, q)  # 1 X, 2 Z, 3 Y
            if p:
                has.add(p)
        if skip_rule >= SKIP_PAPER and has <= {2}:
            continue
        if skip_rule >= SKIP_PAPER and has == {1}:
            pre.append(("H", q, -1))
            continue
        if skip_rule >= SKIP_Y and has == {3}:
            pre.append(("S", q, -1))
            pre.append(("H", q, -1))
            continue
        active.append(q)
    nA = len(active)
    syn = []
    if nA:
        def restrict(v):
            out = 0
            for i, q in enumerate(active):
                out |= _bit(v, q) << i
            return out

        lx = [restrict(v) for v in xs]
        lz = [restrict(v) for v in zs]
        packed = [_pack(a, b, nA) for a, b in zip(lx, lz)]
        indep = linearly_independent_terms(packed, 2 * nA)
        gen = [packed[i] for i in indep]
        gen = complete_generators(gen, nA)
        mask = (1 << nA) - 1
        T = [[g & mask, g >> nA, 0] for g in gen]
        xrank, apply = _local_tableau_ops(nA)

        def H(i):
            apply(T, ("H", i, -1))
            syn.append(("H", i, -1))

        # (i) Algorithm 2: maximise the rank of the X block with H gates
        for i in reversed(range(nA)):
            r0 = xrank(T)
            trial = [[row[0], row[1], row[2]] for row in T]
            for row in trial:
                row[0], row[1], row[2] = apply_gate_row(("H", i, -1), *row)
            if r0 < xrank(trial):
                H(i)
        # (ii) Algorithm 3: zero the upper triangle of the X block with CNOTs
        for i in range(nA):
            if not _bit(T[i][0], i):
                j = next((j for j in range(i + 1, nA) if _bit(T[j][0], i)), None)
                if j is None:
                    continue
                T[i], T[j] = T[j], T[i]
            for j in range(i + 1, nA):
                if _bit(T[i][0], j):
                    apply(T, ("CNOT", i, j))
                    syn.append(("CNOT", i, j))
        # (iii) Algorithm 4: zero the Z block with CZ then S
        for i in range(nA):
            for j in range(nA):
                if j != i and _bit(T[i][1], j):
                    apply(T, ("CZ", i, j))
                    syn.append(("CZ", i, j))
            if _bit(T[i][1], i):
                apply(T, ("S", i, -1))
                syn.append(("S", i, -1))
        # (iv) Algorithm 5: X components to Z with H
        for i in range(nA):
            if any(_bit(row[0], i) for row in T):
                H(i)
        if any(row[0] for row in T):
            raise SynthesisError("X block not cleared")
        syn = [(k, active[a], active[b] if b >= 0 else -1) for k, a, b in syn]
    gates = pre + syn
    X, Z, R = apply_gates_rows(gates, xs, zs)
    if np.any(X):
        raise SynthesisError("a term is not diagonal after the circuit")
    return gates, [int(v) for v in Z], [int(v) for v in R]


def cnot_layer_matrix(gates, n):
    """Columns A e_q of the GF(2) map x -> A x that the CNOT gates of a
    circuit (in order) apply to basis indices, and of its inverse."""
    cn = [(a, b) for k, a, b in gates if k == "CNOT"]

    def run(seq):
        cols = []
        for q in range(n):
            v = 1 << q
            for c, t in seq:
                v ^= _bit(v, c) << t
            cols.append(v)
        return cols

    return run(cn), run(list(reversed(cn)))


class Plan:
    def __init__(self, n, groups, gates, masks, signs):
        self.n = n
        self.groups = groups
        self.gates = gates
        self.masks = masks
        self.signs = signs


def plan(n, x, z, skip_rule=SKIP_Y, grouping=FIRST_FIT, c=None) -> Plan:
    groups = partition(x, z, grouping, c)
    gates, masks, signs = [], [], []
    for g in groups:
        gt, mk, sg = synthesize_group(n, [x[j] for j in g], [z[j] for j in g], skip_rule)
        gates.append(gt)
        masks.append(mk)
        signs.append(sg)
    return Plan(n, groups, gates, masks, signs)


# ------------------------------------------------------------ Trotter order

def trotter_sequence(groups, order: int):
    """One Trotter step as a list of (term, dt multiplier) in application
    order.  First order (Eq. trotter_simul_diag): groups 1..G, terms of a
    group in input order.  Second order (Strang splitting, not in the
    paper): groups 1..G-1 at dt/2, group G at dt, groups G-1..1 at dt/2."""
    if order == 1:
        return [(j, 1.0) for g in groups for j in g]
    if order != 2:
        raise ValueError("order must be 1 or 2")
    G = len(groups)
    seq = []
    for gi in range(G - 1):
        seq += [(j, 0.5) for j in groups[gi]]
    seq += [(j, 1.0) for j in groups[G - 1]]
    for gi in reversed(range(G - 1)):
        seq += [(j, 0.5) for j in groups[gi]]
    return seq
