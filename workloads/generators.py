"""Seeded generators for the synthetic Hamiltonians and initial states.

Encoding.  A Pauli string on n qubits is a pair of n-bit masks (x, z): on
qubit q the operator is I for (0,0), X for (1,0), Z for (0,1) and Y for
(1,1).  Bit q of a mask is qubit q (qubit 1 of the paper is bit 0), and in a
text string character q is qubit q, so "XIZY" has X on qubit 0 and Y on
qubit 3.  Amplitude index bit q is the computational-basis value of qubit q.

A Hamiltonian is returned as ``Hamiltonian(n, x, z, c)`` with numpy arrays
x, z (uint64) and c (float64) of length m.

Seeds follow one rule so that every consumer draws identical inputs:
``numpy.random.default_rng(seed)`` with seed 1000 + workload index for the
five workloads below and 2000 + i for instance i of the random batch.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "Hamiltonian", "pauli_to_masks", "masks_to_pauli", "from_strings",
    "tfim_chain", "heisenberg_lattice", "lattice_sites", "neel_index",
    "random_klocal", "batch_instances", "jw_like", "gradient_2local",
    "tfim_fully_connected", "majorana_strings", "syk_majorana",
    "product_state", "haar_product_factors", "plus_state", "basis_state",
    "z_average_observable", "SEED_BASE", "BATCH_SEED_BASE",
]

SEED_BASE = 1000
BATCH_SEED_BASE = 2000

_PX = {"I": (0, 0), "X": (1, 0), "Z": (0, 1), "Y": (1, 1)}


@dataclass
class Hamiltonian:
    n: int
    x: np.ndarray  # uint64[m]
    z: np.ndarray  # uint64[m]
    c: np.ndarray  # float64[m]

    @property
    def m(self) -> int:
        return int(self.c.shape[0])

    def strings(self):
        return [masks_to_pauli(self.n, int(a), int(b))
                for a, b in zip(self.x, self.z)]


def pauli_to_masks(s: str):
    """Text Pauli string (character q = qubit q) to (x, z) integer masks."""
    x = z = 0
    for q, ch in enumerate(s.upper()):
        bx, bz = _PX[ch]
        x |= bx << q
        z |= bz << q
    return x, z


def masks_to_pauli(n: int, x: int, z: int) -> str:
    out = []
    for q in range(n):
        bx, bz = (x >> q) & 1, (z >> q) & 1
        out.append("IXZY"[bx + 2 * bz])
    return "".join(out)


def from_strings(strings, coeffs) -> Hamiltonian:
    n = len(strings[0])
    xs, zs = zip(*(pauli_to_masks(s) for s in strings))
    return Hamiltonian(n, np.array(xs, dtype=np.uint64),
                       np.array(zs, dtype=np.uint64),
                       np.asarray(coeffs, dtype=np.float64))


def _build(n, terms):
    """terms: list of (dict qubit->'X'|'Y'|'Z', coeff)."""
    x = np.zeros(len(terms), dtype=np.uint64)
    z = np.zeros(len(terms), dtype=np.uint64)
    c = np.zeros(len(terms), dtype=np.float64)
    for k, (ops, coef) in enumerate(terms):
        xv = zv = 0
        for q, p in ops.items():
            bx, bz = _PX[p]
            xv |= bx << q
            zv |= bz << q
        x[k], z[k], c[k] = xv, zv, coef
    return Hamiltonian(n, x, z, c)


# ---------------------------------------------------------------- workloads

def tfim_chain(n: int = 10, J: float = 1.0, h: float = 0.9) -> Hamiltonian:
    """Open transverse-field Ising chain: all J Z_i Z_{i+1} terms (i
    ascending), then all h X_i terms; first-fit grouping gives two groups."""
    terms = [({i: "Z", i + 1: "Z"}, J) for i in range(n - 1)]
    terms += [({i: "X"}, h) for i in range(n)]
    return _build(n, terms)


def lattice_sites(rows: int, cols: int, drop_corners: bool = False):
    """Sites (r, c) of a rows x cols open lattice in row-major order,
    optionally without the four corner sites; qubit k is the k-th site."""
    corners = {(0, 0), (0, cols - 1), (rows - 1, 0), (rows - 1, cols - 1)}
    return [(r, c) for r in range(rows) for c in range(cols)
            if not (drop_corners and (r, c) in corners)]


def heisenberg_lattice(rows: int = 5, cols: int = 6, J: float = 1.0,
                       drop_corners: bool = False) -> Hamiltonian:
    """Nearest-neighbour XXX model on an open lattice.  Term order: J X_aX_b
    for every edge (a<b, edges sorted by (a, b)), then all YY, then all ZZ,
    which first-fit grouping turns into exactly three groups."""
    sites = lattice_sites(rows, cols, drop_corners)
    idx = {s: k for k, s in enumerate(sites)}
    edges = []
    for (r, c), a in idx.items():
        for nb in ((r, c + 1), (r + 1, c)):
            if nb in idx:
                b = idx[nb]
                edges.append((min(a, b), max(a, b)))
    edges.sort()
    terms = []
    for p in "XYZ":
        terms += [({a: p, b: p}, J) for a, b in edges]
    return _build(len(sites), terms)


def neel_index(rows: int = 5, cols: int = 6, drop_corners: bool = False) -> int:
    """Basis-state index of the Neel state: qubit = 1 where r + c is odd."""
    v = 0
    for k, (r, c) in enumerate(lattice_sites(rows, cols, drop_corners)):
        if (r + c) % 2 == 1:
            v |= 1 << k
    return v


def random_klocal(n: int, m: int, rng: np.random.Generator,
                  weights=(2, 3, 4)) -> Hamiltonian:
    """m terms of weight drawn uniformly from `weights` on distinct uniformly
    random qubits with uniformly random X/Y/Z; coefficients N(0,1) scaled so
    that sum |c| = n."""
    terms = []
    for _ in range(m):
        w = int(rng.choice(weights))
        qs = rng.choice(n, size=w, replace=False)
        ps = rng.integers(0, 3, size=w)
        terms.append(({int(q): "XYZ"[int(p)] for q, p in zip(qs, ps)}, 0.0))
    c = rng.standard_normal(m)
    c *= n / np.abs(c).sum()
    h = _build(n, terms)
    h.c[:] = c
    return h


def batch_instances(count: int = 64, m: int = 2000, nmin: int = 16,
                    nmax: int = 24, seed_base: int = BATCH_SEED_BASE):
    """The random k-local batch: instance i draws from seed seed_base + i its
    qubit count (uniform in [nmin, nmax]), its Hamiltonian and its Haar-random
    product initial state (returned as per-qubit factors)."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed_base + i)
        n = int(rng.integers(nmin, nmax + 1))
        h = random_klocal(n, m, rng)
        factors = haar_product_factors(n, rng)
        out.append((h, factors))
    return out


def jw_like(n: int = 26, m: int = 20000, rng: np.random.Generator | None = None,
            z_fraction: float = 0.25) -> Hamiltonian:
    """Jordan-Wigner-style Hamiltonian: first round(z_fraction*m) Z terms of
    weight 1 or 2 (probability 1/2 each, distinct random qubits), then hopping
    terms X_i Z..Z X_j or Y_i Z..Z Y_j (probability 1/2 each) for a random
    pair i < j with Z on every qubit strictly between.  Coefficients have a
    random sign and magnitude 10**U(-4, 0)."""
    if rng is None:
        rng = np.random.default_rng(SEED_BASE + 3)
    nz = int(round(z_fraction * m))
    terms = []
    for _ in range(nz):
        w = 1 if rng.random() < 0.5 else 2
        qs = rng.choice(n, size=w, replace=False)
        terms.append(({int(q): "Z" for q in qs}, 0.0))
    for _ in range(m - nz):
        i, j = sorted(int(v) for v in rng.choice(n, size=2, replace=False))
        p = "X" if rng.random() < 0.5 else "Y"
        ops = {q: "Z" for q in range(i + 1, j)}
        ops[i] = p
        ops[j] = p
        terms.append((ops, 0.0))
    mag = 10.0 ** rng.uniform(-4.0, 0.0, size=m)
    sgn = np.where(rng.random(m) < 0.5, -1.0, 1.0)
    h = _build(n, terms)
    h.c[:] = sgn * mag
    return h


def gradient_2local(n: int = 24, m: int = 200,
                    rng: np.random.Generator | None = None) -> Hamiltonian:
    """m terms P_a Q_b on a uniformly random qubit pair a != b with P, Q
    uniform in {X, Y, Z}; coefficients U[-1, 1]."""
    if rng is None:
        rng = np.random.default_rng(SEED_BASE + 4)
    terms = []
    for _ in range(m):
        a, b = (int(v) for v in rng.choice(n, size=2, replace=False))
        pa, pb = (int(v) for v in rng.integers(0, 3, size=2))
        terms.append(({a: "XYZ"[pa], b: "XYZ"[pb]}, 0.0))
    h = _build(n, terms)
    h.c[:] = rng.uniform(-1.0, 1.0, size=m)
    return h


def tfim_fully_connected(n: int = 30, rng: np.random.Generator | None = None) -> Hamiltonian:
    """Fully connected transverse-field Ising model of the paper's first
    experiment (Sec. 4): H = sum_{i<j} J_ij Z_i Z_j + sum_i h_i X_i with J_ij
    and h_i uniform in [-1, 1]; the ZZ terms (pairs in lexicographic order)
    come first, then the X terms, so first-fit grouping gives 2 groups of
    n(n-1)/2 and n terms."""
    if rng is None:
        rng = np.random.default_rng(SEED_BASE + 5)
    terms = [({i: "Z", j: "Z"}, 0.0) for i in range(n) for j in range(i + 1, n)]
    terms += [({i: "X"}, 0.0) for i in range(n)]
    h = _build(n, terms)
    h.c[:] = rng.uniform(-1.0, 1.0, size=h.m)
    return h


def majorana_strings(n: int):
    """The 2n Majorana operators of n qubits in the Jordan-Wigner form of the
    paper's second experiment (Sec. 4), as (x, z) masks: operator 2q is
    Z_0 ... Z_{q-1} X_q and operator 2q + 1 is Z_0 ... Z_{q-1} Y_q (the
    paper's c_{2i-1}, c_{2i} with qubit i = q + 1)."""
    out = []
    for q in range(n):
        low = (1 << q) - 1
        out.append((1 << q, low))
        out.append((1 << q, low | (1 << q)))
    return out


def _pauli_product(a, b):
    """P_a P_b = i^k P_(xa^xb, za^zb) for Hermitian Pauli strings in the
    (x, z) encoding (Y = i X Z on a qubit); returns (x, z, k mod 4)."""
    (xa, za), (xb, zb) = a, b
    x, z = xa ^ xb, za ^ zb
    k = (bin(xa & za).count("1") + bin(xb & zb).count("1") + 2 * bin(za & xb).count("1")
         - bin(x & z).count("1")) % 4
    return x, z, k


def syk_majorana(n: int = 10, rng: np.random.Generator | None = None) -> Hamiltonian:
    """SYK Majorana model of the paper's second experiment (Sec. 4) on n
    qubits (N = 2n Majorana operators): H = sum_{i<j<k<l} J_ijkl c_i c_j c_k
    c_l with c from ``majorana_strings`` and real J_ijkl ~ N(0, 1), in
    lexicographic (i, j, k, l) order; C(2n, 4) terms.  The paper draws complex
    J with J_ijkl = J*_lkji, which is inconsistent for distinct indices: the
    product of four distinct Majorana operators is Hermitian, so a Hermitian H
    needs real coefficients.  Each product is +-1 times one Pauli string; the
    sign goes into the coefficient."""
    if rng is None:
        rng = np.random.default_rng(SEED_BASE + 6)
    maj = majorana_strings(n)
    N = 2 * n
    xs, zs, sg = [], [], []
    for i in range(N):
        for j in range(i + 1, N):
            xij, zij, kij = _pauli_product(maj[i], maj[j])
            for k in range(j + 1, N):
                x3, z3, k3 = _pauli_product((xij, zij), maj[k])
                for l in range(k + 1, N):
                    x4, z4, k4 = _pauli_product((x3, z3), maj[l])
                    ph = (kij + k3 + k4) % 4
                    if ph % 2:
                        raise AssertionError("a product of four Majorana operators is Hermitian")
                    xs.append(x4)
                    zs.append(z4)
                    sg.append(1.0 if ph == 0 else -1.0)
    J = rng.standard_normal(len(xs))
    return Hamiltonian(n, np.array(xs, dtype=np.uint64), np.array(zs, dtype=np.uint64),
                       J * np.array(sg))


def z_average_observable(n: int):
    """O = sum_i Z_i / n as (x, z, c) arrays."""
    x = np.zeros(n, dtype=np.uint64)
    z = np.array([1 << i for i in range(n)], dtype=np.uint64)
    c = np.full(n, 1.0 / n)
    return x, z, c


# ------------------------------------------------------------ initial states

def haar_product_factors(n: int, rng: np.random.Generator) -> np.ndarray:
    """Per-qubit single-qubit states: two i.i.d. complex normals per qubit,
    normalised.  Row q is (amplitude of |0>, amplitude of |1>) of qubit q."""
    v = rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v.astype(np.complex128)


def product_state(factors: np.ndarray, dtype=np.complex128) -> np.ndarray:
    """Kronecker product with qubit 0 as the least-significant index bit."""
    psi = np.ones(1, dtype=np.complex128)
    for q in range(factors.shape[0]):
        # new index = old index + 2^q * b_q
        psi = np.concatenate([psi * factors[q, 0], psi * factors[q, 1]])
    return psi.astype(dtype)


def plus_state(n: int, dtype=np.complex128) -> np.ndarray:
    return np.full(1 << n, 2.0 ** (-n / 2), dtype=dtype)


def basis_state(n: int, index: int, dtype=np.complex128) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=dtype)
    psi[index] = 1.0
    return psi
