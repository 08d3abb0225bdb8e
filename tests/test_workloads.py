"""Generators of the workloads: the paper's two experiment Hamiltonians
(Sec. 4), checked against their definitions with dense matrices built from
the single-qubit Pauli matrices (not from the generators' (x, z) encoding),
and the generators of the measured configurations, checked against their
recipes."""
import itertools

import numpy as np

from oracle import planner as P
from tests.dense import SX, SY, SZ, pauli, single
from workloads import majorana_strings, syk_majorana, tfim_fully_connected


def _majorana_dense(n):
    """c_{2q} = Z_0..Z_{q-1} X_q, c_{2q+1} = Z_0..Z_{q-1} Y_q as dense matrices."""
    out = []
    for q in range(n):
        zs = np.eye(1 << n, dtype=complex)
        for p in range(q):
            zs = single(n, p, SZ) @ zs
        out.append(zs @ single(n, q, SX))
        out.append(zs @ single(n, q, SY))
    return out


def _dense(h):
    return sum(c * pauli(h.n, int(x), int(z)) for x, z, c in zip(h.x, h.z, h.c))


def test_majorana_operators():
    for n in (2, 3, 4):
        dense = _majorana_dense(n)
        masks = majorana_strings(n)
        for a, (x, z) in zip(dense, masks):
            assert np.allclose(a, pauli(n, x, z))
        for i, j in itertools.product(range(2 * n), repeat=2):
            ac = dense[i] @ dense[j] + dense[j] @ dense[i]
            assert np.allclose(ac, 2 * np.eye(1 << n) * (i == j))


def test_syk_equals_majorana_sum():
    for n in (3, 4):
        h = syk_majorana(n, np.random.default_rng(5))
        N = 2 * n
        assert h.m == N * (N - 1) * (N - 2) * (N - 3) // 24
        dense = _majorana_dense(n)
        rng = np.random.default_rng(5)
        J = rng.standard_normal(h.m)
        H = np.zeros((1 << n, 1 << n), dtype=complex)
        for t, (i, j, k, l) in enumerate(itertools.combinations(range(N), 4)):
            H += J[t] * (dense[i] @ dense[j] @ dense[k] @ dense[l])
        assert np.allclose(H, H.conj().T)
        assert np.allclose(_dense(h), H)


def test_tfim_fully_connected_structure():
    n = 7
    h = tfim_fully_connected(n, np.random.default_rng(1))
    assert h.m == n * (n - 1) // 2 + n
    assert np.all(np.abs(h.c) <= 1.0)
    zz = [(int(x), int(z)) for x, z in zip(h.x, h.z)][: n * (n - 1) // 2]
    assert all(x == 0 and bin(z).count("1") == 2 for x, z in zz)
    groups = P.greedy_partition(h.x, h.z)
    assert len(groups) == 2 and len(groups[0]) == n * (n - 1) // 2


# ---------------------------------------------------------------- the configurations' generators

def _weights(h):
    return np.array([bin(int(x) | int(z)).count("1") for x, z in zip(h.x, h.z)])


def test_configuration_generators_follow_their_recipes():
    """The seeded generators of the measured configurations have the stated
    sizes, structure and coefficient distributions."""
    from workloads import (batch_instances, gradient_2local, heisenberg_lattice, jw_like,
                           neel_index, tfim_chain)
    t = tfim_chain(10)
    assert t.m == 19 and np.all(_weights(t)[:9] == 2) and np.all(_weights(t)[9:] == 1)
    assert np.all(t.c[:9] == 1.0) and np.all(t.c[9:] == 0.9)
    for (rows, cols, corners), n, m in (((5, 6, False), 30, 147), ((6, 6, True), 32, 156)):
        h = heisenberg_lattice(rows, cols, drop_corners=corners)
        assert (h.n, h.m) == (n, m) and np.all(_weights(h) == 2) and np.all(h.c == 1.0)
        assert len(P.greedy_partition(h.x, h.z)) == 3
    assert bin(neel_index(5, 6)).count("1") == 15
    for h, factors in batch_instances(4):
        assert 16 <= h.n <= 24 and h.m == 2000
        assert set(_weights(h)) <= {2, 3, 4} and abs(np.abs(h.c).sum() - h.n) < 1e-9
        assert np.allclose(np.linalg.norm(factors, axis=1), 1.0)
    jw = jw_like()
    w = _weights(jw)
    assert jw.m == 20000 and jw.n == 26
    assert np.all(jw.x[:5000] == 0) and set(w[:5000]) == {1, 2}
    for x, z in zip(jw.x[5000:], jw.z[5000:]):
        x, z = int(x), int(z)
        i, j = (x & -x).bit_length() - 1, x.bit_length() - 1     # the two X/Y ends
        assert bin(x).count("1") == 2
        between = ((1 << j) - 1) & ~((1 << (i + 1)) - 1)
        assert z & between == between and (z >> i & 1) == (z >> j & 1)
    assert np.all((np.abs(jw.c) >= 1e-4) & (np.abs(jw.c) <= 1.0)) and (jw.c < 0).any()
    g = gradient_2local()
    assert (g.n, g.m) == (24, 200) and np.all(_weights(g) == 2) and np.all(np.abs(g.c) <= 1.0)
