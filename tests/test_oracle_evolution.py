"""Pins for the oracle's evolution, expectation and gradient (CPU only).

The oracle applies one rotation exp(-i c_j dt P_j) at a time.  It is pinned
to dense matrix exponentials (scipy.linalg.expm of whole group Hamiltonians,
which equals the product of the group's rotations only if they commute),
to the Trotter error orders, to norm and energy conservation, to Strang
time-reversal symmetry, to closed forms and to central finite differences.
"""
import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from oracle import planner as P
from workloads import random_klocal, product_state, haar_product_factors, from_strings
from tests import dense as D


def _rand_state(rng, n):
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


def test_rotation_matches_expm():
    rng = np.random.default_rng(0)
    n = 4
    for _ in range(30):
        x, z = (int(v) for v in rng.integers(0, 1 << n, size=2))
        th = float(rng.uniform(-2, 2))
        psi = _rand_state(rng, n)
        ref = expm(-1j * th * D.pauli(n, x, z)) @ psi
        assert np.allclose(oracle.apply_rotation(psi, x, z, th), ref, atol=1e-13)
        assert np.allclose(oracle.apply_pauli(psi, x, z), D.pauli(n, x, z) @ psi, atol=1e-14)


@pytest.mark.parametrize("order", [1, 2])
def test_one_step_equals_product_of_group_exponentials(order):
    rng = np.random.default_rng(1 + order)
    for _ in range(6):
        n = int(rng.integers(3, 7))
        h = random_klocal(n, int(rng.integers(5, 25)), rng, weights=(1, 2, 3))
        groups = P.greedy_partition(h.x, h.z)
        dt = 0.3
        Hg = [D.hamiltonian(n, h.x[g], h.z[g], h.c[g]) for g in groups]
        U = np.eye(1 << n, dtype=complex)
        if order == 1:
            for Hk in Hg:
                U = expm(-1j * dt * Hk) @ U
        else:
            G = len(Hg)
            seq = [(k, 0.5) for k in range(G - 1)] + [(G - 1, 1.0)] + \
                  [(k, 0.5) for k in reversed(range(G - 1))]
            for k, f in seq:
                U = expm(-1j * f * dt * Hg[k]) @ U
        psi = _rand_state(rng, n)
        out = oracle.evolve(h, psi, dt, 3, order=order, groups=groups)
        ref = np.linalg.matrix_power(U, 3) @ psi
        assert np.linalg.norm(out - ref) < 1e-12


def test_norm_preserved():
    rng = np.random.default_rng(4)
    h = random_klocal(10, 60, rng)
    psi = _rand_state(rng, 10)
    out = oracle.evolve(h, psi, 0.05, 20, order=2)
    assert abs(np.linalg.norm(out) - 1.0) < 1e-13


def test_trotter_error_orders():
    """One-step error against exp(-iH dt): O(dt^2) first order, O(dt^3)
    second order (log-log slopes)."""
    rng = np.random.default_rng(9)
    n = 6
    h = random_klocal(n, 30, rng, weights=(1, 2))
    groups = P.greedy_partition(h.x, h.z)
    assert len(groups) >= 3
    H = D.hamiltonian(n, h.x, h.z, h.c)
    psi = _rand_state(rng, n)
    dts = np.array([0.04, 0.02, 0.01, 0.005])
    for order, slope in ((1, 2.0), (2, 3.0)):
        err = [np.linalg.norm(oracle.evolve(h, psi, dt, 1, order, groups) - expm(-1j * dt * H) @ psi)
               for dt in dts]
        fit = np.polyfit(np.log(dts), np.log(err), 1)[0]
        assert abs(fit - slope) < 0.15, (order, fit)


def test_single_group_is_exact_and_conserves_energy():
    rng = np.random.default_rng(12)
    n = 6
    h = from_strings(["ZZIIII", "XXIIII", "YYIIII", "XXXXII", "IIZZZI", "IIIIZZ", "IIXXII"],
                     rng.uniform(-1, 1, 7))
    groups = P.greedy_partition(h.x, h.z)
    assert len(groups) == 1
    H = D.hamiltonian(n, h.x, h.z, h.c)
    psi = _rand_state(rng, n)
    out = oracle.evolve(h, psi, 0.1, 40)
    assert np.linalg.norm(out - expm(-1j * 4.0 * H) @ psi) < 1e-12
    e0 = oracle.expect(psi, h.x, h.z, h.c)
    e1 = oracle.expect(out, h.x, h.z, h.c)
    assert abs(e0 - e1) < 1e-12


def test_energy_drift_bounded():
    rng = np.random.default_rng(13)
    n = 8
    h = random_klocal(n, 40, rng, weights=(2,))
    psi = product_state(haar_product_factors(n, rng))
    e0 = oracle.expect(psi, h.x, h.z, h.c)
    drift = {}
    for order in (1, 2):
        dt = 0.02
        st = psi
        worst = 0.0
        for _ in range(10):
            st = oracle.evolve(h, st, dt, 5, order)
            worst = max(worst, abs(oracle.expect(st, h.x, h.z, h.c) - e0))
        drift[order] = worst
    assert drift[2] < drift[1] < 0.05
    assert drift[2] < 1e-3


def test_strang_time_reversal():
    """S2(dt) S2(-dt) = I for the symmetric splitting (not for first order)."""
    rng = np.random.default_rng(14)
    h = random_klocal(7, 40, rng)
    psi = _rand_state(rng, 7)
    back = oracle.evolve(h, oracle.evolve(h, psi, 0.1, 1, 2), -0.1, 1, 2)
    assert np.linalg.norm(back - psi) < 1e-13
    back1 = oracle.evolve(h, oracle.evolve(h, psi, 0.1, 1, 1), -0.1, 1, 1)
    assert np.linalg.norm(back1 - psi) > 1e-4


def test_expect_matches_dense():
    rng = np.random.default_rng(15)
    n = 5
    h = random_klocal(n, 12, rng, weights=(1, 2, 3))
    psi = _rand_state(rng, n)
    H = D.hamiltonian(n, h.x, h.z, h.c)
    assert abs(oracle.expect(psi, h.x, h.z, h.c) - np.vdot(psi, H @ psi).real) < 1e-13


def test_grad_closed_form():
    """H = c Z_0 on |+>: <X_0>(T) = cos(2 c T), d/dc = -2 T sin(2 c T)."""
    h = from_strings(["ZI"], [0.7])
    psi = np.full(4, 0.5, dtype=complex)
    obs = (np.array([1], np.uint64), np.array([0], np.uint64), np.array([1.0]))
    T = 0.05 * 20
    f, g = oracle.grad(h, psi, 0.05, 20, 1, obs)
    assert abs(f - np.cos(2 * 0.7 * T)) < 1e-13
    assert abs(g[0] + 2 * T * np.sin(2 * 0.7 * T)) < 1e-12


@pytest.mark.parametrize("order", [1, 2])
def test_grad_matches_central_differences(order):
    rng = np.random.default_rng(16 + order)
    n = 5
    h = random_klocal(n, 14, rng, weights=(1, 2))
    psi = _rand_state(rng, n)
    ox = np.zeros(n, np.uint64)
    oz = np.array([1 << q for q in range(n)], np.uint64)
    oc = np.full(n, 1.0 / n)
    dt, steps = 0.07, 4
    groups = P.greedy_partition(h.x, h.z)
    f, g = oracle.grad(h, psi, dt, steps, order, (ox, oz, oc), groups)
    hh = 1e-6
    for j in range(h.m):
        cp = h.c.copy(); cp[j] += hh
        cm = h.c.copy(); cm[j] -= hh
        hp = type(h)(n, h.x, h.z, cp)
        hm = type(h)(n, h.x, h.z, cm)
        fp = oracle.expect(oracle.evolve(hp, psi, dt, steps, order, groups), ox, oz, oc)
        fm = oracle.expect(oracle.evolve(hm, psi, dt, steps, order, groups), ox, oz, oc)
        fd = (fp - fm) / (2 * hh)
        assert abs(g[j] - fd) < 1e-7 * max(1.0, abs(g[j]))
    assert abs(f - oracle.expect(oracle.evolve(h, psi, dt, steps, order, groups), ox, oz, oc)) < 1e-13
