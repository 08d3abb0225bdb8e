"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: ||psi_gpu - psi_oracle||_2 <= 1e-10 for complex128 states and
<= 1e-4 for complex64 states (both with the oracle in complex128).  The
oracle applies one rotation at a time in group order; the GPU applies whole
groups through their Clifford frames, so agreement is up to rounding only.
"""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import planner as P
from workloads import (from_strings, heisenberg_lattice, jw_like, neel_index, random_klocal,
                       tfim_chain, basis_state, plus_state, product_state, haar_product_factors,
                       tfim_fully_connected, syk_majorana,
                       gradient_2local, z_average_observable)
from workloads.generators import Hamiltonian

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 1e-4}


@pytest.fixture(scope="module")
def sd():
    import torch
    import paper_2206_11664_gb300 as m
    assert torch.cuda.is_available()
    return m


def _dev(psi, dt):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(psi)).to(torch.complex128 if dt == "c128" else torch.complex64)
    return t.cuda()


def _host(t):
    return t.cpu().numpy().astype(np.complex128)


def _rand_state(rng, n):
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


def _check(sd, h, psi0, dt_, steps, order, dtype, skip_rule=-1, tile_bits=0, pauli=False, jit=0,
           grouping=0, layout=0, prefetch=0):
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan(skip_rule=skip_rule, tile_bits=tile_bits, jit=jit,
                                                grouping=grouping, layout=layout, prefetch=prefetch)
    groups = P.partition(h.x, h.z, grouping, h.c)
    ref = oracle.evolve(h, psi0, dt_, steps, order, groups)
    t = _dev(psi0, dtype)
    if pauli:
        sim.evolve_pauli(t, dt_, steps, order)
    else:
        sim.evolve(t, dt_, steps, order)
    err = np.linalg.norm(_host(t) - ref)
    assert err <= TOL[dtype], (h.n, dtype, order, err)
    return err


# ---------------------------------------------------------------- on-chip path (small n)

@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("order", [1, 2])
def test_small_random(sd, dtype, order):
    rng = np.random.default_rng(100 + order)
    for n in (1, 2, 3, 5, 8, 11):
        h = random_klocal(n, 3 * n + 4, rng, weights=tuple(w for w in (1, 2, 3, 4) if w <= n))
        _check(sd, h, _rand_state(rng, n), 0.07, 5, order, dtype)


def test_worked_example_group(sd):
    ex = ["YIXI", "IXIY", "XZYZ", "YZXZ", "XIYI", "IYIX", "ZXZY", "ZYZX"]
    rng = np.random.default_rng(3)
    h = from_strings(ex, rng.uniform(-1, 1, 8))
    for rule in (0, 1, 2):
        _check(sd, h, _rand_state(rng, 4), 0.2, 3, 1, "c128", skip_rule=rule)


def test_tfim_chain_config(sd):
    """TFIM open chain n=10, J=1, h=0.9, |0..0>, dt=0.01, 100 first-order steps,
    complex128, <Z_0> after every step."""
    import torch
    h = tfim_chain(10)
    psi0 = basis_state(10, 0)
    err = _check(sd, h, psi0, 0.01, 100, 1, "c128")
    assert err < 1e-12
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    t = _dev(psi0, "c128")
    obs = (np.array([0], np.uint64), np.array([1], np.uint64), np.array([1.0]))
    trace = torch.zeros(100, dtype=torch.float64, device="cuda")
    sim.evolve_observe(t, 0.01, 100, obs, trace)
    tr = trace.cpu().numpy()
    groups = P.greedy_partition(h.x, h.z)
    st = psi0
    ref = []
    for k in range(100):
        st = oracle.evolve(h, st, 0.01, 1, 1, groups)
        ref.append(oracle.expect(st, *obs))
    assert np.max(np.abs(tr - np.array(ref))) < 1e-12


# ---------------------------------------------------------------- tile path (several tiles)

@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("rule", [0, 2])
def test_tile_random_klocal(sd, dtype, rule):
    rng = np.random.default_rng(7 + rule)
    for n in (14, 16):
        h = random_klocal(n, 60, rng, weights=(2, 3, 4))
        _check(sd, h, _rand_state(rng, n), 0.05, 2, 2, dtype, skip_rule=rule)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("K", [9, 10, 11, 12, 13])
def test_tile_sizes(sd, dtype, K):
    rng = np.random.default_rng(K)
    n = 15
    h = random_klocal(n, 40, rng, weights=(1, 2, 3))
    _check(sd, h, _rand_state(rng, n), 0.1, 2, 1, dtype, tile_bits=K)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_tile_heisenberg_lattice(sd, dtype):
    h = heisenberg_lattice(4, 4)
    psi0 = basis_state(16, neel_index(4, 4))
    for rule in (0, 1, 2):
        _check(sd, h, psi0, 0.02, 10, 1, dtype, skip_rule=rule)
    # second order over 6 steps: head, one block of 4 merged cores, one core, tail
    _check(sd, h, psi0, 0.02, 6, 2, dtype)


def test_tile_jw_like(sd):
    rng = np.random.default_rng(5)
    h = jw_like(n=15, m=600, rng=rng)
    psi0 = basis_state(15, (1 << 7) - 1)
    _check(sd, h, psi0, 0.05, 3, 2, "c128")
    _check(sd, h, psi0, 0.05, 3, 2, "c64")


@pytest.mark.parametrize("grouping", [1, 2, 3])
def test_grouping_variants(sd, grouping):
    """Largest-first, DSATUR and |c|-ordered partitions evolve like the
    oracle does with the same groups (tile path, both orders)."""
    rng = np.random.default_rng(80 + grouping)
    h = random_klocal(15, 80, rng, weights=(2, 3, 4))
    _check(sd, h, _rand_state(rng, 15), 0.05, 2, 1, "c128", grouping=grouping)
    _check(sd, h, _rand_state(rng, 15), 0.05, 2, 2, "c64", grouping=grouping)


@pytest.mark.parametrize("jit", [-1, 1])
def test_large_diagonal_groups(sd, jit):
    """Groups of Z-strings only (no Clifford): 1500 terms, whose terms the
    passes keep in shared memory, and 5000 terms, read from global memory
    instead; many terms share a slot (class and fixed-position mask)."""
    rng = np.random.default_rng(90)
    n = 16
    for m in (1500, 5000):
        z = rng.integers(1, 1 << n, size=m, dtype=np.uint64) & rng.integers(0, 1 << n, size=m, dtype=np.uint64)
        z[z == 0] = 1
        from workloads import Hamiltonian
        h = Hamiltonian(n, np.zeros(m, dtype=np.uint64), z, rng.uniform(-1, 1, size=m))
        for dtype in ("c128", "c64"):
            _check(sd, h, _rand_state(rng, n), 0.05, 2, 1, dtype, jit=jit)


@pytest.mark.parametrize("order", [1, 2])
def test_split_calls_resume(sd, order):
    """The state is the checkpoint: evolving 3 steps, copying the state to the
    host and back, then evolving 6 more gives the 9-step evolution (each call
    opens and closes its own half steps in second order, and runs its own
    block programs, so only the rounding differs), and both match the oracle."""
    import torch
    h = heisenberg_lattice(4, 5)                      # n = 20: run-time compiled passes
    rng = np.random.default_rng(92 + order)
    psi0 = _rand_state(rng, h.n)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    groups = P.greedy_partition(h.x, h.z)
    ref = oracle.evolve(h, psi0, 0.02, 9, order, groups)
    for dtype in ("c128", "c64"):
        whole = _dev(psi0, dtype)
        sim.evolve(whole, 0.02, 9, order)
        part = _dev(psi0, dtype)
        sim.evolve(part, 0.02, 3, order)
        saved = part.cpu()                             # checkpoint on the host
        part = saved.cuda()
        sim.evolve(part, 0.02, 6, order)
        diff = torch.linalg.vector_norm((whole - part).to(torch.complex128)).item()
        assert diff <= TOL[dtype], (dtype, diff)
        for t in (whole, part):
            assert np.linalg.norm(_host(t) - ref) <= TOL[dtype]


def test_trivial_calls(sd):
    """steps = 0 leaves the state alone; dt = 0 is the identity within the
    tolerance; a Hamiltonian of single-qubit X terms on the tile path."""
    import torch
    h = heisenberg_lattice(4, 4)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    rng = np.random.default_rng(91)
    psi0 = _rand_state(rng, h.n)
    t = _dev(psi0, "c128")
    sim.evolve(t, 0.02, 0, 1)
    assert torch.equal(t, _dev(psi0, "c128"))
    sim.evolve(t, 0.0, 3, 2)
    assert np.linalg.norm(_host(t) - psi0) <= TOL["c128"]
    hx = from_strings(["I" * q + "X" + "I" * (15 - q) for q in range(16)], rng.uniform(-1, 1, 16))
    _check(sd, hx, _rand_state(rng, 16), 0.1, 3, 1, "c64")


def test_paper_models(sd):
    """The paper's two experiment Hamiltonians (Sec. 4): the fully connected
    transverse-field Ising model (2 groups, 10 steps on the tile path, both
    precisions) and the SYK Majorana model on 14 qubits (20475 terms, 816
    groups, tile path)."""
    rng = np.random.default_rng(64)
    h = tfim_fully_connected(16, rng)
    for dtype in ("c128", "c64"):
        _check(sd, h, _rand_state(rng, 16), 0.02, 10, 1, dtype)
    hs = syk_majorana(14, rng)
    groups = P.greedy_partition(hs.x, hs.z)      # one oracle grouping for both checks
    sim = sd.Simulator(hs.n, hs.x, hs.z, hs.c).plan()
    assert sim.plan_view()["n_groups"] == len(groups)
    for dtype, order in (("c128", 1), ("c64", 2)):
        psi0 = _rand_state(rng, 14)
        ref = oracle.evolve(hs, psi0, 0.01, 1, order, groups)
        t = _dev(psi0, dtype)
        sim.evolve(t, 0.01, 1, order)
        err = np.linalg.norm(_host(t) - ref)
        assert err <= TOL[dtype], (dtype, err)


def test_tile_gradient_hamiltonian_plus_state(sd):
    rng = np.random.default_rng(6)
    h = gradient_2local(n=16, m=80, rng=rng)
    _check(sd, h, plus_state(16), 0.01, 5, 1, "c128")


def test_identity_and_single_terms(sd):
    h = from_strings(["IIIIIIIIIIIIII", "XIIIIIIIIIIIII", "IIIIIIIIIIIIIZ", "YYYYYYYYYYYYYY"],
                     [0.3, -0.7, 1.1, 0.4])
    rng = np.random.default_rng(9)
    _check(sd, h, _rand_state(rng, 14), 0.3, 4, 2, "c128")


# ---------------------------------------------------------------- baseline path

@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_per_pauli_path(sd, dtype):
    rng = np.random.default_rng(21)
    for n in (6, 15):
        h = random_klocal(n, 30, rng, weights=(1, 2, 3))
        _check(sd, h, _rand_state(rng, n), 0.05, 2, 2, dtype, pauli=True)


# ---------------------------------------------------------------- expectation, gradient, batch

@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_expectation(sd, dtype):
    rng = np.random.default_rng(31)
    for n in (5, 15):
        h = random_klocal(n, 20, rng, weights=(1, 2, 3))
        psi = _rand_state(rng, n)
        sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
        got = sim.expect(_dev(psi, dtype), (h.x, h.z, h.c))
        ref = oracle.expect(psi, h.x, h.z, h.c)
        assert abs(got - ref) < (1e-12 if dtype == "c128" else 1e-5) * max(1, abs(ref))


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("n", [6, 14])
def test_gradient_vs_oracle(sd, order, n):
    rng = np.random.default_rng(50 + n + order)
    h = gradient_2local(n=n, m=24, rng=rng)
    psi0 = plus_state(n)
    obs = z_average_observable(n)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    t = _dev(psi0, "c128")
    f, g = sim.grad(t, 0.05, 4, obs, order)
    f_ref, g_ref = oracle.grad(h, psi0, 0.05, 4, order, obs)
    assert abs(f - f_ref) < 1e-12
    assert np.max(np.abs(g - g_ref)) < 1e-9 * max(1.0, np.max(np.abs(g_ref)))
    assert np.allclose(_host(t), psi0)   # state0 untouched


def test_gradient_large_group(sd):
    """A commuting group of 120 diagonal terms beside 12 X terms: the adjoint
    kernel sums a group of more than 80 terms per warp instead of per thread;
    value and gradient against the oracle (complex128, both orders)."""
    rng = np.random.default_rng(59)
    n = 12
    z = rng.integers(1, 1 << n, size=120, dtype=np.uint64)
    x = np.array([1 << (i % n) for i in range(12)], dtype=np.uint64)
    h = Hamiltonian(n, np.concatenate([np.zeros(120, dtype=np.uint64), x]),
                    np.concatenate([z, np.zeros(12, dtype=np.uint64)]), rng.uniform(-1, 1, 132))
    psi0 = plus_state(n)
    obs = z_average_observable(n)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    assert max(np.diff(sim.plan_view()["group_offsets"])) > 80
    for order in (1, 2):
        f, g = sim.grad(_dev(psi0, "c128"), 0.05, 3, obs, order)
        f_ref, g_ref = oracle.grad(h, psi0, 0.05, 3, order, obs)
        assert abs(f - f_ref) < 1e-12
        assert np.max(np.abs(g - g_ref)) < 1e-9 * max(1.0, np.max(np.abs(g_ref)))


@pytest.mark.parametrize("jit", [-1, 1])
def test_gradient_complex64(sd, jit):
    """Complex64 states with FP64 reductions in the adjoint: value and
    gradient against the complex128 oracle (tile path, both orders)."""
    rng = np.random.default_rng(57 + jit)
    n = 14
    h = gradient_2local(n=n, m=24, rng=rng)
    psi0 = plus_state(n)
    obs = z_average_observable(n)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan(jit=jit)
    for order in (1, 2):
        f, g = sim.grad(_dev(psi0, "c64"), 0.05, 4, obs, order)
        f_ref, g_ref = oracle.grad(h, psi0, 0.05, 4, order, obs)
        assert abs(f - f_ref) < 1e-5
        assert np.max(np.abs(g - g_ref)) < 1e-4 * max(1.0, np.max(np.abs(g_ref)))


def test_gradient_autograd_function(sd):
    import torch
    rng = np.random.default_rng(77)
    n = 8
    h = gradient_2local(n=n, m=12, rng=rng)
    obs = z_average_observable(n)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    t = _dev(plus_state(n), "c128")
    c = torch.tensor(h.c, dtype=torch.float64, requires_grad=True)
    f = sd.TrotterExpectation.apply(c, sim, t, 0.05, 3, obs, 1)
    f.backward()
    _, g_ref = oracle.grad(h, plus_state(n), 0.05, 3, 1, obs)
    assert np.max(np.abs(c.grad.numpy() - g_ref)) < 1e-9


@pytest.mark.parametrize("dtype,order", [("c64", 2), ("c128", 1), ("c128", 2)])
def test_batch_levels_match_oracle(sd, dtype, order):
    """Tile-path problems of different sizes advanced level by level in shared
    launches (plus one on-chip problem), against the oracle."""
    rng = np.random.default_rng(91 + order)
    sims, states, refs = [], [], []
    for n in (14, 17, 15, 11, 16):
        h = random_klocal(n, 40, rng, weights=(2, 3))
        psi = product_state(haar_product_factors(n, rng))
        sims.append(sd.Simulator(h.n, h.x, h.z, h.c).plan())
        states.append(_dev(psi, dtype))
        refs.append(oracle.evolve(h, psi, 0.01, 3, order))
    sd.evolve_batch(sims, states, 0.01, 3, order)
    for t, r in zip(states, refs):
        assert np.linalg.norm(_host(t) - r) < TOL[dtype]


def test_batch_matches_individual(sd):
    rng = np.random.default_rng(90)
    sims, states, refs = [], [], []
    for i in range(4):
        n = int(rng.integers(9, 15))
        h = random_klocal(n, 40, rng)
        psi = product_state(haar_product_factors(n, rng))
        sims.append(sd.Simulator(h.n, h.x, h.z, h.c).plan())
        states.append(_dev(psi, "c64"))
        refs.append(oracle.evolve(h, psi, 0.005, 3, 2))
    sd.evolve_batch(sims, states, 0.005, 3, 2)
    for t, r in zip(states, refs):
        assert np.linalg.norm(_host(t) - r) < 1e-4


def test_batch_with_large_instance(sd):
    """A batch mixing an instance large enough to run on its own (n = 21,
    passes compiled at run time) with small ones sharing the level launches
    gives what separate sd_evolve calls give."""
    import torch
    rng = np.random.default_rng(93)
    sims, states, refs = [], [], []
    for n in (15, 21, 16):
        h = random_klocal(n, 50, rng, weights=(2, 3))
        psi = _rand_state(rng, n)
        sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
        sims.append(sim)
        states.append(_dev(psi, "c64"))
        r = _dev(psi, "c64")
        sim.evolve(r, 0.01, 3, 2)
        refs.append(r)
    sd.evolve_batch(sims, states, 0.01, 3, 2)
    for t, r in zip(states, refs):
        assert torch.linalg.vector_norm((t - r).to(torch.complex128)).item() < 1e-5


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_autotune_tile_size(sd, dtype):
    """The autotuner times tile sizes on its own scratch state, keeps the
    fastest for the dtype, leaves the caller's state alone, and the tuned
    path still matches the oracle."""
    import torch
    h = heisenberg_lattice(4, 4)
    code = sd.C64 if dtype == "c64" else sd.C128
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    psi0 = basis_state(16, neel_index(4, 4))
    t = _dev(psi0, dtype)
    before = t.clone()
    best, times = sim.autotune(code, 0.02, steps=4, order=1, kmin=10, kmax=13)
    assert torch.equal(t, before)
    assert best in times and min(times, key=times.get) == best
    assert set(times) <= {10, 11, 12, 13} and all(v > 0 for v in times.values())
    assert sim.schedule_stats(code, 1)["tile_bits"] == best
    groups = P.greedy_partition(h.x, h.z)
    ref = oracle.evolve(h, psi0, 0.02, 6, 1, groups)
    sim.evolve(t, 0.02, 6, 1)
    assert np.linalg.norm(_host(t) - ref) <= TOL[dtype]
    with pytest.raises(sd.SDError):
        sim.autotune(code, 0.02, kmin=8, kmax=13)


def test_cuda_graph_capture(sd):
    """Once its programs are built, sd_evolve only launches kernels, and so
    does a prepared sd_evolve_batch: both are captured into a CUDA graph and
    replayed, and must give exactly what the same calls give eagerly."""
    import torch
    rng = np.random.default_rng(65)
    h = heisenberg_lattice(4, 5)                       # n = 20: passes compiled at run time
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    psi0 = _rand_state(rng, h.n)
    ref = _dev(psi0, "c64")
    for _ in range(2):
        sim.evolve(ref, 0.02, 5, 1)
    t = _dev(psi0, "c64")
    sim.prepare(sd.C64, 0.02, 5, 1)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        sim.evolve(t, 0.02, 5, 1)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(t, ref)

    hs = [random_klocal(n, 60, rng, weights=(2, 3)) for n in (12, 15, 17)]   # on chip and tile path
    sims = [sd.Simulator(x.n, x.x, x.z, x.c).plan() for x in hs]
    psis = [_rand_state(rng, x.n) for x in hs]
    refs = [_dev(p, "c128") for p in psis]
    for _ in range(2):
        sd.evolve_batch(sims, refs, 0.03, 3, 2)
    ts = [_dev(p, "c128") for p in psis]
    sd.prepare_batch(sims, ts, 0.03, 3, 2)
    gb = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gb):
        sd.evolve_batch(sims, ts, 0.03, 3, 2)
    for _ in range(2):
        gb.replay()
    torch.cuda.synchronize()
    for a, b in zip(ts, refs):
        assert torch.equal(a, b)
    # capturing a batch whose descriptors were not built is refused, not run
    other = [_dev(p, "c128") for p in psis]
    g2 = torch.cuda.CUDAGraph()
    with pytest.raises(sd.SDError):
        with torch.cuda.graph(g2):
            sd.evolve_batch(sims, other, 0.03, 3, 2)


def test_evolve_host(sd):
    """sd_evolve_host: pinned host state in, the same result as sd_evolve on
    a device copy out; pageable host memory is refused."""
    import torch
    rng = np.random.default_rng(66)
    h = heisenberg_lattice(4, 4)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    psi0 = _rand_state(rng, h.n)
    ref = _dev(psi0, "c64")
    sim.evolve(ref, 0.02, 5, 1)
    host = torch.from_numpy(psi0.astype(np.complex64)).pin_memory()
    work = torch.empty_like(ref)
    sim.evolve_host(host, work, 0.02, 5, 1)
    torch.cuda.synchronize()
    assert torch.equal(host, ref.cpu())
    pageable = torch.from_numpy(psi0.astype(np.complex64))
    with pytest.raises(ValueError):
        sim.evolve_host(pageable, work, 0.02, 1, 1)
    N = sd._native
    st = sim._lib.sd_evolve_host(sim._h, ctypes.c_void_p(pageable.data_ptr()), ctypes.c_void_p(work.data_ptr()),
                                 N.SD_C64, 0.02, 1, 1, None)
    assert st == N.SD_EINVAL


def test_invalid_state_rejected(sd):
    import torch
    h = tfim_chain(10)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    with pytest.raises(TypeError):
        sim.evolve(torch.zeros(1024, dtype=torch.complex64), 0.1, 1)
    with pytest.raises(sd.SDError):
        sim.evolve(torch.zeros(1024, dtype=torch.complex64, device="cuda"), 0.1, 1, order=3)
    # a view that starts 8 bytes into an allocation is refused before any launch
    big = torch.zeros(1025, dtype=torch.complex64, device="cuda")
    with pytest.raises(sd.SDError, match="16-byte aligned"):
        sim.evolve(big[1:], 0.1, 1)


# ---------------------------------------------------------------- run-time specialised passes

@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_jit_heisenberg_and_random(sd, dtype):
    """Passes compiled at run time (NVRTC) against the oracle: Hadamard-type
    layers, CNOT permutations, S/CZ layers, several tiles, both orders."""
    h = heisenberg_lattice(4, 4)
    _check(sd, h, basis_state(16, neel_index(4, 4)), 0.02, 6, 1, dtype, jit=1)
    rng = np.random.default_rng(61)
    h2 = random_klocal(15, 50, rng, weights=(2, 3, 4))
    _check(sd, h2, _rand_state(rng, 15), 0.05, 2, 2, dtype, skip_rule=0, jit=1)
    _check(sd, h2, _rand_state(rng, 15), 0.05, 2, 1, dtype, tile_bits=11, jit=1)


@pytest.mark.parametrize("order", [1, 2])
def test_paired_layout(sd, order):
    """Complex64 passes compiled at run time in the paired layout (qubit 0
    kept in registers, amplitudes packed in f32x2 pairs) against the oracle:
    Hadamard-type layers in 4-step blocks (Heisenberg), CNOT permutations and
    S/CZ layers (random k-local with skip rule 0, whose passes with such
    rounds keep the plain code inside a paired schedule), a 120-term diagonal
    group (fully connected Ising), and a smaller tile size."""
    h = heisenberg_lattice(4, 4)
    _check(sd, h, basis_state(16, neel_index(4, 4)), 0.02, 6, order, "c64", jit=1, layout=1)
    rng = np.random.default_rng(67 + order)
    h2 = random_klocal(15, 50, rng, weights=(2, 3, 4))
    for rule in (0, 2):
        _check(sd, h2, _rand_state(rng, 15), 0.05, 2, order, "c64", skip_rule=rule, jit=1, layout=1)
    _check(sd, h2, _rand_state(rng, 15), 0.05, 3, order, "c64", tile_bits=11, jit=1, layout=1)
    h3 = tfim_fully_connected(16, rng)
    _check(sd, h3, _rand_state(rng, 16), 0.02, 5, order, "c64", jit=1, layout=1)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_two_prefetch_buffers(sd, dtype):
    """Run-time passes with two prefetch buffers (two tiles in flight while a
    block works on a third) against the oracle: Heisenberg blocks, CNOT
    permutations and S/CZ layers, both orders, the paired layout, and a 2^22
    state at the default tile size, where every block runs several tiles
    through both buffers."""
    h = heisenberg_lattice(4, 4)
    _check(sd, h, basis_state(16, neel_index(4, 4)), 0.02, 6, 1, dtype, jit=1, prefetch=2)
    rng = np.random.default_rng(69)
    h2 = random_klocal(15, 50, rng, weights=(2, 3, 4))
    _check(sd, h2, _rand_state(rng, 15), 0.05, 3, 2, dtype, skip_rule=0, jit=1, prefetch=2)
    _check(sd, h2, _rand_state(rng, 15), 0.05, 2, 1, dtype, tile_bits=10, jit=1, prefetch=2)
    if dtype == "c64":
        _check(sd, h, basis_state(16, neel_index(4, 4)), 0.02, 6, 2, dtype, jit=1, layout=1, prefetch=2)
    h3 = heisenberg_lattice(2, 11)
    _check(sd, h3, _rand_state(rng, 22), 0.02, 5, 1, dtype, jit=1, prefetch=2)


def test_autotune_shape(sd, tmp_path):
    """The shape autotuner times tile sizes in both layouts of the run-time
    complex64 passes, keeps the fastest, stores it in a JSON cache that a
    second simulator applies without timing, and the tuned shape still
    matches the oracle."""
    import torch
    h = heisenberg_lattice(4, 5)                      # n = 20: passes compiled at run time
    cache = str(tmp_path / "shapes.json")
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    res = sim.autotune_shape(sd.C64, 0.02, steps=4, order=1, kmin=12, kmax=13, cache=cache)
    assert not res["cached"]
    ms = {tuple(int(v) for v in k.split(",")): t for k, t in res["ms_per_step"].items()}
    assert {lay for _, lay, _ in ms} == {-1, 1} and {pf for _, _, pf in ms} == {1, 3}
    assert all(t > 0 for t in ms.values())
    best = (res["tile_bits"], res["layout"], res["prefetch"])
    assert best in ms and ms[best] == min(ms.values())
    assert sim.schedule_stats(sd.C64, 1)["tile_bits"] == res["tile_bits"]
    again = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    res2 = again.autotune_shape(sd.C64, 0.02, steps=4, order=1, kmin=12, kmax=13, cache=cache)
    assert res2["cached"] and (res2["tile_bits"], res2["layout"], res2["prefetch"]) == best
    assert again.schedule_stats(sd.C64, 1)["tile_bits"] == res["tile_bits"]
    rng = np.random.default_rng(68)
    psi0 = _rand_state(rng, h.n)
    ref = oracle.evolve(h, psi0, 0.02, 5, 1, P.greedy_partition(h.x, h.z))
    for s_ in (sim, again):
        t = _dev(psi0, "c64")
        s_.evolve(t, 0.02, 5, 1)
        assert np.linalg.norm(_host(t) - ref) <= TOL["c64"]


def test_jit_complex128_fixed_point(sd):
    """Complex128 passes compiled at run time compute in 64-bit fixed point
    with one binary exponent per tile: CNOT permutations, S/CZ layers, many
    groups, several tile sizes, tiles that are all zero, and states far from
    unit norm (the exponent is per tile, so the relative error must not
    depend on the scale)."""
    rng = np.random.default_rng(63)
    h = random_klocal(15, 50, rng, weights=(2, 3, 4))
    for rule in (0, 1, 2):
        _check(sd, h, _rand_state(rng, 15), 0.05, 2, 2, "c128", skip_rule=rule, jit=1)
    for K in (10, 11):
        _check(sd, h, _rand_state(rng, 15), 0.05, 5, 1, "c128", tile_bits=K, jit=1)
    hj = jw_like(n=15, m=600, rng=rng)
    _check(sd, hj, basis_state(15, (1 << 7) - 1), 0.05, 3, 2, "c128", jit=1)
    groups = P.greedy_partition(h.x, h.z)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan(jit=1)
    for scale in (1e-30, 1e-3, 1e3, 1e30):
        psi0 = _rand_state(rng, 15) * scale
        ref = oracle.evolve(h, psi0, 0.05, 3, 1, groups)
        t = _dev(psi0, "c128")
        sim.evolve(t, 0.05, 3, 1)
        err = np.linalg.norm(_host(t) - ref) / scale
        assert err <= TOL["c128"], (scale, err)


def test_jit_gradient(sd):
    rng = np.random.default_rng(62)
    n = 14
    h = gradient_2local(n=n, m=20, rng=rng)
    obs = z_average_observable(n)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan(jit=1)
    f, g = sim.grad(_dev(plus_state(n), "c128"), 0.05, 3, obs, 1)
    f_ref, g_ref = oracle.grad(h, plus_state(n), 0.05, 3, 1, obs)
    assert abs(f - f_ref) < 1e-12
    assert np.max(np.abs(g - g_ref)) < 1e-9 * max(1.0, np.max(np.abs(g_ref)))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_full_size_heisenberg_n30(sd, dtype):
    """The benchmark workload at full size (5x6 lattice, n = 30, Neel state,
    dt = 0.02) in the benchmark's launch configuration: the grouped path must
    agree with the independent per-Pauli kernel (itself checked against the
    oracle above) and preserve the norm."""
    import torch
    h = heisenberg_lattice(5, 6)
    cdt = torch.complex64 if dtype == "c64" else torch.complex128
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    steps = 5   # one block of 4 merged steps and a single step, as in the benchmark's calls
    sim.prepare(sd.C64 if dtype == "c64" else sd.C128, 0.02, steps, 1)
    a = torch.zeros(1 << 30, dtype=cdt, device="cuda")
    a[neel_index(5, 6)] = 1
    b = a.clone()
    sim.evolve(a, 0.02, steps, 1)
    sim.evolve_pauli(b, 0.02, steps, 1)
    err = torch.linalg.vector_norm((a - b).to(torch.complex128)).item()
    norm = torch.linalg.vector_norm(a.to(torch.complex128)).item()
    assert err <= TOL[dtype], err
    assert abs(norm - 1.0) < (1e-5 if dtype == "c64" else 1e-12)
    del a, b
    torch.cuda.empty_cache()
