"""Host-side tests of the native library (no GPU needed).

The library loads and exports every symbol of include/sd.h; its planner
(C++) agrees bit for bit with the independent oracle planner (Python) on
groups, gate lists, masks, signs and CNOT index maps; argument validation
returns the documented status codes; the pass scheduler covers every op.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import planner as P
from workloads import (batch_instances, from_strings, gradient_2local, heisenberg_lattice,
                       jw_like, random_klocal, tfim_chain)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sd():
    from paper_2206_11664_gb300 import build
    build.build()
    import paper_2206_11664_gb300 as m
    return m


def test_exports_every_declared_symbol(sd):
    from paper_2206_11664_gb300 import _native
    lib = _native.load()
    hdr = open(os.path.join(ROOT, "include", "sd.h")).read()
    names = set(re.findall(r"\b(sd_[a-z_]+)\s*\(", hdr))
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
        assert name in _native.SIGNATURES, name


KIND = {"H": 0, "S": 1, "CNOT": 2, "CZ": 3}


def _compare(sd, h, rule):
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan(skip_rule=rule)
    v = sim.plan_view()
    pl = P.plan(h.n, h.x, h.z, skip_rule=rule)
    G = v["n_groups"]
    assert G == len(pl.groups)
    for g in range(G):
        a, b = v["group_offsets"][g], v["group_offsets"][g + 1]
        assert v["group_terms"][a:b].tolist() == pl.groups[g]
        assert v["masks"][a:b].tolist() == pl.masks[g]
        assert v["signs"][a:b].tolist() == pl.signs[g]
        ga, gb = v["gate_offsets"][g], v["gate_offsets"][g + 1]
        assert v["gates"][ga:gb].tolist() == [[KIND[k], x, y] for k, x, y in pl.gates[g]]
        A, Ai = P.cnot_layer_matrix(pl.gates[g], h.n)
        assert v["cnot_cols"][g].tolist() == A
        assert v["cnot_inv_cols"][g].tolist() == Ai
    return sim


def test_worked_example_through_abi(sd):
    ex = ["YIXI", "IXIY", "XZYZ", "YZXZ", "XIYI", "IYIX", "ZXZY", "ZYZX"]
    h = from_strings(ex, np.ones(8))
    for rule in (0, 1, 2):
        _compare(sd, h, rule)


@pytest.mark.parametrize("name", ["tfim", "heis30", "heis32", "grad", "jw"])
def test_planner_bit_exact_on_workloads(sd, name):
    h = {"tfim": lambda: tfim_chain(10), "heis30": lambda: heisenberg_lattice(5, 6),
         "heis32": lambda: heisenberg_lattice(6, 6, drop_corners=True),
         "grad": gradient_2local, "jw": jw_like}[name]()
    _compare(sd, h, 2)


def test_planner_bit_exact_on_batch_instances(sd):
    for h, _ in batch_instances(3):
        _compare(sd, h, 2)


@pytest.mark.parametrize("rule", [0, 1, 2])
def test_planner_bit_exact_random(sd, rule):
    rng = np.random.default_rng(40 + rule)
    for _ in range(30):
        n = int(rng.integers(3, 12))
        h = random_klocal(n, int(rng.integers(5, 60)), rng, weights=tuple(w for w in (1, 2, 3, 4) if w <= n))
        _compare(sd, h, rule)


def test_planner_bit_exact_where_completion_uses_the_complement(sd):
    """Groups whose generators no single-qubit Pauli can complete (every
    qubit carries both X and Z), so that both planners must take rows from
    the symplectic complement; embedded in larger registers as well."""
    for texts in (["XXXX", "ZZZZ", "YYYY"], ["XXXXII", "ZZZZII", "IIIIXX"],
                  ["IXXXXI", "IZZZZI", "XIIIIZ", "ZIIIIX"]):
        for rule in (0, 1, 2):
            _compare(sd, from_strings(texts, np.linspace(0.3, 1.1, len(texts))), rule)


def test_argument_validation(sd):
    from paper_2206_11664_gb300 import _native as N
    lib = N.load()
    h = ctypes.c_void_p()
    x = np.array([1 << 5], np.uint64)
    z = np.array([0], np.uint64)
    c = np.array([1.0])
    P64 = ctypes.POINTER(ctypes.c_uint64)
    PD = ctypes.POINTER(ctypes.c_double)
    st = lib.sd_create(3, 1, x.ctypes.data_as(P64), z.ctypes.data_as(P64), c.ctypes.data_as(PD),
                       ctypes.byref(h))
    assert st == N.SD_EINVAL and b"mask bit" in lib.sd_last_error(None)
    st = lib.sd_create(0, 1, x.ctypes.data_as(P64), z.ctypes.data_as(P64), c.ctypes.data_as(PD),
                       ctypes.byref(h))
    assert st == N.SD_EINVAL
    with pytest.raises(sd.SDError):
        sd.Simulator.from_strings(["XQ"], [1.0])
    sim = sd.Simulator.from_strings(["XX", "ZZ"], [1.0, 2.0])
    v = N.PlanView()
    assert lib.sd_get_plan(sim._h, ctypes.byref(v)) == N.SD_ENOPLAN
    with pytest.raises(sd.SDError):
        sim.plan(skip_rule=7)
    with pytest.raises(sd.SDError):
        sim.plan(tile_bits=20)
    sim.plan()
    assert sim.plan_view()["n_groups"] == 1
    c_bad = np.array([np.nan, 1.0])
    with pytest.raises(sd.SDError):
        sim.set_coeffs(c_bad)


def test_schedule_covers_heisenberg_step(sd):
    h = heisenberg_lattice(5, 6)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    s64 = sim.schedule_stats(sd.C64, 1)
    s128 = sim.schedule_stats(sd.C128, 1)
    # three group exponentials per step, far fewer passes than the 147 terms
    assert s64["diag_passes"] == 3 and s64["passes_per_step"] <= 10
    assert s128["passes_per_step"] <= 14


def test_schedule_stats_small_state_is_onchip(sd):
    t = tfim_chain(10)
    sim = sd.Simulator(t.n, t.x, t.z, t.c).plan()
    assert sim.schedule_stats(sd.C128, 1)["onchip"]


def test_count_passes_blocks(sd):
    """Launch counts of sd_evolve: one step is one schedule; longer calls
    merge 4 steps (first order) or 4 cores (second order) into one schedule,
    which needs fewer passes than 4 separate ones; the on-chip path has none."""
    h = heisenberg_lattice(5, 6)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    one = sim.schedule_stats(sd.C64, 1)["passes_per_step"]
    assert sim.count_passes(sd.C64, 1, 0) == 0
    assert sim.count_passes(sd.C64, 1, 1) == one
    four = sim.count_passes(sd.C64, 1, 4)
    assert four < 4 * one
    assert sim.count_passes(sd.C64, 1, 8) == 2 * four
    assert sim.count_passes(sd.C64, 1, 9) == 2 * four + one
    c2 = sim.count_passes(sd.C64, 2, 6)
    assert 0 < c2 < 6 * sim.schedule_stats(sd.C64, 2)["passes_per_step"] + 10
    t = tfim_chain(10)
    small = sd.Simulator(t.n, t.x, t.z, t.c).plan()
    assert small.count_passes(sd.C128, 1, 100) == 0
    with pytest.raises(sd.SDError):
        sim.count_passes(sd.C64, 3, 1)


def test_grouping_variants_match_oracle(sd):
    """The four partition orders of the product planner give the oracle
    planner's groups exactly (and the plans diagonalise them)."""
    rng = np.random.default_rng(72)
    cases = [random_klocal(n, m, rng, weights=(1, 2, 3)) for n, m in ((8, 60), (12, 200), (16, 300))]
    cases.append(jw_like(n=12, m=300, rng=rng))
    for h in cases:
        for g in range(4):
            ref = P.partition(h.x, h.z, g, h.c)
            sim = sd.Simulator(h.n, h.x, h.z, h.c).plan(grouping=g)
            v = sim.plan_view()
            got = [v["group_terms"][v["group_offsets"][i]:v["group_offsets"][i + 1]].tolist()
                   for i in range(v["n_groups"])]
            assert got == ref, (h.n, h.m, g)
    with pytest.raises(sd.SDError):
        sd.Simulator(cases[0].n, cases[0].x, cases[0].z, cases[0].c).plan(grouping=4)


def test_precompile_generated_kernels(sd, tmp_path, monkeypatch):
    """The pass kernels generated at run time compile with NVRTC for sm_103a
    on the host alone (no GPU): the Heisenberg step (complex64), a random
    k-local Hamiltonian with CNOT permutations and S/CZ layers (complex128,
    fixed point), and a large diagonal group; a second call finds them all
    in the on-disk cache."""
    monkeypatch.setenv("SD_JIT_CACHE", str(tmp_path))
    h = heisenberg_lattice(4, 5)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    assert sim.precompile(sd.C64, 1, 1) >= 1
    assert sim.precompile(sd.C64, 1, 1) == 0
    rng = np.random.default_rng(95)
    hr = random_klocal(20, 40, rng, weights=(2, 3))
    simr = sd.Simulator(hr.n, hr.x, hr.z, hr.c).plan(skip_rule=0)
    assert simr.precompile(sd.C128, 1, 1) >= 1
    z = rng.integers(1, 1 << 20, size=1500, dtype=np.uint64)
    hz = sd.Simulator(20, np.zeros(1500, dtype=np.uint64), z, rng.uniform(-1, 1, 1500)).plan()
    assert hz.precompile(sd.C64, 1, 1) >= 1
    assert len(list(tmp_path.glob("*.cubin"))) >= 3
    small = tfim_chain(10)
    assert sd.Simulator(small.n, small.x, small.z, small.c).plan().precompile(sd.C64, 5, 1) == 0


def test_closing_program_shares_the_core_kernels(sd, tmp_path, monkeypatch):
    """A second-order call closes with the core whose last group-1 exponential
    is halved.  Angles are kernel arguments, so that program's generated
    passes are the core's: compiling a 3-step call (opening half step, two
    cores, closing program) compiles one core's worth of NVRTC chunks (12
    passes each), not two."""
    monkeypatch.setenv("SD_JIT_CACHE", str(tmp_path))
    h = heisenberg_lattice(4, 5)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    core = sim.count_passes(sd.C64, 2, 3) - sim.count_passes(sd.C64, 2, 2)
    assert core > 0
    assert sim.precompile(sd.C64, 3, 2) == -(-core // 12)
    assert sim.precompile(sd.C64, 3, 2) == 0


def test_argument_validation_of_the_other_entry_points(sd):
    """Argument errors of the entry points added beside sd_evolve are
    reported before any device work (no GPU needed)."""
    from paper_2206_11664_gb300 import _native as N
    lib = N.load()
    h = heisenberg_lattice(3, 3)
    unplanned = sd.Simulator(h.n, h.x, h.z, h.c)
    best = ctypes.c_int(0)
    cnt = ctypes.c_int64(0)
    assert lib.sd_autotune(unplanned._h, N.SD_C64, 0.1, 4, 1, 11, 13, ctypes.byref(best), None) == N.SD_ENOPLAN
    assert lib.sd_precompile(unplanned._h, N.SD_C64, 1, 1, ctypes.byref(cnt)) == N.SD_ENOPLAN
    assert lib.sd_count_passes(unplanned._h, N.SD_C64, 1, 1, ctypes.byref(cnt)) == N.SD_ENOPLAN
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    for kmin, kmax in ((8, 13), (12, 14), (13, 12)):
        assert lib.sd_autotune(sim._h, N.SD_C64, 0.1, 4, 1, kmin, kmax, ctypes.byref(best), None) == N.SD_EINVAL
    assert lib.sd_autotune(sim._h, N.SD_C64, 0.1, 0, 1, 11, 13, ctypes.byref(best), None) == N.SD_EINVAL
    assert lib.sd_autotune(sim._h, N.SD_C64, float("nan"), 4, 1, 11, 13, ctypes.byref(best), None) == N.SD_EINVAL
    assert lib.sd_autotune(sim._h, 7, 0.1, 4, 1, 11, 13, ctypes.byref(best), None) == N.SD_EINVAL
    assert lib.sd_precompile(sim._h, N.SD_C64, 1, 3, ctypes.byref(cnt)) == N.SD_EINVAL
    assert lib.sd_precompile(sim._h, 7, 1, 1, ctypes.byref(cnt)) == N.SD_EINVAL
    assert lib.sd_precompile(sim._h, N.SD_C64, -1, 1, ctypes.byref(cnt)) == N.SD_EINVAL
    assert lib.sd_count_passes(sim._h, N.SD_C64, 1, -1, ctypes.byref(cnt)) == N.SD_EINVAL
    assert lib.sd_prepare(None, N.SD_C64, 0.1, 1, 1) == N.SD_EINVAL
    assert lib.sd_prepare(sim._h, N.SD_C64, 0.1, 1, 5) == N.SD_EINVAL
    assert lib.sd_prepare(sim._h, N.SD_C64, float("inf"), 1, 1) == N.SD_EINVAL
    assert lib.sd_prepare_batch(None, None, 1, N.SD_C64, 0.1, 1, 1) == N.SD_EINVAL
    hs = (ctypes.c_void_p * 1)(sim._h)
    ps = (ctypes.c_void_p * 1)(None)
    assert lib.sd_prepare_batch(hs, ps, -1, N.SD_C64, 0.1, 1, 1) == N.SD_EINVAL
    assert lib.sd_prepare_batch(hs, ps, 70000, N.SD_C64, 0.1, 1, 1) == N.SD_EINVAL
    assert lib.sd_evolve_host(sim._h, None, None, N.SD_C64, 0.1, 1, 1, None) == N.SD_EINVAL
    tr = N.TuneResult()
    assert lib.sd_autotune_shape(unplanned._h, N.SD_C64, 0.1, 4, 1, 11, 13, ctypes.byref(tr)) == N.SD_ENOPLAN
    assert lib.sd_autotune_shape(sim._h, N.SD_C64, 0.1, 4, 1, 11, 13, None) == N.SD_EINVAL
    for kmin, kmax in ((8, 13), (12, 14), (13, 12)):
        assert lib.sd_autotune_shape(sim._h, N.SD_C64, 0.1, 4, 1, kmin, kmax, ctypes.byref(tr)) == N.SD_EINVAL
    assert lib.sd_autotune_shape(sim._h, N.SD_C64, 0.1, 4, 3, 11, 13, ctypes.byref(tr)) == N.SD_EINVAL
    assert lib.sd_autotune_shape(sim._h, 7, 0.1, 4, 1, 11, 13, ctypes.byref(tr)) == N.SD_EINVAL
    for bad in (-2, 2):
        o = N.PlanOpts(-1, 0, 0, 0, bad)
        assert lib.sd_plan(sim._h, ctypes.byref(o)) == N.SD_EINVAL
    for bad in (-1, 4):
        o = N.PlanOpts(-1, 0, 0, 0, 0, bad)
        assert lib.sd_plan(sim._h, ctypes.byref(o)) == N.SD_EINVAL


def test_paired_layout_schedules(sd, tmp_path, monkeypatch):
    """The paired layout (sd_plan_opts.layout = 1) schedules complex64
    programs compiled at run time with qubit 0 in registers: the benchmark
    calls keep their pass counts, complex128 and interpreter-only programs
    are unaffected, and the paired kernels of the benchmark programs compile
    with NVRTC for sm_103a on the host."""
    monkeypatch.setenv("SD_JIT_CACHE", str(tmp_path))
    h = heisenberg_lattice(5, 6)
    plain = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    paired = sd.Simulator(h.n, h.x, h.z, h.c).plan(layout=1)
    for steps in (1, 4, 20):
        for dt in (sd.C64, sd.C128):
            assert paired.count_passes(dt, 1, steps) == plain.count_passes(dt, 1, steps)
    assert paired.schedule_stats(sd.C64, 1)["rounds_per_step"] > plain.schedule_stats(sd.C64, 1)["rounds_per_step"]
    assert paired.schedule_stats(sd.C128, 1) == plain.schedule_stats(sd.C128, 1)
    assert paired.precompile(sd.C64, 4, 1) >= 1
    small = heisenberg_lattice(3, 5)            # n = 15: interpreter only, layout has no effect
    a = sd.Simulator(small.n, small.x, small.z, small.c).plan()
    b = sd.Simulator(small.n, small.x, small.z, small.c).plan(layout=1)
    assert a.schedule_stats(sd.C64, 1) == b.schedule_stats(sd.C64, 1)


def test_noalloc_argument_validation(sd):
    """sd_expect_noalloc checks its arguments before touching a device: the
    qubit range, null pointers, the dtype, the observable arrays, the fixed
    limit of 4096 terms and mask bits at or above n; an empty observable
    gives 0 without device work."""
    from paper_2206_11664_gb300 import _native as N
    lib = N.load()
    fake = ctypes.c_void_p(0x1000)          # never dereferenced: every call below fails or returns early
    out = ctypes.c_double(7.0)
    m = 4097
    ox = np.zeros(m, np.uint64)
    oz = np.ones(m, np.uint64)
    oc = np.ones(m)

    def call(n, state, dtype, mo, x=ox, z=oz, c=oc, dst=ctypes.byref(out)):
        return lib.sd_expect_noalloc(n, state, dtype, mo, x.ctypes.data_as(N.P_u64),
                                     z.ctypes.data_as(N.P_u64), c.ctypes.data_as(N.P_dbl), dst, None)

    assert call(0, fake, N.SD_C64, 1) == N.SD_EINVAL
    assert call(41, fake, N.SD_C64, 1) == N.SD_EINVAL
    assert call(4, None, N.SD_C64, 1) == N.SD_EINVAL
    assert call(4, fake, N.SD_C64, 1, dst=None) == N.SD_EINVAL
    assert call(4, fake, 7, 1) == N.SD_EINVAL
    assert call(4, fake, N.SD_C64, -1) == N.SD_EINVAL
    assert call(4, fake, N.SD_C64, m) == N.SD_EINVAL
    assert b"4096" in lib.sd_last_error(None)
    bad = oz.copy()
    bad[0] = 1 << 4                         # a mask bit at n = 4
    assert call(4, fake, N.SD_C128, 1, z=bad) == N.SD_EINVAL
    nan = oc.copy()
    nan[0] = float("nan")
    assert call(4, fake, N.SD_C128, 1, c=nan) == N.SD_EINVAL
    assert call(4, fake, N.SD_C128, 0) == N.SD_OK and out.value == 0.0


def test_schedule_stats_report_the_tiles_sd_evolve_uses(sd):
    """A diagonal group with thousands of distinct in-tile masks has more
    term slots than fit beside a 2^13-amplitude complex64 tile in shared
    memory, so the scheduler takes 2^12 tiles; the schedule statistics
    report the tile size and pass count that sd_evolve runs."""
    from workloads import Hamiltonian
    rng = np.random.default_rng(3)
    n, m = 16, 20000
    z = rng.integers(1, 1 << n, size=m, dtype=np.uint64)
    sim = sd.Simulator(n, np.zeros(m, dtype=np.uint64), z, rng.uniform(-1, 1, size=m)).plan()
    st = sim.schedule_stats(sd.C64, 1)
    assert st["tile_bits"] == 12
    assert st["passes_per_step"] == sim.count_passes(sd.C64, 1, 1) == 1
    h = heisenberg_lattice(4, 5)
    small = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    assert small.schedule_stats(sd.C64, 1)["tile_bits"] == 13
    assert small.schedule_stats(sd.C128, 1)["tile_bits"] == 12


def _c_declarations():
    """Function prototypes and struct typedefs of include/sd.h, comments removed."""
    hdr = open(os.path.join(ROOT, "include", "sd.h")).read()
    hdr = re.sub(r"/\*.*?\*/", " ", hdr, flags=re.S)
    funcs = {}
    for ret, name, params in re.findall(r"(sd_status|const char \*|void)\s*(sd_[a-z_]+)\s*\(([^)]*)\)\s*;",
                                        hdr):
        funcs[name] = (ret.replace(" ", ""), [" ".join(p.split()) for p in params.split(",")])
    structs = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(sd_[a-z_]+)\s*;", hdr, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if decl:
                fields.append(decl)
        structs[name] = fields
    return funcs, structs


def _ctype_of(decl):
    """The ctypes type that marshals a C parameter declaration of sd.h."""
    from paper_2206_11664_gb300 import _native as N
    t = re.sub(r"\b[a-z_0-9]+$", "", decl).replace("const", "").replace(" ", "")
    table = {"int": N.c_int, "int64_t": N.c_i64, "double": N.c_dbl, "sd_dtype": N.c_int,
             "void*": N.c_vp, "sd_ctx*": N.c_vp, "sd_ctx**": ctypes.POINTER(N.c_vp),
             "uint64_t*": N.P_u64, "double*": N.P_dbl, "char**": ctypes.POINTER(ctypes.c_char_p),
             "sd_plan_opts*": ctypes.POINTER(N.PlanOpts), "sd_plan_view*": ctypes.POINTER(N.PlanView),
             "sd_schedule_stats*": ctypes.POINTER(N.ScheduleStats), "int*": ctypes.POINTER(N.c_int),
             "sd_tune_result*": ctypes.POINTER(N.TuneResult),
             "int64_t*": ctypes.POINTER(N.c_i64), "void**": ctypes.POINTER(N.c_vp),
             "sd_ctx**const": ctypes.POINTER(N.c_vp)}
    return table[t]


def test_binding_matches_the_header():
    """Every prototype of include/sd.h is bound with the same number and kind
    of arguments and the same result type, and the binding's structures have
    the header's fields in the header's order."""
    from paper_2206_11664_gb300 import _native as N
    funcs, structs = _c_declarations()
    assert set(funcs) == set(N.SIGNATURES)
    results = {"sd_status": N.c_int, "constchar*": ctypes.c_char_p, "void": None}
    for name, (ret, params) in funcs.items():
        res, args = N.SIGNATURES[name]
        assert res is results[ret], name
        assert len(args) == len(params), name
        for decl, a in zip(params, args):
            device_ptr = "*" in decl and decl.split()[-1].lstrip("*").startswith("d_")
            # device addresses (d_...) are passed as plain addresses
            assert _ctype_of(decl) == a or (device_ptr and a is N.c_vp), (name, decl)
    for cname, pyname in (("sd_plan_opts", "PlanOpts"), ("sd_plan_view", "PlanView"),
                          ("sd_schedule_stats", "ScheduleStats"), ("sd_tune_result", "TuneResult")):
        header_fields = [re.sub(r"\[.*\]", "", d).split()[-1].lstrip("*") for d in structs[cname]]
        assert header_fields == [f[0] for f in getattr(N, pyname)._fields_], cname


def test_pass_counts_of_the_benchmark_steps(sd):
    """Tile passes (state sweeps through HBM) of the benchmark workloads, as
    the scheduler plans them on the host; the benchmark's launch count and
    bytes come from these numbers.  5x6 Heisenberg: 7 passes for one step,
    25 for a block of 4 steps (6.25 per step); 6x6 minus corners (n = 32):
    10 and 37.  A change here changes the measured roofline figures."""
    for (rows, cols, corners), one, four in (((5, 6, False), 7, 25), ((6, 6, True), 10, 37)):
        h = heisenberg_lattice(rows, cols, drop_corners=corners)
        sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
        for code in (sd.C64, sd.C128):
            st = sim.schedule_stats(code, 1)
            assert st["passes_per_step"] == one and st["diag_passes"] == 3
            assert sim.count_passes(code, 1, 1) == one
            assert sim.count_passes(code, 1, 20) == 5 * four
            assert sim.count_passes(code, 1, 1000) == 250 * four
            assert sim.count_passes(code, 1, 6) == four + 2 * one


def test_precompile_the_benchmark_programs(sd, tmp_path, monkeypatch):
    """The exact kernels of the benchmark's timed calls (5x6 Heisenberg,
    n = 30, 20 first-order steps: a 25-pass block program, complex64 and
    complex128) are generated and compile with NVRTC for sm_103a on the host
    alone."""
    monkeypatch.setenv("SD_JIT_CACHE", str(tmp_path))
    h = heisenberg_lattice(5, 6)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    for code in (sd.C64, sd.C128):
        assert sim.precompile(code, 20, 1) == 3      # 25 passes in NVRTC programs of 12
        assert sim.precompile(code, 20, 1) == 0      # then all cached


def test_from_strings_arguments(sd):
    """Text input: lower case is accepted and gives the same plan; an empty
    list, a wrong length or a character outside IXYZ is refused."""
    a = sd.Simulator.from_strings(["XXI", "iyy", "ZIZ"], [1.0, 0.5, 0.25]).plan().plan_view()
    b = sd.Simulator.from_strings(["XXI", "IYY", "ZIZ"], [1.0, 0.5, 0.25]).plan().plan_view()
    assert a["n_groups"] == b["n_groups"] and a["masks"].tolist() == b["masks"].tolist()
    with pytest.raises(ValueError):
        sd.Simulator.from_strings([], [])
    with pytest.raises(sd.SDError):
        sd.Simulator.from_strings(["XX", "XYZ"], [1.0, 1.0])
    with pytest.raises(sd.SDError):
        sd.Simulator.from_strings(["XQ"], [1.0])


def test_observable_arrays_must_match(sd):
    """The binding refuses observables whose x, z and c arrays differ in
    length before any call into the library (which reads len(c) of each)."""
    h = heisenberg_lattice(3, 3)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    bad = (np.zeros(2, np.uint64), np.ones(3, np.uint64), np.ones(3))
    with pytest.raises(ValueError):
        sim.expect(None, bad)
    with pytest.raises(ValueError):
        sim.grad(None, 0.1, 1, bad)
    with pytest.raises(ValueError):
        sim.expect(None, (np.zeros((1, 3), np.uint64), np.ones((1, 3), np.uint64), np.ones((1, 3))))
