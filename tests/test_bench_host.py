"""Host-side pieces of the benchmark (no GPU): the CPU-oracle sample that
the benchmark line reports as its CPU baseline, and the reference arm (the
oracle timed on bounded samples of the benchmark step)."""
import json
import subprocess
import sys

import numpy as np

import bench
import oracle


def test_oracle_sample_draws_from_every_group():
    h, neel, name = bench.workload(16)
    assert name == "heisenberg_4x4_n16" and h.m == 72
    groups = oracle.planner.greedy_partition(h.x, h.z)
    picks, m = bench.oracle_sample(h, 5)
    assert m == 72 and len(picks) == 5 * len(groups) == 15
    for g in groups:
        assert len(set(picks) & set(g)) == 5          # evenly spaced inside each group
    picks1, _ = bench.oracle_sample(h, 1)
    assert picks1 == [g[0] for g in groups]


def test_cpu_oracle_sample_all_cores_and_one_core():
    h, neel, _ = bench.workload(16)
    psi = np.zeros(1 << h.n, dtype=np.complex128)
    psi[neel] = 1.0
    all_threads = oracle.num_threads()
    a = bench.cpu_oracle_sample(h, psi, per_group=4)
    b = bench.cpu_oracle_sample(h, psi, per_group=1, threads=1)
    assert a["cores"] == all_threads and b["cores"] == 1
    assert oracle.num_threads() == all_threads          # thread count restored
    for r in (a, b):
        assert r["kind"] == "oracle" and r["unit"] == "steps/s" and r["value"] > 0
        assert "of the 72 rotations" in r["sample"]
    assert "12 of the 72" in a["sample"] and "3 of the 72" in b["sample"]
    # the sample evolves the given state in place with unitary rotations
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-12


def test_reference_arm_reports_the_time_it_spends():
    """The reference arm's steps x ms_per_step is the time it spent timing,
    and value scales the sampled fraction of a Trotter step to whole steps."""
    import time
    t0 = time.perf_counter()
    out = subprocess.run([sys.executable, bench.__file__, "--impl", "reference", "--qubits", "16",
                          "--steps", "3", "--warmup", "1"], capture_output=True, text=True, check=True)
    wall = time.perf_counter() - t0
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 3
    assert line["steps"] * line["ms_per_step"] / 1e3 <= wall
    frac = line["trotter_steps_per_step"]
    assert abs(frac - 21 / 72) < 1e-12
    assert abs(line["value"] - frac / (line["ms_per_step"] / 1e3)) < 1e-9 * line["value"]
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0
