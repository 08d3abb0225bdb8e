"""Host-side pieces of the benchmark (no GPU): the CPU-oracle sample that
the benchmark line reports as its CPU baseline."""
import numpy as np

import bench
import oracle


def test_cpu_oracle_sample_all_cores_and_one_core():
    h, neel, name = bench.workload(16)
    assert name == "heisenberg_4x4_n16" and h.m == 72
    psi = np.zeros(1 << h.n, dtype=np.complex128)
    psi[neel] = 1.0
    all_threads = oracle.num_threads()
    a = bench.cpu_oracle_sample(h, neel, budget_s=0.2, psi=psi)
    b = bench.cpu_oracle_sample(h, neel, budget_s=0.2, psi=psi, threads=1)
    assert a["cores"] == all_threads and b["cores"] == 1
    assert oracle.num_threads() == all_threads          # thread count restored
    for r in (a, b):
        assert r["kind"] == "oracle" and r["unit"] == "steps/s" and r["value"] > 0
        assert "of the 72 rotations" in r["sample"]
    # the sample evolves the given state in place with unitary rotations
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-12
