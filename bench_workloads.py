"""Measurements of the configurations beside the benchmark line
(`python bench.py --workload NAME`): each prints one JSON line of the same
shape as the benchmark's.  Inputs are the seeded synthetic workloads of
workloads/; times are CUDA events on the launching stream, after warm-up.
"""
from __future__ import annotations

import json
import time

import numpy as np


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _time(fn):
    import torch
    e0, e1 = _events()
    torch.cuda.synchronize()
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def _line(metric, value, unit, config, **extra):
    out = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "higher_is_better": True,
           "data": "synthetic", "config": config}
    out.update(extra)
    print(json.dumps(out))


def heisenberg32(args):
    """6x6 lattice minus its corners (n = 32), complex64, dt = 0.02, first order."""
    import torch
    import paper_2206_11664_gb300 as sd
    from workloads import heisenberg_lattice, neel_index
    h = heisenberg_lattice(6, 6, drop_corners=True)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    st = sim.schedule_stats(sd.C64, 1)
    psi = torch.zeros(1 << h.n, dtype=torch.complex64, device="cuda")
    psi[neel_index(6, 6, True)] = 1
    k = max(2, args.steps // 4)
    sim.prepare(sd.C64, 0.02, k, 1)
    sim.evolve(psi, 0.02, args.warmup, 1)
    t = _time(lambda: sim.evolve(psi, 0.02, k, 1))
    tp = _time(lambda: sim.evolve_pauli(psi, 0.02, 1, 1))
    launches = sim.count_passes(sd.C64, 1, k)
    gbs = launches * 2 * (1 << h.n) * 8 / t / 1e9
    _line("Trotter steps/s at n=32", k / t, "steps/s",
          {"workload": "heisenberg_6x6_minus_corners_n32", "n": h.n, "terms": h.m, "dt": 0.02,
           "order": 1, "state": "complex64", "passes_per_step": launches / k,
           "passes_per_single_step": st["passes_per_step"]},
          steps=k, ms_per_step=1e3 * t / k, achieved_gbs=gbs,
          per_pauli={"steps_per_s": 1 / tp, "passes_per_step": h.m},
          speedup_grouped_over_per_pauli=(k / t) * tp)


def tfim10(args):
    """TFIM open chain n = 10, complex128, dt = 0.01, 100 first-order steps with
    <Z_0> recorded after every step (one launch on the on-chip path)."""
    import torch
    import paper_2206_11664_gb300 as sd
    from workloads import tfim_chain
    h = tfim_chain(10)
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    obs = (np.array([0], np.uint64), np.array([1], np.uint64), np.array([1.0]))
    trace = torch.zeros(100, dtype=torch.float64, device="cuda")

    def run():
        psi = torch.zeros(1 << 10, dtype=torch.complex128, device="cuda")
        psi[0] = 1
        sim.evolve_observe(psi, 0.01, 100, obs, trace)
    run()
    t = min(_time(run) for _ in range(5))
    _line("TFIM n=10 Trotter steps/s (100 steps, <Z_0> every step)", 100 / t, "steps/s",
          {"workload": "tfim_chain_n10", "n": 10, "dt": 0.01, "order": 1, "state": "complex128",
           "path": "on-chip, one launch"}, us_per_step=1e6 * t / 100,
          z0_final=float(trace[-1].item()))


def batch(args):
    """64 random k-local instances (n 16..24, 2000 terms), Haar product states,
    complex64, dt = 0.005, second order, one sd_evolve_batch call."""
    import torch
    import paper_2206_11664_gb300 as sd
    from workloads import batch_instances, product_state
    t0 = time.perf_counter()
    inst = batch_instances(64)
    sims, states = [], []
    for h, fac in inst:
        sims.append(sd.Simulator(h.n, h.x, h.z, h.c).plan(tile_bits=getattr(args, "tile_bits", 0)))
        states.append(torch.from_numpy(product_state(fac, np.complex64)).cuda())
    setup = time.perf_counter() - t0
    k = max(2, args.steps // 10)
    sd.evolve_batch(sims, states, 0.005, k, 2)            # builds every program of a k-step call
    t = _time(lambda: sd.evolve_batch(sims, states, 0.005, k, 2))
    nbytes = sum(s.schedule_stats(sd.C64, 2)["passes_per_step"] * 2 * (1 << s.n) * 8 for s in sims)
    _line("batch instance-steps/s (64 instances, second order)", 64 * k / t, "instance-steps/s",
          {"workload": "random_klocal_batch_64", "n_range": [min(s.n for s in sims), max(s.n for s in sims)],
           "terms": 2000, "dt": 0.005, "order": 2, "state": "complex64",
           "tile_bits": getattr(args, "tile_bits", 0) or "default"},
          steps=k, ms_per_batch_step=1e3 * t / k, achieved_gbs=nbytes * k / t / 1e9,
          host_setup_s=setup)


def jw26(args):
    """Jordan-Wigner-style n = 26, 20000 terms, complex64, dt = 0.05, second order."""
    import torch
    import paper_2206_11664_gb300 as sd
    from workloads import jw_like
    h = jw_like()
    t0 = time.perf_counter()
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    plan_s = time.perf_counter() - t0
    st = sim.schedule_stats(sd.C64, 2)
    psi = torch.zeros(1 << h.n, dtype=torch.complex64, device="cuda")
    psi[(1 << 13) - 1] = 1
    k = max(2, args.steps // 4)
    sim.evolve(psi, 0.05, k, 2)                           # builds the head/core/tail programs
    t = _time(lambda: sim.evolve(psi, 0.05, k, 2))
    tp = _time(lambda: sim.evolve_pauli(psi, 0.05, 1, 2))
    launches = sim.count_passes(sd.C64, 2, k)
    _line("JW-style n=26 Trotter steps/s (second order)", k / t, "steps/s",
          {"workload": "jw_like_n26", "n": 26, "terms": h.m, "groups": sim.plan_view()["n_groups"],
           "dt": 0.05, "order": 2, "state": "complex64", "passes_per_step": launches / k,
           "passes_per_core": st["passes_per_step"]},
          steps=k, ms_per_step=1e3 * t / k,
          achieved_gbs=launches * 2 * (1 << 26) * 8 / t / 1e9,
          per_pauli={"steps_per_s": 1 / tp, "passes_per_step": 2 * h.m},
          speedup_grouped_over_per_pauli=(k / t) * tp, plan_s=plan_s)


def grad24(args):
    """Adjoint gradient, random 2-local n = 24 (200 terms), |+...+>, complex128,
    500 first-order steps of dt = 0.01, O = sum_i Z_i / n."""
    import torch
    import paper_2206_11664_gb300 as sd
    from workloads import gradient_2local, z_average_observable
    h = gradient_2local()
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    psi = torch.full((1 << 24,), 2.0 ** -12, dtype=torch.complex128, device="cuda")
    obs = z_average_observable(24)
    steps = int(getattr(args, "grad_steps", 500))
    sim.grad(psi, 0.01, 5, obs, 1)                        # builds the programs
    t0 = time.perf_counter()
    f, g = sim.grad(psi, 0.01, steps, obs, 1)
    t = time.perf_counter() - t0
    _line(f"gradient evaluations/s (n=24, 200 coefficients, {steps} steps)", 1 / t, "evaluations/s",
          {"workload": "gradient_2local_n24", "n": 24, "terms": 200, "dt": 0.01, "steps": steps,
           "order": 1, "state": "complex128"}, seconds=t, value_f=f,
          grad_norm=float(np.linalg.norm(g)))


def _grouped_vs_pauli(h, dt, steps, state_index=0, order=1):
    """Steps/s of the grouped path and of the per-Pauli path on one state
    (complex64), both after a warm-up call; returns a dict."""
    import torch
    import paper_2206_11664_gb300 as sd
    t0 = time.perf_counter()
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan()
    plan_s = time.perf_counter() - t0
    groups = sim.plan_view()["n_groups"]
    psi = torch.zeros(1 << h.n, dtype=torch.complex64, device="cuda")
    psi[state_index] = 1
    sim.prepare(sd.C64, dt, steps, order)
    sim.evolve(psi, dt, steps, order)      # warm-up call of the timed shape (pass graphs of small states)
    t = _time(lambda: sim.evolve(psi, dt, steps, order))
    ps = max(1, steps // 4)
    sim.evolve_pauli(psi, dt, 1, order)
    tp = _time(lambda: sim.evolve_pauli(psi, dt, ps, order))
    passes = sim.count_passes(sd.C64, order, steps)
    return {"n": h.n, "terms": h.m, "groups": groups, "theory_m_over_n_ng": h.m / (h.n * groups),
            "steps_per_s": steps / t, "per_pauli_steps_per_s": ps / tp,
            "speedup": (steps / t) / (ps / tp), "passes_per_step": passes / steps,
            "ms_per_step": 1e3 * t / steps, "plan_s": plan_s}


def tfim_fc(args):
    """Fully connected transverse-field Ising model (the paper's first
    experiment), n = 30, J_ij, h_i ~ U[-1, 1], |0..0>, dt = 0.01, complex64,
    first order: grouped vs per-Pauli on the same GPU."""
    from workloads import tfim_fully_connected
    r = _grouped_vs_pauli(tfim_fully_connected(30), 0.01, max(4, args.steps))
    _line("fully connected TFIM n=30 Trotter steps/s (grouped; per-Pauli beside it)", r["steps_per_s"],
          "steps/s", {"workload": "tfim_fully_connected_n30", "dt": 0.01, "order": 1, "state": "complex64"},
          **r)


def syk(args):
    """SYK Majorana model (the paper's second experiment), n = 20 qubits
    (40 Majorana operators, 91390 terms), |0..0>, dt = 0.01, complex64, first
    order: grouped vs per-Pauli on the same GPU."""
    from workloads import syk_majorana
    r = _grouped_vs_pauli(syk_majorana(20), 0.01, 2)
    _line("SYK n=20 Trotter steps/s (grouped; per-Pauli beside it)", r["steps_per_s"], "steps/s",
          {"workload": "syk_majorana_n20", "dt": 0.01, "order": 1, "state": "complex64"}, **r)


def sweep(args):
    """Speedup of the grouped path over the per-Pauli path against n for the
    paper's two models (its Figs. 5-6 compare the same two methods against
    the cost model m/(n n_g)); one line per point."""
    from workloads import syk_majorana, tfim_fully_connected
    for n in (14, 18, 22, 26, 30):
        r = _grouped_vs_pauli(tfim_fully_connected(n), 0.01, 8)
        _line(f"fully connected TFIM n={n}: grouped vs per-Pauli", r["speedup"], "x",
              {"workload": f"tfim_fully_connected_n{n}", "dt": 0.01, "state": "complex64"}, **r)
    for n in (14, 16, 18, 20):
        r = _grouped_vs_pauli(syk_majorana(n), 0.01, 2)
        _line(f"SYK n={n}: grouped vs per-Pauli", r["speedup"], "x",
              {"workload": f"syk_majorana_n{n}", "dt": 0.01, "state": "complex64"}, **r)


def run(args):
    {"heisenberg32": heisenberg32, "tfim10": tfim10, "batch": batch, "jw26": jw26,
     "grad24": grad24, "tfim_fc": tfim_fc, "syk": syk, "sweep": sweep}[args.workload](args)
