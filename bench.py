"""Benchmark: Trotter steps/s of the grouped (simultaneous-diagonalisation)
path on the 2D Heisenberg XXX model, 5x6 open lattice, n = 30 qubits, 147
terms in 3 commuting groups, Neel initial state, dt = 0.02, first order,
complex64 state with Q0.64 fixed-point phase angles; beside it the plain
per-Pauli path on the same GPU, the complex128 grouped path, an end-to-end
figure through host buffers, the HBM roofline of the pass kernel and the
CPU oracle on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank evolves its own replica (the path has no exchange
step at this size); value = all ranks' steps / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Trotter steps/s at n=30 (grouped vs per-Pauli, same GB300); HBM GB/s vs peak"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--pauli-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip per-Pauli / c128 / e2e legs")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the 2-step comparison of both precisions with the CPU oracle")
    ap.add_argument("--workload", default="heisenberg30",
                    choices=["heisenberg30", "heisenberg32", "tfim10", "batch", "jw26", "grad24",
                             "tfim_fc", "syk", "sweep"],
                    help="heisenberg30 is the benchmark line; the others measure the remaining "
                         "configurations and print their own line")
    ap.add_argument("--grad-steps", dest="grad_steps", type=int, default=500,
                    help="Trotter steps of the gradient workload's timed evaluation (500 in its configuration)")
    ap.add_argument("--tile-bits", dest="tile_bits", type=int, default=0,
                    help="tile size for the batch workload (0 = default)")
    ap.add_argument("--prefetch", type=int, default=0, choices=[0, 1, 2, 3],
                    help="prefetch buffers of the passes compiled at run time (0 = the library's choice; "
                         "3 = two in passes without a group exponential)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the tile size (K = 11..13) and, for complex64, the register layout by "
                         "timing them first (sd_autotune_shape)")
    ap.add_argument("--state", default="c64", choices=["c64", "c128"],
                    help="state precision of the timed leg (c64 is the benchmark line)")
    ap.add_argument("--qubits", type=int, default=30, choices=[16, 20, 24, 25, 28, 30],
                    help="lattice size: 30 is the benchmark workload (5x6); smaller lattices "
                         "are for profiler captures")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = sorted(sm)[len(sm) // 4:] if sm else []
        return {"sm_mhz": float(np.median(loaded)) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_init(backend="nccl"):
    """World size, rank and local rank from the launcher's environment; one
    process group for the timing reduction when there are several ranks."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return ws, rank, local


def max_over_ranks(v, ws, device="cuda"):
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws, steps, t_max):
    """Whole-job throughput: every rank evolves its own replica for `steps`
    steps; the job takes the slowest rank's time."""
    return ws * steps / t_max


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


LATTICES = {16: (4, 4), 20: (4, 5), 24: (4, 6), 25: (5, 5), 28: (4, 7), 30: (5, 6)}


def workload(qubits=30):
    from workloads import heisenberg_lattice, neel_index
    rows = LATTICES[qubits]
    h = heisenberg_lattice(*rows)
    return h, neel_index(*rows), f"heisenberg_{rows[0]}x{rows[1]}_n{h.n}"


DT = 0.02

# DRAM bytes (read + write) per tile-pass launch from ncu: 4.235 GB per launch
# at n = 28 (mean of the 7 passes of a step), scaled by the 4x tile count to
# n = 30.  Taken on the pass kernels as they stand; re-captured when they change.
TRAFFIC_PER_LAUNCH = {28: 4.235e9, 30: 16.94e9}


def oracle_sample(h, per_group):
    """The rotations of one grouped Trotter step that a bounded CPU sample
    times: `per_group` of them, evenly spaced, from every group (so that
    non-diagonal and diagonal rotations are both represented), and the
    number of rotations in the whole step."""
    from oracle import planner as P
    groups = P.greedy_partition(h.x, h.z)
    picks = []
    for g in groups:
        k = min(per_group, len(g))
        picks += [g[(i * len(g)) // k] for i in range(k)]
    return picks, sum(len(g) for g in groups)


def time_oracle_rotations(h, psi, picks):
    """Wall seconds of the oracle applying the picked rotations, one at a
    time, to the 2^n complex128 host state psi (in place)."""
    import ctypes
    import oracle
    lib = oracle.lib()
    ptr = psi.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    t0 = time.perf_counter()
    for j in picks:
        lib.oracle_apply_rotation(h.n, ptr, int(h.x[j]), int(h.z[j]), float(h.c[j] * DT))
    return time.perf_counter() - t0


def cpu_oracle_sample(h, psi, per_group, threads=None):
    """Oracle (one rotation at a time, complex128, OpenMP on the host cores)
    on a bounded sample of one Trotter step (oracle_sample), scaled to whole
    steps: value = (sampled rotations / rotations per step) / seconds.
    threads (default: all cores) sets the OpenMP thread count for this
    sample only."""
    import oracle
    all_threads = oracle.num_threads()
    if threads is not None:
        oracle.set_threads(threads)
    try:
        picks, m = oracle_sample(h, per_group)
        time_oracle_rotations(h, psi, picks[:1])          # first touch, thread start
        t = time_oracle_rotations(h, psi, picks)
        cores = oracle.num_threads()
    finally:
        oracle.set_threads(all_threads)
    return {"value": len(picks) / m / t, "unit": "steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(picks)} of the {m} rotations of one Trotter step at n={h.n} "
                      f"({per_group} evenly spaced from each group), complex128, {t:.1f} s, "
                      f"scaled to a whole step"}


REFERENCE_PER_GROUP = 7   # rotations per group in one step of the reference arm


def run_reference(args):
    """The oracle as the reference arm.  A whole Trotter step of the oracle
    at n = 30 takes about half a minute of the host's cores, so each of the
    arm's steps is a bounded sample of one: REFERENCE_PER_GROUP rotations
    from every group.  ms_per_step is the measured wall time of one such
    sample step; value scales it to whole Trotter steps per second."""
    # The oracle runs on rank 0's host cores only; the other ranks have no
    # work and exit at once, so no process group is needed.
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle
    h, neel, name = workload(args.qubits)
    picks, m = oracle_sample(h, REFERENCE_PER_GROUP)
    psi = np.zeros(1 << h.n, dtype=np.complex128)
    psi[neel] = 1.0
    times = []
    for i in range(args.warmup + args.steps):
        t = time_oracle_rotations(h, psi, picks)
        if i >= args.warmup:
            times.append(t)
    t = float(np.mean(times))
    frac = len(picks) / m
    v = frac / t
    sample = (f"one step = {len(picks)} of the {m} rotations of one Trotter step at n={h.n} "
              f"({REFERENCE_PER_GROUP} evenly spaced from each group), complex128; value = "
              f"{len(picks)}/{m} Trotter steps / measured seconds per step")
    out = {"metric": METRIC, "value": v, "unit": "steps/s", "impl": "reference",
           "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t,
           "trotter_steps_per_step": frac,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
           "data": "synthetic", "config": {"workload": name, "n": h.n, "terms": h.m, "dt": DT,
                                            "order": 1, "initial": "neel"},
           "cpu_baseline": {"value": v, "unit": "steps/s", "kind": "oracle",
                            "cores": oracle.num_threads(), "sample": sample},
           "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def oracle_accuracy(sim, h, neel, dev, steps=2):
    """||psi_gpu - psi_oracle||_2 after `steps` first-order steps from the
    Neel state, for the complex64 and complex128 grouped paths, against the
    oracle (complex128, one rotation at a time) run on the host cores.  The
    comparison runs in chunks, so the host holds the oracle's state and one
    chunk of the GPU's."""
    import torch
    import oracle
    import paper_2206_11664_gb300 as sd
    N = 1 << h.n
    psi0 = np.zeros(N, dtype=np.complex128)
    psi0[neel] = 1.0
    t0 = time.perf_counter()
    ref = oracle.evolve(h, psi0, DT, steps, 1)
    t_oracle = time.perf_counter() - t0
    del psi0
    out = {"steps": steps, "oracle_s": t_oracle, "oracle_cores": oracle.num_threads()}
    chunk = 1 << 26
    for cdt, key in ((torch.complex64, "c64"), (torch.complex128, "c128")):
        s = torch.zeros(N, dtype=cdt, device=dev)
        s[neel] = 1.0
        sim.evolve(s, DT, steps, 1)
        acc = 0.0
        for a in range(0, N, chunk):
            g = s[a:a + chunk].to(torch.complex128).cpu().numpy()
            acc += float(np.sum(np.abs(g - ref[a:a + chunk]) ** 2))
        out["l2_" + key] = acc ** 0.5
        del s
        torch.cuda.empty_cache()
    out["tolerance"] = {"c64": 1e-4, "c128": 1e-10}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "heisenberg30":
        import bench_workloads
        return bench_workloads.run(args)
    import torch
    import paper_2206_11664_gb300 as sd

    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    h, neel, name = workload(args.qubits)
    n = h.n
    sim = sd.Simulator(h.n, h.x, h.z, h.c).plan(prefetch=args.prefetch)
    code = sd.C64 if args.state == "c64" else sd.C128
    cdt = torch.complex64 if args.state == "c64" else torch.complex128
    amp_bytes = 8 if args.state == "c64" else 16
    # shape autotuner: tile sizes 11..13 and, for complex64, both register layouts
    tuned = sim.autotune_shape(code, DT, steps=4, order=1, kmin=11, kmax=13) if args.autotune else None
    st64 = sim.schedule_stats(code, 1)
    launches = sim.count_passes(code, 1, args.steps)   # tile passes of the timed call
    stream = torch.cuda.current_stream()
    N = 1 << n

    def fresh(dtype):
        s = torch.zeros(N, dtype=dtype, device=dev)
        s[neel] = 1.0
        return s

    # ---------------------------------------------------------------- main leg
    state = fresh(cdt)
    sim.prepare(code, DT, args.steps, 1)      # programs of the timed call (run-time compilation)
    sim.evolve(state, DT, args.warmup, 1)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.evolve(state, DT, args.steps, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    t = e0.elapsed_time(e1) / 1e3
    barrier(ws)
    t = max_over_ranks(t, ws)
    value = job_value(ws, args.steps, t)
    norm_err = abs(float(torch.linalg.vector_norm(state.to(torch.complex128)).item()) - 1.0)

    peak, peak_kind = peaks()
    bytes_per_pass = 2 * N * amp_bytes
    avg_launch_s = t / launches
    achieved = bytes_per_pass / avg_launch_s / 1e9
    out = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.state,
           "data": "synthetic",
           "config": {"workload": name, "n": n, "terms": h.m, "groups": 3, "dt": DT, "order": 1,
                      "initial": "neel",
                      "state": ("complex64, Q0.64 phase angles" if args.state == "c64" else
                                "complex128, 64-bit fixed point in the passes, Q0.64 phase angles"),
                      "l2": "state 8 GiB > 129 MB L2, no flush needed" if n == 30 else "small",
                      "parallelism": f"replicas x{ws}", "tile_bits": st64["tile_bits"],
                      "autotune": ({"tile_bits": tuned["tile_bits"], "layout": tuned["layout"],
                                    "prefetch": tuned["prefetch"],
                                    "ms_per_step (K,layout,prefetch)": tuned["ms_per_step"]} if tuned else None),
                      "passes_per_step": launches / args.steps,
                      "passes_per_single_step": st64["passes_per_step"]},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak,
                        "traffic": TRAFFIC_PER_LAUNCH.get(n) if args.state == "c64" else None,
                        "kernel": f"sd_pass_{args.state}_* (one generated kernel per tile pass, "
                                  f"{launches} launches in {args.steps} steps; achieved = mean over them)",
                        "peak_kind": f"{peak_kind} copy bandwidth",
                        "bytes_per_launch": bytes_per_pass},
           "gpu_launches": launches,
           "clocks": ck,
           "norm_error": norm_err}
    if not args.no_extras and args.state == "c64" and ws == 1:
        # accuracy of the timed result: the same warmup + steps in complex128
        # (the complex128 path matches the oracle to 1e-10 in the parity tests)
        ref = fresh(torch.complex128)
        sim.evolve(ref, DT, args.warmup, 1)
        sim.evolve(ref, DT, args.steps, 1)
        diff = float(torch.linalg.vector_norm(state.to(torch.complex128) - ref).item())
        out["accuracy"] = {"l2_vs_complex128": diff, "steps": args.warmup + args.steps,
                           "tolerance": 1e-4}
        del ref
    del state
    torch.cuda.empty_cache()

    if not args.no_extras:
        # per-Pauli baseline on the same GPU and workload
        st = fresh(torch.complex64)
        sim.evolve_pauli(st, DT, 1, 1)
        torch.cuda.synchronize()
        e0.record(stream)
        sim.evolve_pauli(st, DT, args.pauli_steps, 1)
        e1.record(stream)
        torch.cuda.synchronize()
        tp = e0.elapsed_time(e1) / 1e3
        pp = args.pauli_steps / tp
        out["per_pauli"] = {"steps_per_s": pp, "passes_per_step": h.m,
                            "achieved_gbs": h.m * bytes_per_pass * args.pauli_steps / tp / 1e9,
                            "speedup_grouped_over_per_pauli": (value / ws) / pp}
        del st
        torch.cuda.empty_cache()
        # complex128 grouped (one GPU only: with several ranks on one host their
        # run-time compilations would compete for the host cores)
        if ws == 1:
            st = fresh(torch.complex128)
            k128 = max(2, args.steps // 4)
            sim.prepare(sd.C128, DT, k128, 1)
            sim.evolve(st, DT, 1, 1)
            torch.cuda.synchronize()
            e0.record(stream)
            sim.evolve(st, DT, k128, 1)
            e1.record(stream)
            torch.cuda.synchronize()
            t128 = e0.elapsed_time(e1) / 1e3
            l128 = sim.count_passes(sd.C128, 1, k128)
            out["c128"] = {"steps_per_s": k128 / t128, "passes_per_step": l128 / k128,
                           "achieved_gbs": l128 * 2 * N * 16 / t128 / 1e9}
            del st
            torch.cuda.empty_cache()
        # end to end through a pinned host buffer: one sd_evolve_host call copies
        # the state in, runs the steps and copies the result back
        host = torch.zeros(N, dtype=torch.complex64).pin_memory()
        host[neel] = 1.0
        dst = torch.empty(N, dtype=torch.complex64, device=dev)
        torch.cuda.synchronize()
        e0.record(stream)
        sim.evolve_host(host, dst, DT, args.steps, 1)
        e1.record(stream)
        torch.cuda.synchronize()
        te = max_over_ranks(e0.elapsed_time(e1) / 1e3, ws)
        sb = N * 8
        out["e2e"] = {"value": ws * args.steps / te, "unit": "steps/s",
                      "h2d_bytes_per_step": sb / args.steps, "d2h_bytes_per_step": sb / args.steps,
                      "note": f"one sd_evolve_host call = H2D of the {sb} B state, {args.steps} steps, "
                              "D2H of the state"}
        del host, dst
        torch.cuda.empty_cache()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # all host cores, then one core, on the same host state
        psi = np.zeros(N, dtype=np.complex128)
        psi[neel] = 1.0
        cb = cpu_oracle_sample(h, psi, per_group=7)
        one = cpu_oracle_sample(h, psi, per_group=1, threads=1)
        cb["one_core"] = {"value": one["value"], "unit": one["unit"], "cores": one["cores"],
                          "sample": one["sample"]}
        out["cpu_baseline"] = cb
        del psi
    if rank == 0 and ws == 1 and not args.no_oracle_check and args.state == "c64":
        # error of the grouped paths against the oracle on the same workload
        out.setdefault("accuracy", {})["vs_oracle"] = oracle_accuracy(sim, h, neel, dev)
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
