"""GB300 (sm_103a) simulator of Hamiltonian dynamics by simultaneous
diagonalisation of commuting Pauli groups (Kawase & Fujii, arXiv:2206.11664).

Thin binding over the C ABI in include/sd.h: this module only marshals
arguments (numpy host arrays, torch device tensors, CUDA stream handles);
planning runs in the native host library and every state-vector operation
runs in the library's CUDA kernels.  There is no CPU fallback: if the native
library is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as N

__all__ = ["Simulator", "SDError", "evolve_batch", "prepare_batch", "TrotterExpectation", "C64", "C128"]

C64, C128 = N.SD_C64, N.SD_C128


class SDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{N.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _u64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a, t):
    return a.ctypes.data_as(t)


def _obs(obs):
    """(x, z, c) arrays of a Pauli-sum observable, checked for equal length
    (the library reads len(c) entries of each)."""
    ox, oz, oc = _u64(obs[0]), _u64(obs[1]), _f64(obs[2])
    if not (oc.ndim == 1 and ox.shape == oz.shape == oc.shape):
        raise ValueError("observable arrays x, z, c must be 1-D and of equal length")
    return ox, oz, oc


def _dtype_of(state, n=None):
    import torch
    if not isinstance(state, torch.Tensor) or not state.is_cuda:
        raise TypeError("state must be a CUDA torch tensor")
    if n is not None and state.numel() != (1 << n):
        raise ValueError(f"state must hold 2^{n} amplitudes")
    if not state.is_contiguous():
        raise ValueError("state must be contiguous")
    if state.dtype == torch.complex64:
        return N.SD_C64
    if state.dtype == torch.complex128:
        return N.SD_C128
    raise TypeError("state must be complex64 or complex128")


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Simulator:
    """H = sum_j c_j P_j on n qubits; qubit q is amplitude-index bit q and bit
    q of the masks (x, z): I (0,0), X (1,0), Z (0,1), Y (1,1)."""

    def __init__(self, n, x, z, c):
        self._lib = N.load()
        self.n = int(n)
        x, z, c = _u64(x), _u64(z), _f64(c)
        if not (x.shape == z.shape == c.shape) or x.ndim != 1:
            raise ValueError("x, z, c must be 1-D arrays of equal length")
        self.m = int(c.shape[0])
        h = ctypes.c_void_p()
        st = self._lib.sd_create(self.n, self.m, _ptr(x, N.P_u64), _ptr(z, N.P_u64),
                                 _ptr(c, N.P_dbl), ctypes.byref(h))
        if st != N.SD_OK:
            raise SDError(st, self._lib.sd_last_error(None).decode())
        self._h = h

    @classmethod
    def from_strings(cls, strings, coeffs):
        """Terms as text over {I,X,Y,Z}, character q = qubit q (sd_create_str)."""
        self = cls.__new__(cls)
        self._h = None
        self._lib = N.load()
        if len(strings) == 0:
            raise ValueError("need at least one Pauli string")
        self.n = len(strings[0])
        self.m = len(strings)
        c = _f64(coeffs)
        if c.shape != (self.m,):
            raise ValueError("need one coefficient per string")
        arr = (ctypes.c_char_p * self.m)(*[s.encode() for s in strings])
        h = ctypes.c_void_p()
        st = self._lib.sd_create_str(self.n, self.m, arr, _ptr(c, N.P_dbl), ctypes.byref(h))
        if st != N.SD_OK:
            self._h = None
            raise SDError(st, self._lib.sd_last_error(None).decode())
        self._h = h
        return self

    # ------------------------------------------------------------ plumbing
    def _check(self, st):
        if st != N.SD_OK:
            raise SDError(st, self._lib.sd_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ planning
    def plan(self, skip_rule=-1, tile_bits=0, jit=0, grouping=0, layout=0, prefetch=0):
        """Host planning.  jit: 0 automatic, 1 always, -1 never; grouping:
        0 first fit, 1 largest first, 2 DSATUR, 3 by |c|; layout of the
        complex64 run-time passes: 0 default, -1 plain, 1 paired; prefetch
        depth of the run-time passes: 0 default, 1, 2 or 3 (see sd.h)."""
        o = N.PlanOpts(skip_rule, tile_bits, jit, grouping, layout, prefetch)
        self._check(self._lib.sd_plan(self._h, ctypes.byref(o)))
        return self

    def set_coeffs(self, c):
        c = _f64(c)
        if c.shape != (self.m,):
            raise ValueError("need one coefficient per term")
        self._check(self._lib.sd_set_coeffs(self._h, _ptr(c, N.P_dbl)))

    def plan_view(self):
        v = N.PlanView()
        self._check(self._lib.sd_get_plan(self._h, ctypes.byref(v)))
        G, m, n = v.n_groups, v.m, v.n
        goff = np.ctypeslib.as_array(v.group_offsets, (G + 1,)).copy()
        gateoff = np.ctypeslib.as_array(v.gate_offsets, (G + 1,)).copy()
        ng = int(gateoff[-1])
        gates = (np.ctypeslib.as_array(v.gates, (max(ng, 1) * 3,))[: ng * 3].reshape(ng, 3).copy()
                 if ng else np.zeros((0, 3), np.int32))
        return {
            "n_groups": int(G),
            "group_offsets": goff,
            "group_terms": np.ctypeslib.as_array(v.group_terms, (m,)).copy(),
            "masks": np.ctypeslib.as_array(v.masks, (m,)).copy(),
            "signs": np.ctypeslib.as_array(v.signs, (m,)).copy(),
            "gate_offsets": gateoff,
            "gates": gates,
            "cnot_cols": np.ctypeslib.as_array(v.cnot_cols, (G * n,)).copy().reshape(G, n),
            "cnot_inv_cols": np.ctypeslib.as_array(v.cnot_inv_cols, (G * n,)).copy().reshape(G, n),
        }

    def schedule_stats(self, dtype=C64, order=1):
        s = N.ScheduleStats()
        self._check(self._lib.sd_get_schedule(self._h, dtype, order, ctypes.byref(s)))
        return {"tile_bits": s.tile_bits, "passes_per_step": s.passes_per_step,
                "rounds_per_step": s.rounds_per_step, "diag_passes": s.diag_passes,
                "onchip": bool(s.onchip)}

    def prepare(self, dtype, dt, steps, order=1):
        """Build (no launch) the programs evolve(., dt, steps, order) runs on
        a state of `dtype` (C64 / C128), including run-time compiled kernels."""
        self._check(self._lib.sd_prepare(self._h, dtype, float(dt), int(steps), int(order)))
        return self

    def autotune(self, dtype, dt, steps=4, order=1, kmin=None, kmax=None):
        """Time tile sizes kmin..kmax on a scratch state and keep the fastest
        for `dtype`; returns (best K, {K: ms per step}) (best K is 0 when the
        state stays on chip)."""
        kmax = 13 if kmax is None else int(kmax)
        kmin = max(9, kmax - 2) if kmin is None else int(kmin)
        best = ctypes.c_int(0)
        times = np.zeros(kmax - kmin + 1)
        self._check(self._lib.sd_autotune(self._h, dtype, float(dt), int(steps), int(order), kmin, kmax,
                                          ctypes.byref(best), times.ctypes.data_as(N.P_dbl)))
        return best.value, {kmin + i: float(t) for i, t in enumerate(times) if t > 0}

    def autotune_shape(self, dtype, dt, steps=4, order=1, kmin=None, kmax=None, cache=None):
        """Time tile sizes kmin..kmax and, for complex64 passes compiled at
        run time, both register layouts (sd_autotune_shape); the fastest
        shape is kept for `dtype`.  Returns {"tile_bits", "layout",
        "prefetch", "ms_per_step": {"K,layout,prefetch": ms}}.  With `cache` (a JSON file path),
        a shape stored there for this Hamiltonian, dtype, order and dt is
        applied by re-planning with it instead of timing, and a newly timed
        shape is stored."""
        import hashlib
        import json
        import os
        kmax = 13 if kmax is None else int(kmax)
        kmin = max(9, kmax - 2) if kmin is None else int(kmin)
        key = None
        if cache is not None:
            v = self.plan_view()
            hsh = hashlib.sha256()
            for name in ("group_terms", "masks", "signs", "gates"):
                hsh.update(np.ascontiguousarray(v[name]).tobytes())
            key = f"n{self.n}_m{self.m}_{'c128' if dtype == C128 else 'c64'}_o{int(order)}_dt{float(dt)!r}_" \
                  f"s{int(steps)}_k{kmin}-{kmax}_{hsh.hexdigest()[:16]}"
            if os.path.exists(cache):
                with open(cache) as f:
                    known = json.load(f)
                if key in known:
                    got = known[key]
                    self.plan(tile_bits=got["tile_bits"], layout=got["layout"], prefetch=got["prefetch"])
                    got = dict(got)
                    got["cached"] = True
                    return got
        r = N.TuneResult()
        self._check(self._lib.sd_autotune_shape(self._h, dtype, float(dt), int(steps), int(order), kmin, kmax,
                                                ctypes.byref(r)))
        ms = {}
        two = 2 if dtype == C128 else 3        # the dtype's two-buffer form
        for li, (lay, pf) in enumerate(((-1, 1), (-1, two), (1, 1), (1, two))):
            for k in range(kmin, kmax + 1):
                if r.ms[li][k - 9] > 0:
                    ms[f"{k},{lay},{pf}"] = float(r.ms[li][k - 9])
        out = {"tile_bits": r.best_k, "layout": r.best_layout, "prefetch": r.best_prefetch, "ms_per_step": ms,
               "cached": False}
        if key is not None and r.best_k > 0:
            known = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    known = json.load(f)
            known[key] = {"tile_bits": r.best_k, "layout": r.best_layout, "prefetch": r.best_prefetch,
                          "ms_per_step": ms}
            tmp = f"{cache}.tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(known, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return out

    def precompile(self, dtype, steps, order=1):
        """Compile (host only, NVRTC) the kernels evolve(., dt, steps, order)
        compiles at run time into the on-disk cache; returns the number of
        NVRTC programs compiled."""
        out = ctypes.c_int64(0)
        self._check(self._lib.sd_precompile(self._h, dtype, int(steps), int(order), ctypes.byref(out)))
        return out.value

    def count_passes(self, dtype=C64, order=1, steps=1):
        """Tile-pass launches evolve() makes for `steps` steps (0 on chip)."""
        out = ctypes.c_int64(0)
        self._check(self._lib.sd_count_passes(self._h, dtype, order, int(steps), ctypes.byref(out)))
        return out.value

    # ------------------------------------------------------------ dynamics
    def evolve(self, state, dt, steps, order=1, stream=None):
        """In place: `steps` Trotter steps of size dt (order 1 or 2)."""
        self._check(self._lib.sd_evolve(self._h, ctypes.c_void_p(state.data_ptr()),
                                        _dtype_of(state, self.n), float(dt), int(steps), int(order),
                                        _stream(stream)))
        return state

    def evolve_host(self, host_state, work, dt, steps, order=1, stream=None):
        """End to end: copy the pinned host tensor `host_state` into the device
        tensor `work`, evolve it there, copy it back (one asynchronous call)."""
        if not host_state.is_pinned():
            raise ValueError("host_state must be pinned (pin_memory())")
        if host_state.dtype != work.dtype or host_state.numel() != work.numel():
            raise ValueError("work must match host_state in dtype and size")
        self._check(self._lib.sd_evolve_host(self._h, ctypes.c_void_p(host_state.data_ptr()),
                                             ctypes.c_void_p(work.data_ptr()), _dtype_of(work, self.n),
                                             float(dt), int(steps), int(order), _stream(stream)))
        return host_state

    def evolve_pauli(self, state, dt, steps, order=1, stream=None):
        """Baseline: one state pass per term (same product, ungrouped)."""
        self._check(self._lib.sd_evolve_pauli(self._h, ctypes.c_void_p(state.data_ptr()),
                                              _dtype_of(state, self.n), float(dt), int(steps), int(order),
                                              _stream(stream)))
        return state

    def evolve_observe(self, state, dt, steps, obs, trace, order=1, stream=None):
        """Evolve and write <O> after every step into `trace` (CUDA float64, len steps)."""
        import torch
        if trace.dtype != torch.float64 or not trace.is_cuda or trace.numel() < steps:
            raise ValueError("trace must be a CUDA float64 tensor with >= steps entries")
        ox, oz, oc = _obs(obs)
        self._check(self._lib.sd_evolve_observe(
            self._h, ctypes.c_void_p(state.data_ptr()), _dtype_of(state, self.n), float(dt), int(steps),
            int(order), len(oc), _ptr(ox, N.P_u64), _ptr(oz, N.P_u64), _ptr(oc, N.P_dbl),
            ctypes.c_void_p(trace.data_ptr()), _stream(stream)))
        return trace

    def expect(self, state, obs, stream=None):
        ox, oz, oc = _obs(obs)
        out = ctypes.c_double()
        self._check(self._lib.sd_expect(self._h, ctypes.c_void_p(state.data_ptr()), _dtype_of(state, self.n),
                                        len(oc), _ptr(ox, N.P_u64), _ptr(oz, N.P_u64),
                                        _ptr(oc, N.P_dbl), ctypes.byref(out), _stream(stream)))
        return out.value

    def grad(self, state0, dt, steps, obs, order=1, stream=None):
        """(f, df/dc) for f = <psi_T|O|psi_T>, psi_T = evolve(state0); state0 unchanged."""
        ox, oz, oc = _obs(obs)
        g = np.zeros(self.m, np.float64)
        f = ctypes.c_double()
        self._check(self._lib.sd_grad(self._h, ctypes.c_void_p(state0.data_ptr()), _dtype_of(state0, self.n),
                                      float(dt), int(steps), int(order), len(oc), _ptr(ox, N.P_u64),
                                      _ptr(oz, N.P_u64), _ptr(oc, N.P_dbl), ctypes.byref(f),
                                      _ptr(g, N.P_dbl), _stream(stream)))
        return f.value, g


def _batch_args(sims, states):
    if len(sims) != len(states):
        raise ValueError("one state per simulator")
    dts = {_dtype_of(s) for s in states}
    if len(dts) != 1:
        raise ValueError("all states must have the same dtype")
    hs = (ctypes.c_void_p * len(sims))(*[s._h for s in sims])
    ps = (ctypes.c_void_p * len(states))(*[s.data_ptr() for s in states])
    return hs, ps, dts.pop()


def evolve_batch(sims, states, dt, steps, order=1, stream=None):
    """Evolve independent problems (each planned, own state) in one call.
    A repeated call with the same problems, states and arguments only
    launches kernels (capturable in a CUDA graph)."""
    if not sims:
        return
    lib = sims[0]._lib
    hs, ps, dt_code = _batch_args(sims, states)
    st = lib.sd_evolve_batch(hs, ps, len(sims), dt_code, float(dt), int(steps), int(order),
                             _stream(stream))
    if st != N.SD_OK:
        raise SDError(st, lib.sd_last_error(None).decode())


def prepare_batch(sims, states, dt, steps, order=1):
    """Build (no launch) what evolve_batch with these arguments runs."""
    if not sims:
        return
    lib = sims[0]._lib
    hs, ps, dt_code = _batch_args(sims, states)
    st = lib.sd_prepare_batch(hs, ps, len(sims), dt_code, float(dt), int(steps), int(order))
    if st != N.SD_OK:
        raise SDError(st, lib.sd_last_error(None).decode())


try:
    import torch as _torch

    class TrotterExpectation(_torch.autograd.Function):
        """f(c) = <psi_T(c)|O|psi_T(c)> with d f / d c from the adjoint kernel.

        apply(c, sim, state0, dt, steps, obs, order): c is a float64 tensor of the
        m Hamiltonian coefficients (input term order)."""

        @staticmethod
        def forward(ctx, c, sim, state0, dt, steps, obs, order=1):
            sim.set_coeffs(c.detach().cpu().numpy())
            f, g = sim.grad(state0, dt, steps, obs, order)
            ctx.save_for_backward(_torch.from_numpy(g).to(c.device))
            return c.new_tensor(f)

        @staticmethod
        def backward(ctx, gout):
            (g,) = ctx.saved_tensors
            return gout * g, None, None, None, None, None, None
except ImportError:  # torch is required for device memory; keep the ABI importable
    TrotterExpectation = None
