"""CPU ORACLE -- test infrastructure only.

Plain complex128 reference for the simulator: the Trotter product applied
one Pauli rotation at a time (sd_oracle.c, compiled here with gcc), plus an
independent Python planner (planner.py).  Only tests/, the smoke check and
the benchmark's CPU-baseline / reference legs import this package; the
simulator never does, and nothing here imports the simulator.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

from . import planner  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "sd_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sd_oracle.c with gcc (OpenMP) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp",
                               "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _configure(L):
    """Argument and result types of the exported routines."""
    u64p = ctypes.POINTER(ctypes.c_uint64)
    i64p = ctypes.POINTER(ctypes.c_int64)
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_apply_rotation.argtypes = [ctypes.c_int, dp, ctypes.c_uint64,
                                        ctypes.c_uint64, ctypes.c_double]
    L.oracle_apply_pauli.argtypes = [ctypes.c_int, dp, dp, ctypes.c_uint64,
                                     ctypes.c_uint64]
    L.oracle_apply_sequence.argtypes = [ctypes.c_int, dp, u64p, u64p, ctypes.c_int64,
                                        i64p, dp, ctypes.c_int64]
    L.oracle_expect.argtypes = [ctypes.c_int, dp, ctypes.c_int64, u64p, u64p, dp]
    L.oracle_expect.restype = ctypes.c_double
    L.oracle_grad.argtypes = [ctypes.c_int, dp, ctypes.c_int64, u64p, u64p, dp,
                              ctypes.c_int64, i64p, dp, ctypes.c_int64,
                              ctypes.c_int64, u64p, u64p, dp, dp]
    L.oracle_grad.restype = ctypes.c_double
    L.oracle_num_threads.restype = ctypes.c_int
    L.oracle_set_threads.argtypes = [ctypes.c_int]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def library(path: str):
    """Route every wrapper of this module through another build of the C
    routines (a copy with a planted mistake, for the tests that check that
    the pins catch it); the usual library is restored on exit."""
    global _lib
    usual = lib()
    _lib = _configure(ctypes.CDLL(path))
    try:
        yield _lib
    finally:
        _lib = usual


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _state(psi):
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    return psi


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_threads(t: int) -> None:
    lib().oracle_set_threads(int(t))


def apply_rotation(psi, x, z, theta):
    """psi <- exp(-i theta P_(x,z)) psi (returns a new array)."""
    out = _state(psi).copy()
    n = int(out.shape[0]).bit_length() - 1
    lib().oracle_apply_rotation(n, _p(out.view(np.float64), ctypes.c_double),
                                int(x), int(z), float(theta))
    return out


def apply_pauli(psi, x, z):
    psi = _state(psi)
    out = np.empty_like(psi)
    n = int(psi.shape[0]).bit_length() - 1
    lib().oracle_apply_pauli(n, _p(psi.view(np.float64), ctypes.c_double),
                             _p(out.view(np.float64), ctypes.c_double), int(x), int(z))
    return out


def sequence_arrays(groups, c, dt, order):
    seq = planner.trotter_sequence(groups, order)
    term = np.array([j for j, _ in seq], dtype=np.int64)
    dtk = np.array([f * dt for _, f in seq], dtype=np.float64)
    ang = np.array([c[j] * f * dt for j, f in seq], dtype=np.float64)
    return term, dtk, ang


def evolve(ham, psi0, dt, steps, order=1, groups=None, reps=None):
    """Grouped Trotter evolution, one rotation at a time in group order."""
    if groups is None:
        groups = planner.greedy_partition(ham.x, ham.z)
    psi = _state(psi0).copy()
    x = np.ascontiguousarray(ham.x, dtype=np.uint64)
    z = np.ascontiguousarray(ham.z, dtype=np.uint64)
    term, _, ang = sequence_arrays(groups, ham.c, dt, order)
    lib().oracle_apply_sequence(ham.n, _p(psi.view(np.float64), ctypes.c_double),
                                _p(x, ctypes.c_uint64), _p(z, ctypes.c_uint64),
                                len(term), _p(term, ctypes.c_int64),
                                _p(ang, ctypes.c_double), int(steps))
    return psi


def evolve_inplace(ham, psi, dt, steps, order=1, groups=None):
    """As evolve, on psi itself (a C-contiguous complex128 array) instead of
    a copy: for states too large to hold twice in host memory."""
    if groups is None:
        groups = planner.greedy_partition(ham.x, ham.z)
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous:
        raise ValueError("psi must be a C-contiguous complex128 array")
    x = np.ascontiguousarray(ham.x, dtype=np.uint64)
    z = np.ascontiguousarray(ham.z, dtype=np.uint64)
    term, _, ang = sequence_arrays(groups, ham.c, dt, order)
    lib().oracle_apply_sequence(ham.n, _p(psi.view(np.float64), ctypes.c_double),
                                _p(x, ctypes.c_uint64), _p(z, ctypes.c_uint64),
                                len(term), _p(term, ctypes.c_int64),
                                _p(ang, ctypes.c_double), int(steps))
    return psi


def expect(psi, ox, oz, oc):
    psi = _state(psi)
    n = int(psi.shape[0]).bit_length() - 1
    ox = np.ascontiguousarray(ox, dtype=np.uint64)
    oz = np.ascontiguousarray(oz, dtype=np.uint64)
    oc = np.ascontiguousarray(oc, dtype=np.float64)
    return float(lib().oracle_expect(n, _p(psi.view(np.float64), ctypes.c_double),
                                     len(oc), _p(ox, ctypes.c_uint64),
                                     _p(oz, ctypes.c_uint64), _p(oc, ctypes.c_double)))


def grad(ham, psi0, dt, steps, order, obs, groups=None):
    """(f, df/dc) for f = <psi_T|O|psi_T> by a per-rotation reverse sweep."""
    if groups is None:
        groups = planner.greedy_partition(ham.x, ham.z)
    psi0 = _state(psi0)
    x = np.ascontiguousarray(ham.x, dtype=np.uint64)
    z = np.ascontiguousarray(ham.z, dtype=np.uint64)
    c = np.ascontiguousarray(ham.c, dtype=np.float64)
    term, dtk, _ = sequence_arrays(groups, c, dt, order)
    ox, oz, oc = (np.ascontiguousarray(a, dtype=t) for a, t in
                  zip(obs, (np.uint64, np.uint64, np.float64)))
    g = np.zeros(len(c), dtype=np.float64)
    f = lib().oracle_grad(ham.n, _p(psi0.view(np.float64), ctypes.c_double), len(c),
                          _p(x, ctypes.c_uint64), _p(z, ctypes.c_uint64),
                          _p(c, ctypes.c_double), len(term), _p(term, ctypes.c_int64),
                          _p(dtk, ctypes.c_double), int(steps), len(oc),
                          _p(ox, ctypes.c_uint64), _p(oz, ctypes.c_uint64),
                          _p(oc, ctypes.c_double), _p(g, ctypes.c_double))
    return float(f), g
