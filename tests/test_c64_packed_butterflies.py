"""The complex64 pass generator's packed butterflies, checked on the CPU.

The run-time compiler's complex64 passes keep each register slot in one of
eight representations (the stored float pair holds +-re and +-im in either
order), so that most one-qubit Cliffords S^B H S^PA become two packed f32x2
operations, and fold the representations into the group exponential's
rotation and the final store.  tests/pass_source_dump.cpp prints the
generated source of a call's passes; this test interprets every line that
touches the thread's 16 amplitudes -- packed and scalar butterflies, slot
swaps, rotations, returns to the plain representation, quarter-turn layers
and stores -- on random amplitudes, random rotation phases and random
quarter turns, and compares what each round stores with the same round
generated with plain scalar butterflies (SD_C64_SCALAR=1), whose lines
(had_fixed, mono_fixed, diag_rotate) are interpreted by their definitions:
(u, v) -> (u + i^PA v, i^B (u - i^PA v)), (u, v) -> (i^PA v, u) or
(u, i^PA v), and a[s] -> a[s] e_s sc.  Indices, loads and the exchange are
the same in both sources.
"""
import os
import re
import shutil
import struct
import subprocess

import numpy as np
import pytest

from workloads import heisenberg_lattice, jw_like, random_klocal, tfim_chain

HERE = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.join(HERE, "..", "paper_2206_11664_gb300")
CSRC = os.path.join(PKG, "csrc")


@pytest.fixture(scope="module")
def dump(tmp_path_factory):
    cxx = shutil.which("g++")
    cudart = "/usr/local/cuda/lib64"
    if cxx is None or not os.path.isdir(cudart):
        pytest.skip("no host C++ compiler or CUDA runtime library")
    from paper_2206_11664_gb300 import build as B
    os.makedirs(B.OUT, exist_ok=True)
    B._embed_headers()
    exe = str(tmp_path_factory.mktemp("dump") / "pass_source_dump")
    subprocess.check_call([cxx, "-O1", "-std=c++17", "-I", CSRC, "-I", B.OUT, "-I", "/usr/local/cuda/include",
                           os.path.join(HERE, "pass_source_dump.cpp"), os.path.join(CSRC, "planner.cpp"),
                           os.path.join(CSRC, "schedule.cpp"), os.path.join(CSRC, "jit.cpp"),
                           "-L", cudart, "-lcudart", "-ldl", "-lpthread", "-o", exe])
    return exe


def _source(exe, tmp_path, h, scalar, K=13, c=4, order=1, reps=1, skip=2):
    inp = tmp_path / "in.bin"
    with open(inp, "wb") as f:
        f.write(struct.pack("<iqiiiiiqd", h.n, h.m, skip, K, c, order, reps, 1, 0.02))
        f.write(np.ascontiguousarray(h.x, dtype=np.uint64).tobytes())
        f.write(np.ascontiguousarray(h.z, dtype=np.uint64).tobytes())
        f.write(np.ascontiguousarray(h.c, dtype=np.float64).tobytes())
    env = dict(os.environ)
    env.pop("SD_C64_SCALAR", None)
    if scalar:
        env["SD_C64_SCALAR"] = "1"
    r = subprocess.run([exe, str(inp)], capture_output=True, text=True, env=env)
    assert r.returncode == 0, r.stderr
    return r.stdout


def _kernels(src):
    parts = re.split(r'extern "C" __global__ void __launch_bounds__\(\d+\) (sd_pass_c64_\d+)\(', src)
    return [(parts[i], re.split(r"\n    \{ // round \d+\n", parts[i + 1])[1:]) for i in range(1, len(parts), 2)]


A = r"a\[(\d+)\]"
PATTERNS = {
    "pack": re.compile(r"\{ const A u = " + A + r", v = " + A + r"; a\[\d+\] = (.*?); a\[\d+\] = (.*?); \}$"),
    "scalar": re.compile(r"\{ const float s0 = " + A + r"\.x, s1 = a\[\d+\]\.y, t0 = " + A + r"\.x, t1 = a\[\d+\]\.y; "
                         r"a\[\d+\]\.x = (.*?); a\[\d+\]\.y = (.*?); a\[\d+\]\.x = (.*?); a\[\d+\]\.y = (.*?); \}$"),
    "swap": re.compile(r"\{ const A w = " + A + r"; a\[\d+\] = " + A + r"; a\[\d+\] = w; \}$"),
    "signs": re.compile(A + r" = __fmul2_rn\(a\[\d+\], make_float2\((.*?), (.*?)\)\);$"),
    "order": re.compile(A + r" = make_float2\((-?)a\[\d+\]\.y, (-?)a\[\d+\]\.x\);$"),
    "rot_rep": re.compile(A + r" = rotate_tw32_rep<(.*?)>\(a\[\d+\], g\[\d+\], TW, \(T\)(.*?)\);$"),
    "had": re.compile(r"had_fixed<(\d+), (\d+), (\d+)>\(a\);$"),
    "mono": re.compile(r"mono_fixed<(\d+), (\d+), (\d+)>\(a\);$"),
    "rot": re.compile(r"diag_rotate\(a, G, TW, \(T\)(.*?)\);$"),
    "store": re.compile(r"(?:X\[sw \^ 0x[0-9a-f]+u\]|psi\[xf \| 0x[0-9a-f]+ull\]) = " + A + r";$"),
    "store_scaled": re.compile(r"\{ A w = " + A + r"; w\.x \*= \(T\)(.*?); w\.y \*= \(T\)(.*?); psi\[.*?\] = w; \}$"),
    "store_signs": re.compile(r"psi\[.*?\] = __fmul2_rn\(" + A + r", make_float2\(\(T\)(.*?), \(T\)(.*?)\)\);$"),
    "store_order": re.compile(r"psi\[.*?\] = make_float2\(" + A + r"\.y \* \(T\)(.*?), a\[\d+\]\.x \* \(T\)(.*?)\);$"),
    "store_perm": re.compile(r"for \(int s = 0; s < 16; s\+\+\) X\[base"),
    "phase": re.compile(r"phase_apply\(a, xf, gq, kp\.phases\[\d+\]"),
}


def _f(s):
    return float(s.replace("(T)", "").rstrip("f"))


class _Draw(dict):
    """Random draws per key, the same for both sources."""

    def __init__(self, seed, quarter):
        super().__init__()
        self.rng = np.random.default_rng(seed)
        self.quarter = quarter

    def __missing__(self, key):
        v = 1j ** int(self.rng.integers(4)) if self.quarter else np.exp(2j * np.pi * self.rng.random())
        self[key] = v
        return v


def _run_round(text, a, key, E, Q, counts):
    """What the round stores, interpreting its lines from amplitudes a."""
    a = list(a)
    out = []
    nrot = nph = 0

    def ipow(k):
        return 1j ** (k & 3)

    for line in text.split("\n"):
        line = line.strip()
        kind, m = next(((k, p.search(line) if k == "phase" or k == "store_perm" else p.match(line))
                        for k, p in PATTERNS.items() if (p.search(line) if k in ("phase", "store_perm")
                                                           else p.match(line))), (None, None))
        if kind == "pack":
            s, t = int(m[1]), int(m[2])
            u, v = a[s], a[t]

            def ev(e):
                if e == "__fadd2_rn(u, v)":
                    return u + v
                d = re.match(r"__ffma2_rn\(v, make_float2\((.*?), (.*?)\), u\)", e)
                return complex(v.real * _f(d[1]) + u.real, v.imag * _f(d[2]) + u.imag)

            a[s], a[t] = ev(m[3]), ev(m[4])
            counts["packed"] += 1
        elif kind == "scalar":
            s, t = int(m[1]), int(m[2])
            env = {"s0": a[s].real, "s1": a[s].imag, "t0": a[t].real, "t1": a[t].imag}
            v = [eval(m[k], {}, env) for k in (3, 4, 5, 6)]
            a[s], a[t] = complex(v[0], v[1]), complex(v[2], v[3])
            counts["scalar"] += 1
        elif kind == "swap":
            s, t = int(m[1]), int(m[2])
            a[s], a[t] = a[t], a[s]
        elif kind == "signs":
            s = int(m[1])
            a[s] = complex(a[s].real * _f(m[2]), a[s].imag * _f(m[3]))
        elif kind == "order":
            s = int(m[1])
            a[s] = complex(a[s].imag * (-1 if m[2] else 1), a[s].real * (-1 if m[3] else 1))
        elif kind == "rot_rep":
            s = int(m[1])
            swi, sri, sii, swo, sro, sio = (int(x) for x in m[2].split(","))
            p = (a[s].real, a[s].imag)
            r = complex(sri * p[swi], sii * p[1 - swi]) * E[key + (nrot, s)] * _f(m[3])
            a[s] = complex(sio * r.imag, sro * r.real) if swo else complex(sro * r.real, sio * r.imag)
            nrot += s == 15
        elif kind == "rot":
            for s in range(16):
                a[s] *= E[key + (nrot, s)] * _f(m[1])
            nrot += 1
        elif kind == "had":
            i, pa, b = (int(x) for x in m.groups())
            for s in range(16):
                if not (s >> i) & 1:
                    t = s | (1 << i)
                    u, w = a[s], ipow(pa) * a[t]
                    a[s], a[t] = u + w, ipow(b) * (u - w)
            counts["reference"] += 8
        elif kind == "mono":
            i, pa, xx = (int(x) for x in m.groups())
            for s in range(16):
                if not (s >> i) & 1:
                    t = s | (1 << i)
                    w = ipow(pa) * a[t]
                    a[s], a[t] = (w, a[s]) if xx else (a[s], w)
        elif kind == "phase":
            for s in range(16):
                a[s] *= Q[key + (nph, s)]
            nph += 1
        elif kind == "store":
            out.append(a[int(m[1])])
        elif kind in ("store_scaled", "store_signs"):
            s = int(m[1])
            out.append(complex(a[s].real * _f(m[2]), a[s].imag * _f(m[3])))
        elif kind == "store_order":
            s = int(m[1])
            out.append(complex(a[s].imag * _f(m[2]), a[s].real * _f(m[3])))
        elif kind == "store_perm":
            out.extend(a)
        elif re.search(r"\ba\[\d+\](\.[xy])? =", line) and not re.search(r"= (Pf|X)\[", line):
            raise AssertionError("line not understood: " + line)
    return out


def _compare(exe, tmp_path, h, **kw):
    new = _kernels(_source(exe, tmp_path, h, False, **kw))
    ref = _kernels(_source(exe, tmp_path, h, True, **kw))
    assert len(new) == len(ref) > 0
    rng = np.random.default_rng(11)
    E, Q = _Draw(1, False), _Draw(2, True)
    counts = {"packed": 0, "scalar": 0, "reference": 0}
    stores = 0
    for ki, ((nn, rn), (nr, rr)) in enumerate(zip(new, ref)):
        assert nn == nr and len(rn) == len(rr)
        for ri, (tn, tr) in enumerate(zip(rn, rr)):
            a0 = list(rng.standard_normal(16) + 1j * rng.standard_normal(16))
            got = _run_round(tn, a0, (ki, ri), E, Q, counts)
            want = _run_round(tr, a0, (ki, ri), E, Q, counts)
            assert len(got) == len(want), (nn, ri)
            if got:
                assert np.max(np.abs(np.array(got) - np.array(want))) < 1e-12, (nn, ri)
            stores += len(got)
    assert stores > 0
    assert counts["packed"] + counts["scalar"] == counts["reference"]
    return counts


def test_heisenberg_block_program(dump, tmp_path):
    """The 5x6 Heisenberg block of four first-order steps (25 passes): the
    stores agree, and more than 70% of the butterflies are packed."""
    c = _compare(dump, tmp_path, heisenberg_lattice(5, 6), reps=4)
    assert c["packed"] > 0.7 * c["reference"], c


@pytest.mark.parametrize("case", ["heisenberg order 2", "random k-local, CNOT and S/CZ layers",
                                  "random k-local order 2", "JW-style", "TFIM chain"])
def test_other_workloads(dump, tmp_path, case):
    """Schedules with slot swaps (X S^a gates), tile permutations, quarter-turn
    layers and several exponentials per pass, at the default tile size and a
    smaller one."""
    rng = np.random.default_rng(3)
    h, kw = {
        "heisenberg order 2": (heisenberg_lattice(4, 5), dict(order=2)),
        "random k-local, CNOT and S/CZ layers": (random_klocal(16, 40, rng, weights=(2, 3, 4)), dict(skip=0)),
        "random k-local order 2": (random_klocal(18, 60, rng, weights=(2, 3)), dict(order=2, K=11)),
        "JW-style": (jw_like(n=16, m=300, rng=rng), dict()),
        "TFIM chain": (tfim_chain(20), dict(order=2, K=12, c=3)),
    }[case]
    c = _compare(dump, tmp_path, h, **kw)
    assert c["packed"] > 0, c
