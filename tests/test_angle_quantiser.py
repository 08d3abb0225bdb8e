"""The Q0.64 angle quantiser of the pass scheduler, compiled as host C++ and
checked against exact rational arithmetic: a phase of t turns is stored as
the integer nearest to 2^64 (t mod 1) (ties to even), reduced to a signed
64-bit value, so that sums of stored angles are exact modulo one turn."""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2206_11664_gb300", "csrc")


def _exact(t):
    v = Fraction(t) * (1 << 64)
    fl = v.numerator // v.denominator
    rem = v - fl
    r = fl + (1 if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1) else 0)
    r %= 1 << 64
    return r - (1 << 64) if r >= 1 << 63 else r


def test_turns_q64_is_exact(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "q64_host_check")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", CSRC, "-I", "/usr/local/cuda/include",
                           os.path.join(HERE, "q64_host_check.cpp"), os.path.join(CSRC, "schedule.cpp"),
                           os.path.join(CSRC, "planner.cpp"), "-o", exe])
    rng = np.random.default_rng(17)
    ts = [0.0, -0.0, 0.25, -0.25, 0.5, -0.5, 1.5, -1.5, 2.5, 1.0, -1.0, 1e-300, -1e-300,
          2.0 ** -64, 2.0 ** -65, 3 * 2.0 ** -66, 0.5 - 2.0 ** -54, -0.5 + 2.0 ** -54, 1e15 + 0.25]
    ts += list(rng.uniform(-1, 1, 2000))
    ts += list(rng.standard_normal(500) * 1e6)
    ts += list(rng.standard_normal(500) * 1e-9)
    ts += [0.02 * c / (2 * np.pi) for c in rng.standard_normal(500)]   # dt c_j / 2 pi
    out = subprocess.run([exe], input="\n".join(repr(float(t)) for t in ts), capture_output=True,
                         text=True, check=True).stdout.split()
    assert len(out) == len(ts)
    for t, got in zip(ts, out):
        assert int(got) == _exact(t), (t, got, _exact(t))
    # sums of stored angles wrap exactly modulo one turn
    a, b = 0.375, 0.875
    q = (_exact(a) + _exact(b)) % (1 << 64)
    assert q == _exact(0.25) % (1 << 64)
