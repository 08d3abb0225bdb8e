"""The oracle's pins catch plausible mistakes (CPU only).

Each case below plants one mistake in a copy of the oracle's C source -- a
dropped factor, a wrong sign, a wrong index, an operand from the wrong side
of a pair, a reversed product -- builds the copy with gcc, routes the oracle
wrappers through it, and runs the pins of test_oracle_evolution.py.  At
least one pin must fail for every planted mistake, and the unaltered copy,
built the same way, must pass them all.
"""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_evolution as E

SRC = os.path.join(os.path.dirname(oracle.__file__), "sd_oracle.c")

PINS = [
    ("rotation and Pauli action against dense matrices", E.test_rotation_matches_expm, {}),
    ("first-order step against group exponentials",
     E.test_one_step_equals_product_of_group_exponentials, {"order": 1}),
    ("second-order step against group exponentials",
     E.test_one_step_equals_product_of_group_exponentials, {"order": 2}),
    ("norm", E.test_norm_preserved, {}),
    ("Trotter error slopes", E.test_trotter_error_orders, {}),
    ("one commuting group exact", E.test_single_group_is_exact_and_conserves_energy, {}),
    ("energy drift", E.test_energy_drift_bounded, {}),
    ("Strang time reversal", E.test_strang_time_reversal, {}),
    ("expectation against dense", E.test_expect_matches_dense, {}),
    ("gradient closed form", E.test_grad_closed_form, {}),
    ("gradient against central differences, order 1",
     E.test_grad_matches_central_differences, {"order": 1}),
    ("gradient against central differences, order 2",
     E.test_grad_matches_central_differences, {"order": 2}),
]

# (name, text in sd_oracle.c, the same text with the mistake planted)
MUTANTS = [
    ("Y without its factor i",
     "int k = popc64(x & z) + 2 * (popc64(z & (y ^ x)) & 1);",
     "int k = 2 * (popc64(z & (y ^ x)) & 1);"),
    ("Z parity taken on the target index instead of the source",
     "int k = popc64(x & z) + 2 * (popc64(z & (y ^ x)) & 1);",
     "int k = popc64(x & z) + 2 * (popc64(z & y) & 1);"),
    ("i^1 taken as -i",
     "case 1: *re = 0; *im = 1; break;",
     "case 1: *re = 0; *im = -1; break;"),
    ("diagonal rotation with the wrong sign on one component",
     "psi[2 * y] = c * ar + s * sg * ai;",
     "psi[2 * y] = c * ar - s * sg * ai;"),
    ("rotation by -theta",
     "double c = cos(theta), s = sin(theta);",
     "double c = cos(theta), s = -sin(theta);"),
    ("pair phases swapped",
     "double qyr = p1r * br - p1i * bi, qyi = p1r * bi + p1i * br;",
     "double qyr = p2r * br - p2i * bi, qyi = p2r * bi + p2i * br;"),
    ("Pauli action reads the target amplitude",
     "int64_t s = (int64_t)((uint64_t)y ^ x);",
     "int64_t s = (int64_t)y;"),
    ("expectation: conjugate dropped",
     "acc += ar * qr + ai * qi;",
     "acc += ar * qr - ai * qi;"),
    ("expectation: coefficient dropped",
     "total += oc[k] * acc;",
     "total += acc;"),
    ("rotations applied in reverse order",
     "for (int64_t k = 0; k < L; k++)\n            oracle_apply_rotation(n, psi,",
     "for (int64_t k = L - 1; k >= 0; k--)\n            oracle_apply_rotation(n, psi,"),
    ("gradient without the factor 2",
     "grad[j] += 2.0 * im * dtk[k];",
     "grad[j] += im * dtk[k];"),
    ("gradient sweep undoes the rotation in the wrong direction",
     "oracle_apply_rotation(n, phi, x[j], z[j], -a);",
     "oracle_apply_rotation(n, phi, x[j], z[j], a);"),
    ("gradient sweep leaves the adjoint state behind",
     "oracle_apply_rotation(n, lam, x[j], z[j], -a);",
     "(void)lam;"),
]


def _build(tmp_path, text, tag):
    src = tmp_path / f"oracle_{tag}.c"
    so = tmp_path / f"liboracle_{tag}.so"
    src.write_text(text)
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                           str(src), "-o", str(so), "-lm"])
    return str(so)


def _failing_pins(path, stop_at_first):
    failed = []
    with oracle.library(path):
        for name, fn, kw in PINS:
            try:
                fn(**kw)
            except AssertionError:
                failed.append(name)
                if stop_at_first:
                    break
    return failed


def test_unaltered_copy_passes_every_pin(tmp_path):
    with open(SRC) as f:
        text = f.read()
    assert _failing_pins(_build(tmp_path, text, "copy"), stop_at_first=False) == []


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, name, orig, bad):
    with open(SRC) as f:
        text = f.read()
    assert text.count(orig) == 1, f"the text to alter is not unique in the oracle: {orig!r}"
    failed = _failing_pins(_build(tmp_path, text.replace(orig, bad), "mutant"), stop_at_first=True)
    assert failed, f"no pin catches: {name}"


def _seq_mid_half(groups, order):
    """Second order with the middle group at dt/2 instead of dt."""
    return [(j, 0.5 if f == 1.0 and order == 2 else f) for j, f in _usual_seq(groups, order)]


def _seq_reversed_groups(groups, order):
    """Groups applied from last to first."""
    return _usual_seq(list(reversed(groups)), order)


def _seq_no_return(groups, order):
    """Second order without the closing half steps."""
    seq = _usual_seq(groups, order)
    if order == 2:
        last = max(i for i, (_, f) in enumerate(seq) if f == 1.0)
        return seq[:last + 1]
    return seq


_usual_seq = oracle.planner.trotter_sequence


@pytest.mark.parametrize("bad", [_seq_mid_half, _seq_reversed_groups, _seq_no_return],
                         ids=lambda f: f.__doc__.strip().rstrip("."))
def test_planted_sequence_mistake_fails_a_pin(monkeypatch, bad):
    """The same for the Python side of the oracle: the order and the
    fractions of dt in which a Trotter step applies the groups."""
    monkeypatch.setattr(oracle.planner, "trotter_sequence", bad)
    failed = []
    for name, fn, kw in PINS:
        try:
            fn(**kw)
        except AssertionError:
            failed.append(name)
            break
    assert failed


# ---------------------------------------------------------------- the oracle planner

PLANNER_SRC = os.path.join(os.path.dirname(oracle.__file__), "planner.py")

# (name, text in planner.py, the same text with the mistake planted)
PLANNER_MUTANTS = [
    ("H rule without its sign",
     "        xt, zt = _bit(x, a), _bit(z, a)\n        r ^= xt & zt\n        x = (x",
     "        xt, zt = _bit(x, a), _bit(z, a)\n        x = (x"),
    ("S rule moving Z into X",
     "        z ^= xt << a\n",
     "        x ^= zt << a\n"),
    ("CNOT Z rule as printed (z_t ^= z_c)",
     "        z ^= zt << c\n",
     "        z ^= zc << t\n"),
    ("CNOT sign without its last factor",
     "        r ^= xc & zt & (xt ^ zc ^ 1)\n",
     "        r ^= xc & zt & (xt ^ zc)\n"),
    ("CZ rule without its sign",
     "        r ^= xc & xt & (zt ^ zc)\n",
     ""),
    ("vectorised CNOT Z rule as printed",
     "            Z ^= zt << sc\n",
     "            Z ^= zc << st\n"),
    ("Algorithm 2 visiting the qubits first to last",
     "for i in reversed(range(nA)):",
     "for i in range(nA):"),
    ("Algorithm 2 applying H without a strict rank increase",
     "if r0 < xrank(trial):",
     "if r0 <= xrank(trial):"),
    ("Algorithm 6 eliminating above the pivot",
     "        for k in range(ir + 1, N):\n",
     "        for k in range(0, ir):\n"),
    ("Algorithm 4 skipping the S gate",
     "            if _bit(T[i][1], i):\n                apply(T, (\"S\", i, -1))\n"
     "                syn.append((\"S\", i, -1))\n",
     ""),
    ("skip rule leaving only-X qubits alone",
     "        if skip_rule >= SKIP_PAPER and has <= {2}:",
     "        if skip_rule >= SKIP_PAPER and has <= {1, 2}:"),
    ("first fit ignoring anticommutation",
     "            if not anti.any():",
     "            if True:"),
    ("symplectic complement built from (x, z) instead of (z, x)",
     "        cons.append(z | (x << n))\n",
     "        cons.append(x | (z << n))\n"),
    ("complement basis vector without its pivot entries",
     "            if _bit(M[i], f):\n                v |= 1 << pc\n",
     "            pass\n"),
    ("CNOT map inverse taken in the forward order",
     "return run(cn), run(list(reversed(cn)))",
     "return run(cn), run(cn)"),
]


def _planner_pins():
    from tests import test_oracle_planner as T
    pins = []
    for name in sorted(dir(T)):
        fn = getattr(T, name)
        if not name.startswith("test_") or not callable(fn):
            continue
        marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
        if marks:
            argname, values = marks[0].args[0], marks[0].args[1]
            pins += [(f"{name}[{v}]", fn, {argname: v}) for v in values]
        else:
            pins.append((name, fn, {}))
    return T, pins


def _load_planner(tmp_path, text):
    import importlib.util
    path = tmp_path / "planner_copy.py"
    path.write_text(text)
    spec = importlib.util.spec_from_file_location("planner_copy", str(path))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _failing_planner_pins(monkeypatch, mod, stop_at_first):
    T, pins = _planner_pins()
    monkeypatch.setattr(T, "P", mod)
    failed = []
    for name, fn, kw in pins:
        try:
            fn(**kw)
        except (AssertionError, mod.SynthesisError, RuntimeError, ValueError):
            failed.append(name)
            if stop_at_first:
                break
    return failed


def test_unaltered_planner_copy_passes_every_pin(tmp_path, monkeypatch):
    with open(PLANNER_SRC) as f:
        mod = _load_planner(tmp_path, f.read())
    assert len(_planner_pins()[1]) >= 15
    assert _failing_planner_pins(monkeypatch, mod, stop_at_first=False) == []


@pytest.mark.parametrize("name,orig,bad", PLANNER_MUTANTS, ids=[m[0] for m in PLANNER_MUTANTS])
def test_planted_planner_mistake_fails_a_pin(tmp_path, monkeypatch, name, orig, bad):
    with open(PLANNER_SRC) as f:
        text = f.read()
    assert text.count(orig) == 1, f"the text to alter is not unique in the planner: {orig!r}"
    mod = _load_planner(tmp_path, text.replace(orig, bad))
    assert _failing_planner_pins(monkeypatch, mod, stop_at_first=True), f"no pin catches: {name}"
