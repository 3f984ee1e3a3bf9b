"""Planted mistakes in a copy of the oracle: each must make a pin fail.

The pins of ``tests/test_oracle_pins.py`` tie the FP64 oracle to the paper
and to mathematics it does not share code with (numpy/scipy routines, dense
matrices, closed forms, invariants).  To show they would notice a plausible
slip, each case below copies ``oracle/rl_oracle.c``, plants one mistake by an
exact text replacement, compiles the copy with the oracle's own flags and
runs the pin file against it in a fresh process: the run must fail.  The
unmodified copy, built the same way, must pass (so a failure is the pin's,
not the harness's).  Nothing here touches the real oracle library.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rl_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# name -> (exact text in rl_oracle.c, its replacement): one mistake each
MUTANTS = {
    # Eq. 3's convolution read as a correlation (offset sign flipped)
    "forward_offset_sign": (
        "long xx = orc_map((long)x - (i - ax), W, boundary);\n                    acc += w * u[yy * W + xx];",
        "long xx = orc_map((long)x + (i - ax), W, boundary);\n                    acc += w * u[yy * W + xx];"),
    # one column of taps dropped from the forward operator
    "forward_dropped_tap": (
        "double w = h[j * kw + i];\n                    if (w == 0.0) continue;\n"
        "                    long xx = orc_map((long)x - (i - ax), W, boundary);\n"
        "                    acc += w * u[yy * W + xx];",
        "double w = h[j * kw + i];\n                    if (w == 0.0 || i == kw - 1) continue;\n"
        "                    long xx = orc_map((long)x - (i - ax), W, boundary);\n"
        "                    acc += w * u[yy * W + xx];"),
    # the half-sample mirror off by one at the far edge
    "mirror_off_by_one": (
        "return r < n ? r : period - 1 - r;",
        "return r < n ? r : (period - 2 - r < 0 ? 0 : period - 2 - r);"),
    # the adjoint h* taken without reflecting h (Sec. 2)
    "adjoint_not_reflected": (
        "long yy = orc_map((long)y + (j - ay), H, boundary);",
        "long yy = orc_map((long)y - (j - ay), H, boundary);"),
    # the exact transpose scattered to the wrong side
    "transpose_wrong_side": (
        "long xx = orc_map((long)x - (i - ax), W, boundary);\n                    c[yy * W + xx] += w * qv;",
        "long xx = orc_map((long)x + (i - ax), W, boundary);\n                    c[yy * W + xx] += w * qv;"),
    # the ratio of Eq. 3 upside down
    "ratio_inverted": (
        "q[p] = v[p] > 0.0 ? f[p] / v[p] : 0.0;",
        "q[p] = v[p] > 0.0 && f[p] > 0.0 ? v[p] / f[p] : 0.0;"),
    # the stale ratio of Eq. 5 halved
    "stale_ratio_halved": (
        "rs[p] = q[p];",
        "rs[p] = 0.5 * q[p];"),
    # full iterations of the thinning schedule shifted by one (k mod P == 1)
    "reset_shifted": (
        "int full = !thin || (k % P == 0);",
        "int full = !thin || (k % P == 1);"),
    # the relative change rule replaced by the absolute one
    "relative_rule_absolute": (
        "if (use) d = relative ? (u[p] > 0.0 ? fabs(c[p] - 1.0) : 0.0)",
        "if (use) d = relative ? fabs(un - u[p])"),
    # disc support by strict inclusion (dx^2 + dy^2 < r^2)
    "disc_strict_inclusion": (
        "int in = dx * dx + dy * dy <= (long)r * r;",
        "int in = dx * dx + dy * dy < (long)r * r;"),
    # with Q = P the mask rebuilt on every iteration instead of full ones only
    "mask_update_every_iteration": (
        "else if (full)\n                    M[p] = (uint8_t)(d >= tau);",
        "else\n                    M[p] = (uint8_t)(use && d >= tau);"),
    # dense taps left unnormalised
    "taps_not_normalised": (
        "for (int k = 0; k < n; ++k) h[k] /= s;",
        "(void)s;"),
    # motion anchor rounded the other way for even lengths
    "motion_anchor_even": (
        "*kw = length; *kh = 1; *ax = length / 2; *ay = 0;",
        "*kw = length; *kh = 1; *ax = (length - 1) / 2; *ay = 0;"),
}

PLUGIN = """
import oracle
oracle._SRC = {src!r}
oracle._LIB = {lib!r}
oracle._lib = None
"""


def build_copy(tmp_path, name, text):
    """Compile a copy of the oracle source with the oracle's flags; returns
    the directory holding the library and the plugin that points the oracle
    package at it."""
    d = tmp_path / name
    d.mkdir()
    src, lib = d / "rl_oracle.c", d / "_rl_oracle.so"
    src.write_text(text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-o", str(lib), str(src), "-lm"], check=True, capture_output=True)
    os.utime(lib)  # newer than its source: the package will not rebuild it
    (d / f"mutant_{name}.py").write_text(PLUGIN.format(src=str(src), lib=str(lib)))
    return d


def run_pins(d, name):
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([str(d), ROOT, os.environ.get("PYTHONPATH", "")]),
               OMP_NUM_THREADS="2")
    return subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", f"mutant_{name}",
                           "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=600)


def test_unmodified_copy_passes_the_pins(tmp_path):
    d = build_copy(tmp_path, "control", open(SRC).read())
    r = run_pins(d, "control")
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(tmp_path, name):
    text = open(SRC).read()
    old, new = MUTANTS[name]
    assert text.count(old) == 1, f"{name}: the text to mutate is not in rl_oracle.c exactly once"
    d = build_copy(tmp_path, name, text.replace(old, new))
    r = run_pins(d, name)
    assert r.returncode == 1, f"{name}: no pin failed\n{r.stdout[-3000:]}"
    assert " failed" in r.stdout
