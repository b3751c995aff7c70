"""Plant a mistake in a copy of the oracle and check that the pins catch it.

Each case rebuilds oracle.c with one plausible error (a dropped term, a wrong
sign, a transposed index, a missing scale, a double rounding) into a
temporary library, runs every pin against it in a child process (a broken
index may read out of bounds; a crash counts as caught) and requires at least
one pin to fail.  The unmodified oracle must pass them all in the same
harness."""
import os
import subprocess
import sys
import textwrap

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "gemv_plain_dropped_last_term": (
        "for (int64_t j = 0; j < n; ++j) s = s + A[idx(layout, i, j, lda)] * x[j];",
        "for (int64_t j = 0; j < n - 1; ++j) s = s + A[idx(layout, i, j, lda)] * x[j];"),
    "gemv_plain_wrong_sign": (
        "c[i] = c[i] + alpha * s;", "c[i] = c[i] - alpha * s;"),
    "gemv_plain_dropped_initial_c": (
        "c[i] = c[i] + alpha * s;", "c[i] = alpha * s;"),
    "col_major_transposed_index": (
        "return layout == 0 ? i * ld + j : i + j * ld;",
        "return layout == 0 ? i * ld + j : j + i * ld;"),
    "gemv_acc_transposed_operand": (
        "two_prod(A[idx(layout, i, j, lda)], x[j], &h, &r);",
        "two_prod(A[idx(layout, j, i, lda)], x[j], &h, &r);"),
    "gemv_acc_dropped_compensation": (
        "      s = s + (q + r);\n    }\n    /* the row sum",
        "      s = s + q;\n    }\n    /* the row sum"),
    "dot_plain_dropped_initial_alpha": (
        "return alpha + s;", "return s;"),
    "dot_acc_skips_chunk_element": (
        "int64_t lo = k * ORACLE_DOT_CHUNK;", "int64_t lo = k * ORACLE_DOT_CHUNK + 1;"),
    "dot_acc_dropped_chunk_compensation": (
        "S = S + (q + s);", "S = S + q;"),
    "dger_dropped_alpha": (
        "double t = alpha * y[j];", "double t = y[j];"),
    "sger_double_rounding": (
        "C[k] = fmaf(x[i], t, C[k]);", "C[k] = x[i] * t + C[k];"),
    "bf16_ties_always_down": (
        "const uint32_t bias = 0x7FFFu + ((u >> 16) & 1u);", "const uint32_t bias = 0x7FFFu;"),
    "e4m3_ties_half_up": (
        "  if (r < 0.5) return f;\n  return fmod(f, 2.0) == 0.0 ? f : f + 1.0;",
        "  if (r < 0.5) return f;\n  return f + 1.0;"),
    "e4m3_no_saturation": (
        "if (a >= 448.0) return sign | 0x7E;", "if (a >= 480.0) return sign | 0x7E;"),
    "e4m3_wrong_exponent_bias": (
        "const int code = ((e + 7) << 3)", "const int code = ((e + 8) << 3)"),
    "e4m3_scale_not_amax": (
        "const float s = amax / 448.0f;", "const float s = amax / 256.0f;"),
    "gemv_scale_signed_sum": (
        "s = s + fabs(A[idx(layout, i, j, lda)] * x[j]);",
        "s = s + A[idx(layout, i, j, lda)] * x[j];"),
}

RUNNER = textwrap.dedent("""
    import sys
    sys.path[:0] = [{root!r}, {tests!r}]
    import oracle, pins
    O = oracle.load(sys.argv[1])
    failed = []
    for pin in pins.ALL_PINS:
        try:
            pin(O)
        except Exception as e:
            failed.append(pin.__name__)
    print("FAILED:" + ",".join(failed))
""")


def _run_pins(lib_path, tmp_path):
    script = tmp_path / "run_pins.py"
    script.write_text(RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests")))
    r = subprocess.run([sys.executable, str(script), lib_path], capture_output=True, text=True,
                       timeout=300)
    if r.returncode != 0:
        return None  # crashed: the mistake was caught by a crash
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("FAILED:")][-1]
    return [f for f in line[len("FAILED:"):].split(",") if f]


def test_unmodified_oracle_passes_harness(tmp_path):
    lib = str(tmp_path / "liboracle_copy.so")
    oracle.build(out=lib)
    assert _run_pins(lib, tmp_path) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(oracle.SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mutant_src = tmp_path / "oracle_mutant.c"
    mutant_src.write_text(src.replace(old, new))
    lib = str(tmp_path / "liboracle_mutant.so")
    oracle.build(src=str(mutant_src), out=lib)
    failed = _run_pins(lib, tmp_path)
    assert failed is None or len(failed) > 0, f"no pin caught mutant {name}"
