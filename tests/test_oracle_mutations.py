"""The oracle's pins must catch plausible slips.

Each case below plants one mistake in a copy of the C oracle (on the CPU, in
a temporary directory), builds it, and runs the pin suite against it; the
suite has to fail.  The shipped oracle is untouched.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hdda_oracle.c")

MUTANTS = {
    "start_point_not_midpoint": ("float tm = (t + tn) * 0.5f;", "float tm = t;"),
    "no_index_clamp": ("if (i > res - 1)\n                i = res - 1;", ""),
    "closed_upper_face": ("x[c] >= lo[c] && x[c] < hi[c]", "x[c] >= lo[c] && x[c] <= hi[c]"),
    "coarse_level_first": ("for (int l = 0; l < levels; ++l) {\n        const float* lo",
                           "for (int l = levels - 1; l >= 0; --l) {\n        const float* lo"),
    "transposed_lookup": ("((int64_t)l * r + idx[0]) * r + idx[1]) * r + idx[2]",
                          "((int64_t)l * r + idx[2]) * r + idx[1]) * r + idx[0]"),
    "clamp_nesting_swapped": ("fminf(fmaxf(t * cone, step), max_step)",
                              "fmaxf(fminf(t * cone, max_step), step)"),
    "origin_dropped": ("x[c] = o[c] + p;", "x[c] = p;"),
    "stop_rule_strict": ("if (tn > far_t)\n                break;\n            if (k == max_steps)\n                return ORACLE_ERR_STEP_LIMIT;\n            float tm",
                         "if (tn >= far_t)\n                break;\n            if (k == max_steps)\n                return ORACLE_ERR_STEP_LIMIT;\n            float tm"),
    "closed_form_lattice": ("            t = tn;\n            k += 1;",
                            "            k += 1;\n            t = near_t + (float)k * step;"),
    "transmittance_not_updated": ("T *= 1.0 - alpha;", ""),
    "colour_not_weighted_by_T": ("C[c] += T * alpha * (wc[c] / sigma);", "C[c] += alpha * (wc[c] / sigma);"),
    # the compositor's field (Sec. 1's accumulation over a sum of Gaussian blobs)
    "falloff_without_factor_2": ("exp(-d2 / (2.0 * sg * sg))", "exp(-d2 / (sg * sg))"),
    "amplitude_dropped": ("double w = (double)G[4] * exp(", "double w = exp("),
    "colour_not_weighted_by_density": [
        ("wc[c] += w * (double)G[5 + c];", "wc[c] += (double)G[5 + c];"),
        ("C[c] += T * alpha * (wc[c] / sigma);", "C[c] += T * alpha * (wc[c] / n_g);")],
    "field_at_interval_start": ("double tm = 0.5 * (a0 + a1);", "double tm = a0;"),
    "alpha_without_interval_length": ("-expm1(-sigma * (a1 - a0))", "-expm1(-sigma)"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    edits = MUTANTS[name]
    if isinstance(edits, tuple):
        edits = [edits]
    src = open(SRC).read()
    for old, new in edits:
        assert src.count(old) >= 1, f"mutation anchor for {name} not found: {old!r}"
        src = src.replace(old, new)
    with tempfile.TemporaryDirectory() as tmp:
        c = os.path.join(tmp, "m.c")
        so = os.path.join(tmp, "m.so")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                        "-std=c11", "-o", so, c, "-lm"], check=True)
        env = dict(os.environ, ORACLE_SO_OVERRIDE=so)
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                           env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
