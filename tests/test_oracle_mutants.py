"""The pins catch plausible slips: each mutant of the oracle fails at least one.

Each mutant is the oracle's C source with one deliberate mistake, compiled
on the CPU into a temporary library and swapped in for the duration of the
pin run.  Nothing here touches a GPU.
"""
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins  # noqa: E402

SRC = open(os.path.join(os.path.dirname(oracle.__file__), "rp_oracle.c")).read()

MUTANTS = {
    "interpolation weights swapped": ("double sr = (1.0 - w) * a + w * b;",
                                      "double sr = w * a + (1.0 - w) * b;"),
    "self cell dropped": ("double w0 = C * hs * hs;", "double w0 = 0.0;"),
    "self weight C*h instead of C*h^2": ("double w0 = C * hs * hs;", "double w0 = C * hs;"),
    "volume element h^2": ("const double vol = hs * hs * hs;", "const double vol = hs * hs;"),
    "delay one step short": ("long long j0 = (long long)step - (long long)m;",
                             "long long j0 = (long long)step - (long long)m + 1;"),
    "delay rounded down (no interpolation)": ("double w = tau - m; ", "double w = 0.0; "),
    "A missing 1/c": ("out[4 * p + f] = acc_value(&acc[f]) / c;",
                      "out[4 * p + f] = acc_value(&acc[f]);"),
    "A sign flipped": ("out[4 * p + f] = acc_value(&acc[f]) / c;",
                       "out[4 * p + f] = -acc_value(&acc[f]) / c;"),
    "Jx and Jy exchanged": ("out[4 * p + f] = acc_value(&acc[f]) / c;",
                            "out[4 * p + f] = acc_value(&acc[f == 1 ? 2 : (f == 2 ? 1 : f)]) / c;"),
    "distance uses source spacing for target": ("double rx = origin[3 * target + 0] + h[target] * ix;",
                                                "double rx = origin[3 * target + 0] + 1.01 * h[target] * ix;"),
    "clamp ignored": ("        idx = 0;\n", "        idx = 1;\n"),
}

PINS = [pins.test_cube_average_constant, pins.test_static_limit_matches_gaussian_potential,
        pins.test_self_cell_error_constant, pins.test_breathing_monopole_retarded_phase,
        pins.test_lorenz_gauge_condition, pins.test_eq12_delta_s_form_on_4cubed,
        pins.test_reciprocity_equal_spacing, pins.test_linearity_and_time_shift,
        pins.test_constant_source_equals_static_limit, pins.test_history_window_and_clamp]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    assert SRC.count(old) >= 1, f"mutation site for '{name}' not found"
    src = tmp_path / "mutant.c"
    src.write_text(SRC.replace(old, new, 1))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                    str(src), "-o", str(lib), "-lm"], check=True)
    monkeypatch.setattr(oracle, "_lib", oracle._bind(str(lib)))
    failed = []
    for pin in PINS:
        try:
            pin()
        except (AssertionError, oracle.OracleError):
            failed.append(pin.__name__)
    assert failed, f"mutant '{name}' passed every pin"
