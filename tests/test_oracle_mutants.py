"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that the pins
catch each one.  This is what makes the pins evidence: a dropped term, a wrong sign, a
wrong index or exponent anywhere in the oracle must fail at least one of them.
"""
import os

import pytest

import oracle
import tests.test_oracle_pins as pins

# (name, text in pp_oracle.c, replacement, occurrence index or None for all)
MUTANTS = [
    ("dx operands swapped", "double dx = pos[3 * i + 0] - pos[3 * j + 0];",
     "double dx = pos[3 * j + 0] - pos[3 * i + 0];", 0),
    ("softening dropped in field", "double s = dx * dx + dy * dy + dz * dz + eps2;\n            if (s == 0.0) continue;\n            double inv3",
     "double s = dx * dx + dy * dy + dz * dz;\n            if (s == 0.0) continue;\n            double inv3", 0),
    ("inverse-square exponent wrong", "double inv3 = 1.0 / (s * sqrt(s));", "double inv3 = 1.0 / s;", 0),
    ("source weight index i", "double Qj = qe * w[j];", "double Qj = qe * w[i];", 0),
    ("charge sign", "const double qe = -OR_E;", "const double qe = OR_E;", 0),
    ("accel sign", "const double qm = -OR_E / OR_ME;", "const double qm = OR_E / OR_ME;", 0),
    ("drift half missing", "const double half_dt2 = dt * dt / 2.0;", "const double half_dt2 = dt * dt;", 0),
    ("kick uses new accel only", "vel[i] = vel[i] + (acc[i] + scratch[i]) * half_dt;",
     "vel[i] = vel[i] + scratch[i] * dt;", 0),
    ("accel not carried", "            acc[i] = scratch[i];\n", "", 0),
    ("potential double counted", "return 0.5 * k * OR_E * OR_E * total;", "return k * OR_E * OR_E * total;", 0),
    ("potential self pair", "            if (j == i) continue;\n            double dx = pos[3 * i + 0] - pos[3 * j + 0];\n            double dy = pos[3 * i + 1] - pos[3 * j + 1];\n            double dz = pos[3 * i + 2] - pos[3 * j + 2];\n            double s = dx * dx + dy * dy + dz * dz + eps2;\n            if (s == 0.0) continue;\n            acc +=",
     "            double dx = pos[3 * i + 0] - pos[3 * j + 0];\n            double dy = pos[3 * i + 1] - pos[3 * j + 1];\n            double dz = pos[3 * i + 2] - pos[3 * j + 2];\n            double s = dx * dx + dy * dy + dz * dz + eps2;\n            if (s == 0.0) continue;\n            acc +=", 0),
    ("kinetic energy half missing", "ke += 0.5 * m * (vx * vx + vy * vy + vz * vz);", "ke += m * (vx * vx + vy * vy + vz * vz);", 0),
    ("rms radius uncentred", "double dx = pos[3 * i + 0] - cx;", "double dx = pos[3 * i + 0];", 0),
    ("emittance centred", "double x = pos[3 * i + 0];", "double x = pos[3 * i + 0] - cx;", 0),
    ("emittance cross term dropped", "double e2 = mx2 * mvx2 - mxvx * mxvx;", "double e2 = mx2 * mvx2;", 0),
    ("momentum without weight", "px += m * vx;", "px += OR_ME * vx;", 0),
    ("last source skipped", "for (int64_t j = 0; j < N; ++j) {\n            if (j == i) continue;\n            double dx",
     "for (int64_t j = 0; j < N - 1; ++j) {\n            if (j == i) continue;\n            double dx", 0),
    ("z separation from the source's y", "double dz = pos[3 * i + 2] - pos[3 * j + 2];",
     "double dz = pos[3 * i + 2] - pos[3 * j + 1];", 0),
    ("softening not squared", "const double eps2 = eps * eps;", "const double eps2 = eps;", 0),
]

PIN_CALLS = [
    (pins.test_brute_force_exact_fields_small_n, {"n": 17, "eps_frac": 0.0}),
    (pins.test_brute_force_exact_fields_small_n, {"n": 64, "eps_frac": 0.3}),
    (pins.test_two_body_acceleration_closed_form, {"eps": 0.0}),
    (pins.test_two_body_acceleration_closed_form, {"eps": 0.3e-6}),
    (pins.test_ring_on_axis_field, {}),
    (pins.test_regular_tetrahedron, {}),
    (pins.test_third_law_net_force_vanishes, {}),
    (pins.test_translation_rotation_scaling_linearity, {}),
    (pins.test_potential_energy_closed_forms, {}),
    (pins.test_diagnostics_hand_values, {}),
    (pins.test_two_electron_separation_second_order, {}),
    (pins.test_two_electron_energy_and_momentum, {}),
]


def _replace_nth(text, old, new, nth):
    pos = -1
    for _ in range(nth + 1):
        pos = text.find(old, pos + 1)
        if pos < 0:
            raise AssertionError(f"mutation anchor not found: {old!r}")
    return text[:pos] + new + text[pos + len(old):]


@pytest.mark.parametrize("name,old,new,nth", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new, nth):
    src = _replace_nth(oracle.source_text(), old, new, nth)
    lib = oracle.compile_variant(src, os.path.join(str(tmp_path), "mutant.so"))
    caught = []
    with oracle.use_library(lib):
        for fn, kw in PIN_CALLS:
            try:
                fn(**kw)
            except AssertionError:
                caught.append(fn.__name__)
    assert caught, f"no pin caught the planted mistake: {name}"


def test_unmutated_oracle_passes_the_same_pins():
    for fn, kw in PIN_CALLS:
        fn(**kw)
