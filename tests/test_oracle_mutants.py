"""Plant plausible mistakes in copies of the oracle source and check that the
pins in test_oracle_pins.py catch every one of them (CPU only).

Each mutant is the oracle's C source with one edit, compiled into a temporary
library; the pins then run against it through ``oracle.using_library``.
"""
import os
import tempfile

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "nb_oracle.c")

MUTANTS = {
    "jerk factor 3 -> 2": ("3.0 * rv * R[k] / r5", "2.0 * rv * R[k] / r5"),
    "jerk sign": ("V[k] / r3 - 3.0", "V[k] / r3 + 3.0"),
    "force power r^-2": ("double r3 = r2 * r;", "double r3 = r2;"),
    "R reversed": ("R[k] = x[3 * j + k] - x[3 * i + k];", "R[k] = x[3 * i + k] - x[3 * j + k];"),
    "V reversed": ("V[k] = v[3 * j + k] - v[3 * i + k];", "V[k] = v[3 * i + k] - v[3 * j + k];"),
    "boundary <=": ("return rmin < h_i;", "return rmin <= h_i;"),
    "velocity criterion sign": ("R[k] + (*dtr_i) * V[k]", "R[k] - (*dtr_i) * V[k]"),
    "velocity criterion max": ("if (rp < rmin) rmin = rp;", "if (rp > rmin) rmin = rp;"),
    "predictor a dt^2": ("a0[q] * dt2 / 2.0", "a0[q] * dt2"),
    "predictor adot dt^3/2": ("adot0[q] * dt3 / 6.0", "adot0[q] * dt3 / 2.0"),
    "predictor v adot dt^2": ("adot0[q] * dt2 / 2.0;", "adot0[q] * dt2;"),
    "overflow flag >=": ("ovf[a] = count > cap ? 1 : 0;", "ovf[a] = count >= cap ? 1 : 0;"),
    "mass of i": ("add_term(R, V, m[j], Fi, Ji, pot ? &pi : NULL);\n            }\n        }\n        for",
                  "add_term(R, V, m[i], Fi, Ji, pot ? &pi : NULL);\n            }\n        }\n        for"),
    "potential sign": ("*pot += m_j / r;", "*pot -= m_j / r;"),
}


def _pin_calls():
    calls = [lambda c=c: pins.test_two_body_closed_form(c) for c in range(5)]
    calls += [lambda u=u: pins.test_jerk_is_time_derivative_of_force(u) for u in (False, True)]
    calls += [pins.test_newton_third_law]
    calls += [lambda w=w: pins.test_regular_plus_irregular_is_full(w) for w in (False, True)]
    calls += [lambda n=n, w=w: pins.test_neighbour_sets_brute_force(n, w)
              for n in (7, 33) for w in (False, True)]
    calls += [pins.test_overflow_keeps_lowest_indices, pins.test_power_of_two_scaling_is_exact,
              pins.test_translation_and_boost_invariance_exact, pins.test_relabelling_permutes_lists,
              pins.test_zero_radius_and_empty_inputs, pins.test_potential_matches_two_body,
              pins.test_exact_boundary_pair_is_regular, pins.test_predictor_zero_step_is_identity,
              pins.test_predictor_derivatives_at_start, pins.test_predictor_composes_like_a_cubic,
              pins.test_predictor_is_third_order_on_a_kepler_orbit]
    return calls


def test_pins_pass_on_the_real_oracle():
    for call in _pin_calls():
        call()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert old in src, f"mutation anchor not found: {old!r}"
    with tempfile.TemporaryDirectory() as d:
        msrc = os.path.join(d, "mutant.c")
        open(msrc, "w").write(src.replace(old, new))
        lib = oracle.compile_source(msrc, os.path.join(d, "mutant.so"))
        caught = []
        with oracle.using_library(lib):
            for call in _pin_calls():
                try:
                    call()
                except (AssertionError, oracle.OracleError):
                    caught.append(call)
                    break
        assert caught, f"no pin caught the mutant {name!r}"
