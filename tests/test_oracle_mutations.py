"""Planted mistakes: each mutation below is a plausible slip in the oracle
(a dropped term, a wrong index, a wrong sign or bound).  It is planted in a
temporary copy of the oracle's C source, built on the CPU, and the pins of
test_oracle_pins must reject it.  The committed oracle is never modified."""
import ctypes
import importlib.util
import os
import subprocess

import pytest

import oracle
import tests.test_oracle_alg2 as alg2
import tests.test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "qext_oracle.c")

MUTATIONS = {
    "no_reduction": ("if (pbit(sh, q))", "if (0 && pbit(sh, q))"),
    "bit_reversed_element": ("uint64_t t = base + (uint64_t)i * q + j;",
                             "uint64_t t = base + (uint64_t)i * q + (q - 1 - j);"),
    "dropped_first_term": ("for (int i = 0; i < n_p; ++i) {\n        orc_gf_mul",
                           "for (int i = 1; i < n_p; ++i) {\n        orc_gf_mul"),
    "keeps_high_bits": ("if (pbit(z, j)) {", "if (pbit(z, q - m + j)) {"),
    "trinomial_from_2": ("for (int a = 1; a < q; ++a) {", "for (int a = 2; a < q; ++a) {"),
    "rabin_without_gcd": ("if (pdeg(g, ORC_W2) != 0) return 0;", ";"),
    "nmin_off_by_one": ("while ((double)dmin * gap < 24.0 * (double)n) ++dmin;",
                        "while ((double)dmin * gap <= 24.0 * (double)n) ++dmin;"),
    "eps_sign": ("- (k / 4.0 - (double)n / 8.0)", "+ (k / 4.0 - (double)n / 8.0)"),
    "y_for_x": ("if (sbit(y, t)) pset(ys + (size_t)i * ew", "if (sbit(x, t)) pset(ys + (size_t)i * ew"),
    "alg2_cursor_by_first_block": ("i += (uint64_t)ql * (uint64_t)n_p;", "i += (uint64_t)q1 * (uint64_t)n_p;"),
    "alg2_output_by_first_block": ("o += (uint64_t)ql;", "o += (uint64_t)q1;"),
    "alg2_q_step_once": ("ql += dq;", "ql = q1 + dq;"),
}

# fast pins, each a (function, kwargs) pair from test_oracle_pins
CHECKS = [
    (pins.test_fips197_published_products, {}),
    (pins.test_gf_mul_matches_independent_bigint, {"q": 16}),
    (pins.test_np1_is_field_multiplication, {"q": 16}),
    (pins.test_q1_is_textbook_inner_product, {}),
    (pins.test_bilinear_symmetric_zero, {"q": 16, "n_p": 64}),
    (pins.test_concatenation_and_truncation, {}),
    (pins.test_selected_poly_small_q, {"q": 2}),
    (pins.test_rabin_agrees_with_trial_division, {}),
    (pins.test_plan_rejections_and_exact_ceiling, {}),
    (pins.test_theorem31_constant_chain, {}),
    (pins.test_exact_uniformity, {"q": 2, "n_p": 4}),
    (alg2.test_blocks_are_ext_ip_on_closed_form_windows, {"n_p": 27, "q1": 8, "dq": 8, "nb": 6}),
]


def _mutant(name, tmp_path):
    old, new = MUTATIONS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, name
    src = tmp_path / ("m_%s.c" % name)
    src.write_text(text.replace(old, new))
    so = tmp_path / ("m_%s.so" % name)
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", str(src), "-o", str(so), "-lm"], check=True)
    spec = importlib.util.spec_from_file_location("oracle_mutant_" + name, oracle.__file__)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._lib = mod._configure(ctypes.CDLL(str(so)))
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_reject_planted_mistake(name, tmp_path, monkeypatch):
    mod = _mutant(name, tmp_path)
    monkeypatch.setattr(pins, "oracle", mod)
    monkeypatch.setattr(alg2, "oracle", mod)
    caught = []
    for fn, kw in CHECKS:
        try:
            fn(**kw)
        except Exception as e:  # an assertion or an error raised by the mutant
            caught.append((fn.__name__, type(e).__name__))
    assert caught, "no pin caught mutation %s" % name
