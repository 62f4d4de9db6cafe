"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, a transposed
index, a swapped SIC order) in a temporary copy of the oracle's C source,
builds it, and checks that at least one pin of ``test_oracle_pins`` fails.
Nothing here touches the real oracle build.
"""
import os
import subprocess

import pytest

import oracle.oracle as oo
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oo.__file__), "hcran_oracle.c")
SRC_PEN = os.path.join(os.path.dirname(oo.__file__), "hcran_penalty.c")

PIN_SET = [
    pins.test_psi_worked_example,
    lambda: pins.test_scale_bound_tight_and_below(3.7),
    lambda: pins.test_single_link_ee_matches_lambert_w(2e-14, 10.0),
    pins.test_oma_single_rrh_is_waterfilling_at_fixed_E,
    pins.test_kkt_two_interfering_links,
    pins.test_kkt_noma_pair_same_rrh,
    pins.test_kkt_with_streaming_user,
    lambda: pins.test_kkt_sic_multiplier_across_rrhs(300, 1),
    lambda: pins.test_kkt_sic_multiplier_across_rrhs(1054, 2),
    lambda: pins.test_reported_R_P_match_independent_model("small-3x8x6"),
]

MUTANTS = {
    "sic_split_swapped": ("if (c > 0.0) sp += z * c;\n            else sm += z * (-c);",
                          "if (c < 0.0) sp += z * (-c);\n            else sm += z * c;"),
    "sic_coefficient_transposed": ("double c = gain(I, n, j, ka) / gain(I, n, m, ka) - gain(I, n, j, kb) / gain(I, n, m, kb);",
                                   "double c = gain(I, n, m, ka) / gain(I, n, j, ka) - gain(I, n, m, kb) / gain(I, n, j, kb);"),
    "psi_larger_root": ("double psi_hat = 2.0 * lambda_pps * zbar_bits / (b - root);",
                        "double psi_hat = 2.0 * lambda_pps * zbar_bits / (b + root);"),
    "scale_beta_sign": ("*beta = log2(1.0 + z0) - a * log2(z0);",
                        "*beta = log2(1.0 + z0) + a * log2(z0);"),
    "drop_intra_cell": ("return I->sigma + gain(I, n, m, k) * intra + inter_cell(I, Ptot, n, m, k);",
                        "return I->sigma + inter_cell(I, Ptot, n, m, k);"),
    "sic_order_swapped": ("for (int b = 0; b < s; b++)\n    if (st->S[slot(I, n, m, b)] >= 0) intra += st->p[slot(I, n, m, b)];",
                          "for (int b = s + 1; b < I->l; b++)\n    if (st->S[slot(I, n, m, b)] >= 0) intra += st->p[slot(I, n, m, b)];"),
    "victim_gain_transposed": ("acc += pi[slot(I, n, j, b)] * gain(I, n, m, v);",
                               "acc += pi[slot(I, n, j, b)] * gain(I, n, j, v);"),
    "drop_ee_price": ("double den = q * I->eta[m] + st->xi[m] +\n                     victim_price(I, st, w->pi, n, m, k, -1)",
                      "double den = st->xi[m] +\n                     victim_price(I, st, w->pi, n, m, k, -1)"),
    "streaming_ee_price_dropped": ("double den = q * I->eta[m] + st->xi[m] +\n                     victim_price(I, st, w->pi, n, m, k, -1)",
                                   "double den = (k < I->Ke ? q * I->eta[m] : 0.0) + st->xi[m] +\n                     victim_price(I, st, w->pi, n, m, k, -1)"),
    "zeta_step_sign": ("double x = (I->Psi[ks] - r) / (asum > ZETA_ASUM_MIN ? asum : ZETA_ASUM_MIN);",
                       "double x = (r - I->Psi[ks]) / (asum > ZETA_ASUM_MIN ? asum : ZETA_ASUM_MIN);"),
    "power_omits_streaming": ("if (k < 0) continue;\n        tx += I->eta[m] * st->p[e];\n        if (k >= I->Ke) continue;",
                              "if (k < 0 || k >= I->Ke) continue;\n        tx += I->eta[m] * st->p[e];"),
    "interference_price_alpha_dropped": ("pi[e] = weight_c(I, st, m, k) * st->alpha[e] / (LN2 * ie);",
                                         "pi[e] = weight_c(I, st, m, k) / (LN2 * ie);"),
}


def build_mutant(tmp_path, name, find, repl, target=SRC):
    """The oracle library with one replacement in `target` (the other source
    unchanged)."""
    src = open(target).read()
    assert src.count(find) == 1, name
    path = tmp_path / ("m_%s.c" % name)
    path.write_text(src.replace(find, repl))
    others = [f for f in (SRC, SRC_PEN) if f != target]
    so = str(tmp_path / ("m_%s.so" % name))
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-I", os.path.dirname(SRC), "-o", so, str(path), *others, "-lm"])
    return so


def _build_mutant(tmp_path, name):
    find, repl = MUTANTS[name]
    return build_mutant(tmp_path, name, find, repl)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, monkeypatch, name):
    so = _build_mutant(tmp_path, name)
    monkeypatch.setattr(oo, "_lib", None)
    monkeypatch.setattr(oo, "build", lambda force=False: so)
    failed = []
    for pin in PIN_SET:
        try:
            pin()
        except Exception as exc:  # an assertion or a numerical blow-up both count
            failed.append(repr(exc)[:80])
    assert failed, "no pin caught mutant %s" % name
