"""Planted mistakes: each pin of ``test_oracle_pins_glue.py`` must fail on a copy of the
oracle with a plausible mistake in the part it pins (no GPU).

Each case rewrites one expression of ``oracle/nrmg_oracle.c`` (the site must occur exactly
once), compiles the copy into a temporary directory, binds it in place of the oracle for the
duration of the check, and expects the check to fail.  Only arithmetic is changed: no mutant
reads or writes outside the arrays the unmodified oracle touches.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
import test_oracle_pins_glue as pins

# (name, original text, planted text, checks that must catch it)
MUTANTS = [
    ("van Albada weights swapped",
     "((b * b + OR_VA_EPS2) * a + (a * a + OR_VA_EPS2) * b)",
     "((a * a + OR_VA_EPS2) * a + (b * b + OR_VA_EPS2) * b)",
     [pins.check_van_albada_defining_properties, pins.check_van_albada_limiter_function]),
    ("van Albada slope not divided by h",
     "((a * a + b * b + 2.0 * OR_VA_EPS2) * h)", "(a * a + b * b + 2.0 * OR_VA_EPS2)",
     [pins.check_van_albada_defining_properties, pins.check_van_albada_is_second_order_on_smooth_data]),
    ("van Albada one-sided difference reversed",
     "double a = q0 - qm, b = qp - q0;", "double a = q0 - qm, b = q0 - qp;",
     [pins.check_van_albada_defining_properties, pins.check_van_albada_is_second_order_on_smooth_data]),
    ("central slope over h instead of 2h",
     "return (qp - qm) / (2.0 * h);", "return (qp - qm) / h;",
     [pins.check_central_slope_is_exact_on_quadratics, pins.check_van_albada_is_second_order_on_smooth_data]),
    ("face state a full cell width out",
     "f[o] = f[o] + sd * (0.5 * h) * g;", "f[o] = f[o] + sd * h * g;",
     [pins.check_face_states_of_linear_fields, pins.check_face_states_take_the_slope_along_their_axis]),
    ("face state params without the slope",
     "p[q] = p[q] + sd * (0.5 * h) * g;", "p[q] = p[q] + 0.0 * sd * (0.5 * h) * g;",
     [pins.check_face_states_of_linear_fields]),
    ("x-axis slope taken from the y neighbours",
     "int cm = ax == 0 ? c - 1 : c - L->nx;", "int cm = ax == 0 ? c - L->nx : c - 1;",
     [pins.check_face_states_of_linear_fields, pins.check_face_states_take_the_slope_along_their_axis]),
    ("HLL diffusion term with the wrong sign",
     "sL * sR * (ap[o] - am[o])", "sL * sR * (am[o] - ap[o])",
     [pins.check_hll_rusanov_special_case, pins.check_hll_intermediate_state_form]),
    ("HLL speeds swapped in the central term",
     "(sR * xm[o] - sL * xp[o]", "(sL * xm[o] - sR * xp[o]",
     [pins.check_hll_rusanov_special_case, pins.check_hll_intermediate_state_form]),
    ("HLL left speed with theta instead of its root",
     "double sL = fmin(pm[ax] - C * sqrt(pm[3]), pp[ax] - C * sqrt(pp[3]));",
     "double sL = fmin(pm[ax] - C * pm[3], pp[ax] - C * pp[3]);",
     [pins.check_hll_rusanov_special_case, pins.check_hll_intermediate_state_form]),
    ("defect R - r instead of r - R",
     "Lf->D[(size_t)(j * Lf->nx + i) * S->n + o] = -R[o];", "Lf->D[(size_t)(j * Lf->nx + i) * S->n + o] = R[o];",
     [pins.check_fas_restriction_and_coarse_rhs]),
    ("coarse right-hand side R_H - R_bar_H",
     "Lc->rF[q] = Lc->D[q] + Lc->rF[q];", "Lc->rF[q] = Lc->D[q] - Lc->rF[q];",
     [pins.check_fas_restriction_and_coarse_rhs]),
    ("state restricted in place of the defect",
     "RH[o] += wq[q] * tr[o];", "RH[o] += wq[q] * tf[o];",
     [pins.check_fas_restriction_and_coarse_rhs, pins.check_fas_leaves_a_solved_fine_state_unchanged]),
    ("restricted defect summed, not averaged",
     "RH[o] *= mean;", "RH[o] *= 1.0;",
     [pins.check_fas_restriction_and_coarse_rhs]),
    ("coarse temperature from the energy with a wrong factor",
     "pH[3] = (en - rho * (pH[0] * pH[0] + pH[1] * pH[1] + pH[2] * pH[2])) / (3.0 * rho);",
     "pH[3] = (en - rho * (pH[0] * pH[0] + pH[1] * pH[1] + pH[2] * pH[2])) / (2.0 * rho);",
     [pins.check_fas_restriction_and_coarse_rhs]),
    ("coarse-grid update with the coarse terms' signs swapped",
     "g[o] = (fc[o] - tb[o]) + tt[o];", "g[o] = (fc[o] + tb[o]) - tt[o];",
     [pins.check_fas_update_carries_the_coarse_change]),
    ("restricted state re-expanded from the solution's basis",
     "or_transform(S->c.M, Lc->bP + 4 * C, pc, Lc->bF + (size_t)C * n, tb);",
     "or_transform(S->c.M, Lc->P + 4 * C, pc, Lc->bF + (size_t)C * n, tb);",
     [pins.check_fas_update_carries_the_coarse_change]),
    ("coarse solution taken without the fine state",
     "g[o] = (fc[o] - tb[o]) + tt[o];", "g[o] = tt[o];",
     [pins.check_fas_update_carries_the_coarse_change, pins.check_fas_leaves_a_solved_fine_state_unchanged]),
]


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("oracle_mutants")


def build_mutant(directory, k, old, new):
    with open(oracle._SRC) as f:
        src = f.read()
    assert src.count(old) == 1, f"planting site not found exactly once: {old!r}"
    path = os.path.join(directory, f"mutant{k}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(directory, f"libmutant{k}.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-o", so, path, "-lm"])
    return oracle.bind(ctypes.CDLL(so))


def test_every_check_passes_on_the_oracle():
    for check in pins.CHECKS:
        check()


@pytest.mark.parametrize("k", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(k, mutant_dir, monkeypatch):
    name, old, new, checks = MUTANTS[k]
    lib = build_mutant(str(mutant_dir), k, old, new)
    oracle.lib()  # the real library is built before it is swapped out
    monkeypatch.setattr(oracle, "_lib", lib)
    for check in checks:
        with pytest.raises(AssertionError):
            check()
