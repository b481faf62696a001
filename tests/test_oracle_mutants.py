"""Plant plausible slips in a copy of the oracle and check the pins catch them.

Each mutant is a textual edit of oracle/tvlp_oracle.c compiled into a
temporary directory (the real oracle is untouched).  The pins of
test_oracle_pins.py are then run against the mutant library; every mutant
must make at least one pin fail.  Mutations keep every array index in
bounds so a mutant can only compute a wrong value, never crash.
"""
from __future__ import annotations

import os
import subprocess

import pytest

import oracle as O
from tests import test_oracle_coeff_pins as C
from tests import test_oracle_framewise_pins as FW
from tests import test_oracle_pins as P

SRC = open(os.path.join(os.path.dirname(O.__file__), "tvlp_oracle.c")).read()

MUTANTS = {
    "forward drops the order-M term":
        ("for (int i = 1; i <= M; ++i)\n            acc -= a[t * M + (i - 1)] * past_output",
         "for (int i = 1; i < M; ++i)\n            acc -= a[t * M + (i - 1)] * past_output"),
    "forward sign flipped":
        ("acc -= a[t * M + (i - 1)] * past_output", "acc += a[t * M + (i - 1)] * past_output"),
    "forward coefficient order reversed":
        ("acc -= a[t * M + (i - 1)] * past_output", "acc -= a[t * M + (M - i)] * past_output"),
    "initial state read one lag late":
        ("return zi ? zi[(i - t) - 1] : 0.0;", "return zi ? zi[(i - t) > 1 ? (i - t) - 2 : 0] : 0.0;"),
    "initial state ignored":
        ("return zi ? zi[(i - t) - 1] : 0.0;", "return 0.0;"),
    "adjoint without the lag shift":
        ("double a_hat = a[(t + i) * M + (i - 1)];", "double a_hat = a[t * M + (i - 1)];"),
    "adjoint shifted by one sample too few":
        ("double a_hat = a[(t + i) * M + (i - 1)];", "double a_hat = a[(t + i - 1) * M + (i - 1)];"),
    "adjoint drops the last lag":
        ("if (t + i < T) {", "if (t + i < T && i < M) {"),
    "adjoint sign flipped":
        ("acc -= a_hat * ge[t + i];", "acc += a_hat * ge[t + i];"),
    "coefficient gradient sign flipped":
        ("= -ge[t] * past_output(s, zi, t, i);", "= ge[t] * past_output(s, zi, t, i);"),
    "coefficient gradient lag off by one":
        ("= -ge[t] * past_output(s, zi, t, i);", "= -ge[t] * past_output(s, zi, t, i - 1);"),
    "initial-state gradient uses the unshifted coefficient":
        ("acc -= ge[t] * a[t * M + (t + j - 1)];", "acc -= ge[t] * a[t * M + (j - 1)];"),
    "initial-state gradient stops one sample early":
        ("t <= (int64_t)(M - j) && t < T", "t < (int64_t)(M - j) && t < T"),
    # coefficient preparation (Sec. 4.3) and its adjoint
    "step-up pairs a coefficient with itself":
        ("A[m][i] = A[m - 1][i] + km[m] * A[m - 1][m - i];", "A[m][i] = A[m - 1][i] + km[m] * A[m - 1][i];"),
    "step-up sign flipped":
        ("A[m][i] = A[m - 1][i] + km[m] * A[m - 1][m - i];", "A[m][i] = A[m - 1][i] - km[m] * A[m - 1][m - i];"),
    "step-up drops the new reflection coefficient":
        ("        A[m][m] = km[m];", "        A[m][m] = (m < M) ? km[m] : 0.0;"),
    "interpolation weights swapped":
        ("return (1.0 - w) * k[f * M + (m - 1)] + w * k[(f + 1) * M + (m - 1)];",
         "return w * k[f * M + (m - 1)] + (1.0 - w) * k[(f + 1) * M + (m - 1)];"),
    "interpolation anchored one frame late":
        ("return (1.0 - w) * k[f * M + (m - 1)] + w * k[(f + 1) * M + (m - 1)];",
         "return k[(f + 1) * M + (m - 1)];"),
    "adjoint of the step-up drops the direct term":
        ("                    if (j == m)\n                        d += A[m - 1][m - i];",
         "                    if (j == m && m < 0)\n                        d += A[m - 1][m - i];"),
    "adjoint of the step-up misses the pairing":
        ("double d = D[m - 1][i][j] + km[m] * D[m - 1][m - i][j];", "double d = D[m - 1][i][j];"),
    "adjoint of the interpolation swaps the weights":
        ("            gk[f * M + (j - 1)] += (1.0 - w) * g;\n            gk[(f + 1) * M + (j - 1)] += w * g;",
         "            gk[f * M + (j - 1)] += w * g;\n            gk[(f + 1) * M + (j - 1)] += (1.0 - w) * g;"),
    # frame-wise overlap-add approximation
    "frame-wise window not scaled to sum to one":
        ("return 0.25 * (1.0 - cos(", "return 0.5 * (1.0 - cos("),
    "frame-wise frames start one hop late":
        ("const int64_t t0 = (f - 3) * hop;\n        for (int64_t n = 0; n < N; ++n) {",
         "const int64_t t0 = (f - 2) * hop;\n        for (int64_t n = 0; n < N; ++n) {"),
    "frame-wise filter drops the order-M term":
        ("                if (n - i >= 0)\n                    acc -= af", "                if (n - i >= 0 && i < M)\n                    acc -= af"),
    "frame-wise adjoint without the window":
        ("ge[t] += ff_window(n, N) * acc;", "ge[t] += acc;"),
    "frame-wise coefficient gradient lag off by one":
        ("g -= gu[n] * y[f * N + (n - i)];", "g -= gu[n] * y[f * N + (n - i + 1)];"),
}

PINS = [
    (P.test_golden_worked_example_exact, {}),
    (P.test_m1_time_varying_product_form, {}),
    (P.test_m2_resonator_closed_form, {}),
    (P.test_partial_fraction_impulse_response, {"M": 6}),
    (P.test_time_invariant_matches_lfilter_with_initial_state, {"M": 4}),
    (P.test_dense_solve_forward_and_adjoint, {"T": 33, "M": 4}),
    (P.test_finite_differences, {"T": 12, "M": 3}),
    (P.test_iir_expansion_eqs_6_to_10, {"T": 9, "M": 3}),
    (P.test_golf_time_invariant_gradients, {"M": 5}),
    (P.test_adjoint_dot_product_identity, {}),
    (P.test_slicing_with_carried_state, {}),
    (C.test_step_up_is_levinson, {"M": 8}),
    (C.test_closed_forms_at_frame_anchors, {}),
    (C.test_midpoint_is_the_step_up_of_the_mean_frame, {}),
    (C.test_stable_reflection_coefficients_give_minimum_phase, {"M": 10}),
    (C.test_adjoint_finite_differences, {"M": 3, "T": 13, "hop": 4}),
    (C.test_adjoint_closed_form_m1, {}),
    (FW.test_zero_coefficients_identity, {}),
    (FW.test_frames_are_lfilter, {"M": 4}),
    (FW.test_m1_impulse_closed_form, {}),
    (FW.test_adjoint_finite_differences, {}),
    (FW.test_adjoint_dot_product_identity, {}),
]


def _build_mutant(tmp_path, name, old, new):
    assert SRC.count(old) >= 1, f"mutation site not found for {name!r}"
    src = tmp_path / "mutant.c"
    src.write_text(SRC.replace(old, new, 1))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", *O.CFLAGS, str(src), "-o", str(so), *O.LDLIBS], check=True)
    return O.load_library(str(so))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path, monkeypatch):
    lib = _build_mutant(tmp_path, name, *MUTANTS[name])
    monkeypatch.setattr(O, "_lib", lib)
    caught = []
    for fn, kw in PINS:
        try:
            fn(**kw)
        except AssertionError:
            caught.append(fn.__name__)
    assert caught, f"no pin detects the mutant {name!r}"


def test_unmutated_copy_passes_all_pins(tmp_path, monkeypatch):
    lib = _build_mutant(tmp_path, "identity", "#include <stddef.h>", "#include <stddef.h>")
    monkeypatch.setattr(O, "_lib", lib)
    for fn, kw in PINS:
        fn(**kw)
