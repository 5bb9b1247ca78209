"""Plants plausible mistakes in a copy of the oracle's C source (on the CPU)
and checks that the pins of ``test_oracle_pins`` catch every one of them.

Each mutant is a single textual edit of ``oracle/jacobi2d_oracle.c``: a
dropped term, a wrong sign, a wrong neighbour index, a transposed extent, a
wrong weight, an in-place update instead of ping-pong, a written boundary, an
off-by-one step count, and mistakes in the residual / stopping rule.
"""
import os

import pytest

import oracle
from tests.test_oracle_pins import ALL_PINS

SRC = os.path.join(os.path.dirname(oracle.__file__), "jacobi2d_oracle.c")

MUTANTS = {
    "drop_centre": ("double sum = centre + (ns + we);", "double sum = (ns + we);"),
    "sign_east": ("row[j - 1] + row[j + 1]", "row[j - 1] - row[j + 1]"),
    "south_index": ("north[j] + south[j]", "north[j] + south[j + 1]"),
    "west_index": ("row[j - 1] + row[j + 1]", "row[j] + row[j + 1]"),
    "transposed_extent": ("for (i = 1; i < R - 1; ++i) {\n        const double *north",
                          "for (i = 1; i < (C < R ? C : R) - 1; ++i) {\n        const double *north"),
    "weight": ("dst[j] = 0.2 * sum;", "dst[j] = 0.25 * sum;"),
    "in_place": ("        oracle_step(A, B, R, C, nth);\n        tmp = A;",
                 "        oracle_step(A, A, R, C, nth);\n        tmp = A;"),
    "boundary_written": ("for (j = 1; j < C - 1; ++j) {\n            double centre",
                         "for (j = 1; j < C; ++j) {\n            double centre"),
    "off_by_one_T": ("for (t = 1; t <= T; ++t)", "for (t = 1; t < T; ++t)"),
    "residual_squared": ("rel = (r1 > 0.0) ? rt / r1 : 0.0;", "rel = (r1 > 0.0) ? (rt * rt) / (r1 * r1) : 0.0;"),
    "residual_wrong_pair": ("rt = sqrt(oracle_sqdiff(B, A, R, C, rowsum, nth));",
                            "rt = sqrt(oracle_sqdiff(B, B, R, C, rowsum, nth));"),
    "check_phase": ("int is_check = (t % check_stride) == 0;", "int is_check = (t % check_stride) == 1;"),
    "stop_rule": ("if (is_check && tol > 0.0 && rel <= tol)", "if (is_check && tol > 0.0 && rel < tol * tol)"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = src.replace(old, new, 1)
    path = tmp_path / f"mut_{name}.c"
    path.write_text(mutated)
    so = oracle.compile_source(str(path), str(tmp_path / f"libmut_{name}.so"))
    lib = oracle.load_library(so)
    caught = []
    for pin in ALL_PINS:
        try:
            pin(lib)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin caught mutant {name}"


# ---- the Fig. 1 program (oracle_laplace1d) ----------------------------------------
from tests import test_oracle_laplace1d as _l1d  # noqa: E402

LAPLACE_PINS = [_l1d.test_hand_steps, _l1d.test_exact_bruteforce, _l1d.test_eigenvector_closed_form,
                _l1d.test_paper_configuration_runs]

LAPLACE_MUTANTS = {
    "weight_centre": ("src[i] * -2.0", "src[i] * -1.0"),
    "weight_sign": ("src[i - 1] * 1.0 + src[i] * -2.0", "src[i - 1] * 1.0 - src[i] * -2.0"),
    "neighbour_index": ("+ src[i + 1] * 1.0", "+ src[i] * 1.0"),
    "no_ping_pong": ("double *dst = A + ((t + 1) % 2) * N;", "double *dst = A + (t % 2) * N;"),
    "ends_written": ("for (i = 1; i < N - 1; ++i)\n            dst[i]", "for (i = 0; i < N - 1; ++i)\n            dst[i]"),
    "off_by_one_T": ("for (t = 0; t < T; ++t) {\n        const double *src = A + (t % 2) * N;",
                     "for (t = 1; t < T; ++t) {\n        const double *src = A + (t % 2) * N;"),
}


@pytest.mark.parametrize("name", sorted(LAPLACE_MUTANTS))
def test_laplace1d_mutant_is_caught(name, tmp_path):
    old, new = LAPLACE_MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path = tmp_path / f"mut_{name}.c"
    path.write_text(src.replace(old, new, 1))
    lib = oracle.load_library(oracle.compile_source(str(path), str(tmp_path / f"libmut_{name}.so")))
    caught = []
    for pin in LAPLACE_PINS:
        try:
            pin(lib)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin caught mutant {name}"


# ---- the 3-D 7-point oracle (oracle_jacobi3d) --------------------------------------
from tests import test_oracle_jacobi3d as _j3d  # noqa: E402

SRC3D = os.path.join(os.path.dirname(oracle.__file__), "jacobi3d_oracle.c")

JACOBI3D_MUTANTS = {
    "weight": ("static const double ONE_SEVENTH = 1.0 / 7.0;", "static const double ONE_SEVENTH = 1.0 / 6.0;"),
    "drop_planes": ("double sum = centre + ((ns + we) + ud);", "double sum = centre + (ns + we);"),
    "drop_centre": ("double sum = centre + ((ns + we) + ud);", "double sum = (ns + we) + ud;"),
    "plane_stride": ("double ud = row[j - P] + row[j + P];", "double ud = row[j - P] + row[j + C];"),
    "row_index": ("double ns = row[j - C] + row[j + C];", "double ns = row[j - C] + row[j - C];"),
    "sign_west": ("double we = row[j - 1] + row[j + 1];", "double we = row[j + 1] - row[j - 1];"),
    "last_row_skipped": ("for (i = 1; i < R - 1; ++i) {", "for (i = 1; i < R - 2; ++i) {"),
    "in_place": ("        oracle3d_step(A, B, D, R, C, nth);", "        oracle3d_step(A, A, D, R, C, nth);"),
    "off_by_one_T": ("for (t = 1; t <= T; ++t) {", "for (t = 2; t <= T; ++t) {"),
    "shell_written": ("dst[j] = ONE_SEVENTH * sum;", "dst[j] = ONE_SEVENTH * sum;\n                if (j == 1) dst[0] = dst[1];"),
}


@pytest.mark.parametrize("name", sorted(JACOBI3D_MUTANTS))
def test_jacobi3d_mutant_is_caught(name, tmp_path):
    old, new = JACOBI3D_MUTANTS[name]
    src = open(SRC3D).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path = tmp_path / f"mut3d_{name}.c"
    path.write_text(src.replace(old, new, 1))
    lib = oracle.load_library3d(oracle.compile_source(str(path), str(tmp_path / f"libmut3d_{name}.so")))
    caught = []
    for pin in _j3d.ALL_PINS:
        try:
            pin(lib)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin caught mutant {name}"


# ---- the red-black SOR oracle (oracle_sor2d) -------------------------------------------
from tests import test_oracle_sor2d as _sor  # noqa: E402

SRCSOR = os.path.join(os.path.dirname(oracle.__file__), "sor2d_oracle.c")

SOR_MUTANTS = {
    "black_first": ("        sor_colour(out, R, C, 0, a, b);\n        sor_colour(out, R, C, 1, a, b);",
                    "        sor_colour(out, R, C, 1, a, b);\n        sor_colour(out, R, C, 0, a, b);"),
    "colour_parity": ("j = 1 + ((i + 1 + colour) & 1);", "j = 1 + ((i + colour) & 1);"),
    "lexicographic": ("for (; j < C - 1; j += 2) {", "for (j = 1; j < C - 1; j += 1) {"),
    "weight": ("b = 0.25 * omega;", "b = 0.2 * omega;"),
    "relaxation": ("a = 1.0 - omega;", "a = omega - 1.0;"),
    "south_index": ("double q = (north[j] + south[j]) + (row[j - 1] + row[j + 1]);",
                    "double q = (north[j] + south[j + 1]) + (row[j - 1] + row[j + 1]);"),
    "last_row_skipped": ("for (i = 1; i < R - 1; ++i) {", "for (i = 1; i < R - 2; ++i) {"),
    "off_by_one_T": ("for (t = 1; t <= T; ++t) {", "for (t = 2; t <= T; ++t) {"),
}


@pytest.mark.parametrize("name", sorted(SOR_MUTANTS))
def test_sor_mutant_is_caught(name, tmp_path):
    old, new = SOR_MUTANTS[name]
    src = open(SRCSOR).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path = tmp_path / f"mutsor_{name}.c"
    path.write_text(src.replace(old, new, 1))
    lib = oracle.load_library_sor(oracle.compile_source(str(path), str(tmp_path / f"libmutsor_{name}.so")))
    caught = []
    for pin in _sor.ALL_PINS:
        try:
            pin(lib)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin caught mutant {name}"
