"""The oracle's pins are not vacuous: each case copies oracle/mpdet_oracle.c,
plants one plausible mistake (a rounding rule, a dropped sticky bit, a sign,
an index, an operand), compiles the copy and runs the pins that should catch
it against that build in a fresh process (MPDET_ORACLE_LIB).  Every run must
fail, while the same pins pass on the real oracle in the main suite."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "mpdet_oracle.c")

# (name, exact text in the oracle, planted replacement, pins that must fail)
MUTATIONS = [
    ("rounding ties away from zero", "if (rbit && (st || (om[0] & 1u))) {", "if (rbit) {",
     ["test_oracle_ops.py::test_mul_ties_to_even"]),
    ("truncation instead of rounding", "if (rbit && (st || (om[0] & 1u))) {", "if (0) {",
     ["test_oracle_ops.py::test_mul_random_and_specials"]),
    ("reciprocal drops the remainder's sticky bit",
     "rnd(q, L, -(int64_t)p - ea, rem_nz, p, n, sa & 1, os, oe, om);",
     "rnd(q, L, -(int64_t)p - ea, 0, p, n, sa & 1, os, oe, om);", ["test_oracle_ops.py::test_recip"]),
    ("subtraction adds", "  if (sA == sB) addn(X, Y, L);", "  if (1) addn(X, Y, L);",
     ["test_oracle_ops.py::test_addsub_exponent_gaps"]),
    ("far-operand shortcut one bit too early", "if (d >= (int64_t)p + 2) {", "if (d >= (int64_t)p + 1) {",
     ["test_oracle_ops.py::test_addsub_power_of_two_far_operand"]),
    ("L bookkeeping keeps z's sign", "int8_t s = iszero(ze) ? 0 : (int8_t)(zs ^ 1);",
     "int8_t s = iszero(ze) ? 0 : (int8_t)zs;", ["test_oracle_ge.py::test_lastcol_integer_cofactors_and_laplace"]),
    ("update reads the next row as pivot row", "int64_t ij = i * N + j, kj = k * N + j;",
     "int64_t ij = i * N + j, kj = (k + 1) * N + j;", ["test_oracle_ge.py::test_integer_minors_vs_exact"]),
    ("Cauchy entries from x - y", "op_add(c, xs, xe, xm, ys, ye, ym, 0, ts, te, tm);",
     "op_add(c, xs, xe, xm, ys, ye, ym, 1, ts, te, tm);", ["test_oracle_ops.py::test_cauchy_entries"]),
    ("back substitution adds the update",
     "op_add(&c, u->S[ic], u->E[ic], u->M + ic * n, ts, te, t, 1, u->S + ic, u->E + ic, u->M + ic * n);",
     "op_add(&c, u->S[ic], u->E[ic], u->M + ic * n, ts, te, t, 0, u->S + ic, u->E + ic, u->M + ic * n);",
     ["test_oracle_adjoint.py::test_usolve_is_the_inverse"]),
    ("binary64 rounding ties away from zero", "if (rbit && (st || (K & 1))) K += 1;", "if (rbit) K += 1;",
     ["test_oracle_adjoint.py::test_to_f64_is_correctly_rounded"]),
    ("binary64 rounding without subnormals", "int64_t q = (e - 53 < -1074) ? -1074 : e - 53;",
     "int64_t q = e - 53;", ["test_oracle_adjoint.py::test_to_f64_is_correctly_rounded"]),
    ("normalised minors divide by l_N2", "st = op_recip(&c, S[row], E[row], M + row * n, &rs, &re, r);",
     "st = op_recip(&c, S[row + 1], E[row + 1], M + (row + 1) * n, &rs, &re, r);",
     ["test_oracle_ge.py::test_lastcol_integer_cofactors_and_laplace"]),
    ("back substitution runs k upwards", "for (int64_t k = N - 1; k >= 0 && st == OR_OK; --k) {",
     "for (int64_t k = 0; k < N && st == OR_OK; ++k) {",
     ["test_oracle_adjoint.py::test_usolve_brute_force_op_sequence"]),
    ("back substitution divides instead of multiplying by the reciprocal",
     "op_mul(&c, XS[kc], XE[kc], XM + kc * n, rs, re, r, XS + kc, XE + kc, XM + kc * n);",
     "op_div(&c, XS[kc], XE[kc], XM + kc * n, S[kk], E[kk], M + kk * n, XS + kc, XE + kc, XM + kc * n);",
     ["test_oracle_adjoint.py::test_usolve_brute_force_op_sequence"]),
    ("ball subtraction forgets its own rounding error",
     "static rad_t ball_sub(int p, int64_t eu, rad_t rx, rad_t rt) { return rad_add(rad_add(rad_hu(eu, p), rx), rt); }",
     "static rad_t ball_sub(int p, int64_t eu, rad_t rx, rad_t rt) { return rad_add(rx, rt); }",
     ["test_oracle_ball.py::test_ball_brute_force_radius_sequence"]),
    ("ball product drops the radius-times-radius term", "  return rad_add(r, rad_mul(rx, ry, 1));\n}",
     "  return r;\n}", ["test_oracle_ball.py::test_ball_brute_force_radius_sequence"]),
    ("ball product bounds |x| from below", "rad_t r = rad_add(rad_hu(eu, p), rad_mul(rad_mag(ex, mx, n, 1), ry, 1));",
     "rad_t r = rad_add(rad_hu(eu, p), rad_mul(rad_mag(ex, mx, n, 0), ry, 1));",
     ["test_oracle_ball.py::test_ball_brute_force_radius_sequence"]),
    ("radius sum rounds down", "  return rad_from64(A + rad_align_up(b, a.e - b.e), a.e - 63, 1);",
     "  return rad_from64(A + rad_align_up(b, a.e - b.e), a.e - 63, 0);",
     ["test_oracle_ball.py::test_radius_arithmetic_rounds_as_defined"]),
]


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, pins):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for '{name}' not found once in the oracle"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", str(lib), str(mut), "-lm"])
    env = dict(os.environ, MPDET_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        *[os.path.join(HERE, t) for t in pins]], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, f"planted mistake '{name}' passed the pins {pins}:\n{r.stdout[-2000:]}"
    assert "passed" not in r.stdout.splitlines()[-1] or "failed" in r.stdout.splitlines()[-1], r.stdout[-500:]
