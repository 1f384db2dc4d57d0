"""Plant plausible mistakes in a copy of the oracle's C source and check that
the pin suite (test_oracle_pins.py) catches every one of them.

Each mutation is a single textual edit of mpj_oracle.c: a flipped sign, a
transposed rotation, a dropped factor, a wrong index.  The mutated copy is
compiled into a temporary directory and the pins run against it in a child
process; the real oracle is never touched."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "mpj_oracle.c")

MUTATIONS = {
    "tau_sign": ("double tau = (aqq - app) / (2.0 * apq);", "double tau = (app - aqq) / (2.0 * apq);"),
    "t_branch": ("t = 1.0 / (tau + sqrt(1.0 + tau * tau));", "t = 1.0 / (tau - sqrt(1.0 + tau * tau));"),
    "c_formula": ("*c = 1.0 / sqrt(1.0 + t * t);", "*c = 1.0 / sqrt(1.0 + t);"),
    "row_update_sign": ("AT(A, lda, p, k) = c * ap - s * aq;", "AT(A, lda, p, k) = c * ap + s * aq;"),
    "col_update_transposed": ("AT(A, lda, k, p) = c * ap - s * aq;\n    AT(A, lda, k, q) = s * ap + c * aq;",
                              "AT(A, lda, k, p) = c * ap + s * aq;\n    AT(A, lda, k, q) = -s * ap + c * aq;"),
    "v_update_sign": ("AT(V, ldv, k, q) = s * vp + c * vq;", "AT(V, ldv, k, q) = -s * vp + c * vq;"),
    "off_includes_diag": ("if (i != j) s += AT(A, lda, i, j) * AT(A, lda, i, j);", "s += AT(A, lda, i, j) * AT(A, lda, i, j);"),
    "ns_dropped_half": ("AT(X, ldx, i, j) = 0.5 * AT(Y, n, i, j);", "AT(X, ldx, i, j) = AT(Y, n, i, j);"),
    "ns_three_to_two": ("AT(M, n, i, j) = (i == j ? 3.0 : 0.0) - AT(M, n, i, j);", "AT(M, n, i, j) = (i == j ? 2.0 : 0.0) - AT(M, n, i, j);"),
    "gemm_tn_transposed": ("for (int l = 0; l < k; ++l) s += AT(A, lda, l, i) * AT(B, ldb, l, j);",
                           "for (int l = 0; l < k; ++l) s += AT(A, lda, i, l) * AT(B, ldb, l, j);"),
    "rr_pair_offset": ("b = ((r - i) % (m - 1) + (m - 1)) % (m - 1);", "b = ((r - i + 1) % (m - 1) + (m - 1)) % (m - 1);"),
    "skip_rule_inverted": ("if (fabs(apq) > skip_tol * sqrt(fabs(AT(A, lda, p, p) * AT(A, lda, q, q))) && fabs(apq) > skip_abs) {",
                           "if (fabs(apq) < skip_tol * sqrt(fabs(AT(A, lda, p, p) * AT(A, lda, q, q))) && fabs(apq) > skip_abs) {"),
    "threshold_inverted": ("&& fabs(apq) > skip_abs) {", "&& fabs(apq) >= skip_abs * 0.0 + 1e300 * (skip_abs > 0)) {"),
    "backward_gap_sign": ("double gap = W[j] - W[i];", "double gap = W[i] - W[j];"),
    "backward_no_diag": ("g = dW ? dW[i] : 0.0;", "g = 0.0;"),
    "precondition_untransposed": ("orc_gemm_tn_d(n, n, n, Qd, ldq, W, n, Ac, ldc);", "orc_gemm_nn_d(n, n, n, Qd, ldq, W, n, Ac, ldc);"),
    "block_local_map": ("int gy = ly < ORC_BLK ? I * ORC_BLK + ly : J * ORC_BLK + (ly - ORC_BLK);",
                        "int gy = ly < ORC_BLK ? I * ORC_BLK + ly : J * ORC_BLK + ly;"),
    "float_pair_tau": ("float tau = (aqq - app) / (2.0f * apq);", "float tau = (aqq - app) / (apq);"),
    "two_pass_product_order": ("orc_gemm_nn_d(n, n, n, X, n, X2, n, T, n);", "orc_gemm_nn_d(n, n, n, X2, n, X, n, T, n);"),
    "two_pass_transform_on_A": ("orc_precondition_d(n, Ac, n, X2, n, T, n);", "orc_precondition_d(n, A, lda, X2, n, T, n);"),
    "half_not_rounded": ("static float rq(float x, int half) { return half ? orc_round_half(x) : x; }",
                         "static float rq(float x, int half) { return x; }"),
    "half_ns_steps_single": ("if (!half) return n < 52000 ? 2 : 3;", "return n < 52000 ? 2 : 3;"),
    "premise_one_power_step": ("for (int it = 0; it < 200; ++it) {", "for (int it = 0; it < 1; ++it) {"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {name}"
    mutated = src.replace(old, new, 1)
    c = tmp_path / "mut.c"
    so = tmp_path / "libmut.so"
    c.write_text(mutated)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"])
    env = dict(os.environ, MPJ_ORACLE_SO=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(HERE, "test_oracle_pins.py")], cwd=ROOT, env=env,
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutation {name}:\n{r.stdout.decode()[-2000:]}"
