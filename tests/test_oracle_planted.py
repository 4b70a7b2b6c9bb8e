"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins
catch every one of them.

Each mutant is the oracle's C source with one exact substring replaced,
compiled into a temporary library; at least one pin must fail on it.
"""
import os

import pytest

from oracle import oracle as oracle_mod
import pins

SRC = os.path.join(os.path.dirname(oracle_mod.__file__), "panda_oracle.c")

MUTANTS = {
    "tan_drop_abs": ("sqrt(sxx + syy - fabs(sxy))", "sqrt(sxx + syy - sxy)"),
    "tan_wrong_sign": ("sqrt(sxx + syy - fabs(sxy))", "sqrt(sxx + syy + fabs(sxy))"),
    "tan_one_norm_twice": ("sqrt(sxx + syy - fabs(sxy))", "sqrt(sxx + sxx - fabs(sxy))"),
    "w_drop_R": ("alpha / 2.0 * (a + r)", "alpha / 2.0 * (a)"),
    "w_drop_half": ("alpha / 2.0 * (a + r)", "alpha * (a + r)"),
    "w_undamped": ("return (1.0 - alpha) * w +", "return w +"),
    "R_row_of_W": ("oracle_tanimoto(P + i * T, 1, Wt + (long)j * T, 1, T)",
                   "oracle_tanimoto(P + i * T, 1, W + (long)(j % T) * G, 1, T)"),
    "A_uses_old_P_shape": ("oracle_tanimoto(W + i * G, 1, C + (long)j * G, 1, G)",
                           "oracle_tanimoto(W + i * G, 1, C + (long)j * G, 1, G - 1)"),
    "p_from_old_W": ("oracle_p_rows(T, G, Wn, P, alpha, T, idx, Pn, Psim)",
                     "oracle_p_rows(T, G, W, P, alpha, T, idx, Pn, Psim)"),
    "c_from_old_W": ("int rc = oracle_c_rows(T, G, Wn, C,", "int rc = oracle_c_rows(T, G, W, C,"),
    "eq5_half_alpha": ("return (1.0 - alpha) * old + alpha * s;", "return (1.0 - alpha) * old + alpha / 2.0 * s;"),
    "eq5_no_damping": ("return (1.0 - alpha) * old + alpha * s;", "return old + alpha * s;"),
    "p_from_C_row_old": ("v = oracle_eq5_entry(P[i * T + m], alpha,", "v = oracle_eq5_entry(P[m * T + m], alpha,"),
    "diag_multipliers_swapped": ("diag_update(T, (double)G, Pn, P, Psim", "diag_update(T, (double)T, Pn, P, Psim"),
    "diag_t_off_by_one": ("exp(2.0 * alpha * (double)t)", "exp(2.0 * alpha * (double)(t - 1))"),
    "diag_no_damping_old": ("return (1.0 - alpha) * old + gain * mult * sigma * growth;",
                            "return old + gain * mult * sigma * growth;"),
    "diag_sample_std": ("return sqrt(ss / (double)(n - 1));", "return sqrt(ss / (double)(n > 2 ? n - 2 : 1));"),
    "diag_includes_diagonal": ("    double mean = s / (double)(n - 1);",
                               "    s += X[(long)i * n + i];\n    double mean = s / (double)(n - 1);"),
    "diag_d2_sigma_of_entries": ("const double *src = (rule == ORACLE_DIAG_D2) ? sim : Xn;",
                                 "const double *src = Xn;"),
    "diag_d0_damped_like_d1": ("double gain = (rule == ORACLE_DIAG_D0) ? 1.0 : alpha;", "double gain = alpha;"),
    "h_not_mean": ("*h = s / ((double)T * (double)G);", "*h = s / ((double)T);"),
    "zscore_sample_std": ("double sd = sqrt(ss / (double)n);", "double sd = sqrt(ss / (double)(n - 1));"),
    "stop_not_strict": ("if (h < tol) {", "if (h <= tol) {"),
    "pearson_uncentred": ("s += (x[k] - mean[g]) * (y[k] - mean[h]);", "s += x[k] * y[k];"),
    "pearson_one_norm_twice": ("const double r = s / sqrt(ss[g] * ss[h]);", "const double r = s / ss[g];"),
    "pearson_mean_off_by_one": ("        m /= (double)N;", "        m /= (double)(N - 1);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} must be unique"
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    lib = oracle_mod.compile_library(str(mpath), str(tmp_path / "libmutant.so"))
    orc = oracle_mod.Oracle(oracle_mod.load(lib))
    failed = []
    for pin in pins.PINS:
        try:
            pin(orc)
        except (AssertionError, ValueError):
            failed.append(pin.__name__)
    assert failed, f"no pin caught the planted mistake {name}"
