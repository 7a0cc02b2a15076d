"""Planted mistakes in a copy of the oracle must each break at least one pin.

Each mutant is a one-token change of ``oracle/fcm_oracle.c`` of the kind a
reader could miss (a dropped term, a wrong sign, index or exponent, a
transposed operand, a loose comparison). The copy is compiled into a temporary
directory on the CPU; the real oracle is never touched.
"""
import os

import pytest

import oracle
from oracle_pins import ALL_PINS

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "fcm_oracle.c")

MUTANTS = {
    "exponent_1_over_m-1": ("    const double e = 2.0 / (m - 1.0);\n    for (int j = 0; j < C; ++j) {\n        const double dij",
                            "    const double e = 1.0 / (m - 1.0);\n    for (int j = 0; j < C; ++j) {\n        const double dij"),
    "ratio_transposed": ("s += pow(dij / dik, e);", "s += pow(dik / dij, e);"),
    "center_weight_not_powered": ("            const double w = pow(Uj[i], m);\n            num += w * x[i];",
                                  "            const double w = Uj[i];\n            num += w * x[i];"),
    "center_numerator_drops_x": ("num += w * x[i];", "num += w;"),
    "objective_not_powered": ("J += pow(U[(int64_t)j * n + i], m) * d * d;", "J += U[(int64_t)j * n + i] * d * d;"),
    "objective_wrong_sign": ("const double d = x[i] - V[j];", "const double d = x[i] + V[j];"),
    "objective_wrong_index": ("J += pow(U[(int64_t)j * n + i], m) * d * d;", "J += pow(U[(int64_t)j * n], m) * d * d;"),
    "stop_not_strict": ("        if (delta < eps) { status = ORACLE_CONVERGED; break; }\n        if (k == max_iter) break;\n        empty += oracle_centers",
                        "        if (delta <= eps) { status = ORACLE_CONVERGED; break; }\n        if (k == max_iter) break;\n        empty += oracle_centers"),
    "zero_distance_share_not_split": ("u[j] = (xi == V[j]) ? 1.0 / nzero : 0.0;", "u[j] = (xi == V[j]) ? 1.0 : 0.0;"),
    "no_swap_of_previous_U": ("memcpy(V, Vnext, sizeof(double) * C);\n        double* t = Uprev; Uprev = Ucur; Ucur = t;",
                              "memcpy(V, Vnext, sizeof(double) * C);\n        double* t = Ucur; (void)t;"),
    "multi_squared_distance_as_norm": ("dist[j] = sqrt(s);", "dist[j] = s;"),
    "multi_center_ignores_channel": ("for (int d = 0; d < D; ++d) num[d] += w * x[(int64_t)d * n + i];",
                                     "for (int d = 0; d < D; ++d) num[d] += w * x[i];"),
    "delta_without_abs": ("const double d = fabs(a[t] - b[t]);", "const double d = (a[t] - b[t]);"),
    "labels_ties_to_highest": ("if (u > bu) { bu = u; best = j; }", "if (u >= bu) { bu = u; best = j; }"),
    "quantized_drops_count": ("                num += h[b] * w * val[b];\n                den += h[b] * w;\n            }\n            if (den > 0.0) Vnext",
                              "                num += w * val[b];\n                den += h[b] * w;\n            }\n            if (den > 0.0) Vnext"),
    "quantized_first_delta_vs_wrong_pixel": ("fabs(Ub[xq[i] * C + j] - init[(int64_t)j * n + i])", "fabs(Ub[xq[i] * C + j] - init[(int64_t)j * n])"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = oracle.build(str(path), str(tmp_path / "libmutant.so"))
    L = oracle.load_library(so)
    caught = []
    for pin in ALL_PINS:
        try:
            fails = pin(L)
        except Exception as e:  # a crash or a rejected run also counts as caught
            fails = [f"{type(e).__name__}: {e}"]
        if fails:
            caught.append(pin.__name__)
            break
    assert caught, f"mutant {name} passed every pin"
