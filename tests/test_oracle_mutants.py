"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/farm_oracle.c (on the CPU),
compiles it, and runs the pin suites (test_oracle_pins.py,
test_oracle_pins_more.py, test_oracle_pins_mc.py, test_oracle_pins_between.py,
test_oracle_pins_assoc.py) against it in a subprocess: they must fail.  A pin set that passes a planted mistake is not pinning that part.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "farm_oracle.c")

MUTANTS = {
    "above_sign": ("return orc_sigmoid(dz / p->tau_v);", "return orc_sigmoid(-dz / p->tau_v);"),
    "near_width": ("exp(-d2 / (2.0 * p->sigma_near * p->sigma_near))", "exp(-d2 / (p->sigma_near * p->sigma_near))"),
    "left_right_sign": ("acc += orc_sigmoid(sign * (ua - ue) / p->tau_h);",
                        "acc += orc_sigmoid(sign * (ue - ua) / p->tau_h);"),
    "view_validity_or": ("if (!(Ze > p->z_min && Za > p->z_min)) continue;",
                         "if (!(Ze > p->z_min || Za > p->z_min)) continue;"),
    "rank_tie_reversed": ("    return a < b;\n}", "    return a > b;\n}"),
    "rank_off_by_one": ("ssem[j] = class_factor(s, p, c_t, j) / (p->mu + (double)rank[j]);",
                        "ssem[j] = class_factor(s, p, c_t, j) / (p->mu + (double)rank[j] - 1.0);"),
    "class_factor_inverted": ("return (c_t >= 0 && s->cls[j] != c_t) ? p->class_mis : 1.0;",
                              "return (c_t >= 0 && s->cls[j] == c_t) ? p->class_mis : 1.0;"),
    "next_to_width": ("exp(-dist2(s, e, a) / (2.0 * p->sigma_next * p->sigma_next))",
                      "exp(-dist2(s, e, a) / (2.0 * p->sigma_near * p->sigma_near))"),
    "on_gap_from_centres": ("double gap = (center(s, 2, e) - 0.5 * box_size(s, 2, e)) - (center(s, 2, a) + 0.5 * box_size(s, 2, a));",
                            "double gap = center(s, 2, e) - center(s, 2, a);"),
    "front_depth_sign": ("acc += orc_sigmoid(sign * (Za - Ze) / p->tau_d);",
                         "acc += orc_sigmoid(sign * (Ze - Za) / p->tau_d);"),
    "closest_tie_reversed": ("if (dj < de || (dj == de && j < e)) closer += 1;",
                             "if (dj < de || (dj == de && j > e)) closer += 1;"),
    "farthest_counts_anchor": ("        if (j == a) continue;\n        members += 1;\n        double dj",
                               "        members += 1;\n        double dj"),
    "landmark_may_be_target": ("                if (a == e) continue;\n                double r = orc_relation_in(s, p, preds[i], e, a, cset, n_cset);\n                if (arg < 0",
                               "                double r = orc_relation_in(s, p, preds[i], e, a, cset, n_cset);\n                if (arg < 0"),
    "product_not_geometric_mean": ("gbar = zero ? 0.0 : exp(lsum / (double)m);", "gbar = zero ? 0.0 : exp(lsum);"),
    "hellinger_variance_not_box_moment": ("bc *= sqrt(2.0 * se * sa / q) * exp(-3.0 * d * d / q);",
                                          "bc *= sqrt(2.0 * se * sa / q) * exp(-d * d / q);"),
    "hellinger_det_factor_dropped": ("bc *= sqrt(2.0 * se * sa / q) * exp(-3.0 * d * d / q);",
                                     "bc *= exp(-3.0 * d * d / q);"),
    "inside_divides_by_anchor": ("frac *= ov / (2.0 * he);", "frac *= ov / (2.0 * ha);"),
    "fusion_weight_dropped": ("for (int64_t j = 0; j < s->n; ++j) F[j] += ch_w[c] / (p->mu + (double)rank[j]);",
                              "for (int64_t j = 0; j < s->n; ++j) F[j] += 1.0 / (p->mu + (double)rank[j]);"),
    "fusion_class_factor_dropped": ("for (int64_t j = 0; j < n; ++j) ssem[j] = class_factor(s, p, c_t, j) * F[j];",
                                    "for (int64_t j = 0; j < n; ++j) ssem[j] = F[j];"),
    "fusion_landmarks_from_target": ("        if ((rc = fused_scores(s, spaces, n_spaces, p, n_ch, ch_space, ch_w, emb, Fl, cos, rank)) != ORC_OK)\n            goto out;\n        sort_by_value(n, Fl, order, tmp);",
                                     "        if ((rc = fused_scores(s, spaces, n_spaces, p, n_ch, ch_space, ch_w, emb, Fl, cos, rank)) != ORC_OK)\n            goto out;\n        sort_by_value(n, F, order, tmp);"),
    "between_off_line_term_dropped": ("return orc_sigmoid(t / tau_b) * orc_sigmoid((1.0 - t) / tau_b) * exp(-0.5 * d2 / (sg * sg));",
                                      "return orc_sigmoid(t / tau_b) * orc_sigmoid((1.0 - t) / tau_b) + 0.0 * sg;"),
    "between_pair_counted_twice": ("if (preds[i] != ORC_BETWEEN_AND) f[k++] = t[i];", "f[k++] = t[i];"),
    "between_same_landmark_twice": ("            if (aq == e || aq == ap) continue;\n            double r = orc_between(s, p, e, ap, aq);\n            if (bp < 0",
                                    "            if (aq == e) continue;\n            double r = orc_between(s, p, e, ap, aq);\n            if (bp < 0"),
    "assoc_winner_lightest": ("if (win[r] < 0 || ent_w[e] > ent_w[win[r]]", "if (win[r] < 0 || ent_w[e] < ent_w[win[r]]"),
    "assoc_spread_dropped": ("w * (CV(t, k) + dm[ix[k][0]] * dm[ix[k][1]]);", "w * (CV(t, k) + 0.0 * dm[ix[k][0]]);"),
    "assoc_hellinger_exponent": ("* exp(-q / 8.0);", "* exp(-q / 4.0);"),
    "full_product_not_blend": ("return s_sem * ((1.0 - p->w) + p->w * gbar);", "return s_sem * gbar;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(lib), str(mutant), "-lm"],
                   check=True)
    env = dict(os.environ, FARM_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_pins_more.py"),
                        os.path.join(ROOT, "tests", "test_oracle_pins_mc.py"),
                        os.path.join(ROOT, "tests", "test_oracle_pins_between.py"),
                        os.path.join(ROOT, "tests", "test_oracle_pins_assoc.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins pass with mutant {name}:\n{r.stdout[-2000:]}"
