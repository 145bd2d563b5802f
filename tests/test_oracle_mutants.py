"""Plant plausible mistakes in copies of the oracle source (on the CPU) and
check that some pin catches each one."""
import pytest

import oracle
import oracle_pins

# (name, text in qwlsh_oracle.c, replacement, pins expected to catch it)
MUTANTS = [
    ("hash_drops_offset", "double u = (t[i] + (double)b[i]) / (double)w;",
     "double u = (t[i]) / (double)w;", ["pin_hash_exact_sum"]),
    ("hash_truncates", "double u = (t[i] + (double)b[i]) / (double)w;\n            double f = floor(u);",
     "double u = (t[i] + (double)b[i]) / (double)w;\n            double f = trunc(u);",
     ["pin_hash_exact_sum"]),
    ("level_floor_division_truncates", "if ((a % R != 0) && (a < 0)) q -= 1;", "",
     ["pin_collision_counts", "pin_t3_fixpoint", "pin_workload_semantics",
      "pin_hand_worked_golden"]),
    ("threshold_strict", "for (int64_t j = 0; j < n; ++j) if (col[j] >= l) ncand += 1;",
     "for (int64_t j = 0; j < n; ++j) if (col[j] > l) ncand += 1;",
     ["pin_workload_semantics", "pin_v_ge_n_exact", "pin_hand_worked_golden"]),
    ("truncation_fewest_collisions_first", "if (a->col != b->col) return a->col > b->col ? -1 : 1;",
     "if (a->col != b->col) return a->col < b->col ? -1 : 1;",
     ["pin_workload_semantics", "pin_hand_worked_golden"]),
    ("truncation_ignores_previous_level",
     "truncated to k + v */\n        int64_t nc = 0;\n        for (int64_t j = 0; j < n; ++j) {\n            if (col[j] >= l) {\n                cs[nc].prev = prev[j];",
     "truncated to k + v */\n        int64_t nc = 0;\n        for (int64_t j = 0; j < n; ++j) {\n            if (col[j] >= l) {\n                cs[nc].prev = 0;",
     ["pin_workload_semantics", "pin_hand_worked_golden"]),
    ("truncation_larger_id_first",
     "if (a->col != b->col) return a->col > b->col ? -1 : 1;\n    if (a->id != b->id) return a->id < b->id ? -1 : 1;",
     "if (a->col != b->col) return a->col > b->col ? -1 : 1;\n    if (a->id != b->id) return a->id > b->id ? -1 : 1;",
     ["pin_hand_worked_golden"]),
    ("stop_rule_strict", "if (ncand >= cap) { term = 2; break; }\n            if (R > top)",
     "if (ncand > cap) { term = 2; break; }\n            if (R > top)", ["pin_hand_worked_golden"]),
    ("probes_ignored", "lo[i] = (beta - probes) * R;", "lo[i] = beta * R;",
     ["pin_hand_worked_golden", "pin_multi_probe_semantics"]),
    ("probes_radius_rule_ignores_negative_ids", "if (probes > 0 && -g > top) top = -g;", "",
     ["pin_multi_probe_semantics"]),
    ("radius_grows_additively", "if (R > top) { term = 3; break; }\n            nprev = ncand;\n            for (int64_t j = 0; j < n; ++j) prev[j] = (char)(col[j] >= l);\n            R *= c;",
     "if (R > top) { term = 3; break; }\n            nprev = ncand;\n            for (int64_t j = 0; j < n; ++j) prev[j] = (char)(col[j] >= l);\n            R += 1;",
     ["pin_workload_semantics", "pin_hand_worked_golden"]),
    ("distance_not_squared", "s = s + diff * diff;", "s = s + fabs(diff);",
     ["pin_bruteforce", "pin_v_ge_n_exact"]),
    ("ties_by_larger_id",
     "if (a->dist != b->dist) return a->dist < b->dist ? -1 : 1;\n    if (a->id != b->id) return a->id < b->id ? -1 : 1;",
     "if (a->dist != b->dist) return a->dist < b->dist ? -1 : 1;\n    if (a->id != b->id) return a->id > b->id ? -1 : 1;",
     ["pin_duplicates_tie_by_id", "pin_hand_worked_golden"]),
    ("index_not_anchored", "p[j].bid = H[(size_t)j * m + i] - o[i];", "p[j].bid = H[(size_t)j * m + i];",
     ["pin_index_sorted_arrays"]),
    ("eq1_tail_sign", "return 1.0 - two_phi_neg - tail;", "return 1.0 - two_phi_neg + tail;",
     ["pin_collision_prob_quadrature"]),
    ("alpha_swaps_p1_p2", "return (z * p1 + p2) / (1.0 + z);", "return (z * p2 + p1) / (1.0 + z);",
     ["pin_threshold_balance"]),
    ("qalsh_interval_open", "if (fabs(dlt) <= half) cnt += 1;", "if (fabs(dlt) < half) cnt += 1;",
     ["pin_qalsh_hand_worked"]),
    ("qalsh_interval_full_width", "const double half = 0.5 * w * (double)R;\n    for (int64_t j",
     "const double half = w * (double)R;\n    for (int64_t j", ["pin_qalsh_hand_worked", "pin_qalsh_semantics"]),
    ("qalsh_prob_drops_sqrt2", "return erf(w / (2.0 * sqrt(2.0) * r));", "return erf(w / (2.0 * r));",
     ["pin_qalsh_prob_quadrature"]),
    ("qalsh_truncation_ignores_previous_level",
     "as in orc_query */\n        int64_t nc = 0;\n        for (int64_t j = 0; j < n; ++j) {\n            if (col[j] >= l) {\n                cs[nc].prev = prev[j];",
     "as in orc_query */\n        int64_t nc = 0;\n        for (int64_t j = 0; j < n; ++j) {\n            if (col[j] >= l) {\n                cs[nc].prev = 0;",
     ["pin_qalsh_hand_worked", "pin_qalsh_semantics"]),
    ("qalsh_radius_rule_one_sided",
     "if (!(fabs(pmin[i] - pq[i]) <= half && fabs(pmax[i] - pq[i]) <= half)) all = 0;",
     "if (!(fabs(pmax[i] - pq[i]) <= half)) all = 0;", ["pin_qalsh_v_ge_n_exact", "pin_qalsh_semantics"]),
    ("qalsh_threshold_uses_e2lsh_probability",
     "double p1 = orc_qalsh_prob(1.0, w);\n    double p2 = orc_qalsh_prob(c, w);",
     "double p1 = orc_collision_prob(1.0, w);\n    double p2 = orc_collision_prob(c, w);",
     ["pin_qalsh_threshold_balance"]),
    ("project_transposed", "const float *a = A + (size_t)i * d;", "const float *a = A + (size_t)i;",
     ["pin_qalsh_project_exact", "pin_qalsh_hand_worked"]),
    ("query_not_anchored", "int64_t g = (int64_t)hq[i] - (int64_t)o[i];\n        int64_t beta",
     "int64_t g = (int64_t)hq[i];\n        int64_t beta", ["pin_collision_counts", "pin_single_projection_is_e2lsh"]),
]


@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new, pins):
    src = open(oracle.SOURCE).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = oracle.compile_oracle(str(mutated), out=str(tmp_path / "libmutant.so"))
    orc = oracle.Oracle(lib)
    caught = []
    for pname in pins:
        fails = getattr(oracle_pins, pname)(orc)
        if fails:
            caught.append(pname)
    assert caught, f"mutant {name} survived pins {pins}"
    # the hand-worked case alone pins the stop rule and the truncation order,
    # independently of the numpy restatement of the level loop
    if "pin_hand_worked_golden" in pins:
        assert "pin_hand_worked_golden" in caught, f"the hand-worked case misses {name}"
