"""The pins must catch plausible mistakes in the oracle.

Each mutant is a copy of ``oracle/orca_oracle.c`` with one deliberate error (a dropped
term, a flipped sign or comparison, a transposed operand, a wrong index), compiled into a
temporary library.  The pin tests of the other ``test_oracle_*`` modules run against it
(on the CPU) and at least one of them must fail.  The unmodified source must pass them.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
import test_oracle_conditioning as C
import test_oracle_halfplane as H
import test_oracle_knn as K
import test_oracle_lp as LP
import test_oracle_obstacles as OB
import test_oracle_population as POP
import test_oracle_spawn as SP
import test_oracle_step as ST

SRC = os.path.join(os.path.dirname(oracle.__file__), "orca_oracle.c")

MUTANTS = {
    "half_u_dropped": ("L.P = add(va, scl(u, 0.5));", "L.P = add(va, u);"),
    "relative_velocity_transposed": ("v2 p = sub(pb, pa), v = sub(va, vb);",
                                     "v2 p = sub(pb, pa), v = sub(vb, va);"),
    "left_leg_sign": ("L.d = scl(mk(p.x * leg - p.y * R, p.x * R + p.y * leg), 1.0 / p2);",
                      "L.d = scl(mk(p.x * leg + p.y * R, p.x * R + p.y * leg), 1.0 / p2);"),
    "cutoff_test_sign": ("if (wp < 0.0 && wp * wp > R2 * w2) {", "if (wp > 0.0 && wp * wp > R2 * w2) {"),
    "overlap_uses_tau": ("v2 w = sub(v, scl(p, 1.0 / dt));", "v2 w = sub(v, scl(p, 1.0 / tau));"),
    "lp1_bound_sides_swapped": ("if (den >= 0.0) { if (t < tR) tR = t; }",
                                "if (den < 0.0) { if (t < tR) tR = t; }"),
    "lp1_disc_dropped_square": ("double D = a * a + V * V - dot(L[i].P, L[i].P);",
                                "double D = a * a + V - dot(L[i].P, L[i].P);"),
    "lp2_violation_sign": ("if (viol > 0.0) {", "if (viol < 0.0) {"),
    "lp1_dir_mode_end": ("*x = add(L[i].P, scl(L[i].d, od > 0.0 ? tR : tL));",
                         "*x = add(L[i].P, scl(L[i].d, od > 0.0 ? tL : tR));"),
    "lp3_bisector_direction": ("v2 dd = sub(L[j].d, L[i].d);", "v2 dd = sub(L[i].d, L[j].d);"),
    "lp3_wrong_index": ("q.P = add(L[i].P, scl(L[i].d, det2(L[j].d, sub(L[i].P, L[j].P)) / den));",
                        "q.P = add(L[j].P, scl(L[i].d, det2(L[j].d, sub(L[i].P, L[j].P)) / den));"),
    "knn_radius_not_strict": ("if (d2 < nd2f) cand_insert", "if (d2 <= nd2f) cand_insert"),
    "knn_tie_break_reversed": ("return d2a < d2b || (d2a == d2b && ja < jb);",
                               "return d2a < d2b || (d2a == d2b && ja > jb);"),
    "pref_velocity_no_clamp": ("if (dist > pref_speed * dt) return scl(g, pref_speed / dist);",
                               "if (dist > 0.0) return scl(g, pref_speed / dist);"),
    "integrate_old_velocity": ("pos_out[0] = pa.x + x.x * S->dt;", "pos_out[0] = pa.x + va.x * S->dt;"),
    "knn_wrong_agent": ("float dx = pf[2 * j] - pf[2 * i];", "float dx = pf[2 * j] - pf[2 * j + 1];"),
    "arrival_strict": ("arrived[i] = d2 <= r2;", "arrived[i] = d2 < r2;"),
    "arrival_mixed_square": ("float dy2 = dy * dy;", "float dy2 = dx * dy;"),
    "arrival_radius_not_squared": ("float r2 = radius[i] * radius[i];", "float r2 = radius[i];"),
    "obstacle_radius_dropped": ("c = d > ra ? -(d - ra) / tau_o : -(d - ra) / dt;",
                                "c = d > ra ? -d / tau_o : -(d - ra) / dt;"),
    "obstacle_uses_dt": ("c = d > ra ? -(d - ra) / tau_o : -(d - ra) / dt;",
                         "c = d > ra ? -(d - ra) / dt : -(d - ra) / dt;"),
    "obstacle_normal_sign": ("if (d > 0.0) n = scl(q, -1.0 / d);", "if (d > 0.0) n = scl(q, 1.0 / d);"),
    # the conditioning tags that decide which agents the GPU parity gate may excuse
    "sens_ulp_scale": ("double eta_c = ldexp(1.0, e2 - 22);", "double eta_c = ldexp(1.0, e2 - 21);"),
    "sens_turn_angle": ("const double eta_r = ldexp(1.0, -22);", "const double eta_r = ldexp(1.0, -21);"),
    "sens_perturbs_wrong_line": ("Q[q].P = scl(nn, cc);", "Q[0].P = scl(nn, cc);"),
    "sens_offset_from_wrong_point": ("double c = dot(nq, L[q].P);", "double c = dot(nq, L[q].d);"),
    "margin_overlap_scale": ("note(tg, p2, R2, R2);", "note(tg, p2, R2, 1.0);"),
    "margin_leg_scale": ("note(tg, side, 0.0, sqrt(p2 * w2));", "note(tg, side, 0.0, p2);"),
    # spawning without overlap
    "spawn_strict": ("    return d2 <= reach2;", "    return d2 < reach2;"),
    "spawn_speed_of_neighbour_dropped": ("    float ss = vc + sj;", "    float ss = vc;"),
    "spawn_radius_sum_wrong": ("    float rr = rc + rj;", "    float rr = rc + rc;"),
    "spawn_window_dropped": ("    float travel = ss * window;", "    float travel = ss;"),
    "spawn_ignores_earlier_candidates": ("            if (accepted[e] && spawn_conflict(",
                                         "            if (0 && spawn_conflict("),
    "spawn_blocked_by_rejected": ("            if (accepted[e] && spawn_conflict(",
                                  "            if (1 && spawn_conflict("),
    "obstacle_lines_not_hard_in_lp3": ("for (int j = 0; j < nobst && j < OR_MAXK; ++j) proj[m++] = L[j];",
                                       "for (int j = 0; j < 0; ++j) proj[m++] = L[j];"),
}


def _pins():
    """Quick versions of the pins: (name, callable raising AssertionError on failure)."""
    o = oracle
    return [
        ("sens_shift", C.test_single_line_shift_moves_the_answer_by_four_ulps),
        ("sens_turn", C.test_single_line_turn_dominates_far_from_the_line),
        ("sens_parallel", lambda: C.test_near_parallel_vertex_is_tagged(1e-3)),
        ("sens_tangent", C.test_near_tangent_line_is_tagged),
        ("sens_vertex", C.test_well_separated_vertex_is_not_tagged),
        ("sens_lp3", C.test_least_penetration_answer_is_probed_too),
        ("margin_overlap", lambda: [C.test_overlap_decision_margin(d) for d in (3e-5, -3e-5)]),
        ("margin_leg", lambda: C.test_leg_side_margin(2e-5)),
        ("head_on", lambda: H.test_head_on_pair_closed_form(o)),
        ("cutoff", lambda: H.test_resting_pair_cutoff_closed_form(o)),
        ("overlap", lambda: [H.test_resting_overlap_closed_form(o, dt, v)
                             for dt, v in ((0.25, 2.0), (1 / 60, 1.5))]),
        ("vo_distance", lambda: H.test_u_is_shortest_vector_to_vo_boundary(o, 0)),
        ("overlap_disc", lambda: H.test_overlap_uses_one_step_disc(o, 0)),
        ("lp2_enum", lambda: LP.test_lp2_matches_vertex_enumeration(o, 0)),
        ("lp2_dir", lambda: LP.test_lp2_direction_mode_matches_enumeration(o, 0)),
        ("lp3_minimax", lambda: LP.test_lp3_reaches_minimax_penetration(o, 0)),
        ("lp3_single", lambda: LP.test_lp3_single_unreachable_line(o)),
        ("knn_numpy", lambda: K.test_knn_brute_matches_numpy_definition(o, 0)),
        ("knn_ties", lambda: K.test_knn_ties_break_by_index(o)),
        ("knn_strict", lambda: K.test_knn_strict_radius_and_padding(o)),
        ("lone_agent", lambda: (ST.test_lone_agent_prefers_goal_direction(o),
                                ST.test_lone_agent_lands_on_goal(o))),
        ("collision_free", lambda: ST.test_feasible_mutual_pairs_do_not_collide_within_tau(o, 0)),
        ("arrival_boundary", POP.test_boundary_cases),
        ("obstacle_wall", OB.test_wall_ahead_closed_form),
        ("obstacle_endpoint", OB.test_nearest_endpoint_closed_form),
        ("obstacle_overlap", OB.test_overlap_pushes_out_within_one_step),
        ("obstacle_lp3", OB.test_lp3_keeps_obstacle_lines_hard_and_minimises_the_rest),
        ("obstacle_lone_agent", OB.test_lone_agent_into_a_wall_closed_form),
        ("arrival_exact", POP.test_matches_exact_arithmetic_away_from_the_boundary),
        ("spawn_boundary", SP.test_touching_exactly_at_the_reach_is_a_conflict),
        ("spawn_earlier", SP.test_earlier_accepted_candidates_block_later_ones),
        ("spawn_reasons", SP.test_accepted_set_is_clear_and_every_rejection_has_a_reason),
        ("spawn_physics", SP.test_accepted_candidates_cannot_touch_anyone_within_the_window),
    ]


def _failing_pins(lib_path, first_only=False):
    """Names of the pins that fail against the library (stopping at the first failure
    when first_only: a mutant needs only one pin to catch it)."""
    failed = []
    with oracle.use_library(lib_path):
        for name, fn in _pins():
            try:
                fn()
            except (AssertionError, ValueError, FloatingPointError, ZeroDivisionError):
                failed.append(name)
                if first_only:
                    break
    return failed


def test_unmodified_oracle_passes_quick_pins():
    assert _failing_pins(oracle.build()) == []


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_mutant_is_caught(mutant):
    old, new = MUTANTS[mutant]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found once: {old!r}"
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "mut.c")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        lib = oracle.compile_source(path, os.path.join(td, f"lib_{mutant}.so"))
        with np.errstate(all="ignore"):
            failed = _failing_pins(lib, first_only=True)
    assert failed, f"no pin catches mutant {mutant}"
