"""Planted mistakes in the oracle must fail its pins (CPU only).

Each mutant is a copy of the oracle's C++ sources, or of its dense driver sim.py, with one
plausible mistake planted by a text substitution: a flipped sign, a dropped or wrong term,
a wrong index or operand.  The copy is compiled beside the real oracle (or loaded as a
module) and bound in its place, and the pins that guard the mistaken step run against it;
at least one of them must fail.  A mutant that passed all of its pins would show a step of
the oracle that is checked only against itself.

Every mutant keeps memory accesses in bounds and loops bounded (the Jacobi sweeps and the
conservative advancement carry their own caps), so a mutant can fail a pin but not crash.
Changes that cannot alter any output are left out.  Three examples: the second derivative
of 1/x, which reaches the distances only through the parameters of closest points, where
the squared distance is stationary; where a segment clamps t above 1, since the closest
point is then also the start of the next edge; and, in the coplanar case of the exact
intersection test, the check that the segment's second endpoint lies in the triangle and
the closed upper bounds of the collinear on-segment test, which the edge crossings and the
same test with edge and triangle exchanged repeat.
"""
import concurrent.futures
import ctypes
import functools
import hashlib
import importlib
import os
import sys
import types

import pytest

import oracle

_SRC = os.path.dirname(os.path.abspath(oracle.__file__))
_OUT = os.path.join(_SRC, "_build", "mutants")

# a pin: (test module, test function, argument tuples to run it with)
GEO_PT = ("test_oracle_geometry", "test_pt_distance_vs_sampling", [(t,) for t in range(40)])
GEO_EE = ("test_oracle_geometry", "test_ee_distance_vs_sampling", [(t,) for t in range(40)])
GEO_PT_CF = ("test_oracle_geometry", "test_pt_closed_forms", [()])
GEO_EE_CF = ("test_oracle_geometry", "test_ee_closed_forms", [()])
GEO_EE_PAR = ("test_oracle_geometry", "test_ee_near_parallel_interior_minimum", [()])
GEO_DEGEN = ("test_oracle_geometry", "test_degenerate_primitives", [()])
GEO_EXACT = ("test_oracle_geometry", "test_intersection_test_on_exact_configurations", [()])
BARRIER = ("test_oracle_potentials", "test_barrier_closed_form_and_boundary", [()])
F0 = ("test_oracle_potentials", "test_f0_matches_integral_of_f1", [()])
PAIR_FD = ("test_oracle_potentials", "test_barrier_derivatives_vs_central_differences",
           [(p, r) for p in (0, 1) for r in ("face", "edge", "vertex")])
PP_HESS = ("test_oracle_potentials", "test_point_point_hessian_closed_form", [()])
PSD = ("test_oracle_potentials", "test_psd_projection_properties", [()])
PSD_PAIR = ("test_oracle_potentials", "test_projected_barrier_hessian_is_psd_and_nearest", [()])
FRICTION = ("test_oracle_potentials", "test_friction_derivatives_and_invariants", [()])
FRICTION_ZERO = ("test_oracle_potentials", "test_friction_hessian_at_zero_slip_is_the_limit", [()])
EMBED = ("test_oracle_scene", "test_embedding_reproduces_rest_positions", [()])
REDUCE = ("test_oracle_scene", "test_reduction_equals_dense_JT_H_J_config1", [()])
INVARIANTS = ("test_oracle_scene", "test_reduced_invariants_all_embedded", [()])
IDENTITY = ("test_oracle_scene", "test_identity_embedding_is_full_space_ipc", [()])
REDUCED_FD = ("test_oracle_scene", "test_reduced_gradient_and_hessian_vs_finite_differences", [()])
PAIRS = ("test_oracle_scene", "test_pair_set_properties_config1", [()])
PAIRS_KNOWN = ("test_oracle_scene", "test_pair_set_known_configuration", [()])
CA_PP = ("test_oracle_scene", "test_ca_point_plane_constant_velocity", [()])
CA_EDGES = ("test_oracle_scene", "test_ca_separating_and_edges", [()])
CA_STEPS = ("test_oracle_scene", "test_ca_advances_by_the_speed_bound_until_s_d0", [()])
CA_CAP = ("test_oracle_scene", "test_ca_iteration_cap_returns_safe_time", [()])
ACCD = ("test_oracle_scene", "test_accd_no_penetration_after_accepted_step_config1", [()])
CA_REL = ("test_oracle_scene", "test_ca_bound_depends_only_on_relative_motion", [()])
ACCD_SAMPLED = ("test_oracle_scene", "test_restricted_step_bounds_match_the_full_one", [()])
PAIRS_EE_SAMPLED = ("test_oracle_scene", "test_restricted_edge_pairs_match_the_full_set", [()])
NO_PENETRATION = ("test_oracle_scene", "test_trajectories_are_intersection_free_small", [()])
LAG = ("test_oracle_scene", "test_friction_lag_is_the_lagged_contact_force", [()])
HVP_FD = ("test_oracle_hvp", "test_hvp_matches_central_differences_of_the_gradient", [()])
HVP_KIN = ("test_oracle_hvp", "test_hvp_of_a_kinematic_shift_matches_central_differences", [()])
HVP_H = ("test_oracle_hvp", "test_hvp_equals_the_unprojected_reduced_hessian", [()])
HVP_BALANCE = ("test_oracle_hvp", "test_kinematic_sum_balances_the_reduced_rows", [()])
DEDUP_RIDGE = ("test_oracle_dedup", "test_point_above_a_ridge_counts_once", [()])
DEDUP_APEX = ("test_oracle_dedup", "test_point_above_a_pyramid_apex_counts_once", [()])
DEDUP_FACE = ("test_oracle_dedup", "test_point_above_a_face_interior_is_kept", [()])
DEDUP_SCENES = ("test_oracle_dedup", "test_dedup_invariants_on_scenes", [(1,), (2,)])
MOLL_CF = ("test_oracle_mollifier", "test_energy_matches_the_closed_form", [()])
MOLL_FD = ("test_oracle_mollifier", "test_derivatives_match_central_differences", [()])
MOLL_EDGE = ("test_oracle_mollifier", "test_no_change_above_the_threshold_and_continuity_at_it", [()])
MOLL_SCENE = ("test_oracle_mollifier", "test_scene_energy_and_lag_with_the_mollifier", [()])

SIM_REST = ("test_oracle_sim", "test_energy_is_zero_and_stress_free_at_rest_and_rotation_invariant", [()])
SIM_POLAR = ("test_oracle_sim", "test_polar_rotation_matches_the_svd", [()])
SIM_LAME = ("test_oracle_sim", "test_lame_parameters_give_back_youngs_modulus_and_poissons_ratio", [()])
SIM_SMALL_STRAIN = ("test_oracle_sim", "test_small_strain_limit_is_linear_elasticity", [()])
SIM_STRESS = ("test_oracle_sim", "test_stress_is_the_complex_step_derivative_of_the_energy", [()])
SIM_DSTRESS = ("test_oracle_sim", "test_stress_differential_matches_central_differences", [()])
SIM_VOLUMES = ("test_oracle_sim", "test_volumes_mass_and_weight", [()])
SIM_VOLUME_SPLIT = ("test_oracle_sim", "test_vertex_volumes_of_an_offset_octahedron", [()])
SIM_MASS = ("test_oracle_sim", "test_reduced_mass_is_the_kinetic_energy_through_the_embedding", [()])
SIM_FLIGHT = ("test_oracle_sim", "test_free_flight_of_a_rigid_translation_is_exact", [()])
SIM_ELASTIC = ("test_oracle_sim", "test_elastic_gradient_and_hessian_match_central_differences", [()])
SIM_NEWTON = ("test_oracle_sim", "test_newton_step_converges_and_keeps_surfaces_apart", [()])
SIM_ADJOINT = ("test_oracle_sim", "test_adjoint_matches_central_differences_of_the_trajectory", [()])

# (name, file, original text, planted text, pins that must catch it)
MUTANTS = [
    # the barrier of Eq. 7 and f0 of Sec. III-B
    ("barrier_sign", "geometry.hpp", "return -(m * m) * log(d / T(dhat));",
     "return (m * m) * log(d / T(dhat));", [BARRIER]),
    ("barrier_log_scale", "geometry.hpp", "return -(m * m) * log(d / T(dhat));",
     "return -(m * m) * log(d / T(2.0 * dhat));", [BARRIER]),
    ("f0_quadratic_term", "geometry.hpp", "+ (y * y) / T(eps) +", "+ (y * y) / T(2.0 * eps) +", [F0]),
    ("f0_constant", "geometry.hpp", "T(eps / 3.0)", "T(eps / 2.0)", [F0]),
    ("f0_branch_point", "geometry.hpp", "if (val(y) >= eps) return y;", "if (val(y) >= 2.0 * eps) return y;",
     [F0]),
    # forward-mode differentiation rules
    ("ad_product_cross_term", "ad.hpp", "+ a.g[i] * b.g[j] + b.g[i] * a.g[j];",
     "+ 2.0 * a.g[i] * b.g[j];", [PAIR_FD, PP_HESS]),
    ("ad_sqrt_curvature", "ad.hpp", "-0.25 / (s * a.v)", "0.25 / (s * a.v)", [PAIR_FD, PP_HESS]),
    ("ad_inverse_slope", "ad.hpp", "-1.0 / (x * x)", "-2.0 / (x * x)", [PAIR_FD, PP_HESS]),
    ("ad_log_curvature", "ad.hpp", "-1.0 / (a.v * a.v)", "1.0 / (a.v * a.v)", [BARRIER, PAIR_FD]),
    ("ad_chain_drops_inner_hessian", "ad.hpp",
     "for (int j = 0; j < NV; ++j) r.h[i][j] = d1 * a.h[i][j] + d2 * a.g[i] * a.g[j];",
     "for (int j = 0; j < NV; ++j) r.h[i][j] = d2 * a.g[i] * a.g[j];", [PAIR_FD, PP_HESS]),
    ("ad_difference_hessian", "ad.hpp", "for (int j = 0; j < NV; ++j) r.h[i][j] = a.h[i][j] - b.h[i][j];",
     "for (int j = 0; j < NV; ++j) r.h[i][j] = a.h[i][j] + b.h[i][j];", [PAIR_FD, PP_HESS]),
    ("ad_log_slope", "ad.hpp", "return chain(a, std::log(a.v), 1.0 / a.v, -1.0 / (a.v * a.v));",
     "return chain(a, std::log(a.v), 2.0 / a.v, -1.0 / (a.v * a.v));", [BARRIER, PAIR_FD]),
    # distances
    ("pt_barycentric_operand", "geometry.hpp", "T b2 = (a * e - b * d) / det;",
     "T b2 = (a * e - b * e) / det;", [GEO_PT, GEO_PT_CF]),
    ("pt_edge_orientation", "geometry.hpp", "point_segment_d2(p, *tv[k], *tv[(k + 1) % 3], &tp);",
     "point_segment_d2(p, *tv[(k + 1) % 3], *tv[k], &tp);", [GEO_PT, GEO_PT_CF, FRICTION, DEDUP_RIDGE]),
    ("ee_stationary_sign", "geometry.hpp", "T t = (A * E - B * D) / nn;", "T t = (A * E + B * D) / nn;",
     [GEO_EE, GEO_EE_CF]),
    ("ee_endpoint_weights", "geometry.hpp", "c[2] = -(1.0 - t); c[3] = -t;", "c[2] = -t; c[3] = -(1.0 - t);",
     [GEO_EE, GEO_EE_CF, FRICTION, DEDUP_SCENES]),
    ("segment_no_lower_clamp", "geometry.hpp", "  if (val(t) <= 0.0) {\n    t = T(0.0);",
     "  if (val(t) <= -1e300) {\n    t = T(0.0);", [GEO_PT, GEO_EE]),
    ("pt_face_without_edge_check", "geometry.hpp", "if (!(edges < val(d2) * (1.0 - 1e-13))) {",
     "if (!(edges < -1.0)) {", [GEO_DEGEN]),
    ("segment_zero_length", "geometry.hpp", "if (val(dot(e, e)) == 0.0) {", "if (val(dot(e, e)) < 0.0) {",
     [GEO_DEGEN]),
    ("pt_vertex_region", "geometry.hpp", "*region = 4 + best_k;", "*region = 4 + (best_k + 1) % 3;",
     [GEO_PT_CF, DEDUP_APEX, DEDUP_SCENES]),
    ("ee_corner_region", "geometry.hpp", "*region = 5 + ia * 2 + ib;", "*region = 5 + ib * 2 + ia;",
     [GEO_EE_CF, DEDUP_SCENES]),
    ("pt_face_stencil", "geometry.hpp",
     "c[0] = 1.0; c[1] = -(1.0 - val(b1) - val(b2)); c[2] = -val(b1); c[3] = -val(b2);",
     "c[0] = 1.0; c[1] = -(1.0 - val(b1)); c[2] = -val(b1); c[3] = -val(b2);", [GEO_PT_CF, LAG, FRICTION]),
    ("ee_parallel_threshold", "geometry.hpp", "if (val(nn) > 1e-20 * val(A) * val(C)) {",
     "if (val(nn) > 1e-2 * val(A) * val(C)) {", [GEO_EE, GEO_EE_CF, GEO_EE_PAR]),
    ("ee_interior_weights", "geometry.hpp",
     "c[0] = 1.0 - val(s); c[1] = val(s); c[2] = -(1.0 - val(t)); c[3] = -val(t);",
     "c[0] = 1.0 - val(s); c[1] = val(s); c[2] = -val(t); c[3] = -(1.0 - val(t));", [GEO_EE_CF, LAG, FRICTION]),
    # projection to the nearest PSD matrix (Sec. III-C)
    ("jacobi_rotation_sign", "oracle.cpp", "A[k * n + q] = s * akp + c * akq;",
     "A[k * n + q] = s * akp - c * akq;", [PSD, PSD_PAIR]),
    ("psd_absolute_value", "oracle.cpp", "if (lam[k] > 0) s += V[i * n + k] * lam[k] * V[j * n + k];",
     "s += V[i * n + k] * std::fabs(lam[k]) * V[j * n + k];", [PSD, PSD_PAIR]),
    ("jacobi_eigenvector_sign", "oracle.cpp", "V[k * n + q] = s * vkp + c * vkq;",
     "V[k * n + q] = s * vkp - c * vkq;", [PSD, PSD_PAIR]),
    ("jacobi_loose_stop", "oracle.cpp", "if (off <= 1e-34 * fro || off == 0.0) break;",
     "if (off <= 1e-4 * fro || off == 0.0) break;", [PSD, PSD_PAIR]),
    ("psd_eigenvector_index", "oracle.cpp", "if (lam[k] > 0) s += V[i * n + k] * lam[k] * V[j * n + k];",
     "if (lam[k] > 0) s += V[i * n + k] * lam[k] * V[k * n + j];", [PSD, PSD_PAIR]),
    # the embedding (Eq. 14) and the reduction (Eq. 17)
    ("embed_index", "oracle.cpp", "s += w[4 * v + j] * q[3 * idx[4 * v + j] + k];",
     "s += w[4 * v + j] * q[3 * idx[4 * v + 3 - j] + k];", [EMBED]),
    ("embed_kinematic_row", "oracle.cpp", "for (int k = 0; k < 3; ++k) x[3 * v + k] = x_kin[3 * v + k];",
     "for (int k = 0; k < 3; ++k) x[3 * v + k] = x_kin[3 * v];", [EMBED, PAIRS_KNOWN, ACCD, NO_PENETRATION]),
    ("reduce_gradient_weight", "oracle.cpp", "R.g[3 * I + k] += wa * L.g[3 * a + k];",
     "R.g[3 * I + k] += L.g[3 * a + k];", [REDUCE, INVARIANTS]),
    ("reduce_hessian_weight", "oracle.cpp", "+= wa * wb * L.H[", "+= wa * wa * L.H[", [REDUCE, INVARIANTS]),
    ("reduce_drops_friction", "oracle.cpp", "      scatter(L.v, idx, w, F, res->R);\n",
     "\n", [REDUCE]),
    ("eval_projection_switch", "oracle.cpp", "    if (project) {", "    if (!project) {",
     [REDUCE, REDUCED_FD]),
    ("eval_friction_energy_dropped", "oracle.cpp", "      res->R.E += F.E;", "      res->R.E += 0.0 * F.E;",
     [REDUCE]),
    # the contact set B (Sec. III-B)
    ("pairs_ee_range", "oracle.cpp", "else if (d < dhat) part[tid].push_back({1,",
     "else if (d < 1.5 * dhat) part[tid].push_back({1,", [PAIRS, PAIRS_KNOWN]),
    ("pairs_pt_range", "oracle.cpp", "else if (d < dhat) part[tid].push_back({0,",
     "else if (d < 1.5 * dhat) part[tid].push_back({0,", [PAIRS, PAIRS_KNOWN]),
    ("pairs_order", "oracle.cpp", "    return j < o.j;\n", "    return j > o.j;\n", [PAIRS]),
    ("incident_ee_partial", "oracle.cpp",
     "return v[0] == v[2] || v[0] == v[3] || v[1] == v[2] || v[1] == v[3];",
     "return v[0] == v[2] || v[0] == v[3] || v[1] == v[2];", [PAIRS, PAIRS_KNOWN, NO_PENETRATION]),
    ("prim_box_upper_corner", "oracle.cpp", "b.hi[k] = std::max(b.hi[k], x[3 * v[t] + k]);",
     "b.hi[k] = std::min(b.hi[k], x[3 * v[t] + k]);", [PAIRS, PAIRS_KNOWN, PAIRS_EE_SAMPLED]),
    ("box_overlap_pad_sign", "oracle.cpp",
     "if (a.lo[k] - pad > b.hi[k] || b.lo[k] - pad > a.hi[k]) return false;",
     "if (a.lo[k] + pad > b.hi[k] || b.lo[k] + pad > a.hi[k]) return false;", [PAIRS, PAIRS_KNOWN, PAIRS_EE_SAMPLED]),
    ("enumeration_pad", "oracle.cpp", "const double pad = dhat * (1.0 + 1e-9);\n  bool ok = true;",
     "const double pad = dhat * 0.5;\n  bool ok = true;", [PAIRS, PAIRS_KNOWN, PAIRS_EE_SAMPLED]),
    # lagged friction (Sec. III-B)
    ("lag_force_magnitude", "oracle.cpp", "llambda[k] = kappa * mk * std::fabs(bb[1]);",
     "llambda[k] = kappa * mk * std::fabs(bb[0]);", [LAG]),
    ("lag_anchor", "oracle.cpp", "lanchor[3 * k + q] = r[q];", "lanchor[3 * k + q] = 0.5 * r[q];", [LAG]),
    ("lag_normal", "oracle.cpp", "ln[3 * k + q] = r[q] / rn;", "ln[3 * k + q] = r[(q + 1) % 3] / rn;", [LAG]),
    ("friction_tangent_projection", "oracle.cpp", "for (int k = 0; k < 3; ++k) w[k] = v[k] - vn * AD(L.n[k]);",
     "for (int k = 0; k < 3; ++k) w[k] = v[k];", [FRICTION]),
    ("friction_without_mu", "oracle.cpp", "double ml = mu * L.lambda;", "double ml = L.lambda;", [FRICTION]),
    ("friction_zero_slip_curvature", "oracle.cpp", "ml * (2.0 / eps) * L.gamma[a] * L.gamma[b]",
     "ml * (1.0 / eps) * L.gamma[a] * L.gamma[b]", [FRICTION_ZERO]),
    # the step bound (Sec. III-C)
    ("ca_no_safety_factor", "oracle.cpp", "double tn = t + (1.0 - s) * d / L;", "double tn = t + d / L;",
     [CA_PP, CA_EDGES]),
    ("ca_speed_bound", "oracle.cpp", "double L = La + Lb;", "double L = std::max(La, Lb);",
     [CA_PP, CA_EDGES, ACCD]),
    ("ca_mean_motion", "oracle.cpp", "for (int k = 0; k < 3; ++k) mean[k] /= 4.0;",
     "for (int k = 0; k < 3; ++k) mean[k] /= 2.0;", [CA_REL]),
    ("ca_stop_threshold", "oracle.cpp", "if (d <= s * d0) return t;", "if (d <= 0.5 * s * d0) return t;",
     [CA_PP, CA_EDGES, CA_STEPS]),
    ("ca_cap_off_by_one", "oracle.cpp", "if (*iters >= max_iter) { *capped = true; return t; }",
     "if (*iters > max_iter) { *capped = true; return t; }", [CA_CAP]),
    ("ca_point_speed_dropped", "oracle.cpp", "La = norm3(0);", "La = 0.0;", [CA_PP, CA_EDGES, ACCD]),
    ("accd_unswept_boxes", "oracle.cpp",
     "Box a = prim_box(m0, type, i, side_a, x), b = prim_box(m1, type, i, side_a, x1.data());",
     "Box a = prim_box(m0, type, i, side_a, x), b = a;", [ACCD]),
    ("accd_sampled_update", "oracle.cpp", "++ncand; iters += n;\n      if (t < alpha) alpha = t;",
     "++ncand; iters += n;\n      if (t < 0.0) alpha = t;", [ACCD_SAMPLED]),
    ("accd_list_update", "oracle.cpp", "iters += n;\n    if (t < alpha) alpha = t;",
     "iters += n;\n    if (t < 0.0) alpha = t;", [ACCD_SAMPLED]),
    ("accd_min_update", "oracle.cpp", "    if (t < a) a = t;", "    if (t < 0.0) a = t;", [ACCD, ACCD_SAMPLED]),
    ("intersection_incident_skip", "oracle.cpp",
     "if (a == t[0] || a == t[1] || a == t[2] || b == t[0] || b == t[1] || b == t[2]) continue;",
     "if (a == t[0] || a == t[1] || a == t[2] || b == t[0] || b == t[1]) continue;", [NO_PENETRATION, ACCD]),
    ("pairs_sampled_order", "oracle.cpp", "if (type == 1 && j < i) std::swap(i, j);\n      int32_t s[4];",
     "int32_t s[4];", [PAIRS_EE_SAMPLED]),
    ("pairs_sampled_range", "oracle.cpp", "if (d > 0.0 && d < dhat) out.push_back",
     "if (d > 0.0 && d < 1.5 * dhat) out.push_back", [PAIRS_EE_SAMPLED, PAIRS]),
    ("exact_product_error_dropped", "predicates.hpp", "    h = grow(h, err);\n    h = grow(h, p);",
     "    h = grow(h, p);", [GEO_EXACT]),
    ("exact_sum_error_dropped", "predicates.hpp", "    if (err != 0.0) h.push_back(err);\n", "",
     [GEO_EXACT]),
    ("intersection_decision", "predicates.hpp", "return !(has_pos && has_neg);", "return has_pos && has_neg;",
     [ACCD, NO_PENETRATION]),
    ("segment_plane_touch", "predicates.hpp", "if (sp * sq > 0) return false;", "if (sp * sq >= 0) return false;",
     [GEO_EXACT]),
    ("segments_meet_or", "predicates.hpp", "if (o1 * o2 < 0 && o3 * o4 < 0) return true;",
     "if (o1 * o2 < 0 || o3 * o4 < 0) return true;", [GEO_EXACT]),
    ("orient3d_cofactor_sign", "predicates.hpp", "Expansion cy = add(mul(bd[2], cd[0]), neg(mul(bd[0], cd[2])));",
     "Expansion cy = add(mul(bd[0], cd[2]), neg(mul(bd[2], cd[0])));", [GEO_EXACT, ACCD]),
    ("two_sum_error_term", "predicates.hpp", "y = (a - av) + (b - bv);", "y = (a - av);", [GEO_EXACT]),
    # the exact Hessian-vector product
    ("hvp_operand", "oracle.cpp", "acc += L.H[i * 12 + j] * u4[j];", "acc += L.H[i * 12 + j] * u4[i];",
     [HVP_FD, HVP_H]),
    ("hvp_drops_friction", "oracle.cpp", "      apply(L.v, F);\n", "\n", [HVP_FD, HVP_H]),
    ("hvp_kinematic_sign", "oracle.cpp", "out_kin[k] += y[3 * a + k];", "out_kin[k] -= y[3 * a + k];",
     [HVP_KIN, HVP_BALANCE]),
    ("hvp_reduction_weight", "oracle.cpp", "+= w[4 * a + i] * y[3 * a + k];", "+= y[3 * a + k];",
     [HVP_FD, HVP_H]),
    # mollifier and deduplication variants
    ("mollifier_curvature", "oracle.cpp", "c * T(1.0 / (eps * eps))", "c * T(2.0 / (eps * eps))",
     [MOLL_CF, MOLL_EDGE]),
    ("mollifier_threshold", "oracle.cpp", "if (val(c) >= eps) return T(1.0);",
     "if (val(c) >= 2.0 * eps) return T(1.0);", [MOLL_CF, MOLL_EDGE]),
    ("mollifier_rest_lengths", "oracle.cpp", "g_moll_factor * g_rest_len2[i] * g_rest_len2[j]",
     "g_moll_factor * g_rest_len2[i] * g_rest_len2[i]", [MOLL_SCENE]),
    ("lag_ignores_mollifier", "oracle.cpp", "llambda[k] = kappa * mk * std::fabs(bb[1]);",
     "llambda[k] = kappa * std::fabs(bb[1]);", [MOLL_SCENE]),
    ("dedup_face_key", "oracle.cpp", "key = {0, pj[k], pi[k]};", "key = {0, pj[k], 0};",
     [DEDUP_FACE, DEDUP_SCENES]),
    ("dedup_edge_key", "oracle.cpp", "edge_id(v[1 + e], v[1 + (e + 1) % 3])", "edge_id(v[1 + e], v[1 + (e + 2) % 3])",
     [DEDUP_RIDGE, DEDUP_SCENES]),
    ("dedup_vertex_key", "oracle.cpp", "key = {2, std::min(v[0], t), std::max(v[0], t)};",
     "key = {2, v[0], v[0]};", [DEDUP_APEX, DEDUP_SCENES]),
    ("dedup_ee_interior_key", "oracle.cpp", "key = {3, pi[k], pj[k]};", "key = {3, pi[k], pi[k]};",
     [DEDUP_SCENES]),
    ("dedup_ee_endpoint_edge", "oracle.cpp",
     "key = e < 2 ? std::array<int64_t, 3>{1, v[e], pj[k]} : std::array<int64_t, 3>{1, v[e], pi[k]};",
     "key = e < 2 ? std::array<int64_t, 3>{1, v[e], pi[k]} : std::array<int64_t, 3>{1, v[e], pj[k]};",
     [DEDUP_SCENES]),
    ("dedup_ee_corner_key", "oracle.cpp", "key = {2, std::min(v[ia], v[2 + ib]), std::max(v[ia], v[2 + ib])};",
     "key = {2, std::min(v[ia], v[2 + ia]), std::max(v[ia], v[2 + ia])};", [DEDUP_SCENES]),
    ("mollifier_cross_operand", "oracle.cpp", "    V3<AD> n = cross(p[1] - p[0], p[3] - p[2]);",
     "    V3<AD> n = cross(p[1] - p[0], p[2] - p[0]);", [MOLL_CF, MOLL_FD, MOLL_SCENE]),
]

# the dense driver and adjoint (oracle/sim.py): (name, original, planted, pins)
SIM_MUTANTS = [
    ("psi_volumetric_factor", "0.5 * lam * (tr - 3.0) ** 2", "lam * (tr - 3.0) ** 2", [SIM_SMALL_STRAIN, SIM_STRESS]),
    ("stress_shear_factor", "return 2.0 * mu3 * (F - R)", "return mu3 * (F - R)", [SIM_STRESS, SIM_SMALL_STRAIN]),
    ("polar_step", "Rn = 0.5 * (R + _inv_transpose(R))", "Rn = 0.5 * (R + np.swapaxes(R, -1, -2))",
     [SIM_POLAR, SIM_REST]),
    ("volume_split", "np.add.at(V, tri[:, k], vol / 3.0)", "np.add.at(V, tri[:, k], vol / 2.0)", [SIM_VOLUMES]),
    ("lumped_mass", "M[np.ix_(idx, idx)] += m * np.outer(w, w)", "M[np.ix_(idx, idx)] += m * np.diag(w)",
     [SIM_VOLUMES, SIM_MASS]),
    ("gravity_weights", "f[idx] += m * w[:, None] * sc.gravity[None, :]", "f[idx] += m * sc.gravity[None, :]",
     [SIM_VOLUMES, SIM_FLIGHT]),
    ("tet_hessian_node0", "dDs[:, c, :] = -1.0", "dDs[:, c, :] = 1.0", [SIM_ELASTIC]),
    ("tet_force_node0", "np.add.at(out, t[:, 0], -G.sum(axis=2))", "np.add.at(out, t[:, 0], G.sum(axis=2))",
     [SIM_ELASTIC]),
    ("inertia_target", "q_tilde = 2.0 * q_prev - q_prev2", "q_tilde = q_prev", [SIM_FLIGHT]),
    ("external_force_sign", "g = Md + h2 * (ge - m.f_ext + r[\"g\"])", "g = Md + h2 * (ge + m.f_ext + r[\"g\"])",
     [SIM_FLIGHT, SIM_NEWTON]),
    ("adjoint_second_history_term", "qbar[n - 2] -= MZ", "qbar[n - 2] += MZ", [SIM_ADJOINT]),
    ("volume_apex_origin", "c = x[members].mean(0)", "c = np.zeros(3)", [SIM_VOLUME_SPLIT]),
    ("lame_lambda", "E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))", "E * nu / ((1.0 + nu) * (1.0 - nu))",
     [SIM_LAME]),
    ("lame_mu", "return E / (2.0 * (1.0 + nu)),", "return E / (1.0 + nu),", [SIM_LAME]),
    ("pk_volumetric_direction", "(np.asarray(lam) * (tr - 3.0))[..., None, None] * R",
     "(np.asarray(lam) * (tr - 3.0))[..., None, None] * F", [SIM_STRESS, SIM_REST]),
    ("deformation_edge_vector", "q[t[:, 3]] - q[t[:, 0]]], axis=2)", "q[t[:, 3]] - q[t[:, 1]]], axis=2)",
     [SIM_ELASTIC, SIM_FLIGHT, SIM_NEWTON]),
    ("adjoint_first_history_term", "qbar[n - 1] += 2.0 * MZ", "qbar[n - 1] += MZ", [SIM_ADJOINT]),
    ("adjoint_theta_partial_sign", "tbar -= h2 * float(np.sum(Z * hk))", "tbar += h2 * float(np.sum(Z * hk))",
     [SIM_ADJOINT]),
    ("adjoint_kappa_partial_scale", "kbar -= h2 * float(np.sum(Z * r[\"g\"])) / kappa",
     "kbar -= h2 * float(np.sum(Z * r[\"g\"]))", [SIM_ADJOINT]),
]


def _mutant_dir(name):
    return os.path.join(_OUT, name)


def _build_one(mutant):
    name, fname, old, new, _ = mutant
    d = _mutant_dir(name)
    os.makedirs(d, exist_ok=True)
    texts = {}
    for f in oracle._SRCS:
        with open(os.path.join(_SRC, f)) as fh:
            texts[f] = fh.read()
    assert texts[fname].count(old) == 1, f"{name}: the original text must occur once in {fname}"
    texts[fname] = texts[fname].replace(old, new)
    digest = hashlib.sha256("\0".join(texts[f] for f in oracle._SRCS).encode()).hexdigest()[:16]
    so = os.path.join(d, f"liboracle_{digest}.so")       # a new path per source: dlopen caches by path
    for old_so in os.listdir(d):                         # builds of earlier sources
        if old_so.startswith("liboracle_") and old_so.endswith(".so") and old_so != os.path.basename(so):
            os.remove(os.path.join(d, old_so))
    if not os.path.exists(so):
        for f in oracle._SRCS:
            with open(os.path.join(d, f), "w") as fh:
                fh.write(texts[f])
        oracle.compile_so(d, so)
    return name, so


@pytest.fixture(scope="module")
def mutant_libs():
    with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        built = dict(ex.map(_build_one, MUTANTS))
    return built


def _clear_caches(mod):
    for v in vars(mod).values():
        if isinstance(v, functools._lru_cache_wrapper):
            v.cache_clear()


def _run_pins(pins):
    """Runs pins until one fails; returns (pin, args, exception) of the first failure."""
    for mod_name, fn_name, arg_sets in pins:
        mod = importlib.import_module(mod_name)
        fn = getattr(mod, fn_name)
        for args in arg_sets:
            _clear_caches(mod)
            try:
                fn(*args)
            except Exception as e:           # an assertion, or an error the wrapper raises
                return (fn_name, args, e)
            finally:
                _clear_caches(mod)
    return None


def _sim_mutant(name, old, new):
    """oracle/sim.py with one planted mistake, loaded as a module of the oracle package."""
    with open(os.path.join(_SRC, "sim.py")) as fh:
        text = fh.read()
    assert text.count(old) == 1, f"{name}: the original text must occur once in sim.py"
    mod = types.ModuleType(f"oracle._sim_{name}")
    mod.__package__ = "oracle"
    sys.modules[mod.__name__] = mod        # dataclasses look their module up by name
    try:
        exec(compile(text.replace(old, new), f"<sim.py mutant {name}>", "exec"), mod.__dict__)
    finally:
        del sys.modules[mod.__name__]
    return mod


@pytest.mark.parametrize("mutant", SIM_MUTANTS, ids=[m[0] for m in SIM_MUTANTS])
def test_planted_mistake_in_the_driver_fails_a_pin(mutant, monkeypatch):
    name, old, new, pins = mutant
    tmod = importlib.import_module("test_oracle_sim")
    monkeypatch.setattr(tmod, "sim", _sim_mutant(name, old, new))
    try:
        caught = _run_pins(pins)
    finally:
        _clear_caches(tmod)
    assert caught is not None, f"mutant {name} passed every pin it names"


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(mutant, mutant_libs, monkeypatch):
    name, _, _, _, pins = mutant
    L = oracle.bind(ctypes.CDLL(mutant_libs[name]))
    monkeypatch.setattr(oracle, "_lib", L)
    caught = _run_pins(pins)
    assert caught is not None, f"mutant {name} passed every pin it names"


def test_unmutated_oracle_passes_the_same_pins():
    """The pins the mutants fail pass on the oracle as committed (the harness itself plants
    nothing by accident)."""
    seen = []
    for pins in [m[4] for m in MUTANTS] + [m[3] for m in SIM_MUTANTS]:
        for p in pins:
            if p not in seen:
                seen.append(p)
    # each pin on its first argument set; the slow trajectory pins run in their own module
    seen = [p for p in seen if p not in (SIM_ADJOINT, SIM_NEWTON)]
    assert _run_pins([(mod, fn, args[:1]) for mod, fn, args in seen]) is None
