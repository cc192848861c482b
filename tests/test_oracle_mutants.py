"""Planted mistakes: each mutant is a copy of the oracle source with one
plausible slip; the pin named beside it must fail on the mutant (and passes on
the real oracle).  CPU only; nothing here touches the CUDA path."""
import pytest

import oracle as _oracle
import test_oracle_adjoint as adj
import test_oracle_error_bounds as eb
import test_oracle_mask_pins as mask
import test_oracle_pins as pins
import test_oracle_pins_capsule as capsule
import test_oracle_pins_drive as drive

MUTANTS = [
    ("dropped dilation", "#define DILATION 0.3", "#define DILATION 0.0",
     lambda o: pins.test_single_gaussian_closed_form(o, 3.0, -2.5, 0.3, 16.5)),
    ("no discriminant floor", "if (disc < 0.1) disc = 0.1;", "",
     lambda o: pins.test_single_gaussian_closed_form(o, 5.0, -1.5, -1.0, 16.0)),
    ("no 0.99 clamp", "double a_raw = g->o * G;\n    double alpha = a_raw < ALPHA_MAX ? a_raw : ALPHA_MAX;",
     "double a_raw = g->o * G;\n    double alpha = a_raw;",
     lambda o: pins.test_single_gaussian_closed_form(o, 2.0, -3.0, 5.0, 24.0)),
    ("no 1/255 skip", "if (alpha < ALPHA_MIN) return;", "if (alpha <= 0.0) return;",
     lambda o: pins.test_single_gaussian_closed_form(o, 3.0, -2.5, 0.3, 16.5)),
    ("radius one pixel too wide", "o->r = (int32_t)ceil(o->r3);", "o->r = (int32_t)ceil(o->r3) + 1;",
     pins.test_elongated_gaussian_square_footprint_closed_form),
    ("stop tested on T before the step", "if (Tn < T_STOP) {", "if (s->T < T_STOP) {",
     pins.test_stop_rule_never_blends_below_threshold),
    ("n_contrib counts covered instead of blended", "s->n += 1;", "s->n = s->ncov;",
     pins.test_contributor_counts_closed_form),
    ("n_covered stops at the first blended", "s->ncov_last = s->ncov;", "if (!s->ncov_last) s->ncov_last = s->ncov;",
     pins.test_contributor_counts_closed_form),
    ("depth weighted by alpha only", "s->D += g->z * w;", "s->D += g->z * alpha;", pins.test_transmittance_invariant),
    ("Jacobian sign", "J[0] = k->fx / pz; J[1] = 0.0; J[2] = -k->fx * tx / pz;",
     "J[0] = k->fx / pz; J[1] = 0.0; J[2] = k->fx * tx / pz;", pins.test_ewa_covariance_is_linearised_pinhole),
    ("no lateral clamp", "if (tx > limx) tx = limx;", "", pins.test_lateral_clamp_of_jacobian),
    ("quaternion entry sign", "R[1] = 2.0 * (x * y - w * z);", "R[1] = 2.0 * (x * y + w * z);",
     pins.test_quaternion_rotation),
    ("SH degree-1 sign", "c[1] = -c1;", "c[1] = c1;", pins.test_sh_matches_scipy_real_harmonics),
    ("SH degree-3 constant", "c[12] = 0.25 * sqrt(7.0 / pi);", "c[12] = 0.5 * sqrt(7.0 / pi);",
     pins.test_sh_orthonormal_by_quadrature),
    ("no colour clamp", "o->rgb[ch] = acc < 0.0 ? 0.0 : acc;", "o->rgb[ch] = acc;",
     pins.test_colour_clamped_at_zero_and_direction_dependent),
    ("camera centre added", "for (int i = 0; i < 3; ++i) o->d[i] = mu[i] - k->C[i];",
     "for (int i = 0; i < 3; ++i) o->d[i] = mu[i] + k->C[i];", pins.test_camera_translation_equivariance),
    ("view rotation transposed",
     "o->p[r] = k->R[3 * r] * o->d[0] + k->R[3 * r + 1] * o->d[1] + k->R[3 * r + 2] * o->d[2];",
     "o->p[r] = k->R[r] * o->d[0] + k->R[r + 3] * o->d[1] + k->R[r + 6] * o->d[2];",
     pins.test_camera_rotation_equivariance),
    ("tie-break reversed", "return (x->idx < y->idx) ? -1 : (x->idx > y->idx);",
     "return (x->idx > y->idx) ? -1 : (x->idx < y->idx);", pins.test_equal_depth_ties_follow_index),
    ("LBS drops translation", "mu[2] + A[4 * r + 3];", "mu[2];", pins.test_lbs_common_rigid_transform_and_no_renormalisation),
    ("LBS renormalises weights", "for (int e = 0; e < 12; ++e) A[e] += w[kk] * Gj[e];",
     "for (int e = 0; e < 12; ++e) A[e] += w[kk] / (w[0] + w[1] + w[2] + w[3]) * Gj[e];",
     pins.test_lbs_common_rigid_transform_and_no_renormalisation),
    ("adjoint: conic derivative sign", "gr->gB * (b * c / d2)", "gr->gB * (-b * c / d2)",
     adj.test_adjoint_matches_finite_differences),
    ("adjoint: clamp passes gradient", "if (a_raw < ALPHA_MAX) {\n                    q->go", "if (1) {\n                    q->go",
     adj.test_adjoint_matches_finite_differences),
    ("capsule distance to the infinite line", "    if (t < 0.0) t = 0.0;\n    if (t > 1.0) t = 1.0;", "",
     capsule.test_distance_and_nearest_against_sampling),
    ("first contact bisects towards the last crossing", "if (PT(m) <= R) b = m;\n                else a = m;",
     "if (PT(m) <= R) a = m;\n                else b = m;", capsule.test_first_contact_against_sampling),
    ("capsule joint unposed by its translation", "Mj[4 * r + 3];", "0.0;",
     capsule.test_capsules_of_rest_pose_and_rigid_motion),
    ("composite keeps the farther fragment",
     "const int take_a = layer_depth(depth_a[i]) < layer_depth(depth_b[i]);",
     "const int take_a = layer_depth(depth_a[i]) > layer_depth(depth_b[i]);", drive.test_composite_picks_the_nearer_fragment),
    ("composite: empty layer compares as depth 0", "return (d > 0.0 && d <= DBL_MAX) ? d : INFINITY;", "return d;",
     drive.test_composite_picks_the_nearer_fragment),
    ("FK: child offset from the rest joint instead of the bone",
     "acc += GR[9 * p + 3 * r + c] * (rest[3 * j + c] - rest[3 * p + c]);", "acc += GR[9 * p + 3 * r + c] * rest[3 * j + c];",
     drive.test_fk_rigid_invariants),
    ("FK: local rotation applied before the parent's", "mat3_mul(GR + 9 * p, Rl + 9 * j, GR + 9 * j);",
     "mat3_mul(Rl + 9 * j, GR + 9 * p, GR + 9 * j);", drive.test_fk_root_equivariance),
    ("FK: skinning matrix without the rest offset", "t -= GR[9 * j + 3 * r + c] * rest[3 * j + c];", "",
     drive.test_fk_zero_pose_is_identity),
    ("SH direction matrix transposed",
     "dv3[r] = dirmat[3 * r] * o->d[0] + dirmat[3 * r + 1] * o->d[1] + dirmat[3 * r + 2] * o->d[2];",
     "dv3[r] = dirmat[r] * o->d[0] + dirmat[r + 3] * o->d[1] + dirmat[r + 6] * o->d[2];",
     drive.test_sh_direction_matrix),
    ("mesh: barycentric of the wrong edge", "const double l0 = e[1] / area, l1 = e[2] / area, l2 = e[0] / area;",
     "const double l0 = e[0] / area, l1 = e[1] / area, l2 = e[2] / area;",
     drive.test_mesh_depth_is_the_ray_plane_intersection_and_colour_the_surface_point),
    ("mesh: depth interpolated in screen space", "const double z = 1.0 / (w0 + w1 + w2);",
     "const double z = l0 * Z[0] + l1 * Z[1] + l2 * Z[2];",
     drive.test_mesh_depth_is_the_ray_plane_intersection_and_colour_the_surface_point),
    ("mesh: equal depths keep the later triangle", "            if (z < best) {\n                second = best;",
     "            if (z <= best) {\n                second = best;", drive.test_mesh_occlusion_ties_and_near_cull),
    ("interpolation weights swapped", "o[e] = (1.0 - w) * A0[e] + w * A1[e];", "o[e] = w * A0[e] + (1.0 - w) * A1[e];",
     drive.test_interpolation_between_frames),
    ("mask: clamp decision not flagged",
     "if (fabs(power + log(g->o) - log(ALPHA_MAX)) <= dpow + E_ALPHA) s->amb |= AMB_CLAMP;", "",
     mask.test_clamp_threshold_is_flagged),
    ("mask: alpha decision bound dropped", "if (fabs(power + log(g->o) - log(ALPHA_MIN)) <= dpow + E_ALPHA) {",
     "if (fabs(power + log(g->o) - log(ALPHA_MIN)) <= 0.0) {", mask.test_alpha_threshold_is_flagged),
    ("mask: footprint flagged only outside r", "if (m >= g->r_lo - eps && m <= g->r_hi + eps) {",
     "if (m > g->r_hi && m <= g->r_hi + eps) {", mask.test_footprint_threshold_is_flagged),
    ("mask: stop decision bound dropped", "if (fabs(Tn - T_STOP) <= T_STOP * (relTn + U32) + 1e-15) {",
     "if (fabs(Tn - T_STOP) <= 0.0) {", mask.test_stop_threshold_is_flagged),
    ("bound: radius ignores the covariance's error", "const double emid = 0.5 * (e2[0] + e2[2]) + U32 * mid;",
     "const double emid = U32 * mid;", eb.test_fp32_projection_within_the_oracle_bounds),
    ("bound: 3D factor taken as exact",
     "e += et[3 * r + kk] * fabs(M[3 * kk + j]) + fabs(T[3 * r + kk]) * eM[3 * kk + j];",
     "e += et[3 * r + kk] * fabs(M[3 * kk + j]);", eb.test_fp32_projection_within_the_oracle_bounds),
    ("bound: conic ignores the determinant's error", "const double rd = edet / det + 2.0 * U32;",
     "const double rd = 2.0 * U32;", eb.test_fp32_projection_within_the_oracle_bounds),
    ("bound: conic B ignores b's error", "o->eB = fabs(o->conic[1]) * rd + e2[1] / det;",
     "o->eB = fabs(o->conic[1]) * rd;", eb.test_fp32_projection_within_the_oracle_bounds),
    ("adjoint: LBS covariance factor", "gA[4 * r + cc] = gm[r] * mu[cc] + 2.0 * acc;",
     "gA[4 * r + cc] = gm[r] * mu[cc] + acc;", adj.test_lbs_adjoint_matches_finite_differences),
]


@pytest.mark.parametrize("name,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(oracle, name, old, new, pin):
    src = _oracle.source()
    assert src.count(old) == 1, f"mutation site not unique: {name}"
    with _oracle.variant(src.replace(old, new)):
        with pytest.raises(AssertionError):
            pin(_oracle)
