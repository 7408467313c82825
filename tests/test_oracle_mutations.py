"""The oracle's pins must be sharp: plant one plausible mistake at a time in a
copy of the oracle source (on the CPU), rebuild it, and check that at least
one pin fails.  Each mutant names the pins expected to catch it."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import tests.test_oracle_params as params_pins
import tests.test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "linprim_oracle.c")

MUTANTS = {
    "frustum_off": ("if (!(xc >= lox && xc <= hix && yc >= loy && yc <= hiy)) return;",
                    "(void)lox; (void)hix; (void)loy; (void)hiy;", ["frustum"]),
    "frustum_margin_1": ("const float lox = -0.15f * W, hix = 1.15f * W, loy = -0.15f * H, hiy = 1.15f * H;",
                         "const float lox = 0.0f * W, hix = 1.0f * W, loy = 0.0f * H, hiy = 1.0f * H;",
                         ["frustum"]),
    "eq1_drop_099": ("-log1p(-0.99 * P->opacity[i])", "-log1p(-P->opacity[i])",
                     ["thin_axis"]),
    "eq1_drop_factor_2": ("/ (2.0 * pp->dmin);", "/ (pp->dmin);", ["thin_axis"]),
    "stop_threshold": ("if (T < ORC_STOP_T) break;", "if (T < 1e-4) break;", ["early_stop"]),
    "stop_exclusive": ("        T = Tn;\n        /* reading",
                       "        if (Tn < ORC_STOP_T) break;\n        T = Tn;\n        /* reading",
                       ["early_stop"]),
    "blend_drop_T": ("C[ch] += T * o * pp->rgb[ch];", "C[ch] += o * pp->rgb[ch];", ["two_layer"]),
    "order_back_to_front": ("if (zi != zj) return zi < zj ? -1 : 1;",
                            "if (zi != zj) return zi > zj ? -1 : 1;", ["two_layer"]),
    "mtia_swap_uv_depth": ("*depth = (1.0 - u - v) * p0[2] + u * p1[2] + v * p2[2];",
                           "*depth = (1.0 - u - v) * p0[2] + v * p1[2] + u * p2[2];",
                           ["linear_solve"]),
    "mtia_grad_sign": ("dD[0][0] = p2[1] - p1[1];", "dD[0][0] = p1[1] - p2[1];", ["mtia_fd"]),
    "jacobian_sign": ("J[0][2] = -cam->fx * t[0] / (tz * tz);",
                      "J[0][2] = cam->fx * t[0] / (tz * tz);", ["first_order"]),
    "jacobian_row2": ("J[2][0] = t[0] / len;", "J[2][0] = 0.0;", ["chord"]),
    "sh_sign": ("Y[1] = -c1 * y;", "Y[1] = c1 * y;", ["scipy"]),
    "sh_deriv": ("SETD(4, c2a * y, c2a * x, 0.0);", "SETD(4, c2a * x, c2a * y, 0.0);", ["sh_fd"]),
    "chain_transpose_J": ("dtv[k][a] += pp->J[m][a] * gm;", "dtv[k][a] += pp->J[a][m] * gm;",
                          ["fd_tetra"]),
    "chain_drop_tau": ("pg->dsigma += dL_do * c->s * c->tau;", "pg->dsigma += dL_do * c->s;",
                       ["fd_tetra"]),
    "chain_dist_sh": ("dcentre[3 * i + a] += s / pp->dist;", "dcentre[3 * i + a] += s;",
                      ["fd_octa"]),
    "chain_B_recursion": ("B[ch] = c->o * pp->rgb[ch] + c->tau * B[ch];",
                          "B[ch] = c->o * pp->rgb[ch] + B[ch];", ["fd_tetra"]),
    "rect_round": ("fx0 = ceilf(xmin - 0.5f);", "fx0 = floorf(xmin - 0.5f);", ["keyfields"]),
    "key_tie_order": ("return (x->seq > y->seq) - (x->seq < y->seq);",
                      "return (x->seq < y->seq) - (x->seq > y->seq);", ["ties"]),
    "render_tie_order": ("return (i > j) - (i < j);", "return (i < j) - (i > j);", ["ties"]),
    "param_octa_sign": ("*sign = (k % 2) ? -1.0 : 1.0;", "*sign = 1.0;", ["param_scipy"]),
    "param_quat_grad": ("g[0] = 2 * (-z * dR[0][1] + y * dR[0][2]", "g[0] = 2 * (z * dR[0][1] + y * dR[0][2]",
                        ["param_fd"]),
    "param_norm_grad": ("dquat[4 * (size_t)i + 0] = (g[0] - dot * w) / qn;",
                        "dquat[4 * (size_t)i + 0] = g[0] / qn;", ["param_fd"]),
    "param_sigmoid_grad": ("dlogit[i] = dopacity[i] * al * (1.0 - al);", "dlogit[i] = dopacity[i] * al;",
                           ["param_fd"]),
    "aa_octa_full_kernel": ("return (float)(P->nv == 6 ? 0.5 * P->aa_kernel : P->aa_kernel);",
                            "return (float)(P->aa_kernel);", ["aa_span"]),
    "aa_min_side_inward": ("else if (kf->shx[k] < 0) qx = qx - sh;", "else if (kf->shx[k] < 0) qx = qx + sh;",
                           ["aa_rect", "aa_moves"]),
    "aa_box_unmoved": ("pp->p[k][0] += pp->kf.shx[k] * (double)pp->kf.shift;", "pp->p[k][0] += 0.0;",
                       ["aa_span", "aa_moves"]),
    "depth_exit_not_entry": ("if (out->depth == 0.0 && T >= 0.5 && Tn < 0.5) out->depth = i1;",
                             "if (out->depth == 0.0 && T >= 0.5 && Tn < 0.5) out->depth = i2;", ["depth_surface"]),
    "depth_threshold": ("if (out->depth == 0.0 && T >= 0.5 && Tn < 0.5) out->depth = i1;",
                        "if (out->depth == 0.0 && T >= 0.1 && Tn < 0.1) out->depth = i1;", ["depth_layers"]),
    "exact_no_dir_length": ("depth = lam * dl;   /* distance along the ray */", "depth = lam;",
                            ["exact_chord"]),
    "exact_grad_sign": ("for (m = 0; m < 3; ++m) a[m] = (p0[m] - lam * d[m]) / dn;",
                        "for (m = 0; m < 3; ++m) a[m] = (p0[m] + lam * d[m]) / dn;", ["exact_fd"]),
    "aa_rect_unmoved": ("if (kf->shx[k] > 0) qx = qx + sh;", "if (kf->shx[k] > 0) qx = qx;", ["aa_rect"]),
    "colour_clamp_grad_unmasked": ("double gc = pp->rgb_raw[ch] > 0.0 ? pg->drgb[ch] : 0.0;",
                                   "double gc = pg->drgb[ch];", ["clamp"]),
    "colour_offset_dropped": ("pp->rgb_raw[ch] = s + 0.5;", "pp->rgb_raw[ch] = s;", ["two_layer"]),
    "dalpha_drop_099": ("dopacity[i] += pg->dsigma * 0.99 / ((1.0 - 0.99 * P->opacity[i]) * 2.0 * pp->dmin);",
                        "dopacity[i] += pg->dsigma / ((1.0 - 0.99 * P->opacity[i]) * 2.0 * pp->dmin);",
                        ["fd_tetra"]),
    "background_unattenuated": ("for (ch = 0; ch < 3; ++ch) out->rgb[ch] = C[ch] + T * bg[ch];",
                                "for (ch = 0; ch < 3; ++ch) out->rgb[ch] = C[ch] + bg[ch];", ["two_layer"]),
    "near_plane_off": ("    if (!(tc[2] > ORC_NEAR)) return;", "    if (!(tc[2] > -ORC_NEAR)) return;", ["near"]),
    "camera_position_sign": ("campos[m] = -(R[0][m] * T[0] + R[1][m] * T[1] + R[2][m] * T[2]);",
                             "campos[m] = (R[0][m] * T[0] + R[1][m] * T[1] + R[2][m] * T[2]);", ["colour_dir"]),
    "keys_value_not_record": ("E[n].val = (uint32_t)((long long)c * P->n + i);", "E[n].val = (uint32_t)i;",
                              ["keys_multiview"]),
    "keys_tile_base_missing": ("            tile_base += (long long)tiles_x * tiles_y;\n", "", ["keys_multiview"]),
    "keys_last_tile_column": ("for (tx = kf.px0 / tile; tx <= kf.px1 / tile; ++tx) {",
                              "for (tx = kf.px0 / tile; tx < kf.px1 / tile; ++tx) {", ["keys_structure"]),
    "keys_no_depth": ("E[n].key = (gt << 32) | kf.zbits;", "E[n].key = (gt << 32);", ["keys_structure"]),
    "counts_flag_only": ("counts[(size_t)c * P->n + i] = (uint32_t)cnt;", "counts[(size_t)c * P->n + i] = (uint32_t)(cnt > 0);",
                         ["keys_structure"]),
    "rect_clamp_past_image": ("fx1 = fminf(fx1, (float)(cam->width - 1));", "fx1 = fminf(fx1, (float)(cam->width));",
                              ["keyfields"]),
    "aa_tetra_half_kernel": ("return (float)(P->nv == 6 ? 0.5 * P->aa_kernel : P->aa_kernel);",
                             "return (float)(0.5 * P->aa_kernel);", ["aa_moves"]),
    "chain_drop_direction_row": ("            dtc[b] += dJ[2][a] * d_ab / len;\n", "", ["aa_fd"]),
    "exact_near_plane_off": ("if (!(Z > ORC_NEAR)) { kf->visible = 0; return; }",
                             "if (!(Z > -1e30f)) { kf->visible = 0; return; }", ["exact_near"]),
    "silhouette_flag_off": ("if (fabs(c2 - c1) <= 1e-5 * (zhi - zlo)) out->borderline |= 2;",
                            "if (0) out->borderline |= 2;", ["silhouette"]),
    "stop_flag_too_tight": ("if (fabs(Tn - ORC_STOP_T) <= 1e-3 * ORC_STOP_T) out->borderline |= 1;",
                            "if (fabs(Tn - ORC_STOP_T) <= 1e-9 * ORC_STOP_T) out->borderline |= 1;", ["stop_flag"]),
    "depth_flag_off": ("if (fabs(Tn - 0.5) <= 1e-4 * 0.5) out->borderline |= 4;", "if (0) out->borderline |= 4;",
                       ["depth_flag"]),
    "quat_rotation_sign": ("R[0][1] = 2 * (x * y - w * z);", "R[0][1] = 2 * (x * y + w * z);", ["param_scipy"]),
    "quat_not_normalised": ("double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;",
                            "double w = q_in[0], x = q_in[1], y = q_in[2], z = q_in[3];", ["param_scipy"]),
    "opacity_sigmoid_sign": ("opacity[i] = 1.0 / (1.0 + exp(-logit[i]));", "opacity[i] = 1.0 / (1.0 + exp(logit[i]));",
                             ["param_scipy"]),
    "exact_ray_no_principal_point": ("d[0] = (rx - pp->cx) / pp->fx;", "d[0] = rx / pp->fx;", ["exact_chord"]),
    "exact_grad_drop_plane_term": ("for (m = 0; m < 3; ++m) g[0][m] = n[m] / dn - g[1][m] - g[2][m];",
                                   "for (m = 0; m < 3; ++m) g[0][m] = -g[1][m] - g[2][m];", ["exact_fd"]),
    "ray_space_depth_is_z": ("pp->pc[2] = sqrt(pp->tc[0] * pp->tc[0] + pp->tc[1] * pp->tc[1] + pp->tc[2] * pp->tc[2]);",
                             "pp->pc[2] = pp->tc[2];", ["first_order"]),
    "sh_count_wrong": ("static int sh_count(int degree) { return (degree + 1) * (degree + 1); }",
                       "static int sh_count(int degree) { return 3 * degree + 1; }", ["colour_dir"]),
    "frozen_dmin_ignored": ("    if (P->dmin) pp->dmin = P->dmin[i];\n", "", ["fd_tetra"]),
    "aa_y_move_from_x_side": ("pp->p[k][1] += pp->kf.shy[k] * (double)pp->kf.shift;",
                              "pp->p[k][1] += pp->kf.shx[k] * (double)pp->kf.shift;", ["aa_moves"]),
    "backward_T_after_primitive": ("c->i1 = i1; c->i2 = i2; c->s = s; c->tau = tau; c->o = o; c->T = T;",
                                   "c->i1 = i1; c->i2 = i2; c->s = s; c->tau = tau; c->o = o; c->T = Tn;", ["fd_tetra"]),
    "span_grad_sign": ("dL_ds = dL_do * pp->sigma * c->tau;", "dL_ds = -dL_do * pp->sigma * c->tau;", ["fd_tetra"]),
    "octa_face_table": ("    {1, 2, 4}, {1, 2, 5}, {1, 3, 4}, {1, 3, 5}};", "    {1, 2, 4}, {1, 2, 5}, {1, 3, 4}, {0, 3, 5}};",
                        ["chord"]),
    "tetra_face_table": ("static const int TETRA_FACES[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};",
                         "static const int TETRA_FACES[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 3}};",
                         ["chord_tetra"]),
}

CHECKS = {
    "thin_axis": lambda o: [pins.test_thin_axis_opacity_is_099_alpha(o, a) for a in (0.5, 0.9)],
    "early_stop": lambda o: [pins.test_early_stop_at_cumulative_opacity_0999(o, a) for a in (0.5, 0.8)],
    "two_layer": pins.test_two_layer_compositing_and_background,
    "linear_solve": pins.test_mtia_matches_linear_solve,
    "mtia_fd": pins.test_mtia_gradient_fd,
    "first_order": pins.test_ray_space_map_is_first_order_perspective,
    "chord": lambda o: pins.test_span_centre_pixel_equals_world_chord(o, 6),
    "chord_tetra": lambda o: pins.test_span_centre_pixel_equals_world_chord(o, 4),
    "scipy": pins.test_sh_basis_matches_scipy,
    "sh_fd": pins.test_sh_basis_derivative_fd,
    "fd_tetra": pins.test_adjoint_fd_tetrahedra,
    "fd_octa": pins.test_adjoint_fd_octahedra_sh3,
    "keyfields": pins.test_keyfields_are_binary32_replay,
    "frustum": pins.test_view_frustum_cull,
    "keys_structure": pins.test_keys_structure,
    "ties": pins.test_depth_ties_keep_index_order,
    "param_scipy": lambda o: [params_pins.test_vertices_match_scipy_rotation(k) for k in (6, 4)],
    "param_fd": lambda o: [params_pins.test_params_adjoint_fd(k) for k in (6, 4)],
    "depth_surface": pins.test_depth_front_surface_closed_form,
    "exact_chord": lambda o: pins.test_exact_span_is_the_world_chord(o, 6),
    "exact_fd": lambda o: [pins.test_exact_adjoint_fd(o, k) for k in (6, 4)],
    "depth_layers": pins.test_depth_two_layers,
    "aa_span": lambda o: pins.test_aa_filter_octahedron_span_closed_form(o, 4.0),
    "aa_moves": pins.test_aa_filter_moves_box_vertices,
    "aa_rect": pins.test_aa_filter_widens_the_pixel_rectangle,
    "clamp": pins.test_clamped_colour_channel_has_no_gradient,
    "near": pins.test_near_plane_cull,
    "colour_dir": pins.test_colour_direction_is_from_the_camera,
    "keys_multiview": pins.test_keys_multiview_tile_bases,
    "aa_fd": pins.test_aa_filter_adjoint_fd,
    "exact_near": pins.test_exact_culls_primitives_reaching_the_near_plane,
    "silhouette": pins.test_silhouette_grazing_pixels_are_flagged,
    "stop_flag": lambda o: [pins.test_borderline_stop_flag(o, r, f) for r, f in ((2e-4, True), (5e-3, False))],
    "depth_flag": lambda o: [pins.test_borderline_depth_flag(o, x, f) for x, f in ((0.5 + 2e-5, True), (0.501, False))],
}


@pytest.fixture(scope="module")
def tmpdir_mut():
    with tempfile.TemporaryDirectory() as d:
        yield d


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmpdir_mut, orc):
    old, new, checks = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path_c = os.path.join(tmpdir_mut, f"{name}.c")
    path_so = os.path.join(tmpdir_mut, f"{name}.so")
    open(path_c, "w").write(src.replace(old, new))
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", path_c,
                    "-o", path_so, "-lm"], check=True)
    caught = False
    with oracle.use_library(path_so):
        for c in checks:
            try:
                CHECKS[c](oracle)
            except AssertionError:
                caught = True
                break
    assert caught, f"mutant {name} survived {checks}"
