"""The oracle's pins must be discriminating, not only green.

Each mutant below plants ONE plausible mistake into a temporary copy of the oracle: a
dropped term, a wrong sign, a swapped index or operand, a wrong constant, a rule taken in
the wrong order. The oracle's own ``-m "not gpu"`` pin tests (``tests/test_oracle_*.py``)
then run against that copy, and at least one of them must FAIL with an assertion, not with
a crash. A mutant that every pin accepts would be a mistake the GPU parity tests inherit
unseen. The oracle itself is never modified: the copy lives in a temporary directory, and
mutated C code is compiled there.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (id, file under oracle/, original text (must occur exactly once), mutated text)
MUTANTS = [
    # ---- projection (Eq. 2-3, EWA) ----
    ("proj_dilation_dropped", "sg_oracle.c", "double s00 = S[0] + cfg->dilation,", "double s00 = S[0],"),
    ("proj_jacobian_sign", "sg_oracle.c", "J[2] = -cam->fx * xt / z2;", "J[2] = cam->fx * xt / z2;"),
    ("proj_view_rotation_transposed_in_JW", "sg_oracle.c",
     "T[3 * i + j] = J[3 * i] * W[j] + J[3 * i + 1] * W[3 + j] + J[3 * i + 2] * W[6 + j];",
     "T[3 * i + j] = J[3 * i] * W[3 * j] + J[3 * i + 1] * W[3 * j + 1] + J[3 * i + 2] * W[3 * j + 2];"),
    ("proj_mean_rotation_transposed", "sg_oracle.c",
     "t[i] = W[3 * i] * mean[0] + W[3 * i + 1] * mean[1] + W[3 * i + 2] * mean[2] + cam->t[i];",
     "t[i] = W[i] * mean[0] + W[3 + i] * mean[1] + W[6 + i] * mean[2] + cam->t[i];"),
    ("proj_quaternion_sign", "sg_oracle.c", "R[1] = 2 * (x * y - w * z);", "R[1] = 2 * (x * y + w * z);"),
    ("proj_scale_on_rows", "sg_oracle.c", "M[3 * i + j] = R[3 * i + j] * exp(log_scale[j]);",
     "M[3 * i + j] = R[3 * i + j] * exp(log_scale[i]);"),
    ("proj_conic_offdiag_sign", "sg_oracle.c", "out[P_CB] = -s01 / det;", "out[P_CB] = s01 / det;"),
    ("proj_u_uses_fy", "sg_oracle.c", "out[P_U] = cam->fx * t[0] / t[2] + cam->cx;",
     "out[P_U] = cam->fy * t[0] / t[2] + cam->cx;"),
    ("proj_sigmoid_sign", "sg_oracle.c", "double o = 1.0 / (1.0 + exp(-opacity_logit));",
     "double o = 1.0 / (1.0 + exp(opacity_logit));"),
    ("proj_x_extent_from_y_variance", "sg_oracle.c", "out[P_EXTX] = sqrt(2.0 * thr * s00)",
     "out[P_EXTX] = sqrt(2.0 * thr * s11)"),
    ("proj_isotropic_fx_for_y", "sg_oracle.c", "ry = cam->fy * r / t[2];", "ry = cam->fx * r / t[2];"),
    ("proj_depth_key_from_tx", "sg_oracle.c", "out[P_DKEY] = (double)depth_key(mean, cam, t[2], &damb);",
     "out[P_DKEY] = (double)depth_key(mean, cam, t[0], &damb);"),
    ("proj_depth_midpoint_band_ignored", "sg_oracle.c", "*ambiguous = fabs(tz - lo) <= band || fabs(tz - hi) <= band;",
     "*ambiguous = 0;"),
    ("proj_fov_limit_y_uses_W", "sg_oracle.c", "double limy = cfg->fov_clamp * 0.5 * cam->H / cam->fy;",
     "double limy = cfg->fov_clamp * 0.5 * cam->W / cam->fy;"),
    ("proj_fov_limit_x_uses_fy", "sg_oracle.c", "double limx = cfg->fov_clamp * 0.5 * cam->W / cam->fx;",
     "double limx = cfg->fov_clamp * 0.5 * cam->W / cam->fy;"),
    ("proj_det_sign", "sg_oracle.c", "double det = s00 * s11 - s01 * s01;", "double det = s00 * s11 + s01 * s01;"),
    ("proj_conic_diagonal_swapped", "sg_oracle.c", "out[P_CA] = s11 / det;", "out[P_CA] = s00 / det;"),
    ("pack_camera_fx_fy_swapped", "__init__.py", 'return np.array([cam["fx"], cam["fy"], cam["cx"], cam["cy"]',
     'return np.array([cam["fy"], cam["fx"], cam["cx"], cam["cy"]'),
    ("pack_camera_rotation_transposed", "__init__.py", '*np.asarray(cam["R_cw"], np.float64).reshape(9),',
     '*np.asarray(cam["R_cw"], np.float64).T.reshape(9),'),
    ("pack_cfg_alpha_min_T_min_swapped", "__init__.py", 'return np.array([c["alpha_max"], c["alpha_min"], c["T_min"],',
     'return np.array([c["alpha_max"], c["T_min"], c["alpha_min"],'),
    ("proj_v_uses_cx", "sg_oracle.c", "out[P_V] = cam->fy * t[1] / t[2] + cam->cy;",
     "out[P_V] = cam->fy * t[1] / t[2] + cam->cx;"),
    # ---- compositing (Eq. 7-9) ----
    ("comp_depth_order_flag_dropped", "sg_oracle.c", "        if (c->order_amb) fl |= F_DEPTH;\n", "\n"),
    ("comp_stop_band_uses_alpha_tolerance", "sg_oracle.c",
     "if (fabs(Tn - cfg->T_min) <= tol_T * cfg->T_min) fl |= F_STOP;",
     "if (fabs(Tn - cfg->T_min) <= tol * cfg->T_min) fl |= F_STOP;"),
    ("comp_skip_band_dropped", "sg_oracle.c",
     "        if (fabs(c->raw - cfg->alpha_min) <= tol * cfg->alpha_min) fl |= F_SKIP;\n", "\n"),
    ("comp_gather_stops_at_exact_extent", "sg_oracle.c",
     "if (fabs(dx) > p[P_GEXTX] || fabs(dy) > p[P_GEXTY]) continue;", "if (fabs(dx) > p[P_EXTX] || fabs(dy) > p[P_EXTY]) continue;"),
    ("comp_sigma_cross_term_halved", "sg_oracle.c", "+ p[P_CB] * dx * dy;", "+ 0.5 * p[P_CB] * dx * dy;"),
    ("comp_alpha_clamp_dropped", "sg_oracle.c", "double alpha = raw < cfg->alpha_max ? raw : cfg->alpha_max;",
     "double alpha = raw;"),
    ("comp_skip_threshold_halved", "sg_oracle.c", "if (c->alpha < cfg->alpha_min) continue;",
     "if (c->alpha < 0.5 * cfg->alpha_min) continue;"),
    ("comp_stop_after_adding", "sg_oracle.c", "if (Tn < cfg->T_min) break;\n        contrib[m] = k; Tb[m] = T; ++m;",
     "contrib[m] = k; Tb[m] = T; ++m;\n        if (Tn < cfg->T_min) break;"),
    ("comp_depth_weight_alpha_only", "sg_oracle.c", "acc[3] += w * proj", "acc[3] += c->alpha * proj"),
    ("comp_colour_weight_T_only", "sg_oracle.c", "acc[ch] += w * rgb[", "acc[ch] += Tb[j] * rgb["),
    ("comp_back_to_front", "sg_oracle.c", "if (a->dkey < b->dkey) return -1;\n    if (a->dkey > b->dkey) return 1;",
     "if (a->dkey < b->dkey) return 1;\n    if (a->dkey > b->dkey) return -1;"),
    ("comp_ties_by_descending_id", "sg_oracle.c", "return (a->id > b->id) - (a->id < b->id);",
     "return (a->id < b->id) - (a->id > b->id);"),
    ("comp_background_not_weighted_by_T", "sg_oracle.c", "acc[ch] + T * cfg.bg[ch];", "acc[ch] + cfg.bg[ch];"),
    ("comp_extent_filter_too_tight", "sg_oracle.c", "if (fabs(dx) > p[P_GEXTX] || fabs(dy) > p[P_GEXTY]) continue;",
     "if (fabs(dx) > 0.5 * p[P_GEXTX] || fabs(dy) > p[P_GEXTY]) continue;"),
    ("comp_candidates_prefiltered_too_tight", "sg_oracle.c", "if (alpha < cfg->alpha_min * 0.5) continue;",
     "if (alpha < cfg->alpha_min * 2.0) continue;"),
    ("comp_transmittance_update", "sg_oracle.c", "        T = Tn;\n", "        T = T * c->alpha;\n"),
    ("comp_transmittance_unclamped_alpha", "sg_oracle.c", "double Tn = T * (1.0 - c->alpha);",
     "double Tn = T * (1.0 - c->raw);"),
    ("comp_sigma_conic_diagonal_swapped", "sg_oracle.c",
     "double sigma = 0.5 * (p[P_CA] * dx * dx + p[P_CC] * dy * dy) + p[P_CB] * dx * dy;",
     "double sigma = 0.5 * (p[P_CC] * dx * dx + p[P_CA] * dy * dy) + p[P_CB] * dx * dy;"),
    # ---- adjoint (Sec. III-D) ----
    ("bwd_dalpha_missing_T", "sg_oracle.c", "dalpha *= Ti;", "dalpha *= 1.0;"),
    ("bwd_suffix_not_attenuated", "sg_oracle.c", "A[ch] = al * f[ch] + (1.0 - al) * A[ch];",
     "A[ch] = al * f[ch] + A[ch];"),
    ("bwd_dsigma_sign", "sg_oracle.c", "double gsig = -dalpha * p[P_OPAC] * c->G;",
     "double gsig = dalpha * p[P_OPAC] * c->G;"),
    ("bwd_du_wrong_conic_entry", "sg_oracle.c", "gsig * -(ca * dx + cb * dy),", "gsig * -(ca * dx + cc * dy),"),
    ("bwd_conic_inverse_term_dropped", "sg_oracle.c", "(a * c + b * b) * gb", "(a * c) * gb"),
    ("bwd_dT_factor_two", "sg_oracle.c", "gT[3 * i + j] = 2.0 * s;", "gT[3 * i + j] = s;"),
    ("bwd_clamped_jacobian_sign", "sg_oracle.c", "gt[2] += gJ[2] * (-J[2] / tz);", "gt[2] += gJ[2] * (J[2] / tz);"),
    ("bwd_sigmoid_derivative_dropped", "sg_oracle.c", "double o = p[P_OPAC];\n    *g_ol += go * o * (1.0 - o);\n}",
     "double o = p[P_OPAC];\n    *g_ol += go * o;\n}"),
    ("bwd_quat_normalisation_dropped", "sg_oracle.c", "g_q[i] += (gqh[i] - qh[i] * dot) / qn;",
     "g_q[i] += gqh[i] / qn;"),
    ("bwd_rotation_adjoint_sign", "sg_oracle.c", "double gw = 2 * (-z * gR[1]", "double gw = 2 * (z * gR[1]"),
    ("bwd_log_scale_index_transposed", "sg_oracle.c", "s += gM[3 * i + j] * R[3 * i + j] * e;",
     "s += gM[3 * j + i] * R[3 * i + j] * e;"),
    ("bwd_mean_rotation_transposed", "sg_oracle.c",
     "/* t = W mu + t_cw */\n    for (int j = 0; j < 3; ++j) g_mean[j] += W[j] * gt[0] + W[3 + j] * gt[1] + W[6 + j] * gt[2];",
     "/* t = W mu + t_cw */\n    for (int j = 0; j < 3; ++j) g_mean[j] += W[3 * j] * gt[0] + W[3 * j + 1] * gt[1] + W[3 * j + 2] * gt[2];"),
    ("bwd_depth_channel_dropped", "sg_oracle.c", "gt[2] += -gu * fx * t[0] / tz2 - gv * fy * t[1] / tz2 + gd;",
     "gt[2] += -gu * fx * t[0] / tz2 - gv * fy * t[1] / tz2;"),
    ("bwd_colour_weight_alpha_only", "sg_oracle.c", "grgb[3 * (size_t)c->id + ch] += w * g[ch];",
     "grgb[3 * (size_t)c->id + ch] += al * g[ch];"),
    ("bwd_gradient_through_clamp", "sg_oracle.c", "if (c->raw >= cfg.alpha_max) continue;",
     "if (c->raw >= 1e30) continue;"),
    ("bwd_isotropic_radius_chain", "sg_oracle.c", "g_ls[0] += gr * r;", "g_ls[0] += gr;"),
    ("bwd_background_suffix_dropped", "sg_oracle.c", "A[ch] = ch < 3 ? cfg.bg[ch] : 0.0;", "A[ch] = 0.0;"),
    ("bwd_dopacity_missing_G", "sg_oracle.c", "double go = dalpha * c->G;", "double go = dalpha;"),
    ("bwd_semantic_channel_offset", "sg_oracle.c", "gsem[(size_t)C * c->id + ch] += w * g[4 + ch];",
     "gsem[(size_t)C * c->id + ch] += w * g[3 + ch];"),
    ("bwd_clamped_jacobian_y_sign", "sg_oracle.c", "gt[2] += gJ[5] * (-J[5] / tz);", "gt[2] += gJ[5] * (J[5] / tz);"),
    ("bwd_unclamped_y_wrong_coordinate", "sg_oracle.c", "gt[2] += gJ[5] * (2.0 * fy * t[1] / tz3);",
     "gt[2] += gJ[5] * (2.0 * fy * t[0] / tz3);"),
    ("bwd_isotropic_depth_uses_fx_for_y", "sg_oracle.c", "- gS11 * 2.0 * fy * fy * r * r / tz3",
     "- gS11 * 2.0 * fx * fx * r * r / tz3"),
    ("bwd_conic_inverse_wrong_entry", "sg_oracle.c", "double gS00 = -(a * a * ga + a * b * gb + b * b * gc);",
     "double gS00 = -(a * a * ga + a * b * gb + b * c * gc);"),
    ("bwd_symmetric_gradient_not_halved", "sg_oracle.c", "double G[4] = {gS00, 0.5 * gS01, 0.5 * gS01, gS11};",
     "double G[4] = {gS00, gS01, gS01, gS11};"),
    ("bwd_dconic_a_factor", "sg_oracle.c", "gsig * 0.5 * dx * dx,", "gsig * dx * dx,"),
    ("bwd_isotropic_v_uses_fx", "sg_oracle.c", "double gt[3] = {gu * fx / tz, gv * fy / tz,",
     "double gt[3] = {gu * fx / tz, gv * fx / tz,"),
    ("bwd_dalpha_sign", "sg_oracle.c", "dalpha += g[ch] * (f[ch] - A[ch]);", "dalpha += g[ch] * (A[ch] - f[ch]);"),
    # ---- SSIM (Eq. 10, 12) ----
    ("ssim_C1_for_C2", "sg_oracle.c", "A2 = 2 * sxy + C2;", "A2 = 2 * sxy + C1;"),
    ("ssim_window_sigma", "sg_oracle.c", "/ (2.0 * 1.5 * 1.5));", "/ (2.0 * 1.5));"),
    ("ssim_covariance_mx_mx", "sg_oracle.c", "sxy = exy - mx * my;", "sxy = exy - mx * mx;"),
    ("ssim_adjoint_factor_two", "sg_oracle.c", "Gd[o] = a + 2.0 * X[o] * bq + Y[o] * cr;",
     "Gd[o] = a + X[o] * bq + Y[o] * cr;"),
    ("ssim_dmu_term_dropped", "sg_oracle.c", "double ds_dmx = 2 * my * A2 / (B1 * B2) - ss * 2 * mx / B1;",
     "double ds_dmx = 2 * my * A2 / (B1 * B2);"),
    ("ssim_mean_over_one_channel", "sg_oracle.c", "double norm = 1.0 / ((double)nch * (double)P);",
     "double norm = 1.0 / (double)P;"),
    ("ssim_window_product_index", "sg_oracle.c", "double w = g1[i + 5] * g1[j + 5];\n                        double xv",
     "double w = g1[i + 5] * g1[i + 5];\n                        double xv"),
    ("ssim_replicate_padding", "sg_oracle.c",
     "                        int cc = q + j;\n                        if (cc < 0 || cc >= W) continue;\n                        double w = g1[i + 5] * g1[j + 5];\n                        double xv",
     "                        int cc = q + j;\n                        if (cc < 0 || cc >= W) cc = cc < 0 ? 0 : W - 1;\n                        double w = g1[i + 5] * g1[j + 5];\n                        double xv"),
    # ---- pyramid (Eq. 4-6) ----
    ("pyr_principal_point_no_half_pixel", "__init__.py", 'cx=(p["cx"] - 0.5) / 2,', 'cx=p["cx"] / 2,'),
    ("pyr_depth_mean_over_invalid", "__init__.py", "(d * valid).sum(axis=(1, 3)) / np.maximum(cnt, 1)",
     "(d * valid).sum(axis=(1, 3)) / 4"),
    ("pyr_label_ties_to_highest", "__init__.py", "if cc > bc:", "if cc >= bc:"),
    ("pyr_subsample_instead_of_mean", "__init__.py", "rgb2 = r.mean(axis=(2, 4))", "rgb2 = r[:, :, 0, :, 0]"),
    ("pyr_size_rounds_up", "__init__.py", 'W=p["W"] // 2,', 'W=(p["W"] + 1) // 2,'),
    ("pyr_label_ties_sorted_descending", "__init__.py", "for v in sorted(set(vals)):", "for v in sorted(set(vals), reverse=True):"),
    # ---- losses (Eq. 10-13) ----
    ("loss_ssim_not_dissimilarity", "__init__.py", "L_r = (1 - lambda_r) * lr + lambda_r * (1 - s_val)",
     "L_r = (1 - lambda_r) * lr + lambda_r * s_val"),
    ("loss_ce_gradient_without_softmax", "__init__.py", "grad = e / ssum", "grad = e"),
    ("loss_depth_unmasked", "__init__.py", "ld, g_d = l1(r_depth, gt_depth, mask=np.asarray(gt_depth) > 0)",
     "ld, g_d = l1(r_depth, gt_depth)"),
    ("loss_paper_mode_uses_lambda_r", "__init__.py", "L_s = w_sem * ((1 - lambda_s) * ls + lambda_s * (1 - ss))",
     "L_s = w_sem * ((1 - lambda_r) * ls + lambda_r * (1 - ss))"),
    ("loss_decoder_gradient_unweighted", "__init__.py", 'grads["decoder"] = w_sem * np.einsum(',
     'grads["decoder"] = np.einsum('),
    ("loss_depth_weight_missing_in_value", "__init__.py", "L_d = w_depth * ld", "L_d = ld"),
    ("loss_rgb_ssim_gradient_sign", "__init__.py", "g_rgb = (1 - lambda_r) * g_l1 - lambda_r * g_s",
     "g_rgb = (1 - lambda_r) * g_l1 + lambda_r * g_s"),
    ("loss_ce_label_zero_ignored", "__init__.py", "valid = lab >= 0", "valid = lab > 0"),
    ("loss_ce_without_max_shift_in_log", "__init__.py", "logp = z - zmax - np.log(ssum)", "logp = z - np.log(ssum)"),
    ("loss_l1_mask_count", "__init__.py", "n = int(mask.sum())", "n = mask.size"),
    # ---- SH colour and semantic features (Sec. III-B) ----
    ("sh_l1_without_condon_shortley", "__init__.py", "out += [-c1 * y, c1 * z, -c1 * x]",
     "out += [c1 * y, c1 * z, c1 * x]"),
    ("sh_l2_m0_polynomial", "__init__.py", "b * (2 * z * z - x * x - y * y), -a * x * z",
     "b * (3 * z * z - x * x - y * y), -a * x * z"),
    ("sh_basis_gradient_entry", "__init__.py", "(-2 * b * x, -2 * b * y, 4 * b * z)",
     "(-2 * b * x, -2 * b * y, 2 * b * z)"),
    ("sh_camera_centre_untransposed", "__init__.py", 'c = -R.T @ np.asarray(cam["t_cw"]',
     'c = -R @ np.asarray(cam["t_cw"]'),
    ("sh_mean_gradient_not_tangent", "__init__.py", "gdir -= sh_d * (gdir * sh_d).sum(1, keepdims=True)",
     "gdir = gdir + 0.0"),
    ("sh_l3_gradient_entry", "__init__.py", "(f * y * z, f * x * z, f * x * y)", "(f * y * z, f * x * z, f * x * z)"),
    ("sh_mean_gradient_not_divided_by_distance", "__init__.py", 'out["mean"] += gdir / sh_n[:, None]',
     'out["mean"] += gdir'),
    ("sh_adjoint_overwrites_colour_part", "__init__.py", "w += np.einsum(\"nkc,nc->nk\"", "w = w * 0 + np.einsum(\"nkc,nc->nk\""),
    ("sh_l3_constant", "__init__.py", "e, f, h = np.sqrt(35 / (2 * pi)) / 4, np.sqrt(105 / pi) / 2, np.sqrt(21 / (2 * pi)) / 4\n        k, m = np.sqrt(7 / pi) / 4, np.sqrt(105 / pi) / 4\n        out",
     "e, f, h = np.sqrt(35 / (2 * pi)) / 4, np.sqrt(105 / pi) / 2, np.sqrt(21 / (2 * pi)) / 4\n        k, m = np.sqrt(7 / pi) / 2, np.sqrt(105 / pi) / 4\n        out"),
    ("sh_direction_not_unit", "__init__.py", "    d = v / n[:, None]\n    return d, n, sh_basis(d, D)",
     "    d = v\n    return d, n, sh_basis(d, D)"),
    # ---- tile lists ----
    ("tiles_record_before_depth", "__init__.py", "order = np.lexsort((recs, dbits, tiles))",
     "order = np.lexsort((dbits, recs, tiles))"),
    ("tile_reach_cross_term_halved", "__init__.py", "sig = 0.5 * (a[:, None] * dx * dx + c[:, None] * dy * dy) + b[:, None] * dx * dy",
     "sig = 0.5 * (a[:, None] * dx * dx + c[:, None] * dy * dy) + 0.5 * b[:, None] * dx * dy"),
    ("tile_reach_last_pixel_column_dropped", "__init__.py", "inside = (xs <= X1[:, None])", "inside = (xs < X1[:, None])"),
    ("tile_reach_edge_minimum_unclamped", "__init__.py", "best = np.minimum(best, q(x, np.clip(-B * x / C, y0, y1)))",
     "best = np.minimum(best, q(x, -B * x / C))"),
    ("tile_pairs_y_extent_from_x", "__init__.py", 'u, v, ex, ey = p[i, P["U"]], p[i, P["V"]], p[i, P["EXTX"]], p[i, P["EXTY"]]',
     'u, v, ex, ey = p[i, P["U"]], p[i, P["V"]], p[i, P["EXTX"]], p[i, P["EXTX"]]'),
    ("tiles_rectangle_row_past_end", "__init__.py", "for ty in range(ty0, ty1):", "for ty in range(ty0, ty1 + 1):"),
    ("tiles_view_offset_ignored", "__init__.py", "tiles.append(tile_offset[v] + ty * n_tiles_x[v] + tx)",
     "tiles.append(tile_offset[0] + ty * n_tiles_x[v] + tx)"),
    ("tiles_row_width_of_first_view", "__init__.py", "tiles.append(tile_offset[v] + ty * n_tiles_x[v] + tx)",
     "tiles.append(tile_offset[v] + ty * n_tiles_x[0] + tx)"),
    ("tiles_empty_range_not_zeroed", "__init__.py", "        ranges[empty] = 0\n", "        pass\n"),
    # ---- insertion: heuristic initializer, patch features, network outputs ----
    ("init_mean_rotation_untransposed", "init.py", "mean = (pc - t) @ R            # rows: R^T (p - t)",
     "mean = (pc - t) @ R.T"),
    ("init_backprojection_fx_for_y", "init.py", "(ys - cam[\"cy\"]) / cam[\"fy\"] * D, D], 1)",
     "(ys - cam[\"cy\"]) / cam[\"fx\"] * D, D], 1)"),
    ("init_scale_not_one_pixel", "init.py", "ls = np.log(D / cam[\"fx\"])", "ls = np.log(D)"),
    ("patch_neighbours_column_major", "init.py", "x = x0 + n % PATCH - PATCH // 2\n            y = y0 + n // PATCH - PATCH // 2",
     "x = x0 + n // PATCH - PATCH // 2\n            y = y0 + n % PATCH - PATCH // 2"),
    ("patch_ray_not_normalised", "init.py", "f[36:39] = ray / np.linalg.norm(ray)", "f[36:39] = ray"),
    ("patch_label_offset", "init.py", "f[4 + int(label[y, x])] = 1.0", "f[3 + int(label[y, x])] = 1.0"),
    ("apply_sem_offset", "init.py", "sem[:, :n] = V[:, 4:4 + n]", "sem[:, :n] = V[:, 3:3 + n]"),
    # ---- learned-initializer MLP ----
    ("mlp_relu_mask_wrong_layer", "mlp.py", "dH1 = r((dH2 @ W2) * (H1 > 0))", "dH1 = r((dH2 @ W2) * (H2 > 0))"),
    ("mlp_weight_gradient_transposed", "mlp.py", "W2=dH2.T @ H1", "W2=H1.T @ dH2"),
    ("mlp_second_layer_weight_transposed", "mlp.py", "H2 = r(np.maximum(H1 @ W2.T + b2, 0.0))",
     "H2 = r(np.maximum(H1 @ W2 + b2, 0.0))"),
    ("mlp_bias_after_relu", "mlp.py", "H1 = r(np.maximum(X @ W1.T + b1, 0.0))", "H1 = r(np.maximum(X @ W1.T, 0.0) + b1)"),
    ("mlp_loss_normalised_per_output", "mlp.py", "L = float((w[None] * (Y - T) ** 2).sum() / B)",
     "L = float((w[None] * (Y - T) ** 2).sum() / (B * Y.shape[1]))"),
    ("mlp_loss_weight_missing_in_gradient", "mlp.py", "dY = r(2.0 * w[None] * (Y - T) / B)",
     "dY = r(2.0 * (Y - T) / B)"),
]

PIN_FILES = sorted(f for f in os.listdir(os.path.join(ROOT, "tests"))
                   if f.startswith("test_oracle_") and f.endswith(".py") and f != os.path.basename(__file__))


def _copy_tree(dst):
    """The oracle, the seeded generators, the pin tests and their configuration."""
    for sub, names in (("oracle", ["__init__.py", "mlp.py", "init.py", "sg_oracle.c"]),
                       ("synthetic", ["__init__.py"]),
                       ("tests", ["conftest.py", "helpers.py"] + PIN_FILES)):
        os.makedirs(os.path.join(dst, sub), exist_ok=True)
        for n in names:
            shutil.copyfile(os.path.join(ROOT, sub, n), os.path.join(dst, sub, n))
    shutil.copyfile(os.path.join(ROOT, "pytest.ini"), os.path.join(dst, "pytest.ini"))


def _run_mutant(base, mutant):
    mid, fname, old, new = mutant
    work = os.path.join(base, mid)
    _copy_tree(work)
    path = os.path.join(work, "oracle", fname)
    src = open(path).read()
    if src.count(old) != 1:
        return mid, "bad", f"original text occurs {src.count(old)} times in {fname}"
    open(path, "w").write(src.replace(old, new))
    if fname.endswith(".c"):  # the mutant must still compile: a build error is no catch
        cp = subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
                             "-ffp-contract=off", path, "-o", os.path.join(work, "oracle", "libsg_oracle.so"),
                             "-lm"], capture_output=True, text=True)
        if cp.returncode:
            return mid, "bad", "mutant does not compile:\n" + cp.stderr[-2000:]
    env = {k: v for k, v in os.environ.items() if k not in ("PYTHONPATH",)}
    env["OMP_NUM_THREADS"] = "1"
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-rfE", "-p", "no:cacheprovider", "-m", "not gpu",
           *[os.path.join("tests", f) for f in PIN_FILES]]
    pr = subprocess.run(cmd, cwd=work, env=env, capture_output=True, text=True, timeout=900)
    out = pr.stdout[-3000:] + pr.stderr[-1000:]
    if pr.returncode == 0:
        return mid, "survived", out
    failed = [ln for ln in pr.stdout.splitlines() if ln.startswith("FAILED ")]
    if pr.returncode == 1 and failed and not any(ln.startswith("ERROR ") for ln in pr.stdout.splitlines()):
        return mid, "caught", failed[0]
    return mid, "bad", out


@pytest.fixture(scope="module")
def mutant_results(tmp_path_factory):
    base = str(tmp_path_factory.mktemp("oracle_mutants"))
    workers = max(1, min(len(MUTANTS), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        res = list(ex.map(lambda m: _run_mutant(base, m), MUTANTS))
    return {mid: (status, detail) for mid, status, detail in res}


def test_pin_files_found():
    assert {"test_oracle_projection.py", "test_oracle_render.py", "test_oracle_backward.py",
            "test_oracle_loss.py", "test_oracle_pyramid_tiles.py", "test_oracle_sh.py",
            "test_oracle_mlp.py"} <= set(PIN_FILES)


@pytest.mark.parametrize("mid", [m[0] for m in MUTANTS])
def test_some_pin_catches_mutant(mutant_results, mid):
    status, detail = mutant_results[mid]
    assert status == "caught", f"{mid}: {status}\n{detail}"
