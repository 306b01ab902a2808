"""Planted mistakes: checks of the oracle's pins, not of the oracle.

Each entry copies the oracle with one plausible slip -- a dropped factor, a
flipped sign, a swapped operand, an off-by-one, a wrong tie rule -- builds
(C++) or loads (Python) that copy on the CPU, and runs the pins named beside
it in a fresh interpreter.  An entry passes when those pins FAIL: every slip
listed here must be caught by at least one check that is independent of the
oracle's own formulas (a closed form, a limit, a textbook special case, a
published value, finite differences, brute force).  The oracle itself is
never touched; the copies live in pytest's temporary directory, and a control
copy without a slip must pass the same pins.  CPU only."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")
CPP = "nrt_oracle.cpp"

T_GEO = "tests/test_oracle_geometry.py"
T_EM = "tests/test_oracle_em.py"
T_PATHS = "tests/test_oracle_paths.py"
T_LAB = "tests/test_oracle_labels.py"
T_POL = "tests/test_oracle_polarisation.py"
T_DIF = "tests/test_oracle_diffraction.py"
T_SDF = "tests/test_oracle_sdf.py"
T_CFR = "tests/test_oracle_cfr.py"
T_MLP = "tests/test_oracle_mlp.py"

# (name, file, original text, planted text, pins expected to notice)
MUTANTS = [
    # Sec. II-C: ray/disc intersection, Eq. 3 / Eq. 4
    ("eq3_gaussian_width", CPP, "std::exp(-e.r * e.r / (2.0 * rp * rp)) * std::exp(",
     "std::exp(-e.r * e.r / (rp * rp)) * std::exp(", [f"{T_GEO}::test_gaussian_weight_closed_form"]),
    ("eq4_depth_factor_dropped", CPP,
     "double w = std::exp(-e.r * e.r / (2.0 * rp * rp)) * std::exp(-S.lambda_d * norm(e.q - qmin));",
     "double w = std::exp(-e.r * e.r / (2.0 * rp * rp));",
     [f"{T_GEO}::test_depth_attenuation_closed_form"]),
    ("normal_not_turned_to_the_ray", CPP, "if (dot(h.n, d) > 0) h.n = -1.0 * h.n;",
     "if (dot(h.n, d) < 0) h.n = -1.0 * h.n;", [f"{T_GEO}::test_single_disc_hit_and_miss"]),
    ("tie_rule_larger_index", CPP, "(e.t == best_t && i < best_i)", "(e.t == best_t && i > best_i)",
     [f"{T_GEO}::test_tie_rule_smaller_index"]),
    ("disc_radius_doubled", CPP, "if (e.t > cfg.t_min && e.t < t_max && e.r <= rp) {",
     "if (e.t > cfg.t_min && e.t < t_max && e.r <= 2.0 * rp) {",
     [f"{T_GEO}::test_single_disc_hit_and_miss"]),
    ("eq3_point_unweighted", CPP, "    sq = sq + w * e.q;", "    sq = sq + e.q;",
     [f"{T_GEO}::test_depth_attenuation_closed_form"]),
    ("eq3_normal_unweighted", CPP, "    sn = sn + w * S.N[i];\n  }\n  h.q = (1.0 / sw) * sq;",
     "    sn = sn + S.N[i];\n  }\n  h.q = (1.0 / sw) * sq;",
     [f"{T_GEO}::test_gaussian_weight_closed_form"]),
    ("incidence_cosine_from_z", CPP, "  h.cos_in = std::fabs(dot(d, h.n));",
     "  h.cos_in = std::fabs(d.z);",
     [f"{T_EM}::test_diffuse_power_off_a_plane_is_the_lambertian_integral"]),
    # Sec. II-A voxelisation, Sec. II-B launch
    ("voxel_rounded_not_floored", CPP, "return (int)std::floor((float)s);",
     "return (int)std::lround((float)s);", [f"{T_GEO}::test_voxelisation_matches_float32_floor"]),
    ("fibonacci_half_offset_dropped", CPP, "double a = (2.0 * (double)i + 1.0) / (double)n;",
     "double a = (2.0 * (double)i) / (double)n;", [f"{T_GEO}::test_fibonacci_directions"]),
    ("fibonacci_half_turn", CPP, "double phi = 2.0 * kPi * std::ldexp((double)u, -64);",
     "double phi = kPi * std::ldexp((double)u, -64);", [f"{T_GEO}::test_fibonacci_directions"]),
    # Sec. II-B: continuation, visibility, capture, dedup
    ("dps_launch_not_in_morton_order", CPP,
     "  if (sim.p.launch == 1) return unit(sim.S->recv[sim.S->dps_morton[rid]] - sim.tx);",
     "  if (sim.p.launch == 1) return unit(sim.S->recv[rid] - sim.tx);",
     [f"{T_GEO}::test_dps_directed_launch_hits_its_target_dps"]),
    ("continuation_projects_not_mirrors", CPP,
     "d = d - 2.0 * dot(d, h.n) * h.n;  // specular continuation",
     "d = d - dot(d, h.n) * h.n;  // specular continuation",
     [f"{T_PATHS}::test_shoebox_image_sources"]),
    ("visibility_cast_to_the_centre", CPP, "double t_max = s - rx_margin(S);", "double t_max = s;",
     [f"{T_PATHS}::test_rough_wall_fully_visible_from_the_front"]),
    ("receiver_inside_a_dps_sees_nothing", CPP, "  if (t_max <= cfg.t_min) return {true,",
     "  if (t_max <= cfg.t_min) return {false,",
     [f"{T_PATHS}::test_rough_wall_fully_visible_from_the_front"]),
    ("dedup_highest_ray_first", CPP, "return a.ray < b.ray;", "return a.ray > b.ray;",
     [f"{T_LAB}::test_dedup_tries_lowest_ray_ids_first"]),
    ("dedup_one_try", CPP,
     "sim.p.rep_tries > 0 ? std::min<int64_t>(cl.size(), sim.p.rep_tries) : (int64_t)cl.size();",
     "std::min<int64_t>(cl.size(), 1);", [f"{T_LAB}::test_dedup_tries_lowest_ray_ids_first"]),
    ("dedup_cap_ignored", CPP,
     "sim.p.rep_tries > 0 ? std::min<int64_t>(cl.size(), sim.p.rep_tries) : (int64_t)cl.size();",
     "(int64_t)cl.size();", [f"{T_LAB}::test_dedup_tries_lowest_ray_ids_first"]),
    ("dedup_uncapped_stops_at_8", CPP,
     "sim.p.rep_tries > 0 ? std::min<int64_t>(cl.size(), sim.p.rep_tries) : (int64_t)cl.size();",
     "std::min<int64_t>(cl.size(), sim.p.rep_tries > 0 ? sim.p.rep_tries : 8);",
     [f"{T_LAB}::test_dedup_tries_lowest_ray_ids_first"]),
    # Sec. II-B-1 diffuse, Sec. II-B-2 specular refinement (Eq. 1)
    ("diffuse_accepts_rx_behind", CPP, "if (cs <= 0.0) return v;", "if (cs < -1.0) return v;",
     [f"{T_PATHS}::test_adjoint_matches_central_differences"]),
    ("image_source_not_mirrored", CPP,
     "img[m + 1] = img[m] - 2.0 * dot(img[m] - Pp[m], Pn[m]) * Pn[m];",
     "img[m + 1] = img[m] - dot(img[m] - Pp[m], Pn[m]) * Pn[m];",
     [f"{T_PATHS}::test_shoebox_image_sources"]),
    ("refinement_accepts_either_criterion", CPP, "if (!(c >= cos_ta && dist <= sim.p.t_d)) {",
     "if (!(c >= cos_ta || dist <= sim.p.t_d)) {",
     [f"{T_PATHS}::test_refinement_converges_on_a_cylinder"]),
    ("refinement_never_retries", CPP, "if (attempt == sim.p.kappa) return v;",
     "if (attempt == 0) return v;", [f"{T_PATHS}::test_refinement_converges_on_a_cylinder"]),
    ("side_check_dropped", CPP, "if (!(a * b > 0.0)) return v;", "if (false) return v;",
     [f"{T_PATHS}::test_valid_paths_are_physical"]),
    ("last_leg_unchecked", CPP, "if (hf.hit) return v;", "if (false) return v;",
     [f"{T_PATHS}::test_valid_paths_are_physical"]),
    ("surface_label_unchecked", CPP, "if (!h.hit || S.surf[h.idx] != labels[m - 1]) {",
     "if (!h.hit) {", [f"{T_PATHS}::test_valid_paths_are_physical"]),
    ("diffuse_shadow_unchecked", CPP,
     "  Hit h = cast(S, hk.q, w, hk.dps, rs, false, cfg);\n  if (h.amb) v.amb = true;\n  if (h.hit) return v;",
     "  Hit h = cast(S, hk.q, w, hk.dps, rs, false, cfg);\n  if (h.amb) v.amb = true;",
     [f"{T_PATHS}::test_valid_paths_are_physical"]),
    ("diffuse_length_last_segment", CPP, "ri += hm.t;", "ri = hm.t;",
     [f"{T_PATHS}::test_valid_paths_are_physical"]),
    ("capture_before_segment_start", CPP, "ts = std::min(std::max(ts, 0.0), t_end);",
     "ts = std::min(ts, t_end);", [f"{T_LAB}::test_capture_stops_at_the_segment_ends"]),
    ("capture_past_segment_end", CPP, "ts = std::min(std::max(ts, 0.0), t_end);",
     "ts = std::max(ts, 0.0);", [f"{T_LAB}::test_capture_stops_at_the_segment_ends"]),
    ("hits_below_t_min", CPP, "if (e.t > cfg.t_min && e.t < t_max && e.r <= rp) {",
     "if (e.t > 0.0 && e.t < t_max && e.r <= rp) {", [f"{T_GEO}::test_single_disc_hit_and_miss"]),
    # EM readings
    ("fresnel_te_sign", CPP, "if (pol == 0) return (cos_t - s) / (cos_t + s);",
     "if (pol == 0) return (s - cos_t) / (cos_t + s);", [T_EM]),
    ("fresnel_tm_form", CPP, "return (eta * cos_t - s) / (eta * cos_t + s);",
     "return (cos_t - eta * s) / (cos_t + eta * s);", [f"{T_EM}::test_brewster_zero_lossless_tm"]),
    ("permittivity_loss_sign", CPP, "return cd(eps_r, -sigma / (2.0 * kPi * f * kEps0));",
     "return cd(eps_r, sigma / (2.0 * kPi * f * kEps0));", [T_EM]),
    ("fresnel_derivative_sign", CPP, "return -cos_t / (s * den * den);",
     "return cos_t / (s * den * den);", [f"{T_EM}::test_fresnel_derivative_complex_step"]),
    ("fresnel_tm_derivative", CPP, "return cos_t * (eta - 2.0 * sin2) / (s * den * den);",
     "return cos_t * (eta - sin2) / (s * den * den);",
     [f"{T_EM}::test_fresnel_derivative_complex_step"]),
    ("los_delay_doubled", CPP, "P.tau = d / kC0;", "P.tau = 2.0 * d / kC0;",
     [f"{T_EM}::test_los_amplitude_and_delay"]),
    ("specular_delay_halved", CPP, "P.tau = len / kC0;", "P.tau = 0.5 * len / kC0;",
     [f"{T_PATHS}::test_shoebox_image_sources"]),
    ("los_two_pi", CPP, "P.geo = lam / (4.0 * kPi * d);", "P.geo = lam / (2.0 * kPi * d);",
     [f"{T_EM}::test_los_amplitude_and_delay"]),
    ("specular_spreading_squared", CPP, "P.geo = lam / (4.0 * kPi * len);",
     "P.geo = lam / (4.0 * kPi * len * len);", [f"{T_PATHS}::test_single_wall_amplitude_snell_form"]),
    ("diffuse_incidence_cosine_dropped", CPP, "std::sqrt(S.rho * S.rho * hk.cos_in * cs / kPi)",
     "std::sqrt(S.rho * S.rho * cs / kPi)",
     [f"{T_EM}::test_diffuse_power_off_a_plane_is_the_lambertian_integral"]),
    ("roughness_not_energy_conserving", CPP,
     "double f = last_diffuse ? sca[l] : std::sqrt(std::max(0.0, 1.0 - sca[l] * sca[l]));",
     "double f = last_diffuse ? sca[l] : 1.0 - sca[l];",
     [f"{T_PATHS}::test_adjoint_matches_central_differences"]),
    # Sec. III-B adjoint
    ("adjoint_roughness_sign", CPP, "dc[m] = last_diffuse ? 1.0 : (R > 0.0 ? -sca[l] / R : 0.0);",
     "dc[m] = last_diffuse ? 1.0 : (R > 0.0 ? sca[l] / R : 0.0);",
     [f"{T_PATHS}::test_adjoint_matches_central_differences"]),
    ("adjoint_factor_dropped", CPP, "da_deta[m] = others * (c[m] * dG[m][0]);",
     "da_deta[m] = others * dG[m][0];", [f"{T_PATHS}::test_adjoint_matches_central_differences"]),
    # vector polarisation
    ("theta_hat_sign", CPP, "return {d.z * d.x / st, d.z * d.y / st, -st};",
     "return {d.z * d.x / st, d.z * d.y / st, st};", [f"{T_POL}::test_floor_reflection_is_tm"]),
    ("p_basis_handedness", CPP, "pout[m] = cross(sv[m], d[m + 1]);",
     "pout[m] = cross(d[m + 1], sv[m]);", [f"{T_POL}::test_floor_reflection_is_tm"]),
    ("jones_e0_basis", CPP, "J.e0[1] = dot(t0, pin[0]);", "J.e0[1] = dot(t0, pout[0]);", [T_POL]),
    ("jones_basis_change_transposed", CPP, "J.B[m][0][1] = dot(sv[m + 1], pout[m]);",
     "J.B[m][0][1] = dot(pin[m + 1], sv[m]);", [T_POL]),
    ("jones_rx_basis", CPP, "J.r[1] = dot(tr, pout[k - 1]);", "J.r[1] = dot(tr, pin[k - 1]);", [T_POL]),
    ("jones_partial_forward_index", CPP, "    dA[m][0] = w[0] * fwd[m][0];",
     "    dA[m][0] = w[1] * fwd[m][0];", [T_POL]),
    ("jones_partial_backward_transpose", CPP,
     "      w[0] = u0 * J.B[m - 1][0][0] + u1 * J.B[m - 1][1][0];",
     "      w[0] = u0 * J.B[m - 1][0][0] + u1 * J.B[m - 1][0][1];", [T_POL]),
    # Sec. II-B-3 edge diffraction
    ("utd_constant_sign", CPP, "const cd K = -std::exp(cd(0.0, -kPi / 4.0)) / (2.0 * nw",
     "const cd K = std::exp(cd(0.0, -kPi / 4.0)) / (2.0 * nw",
     [f"{T_DIF}::test_half_plane_pec_matches_the_textbook_form"]),
    ("utd_cot_argument", CPP, "const cd T3 = cot((kPi - bp) / (2.0 * nw))",
     "const cd T3 = cot((kPi + bp) / (2.0 * nw))",
     [f"{T_DIF}::test_half_plane_pec_matches_the_textbook_form"]),
    ("transition_function_phase", CPP,
     "0.5 * std::sqrt(kPi) * std::exp(cd(0.0, -kPi / 4.0)) - acc;",
     "0.5 * std::sqrt(kPi) * std::exp(cd(0.0, kPi / 4.0)) - acc;",
     [f"{T_DIF}::test_transition_function_limits"]),
    ("diffraction_point_weights_swapped", CPP, "G.tpar = (at * br + ar * bt) / (bt + br);",
     "G.tpar = (at * bt + ar * br) / (bt + br);",
     [f"{T_DIF}::test_keller_point_minimises_the_path_length"]),
    ("distance_parameter_sin2_dropped", CPP,
     "const double L = G.s_in * G.s_out * G.sinb * G.sinb / (G.s_in + G.s_out);",
     "const double L = G.s_in * G.s_out / (G.s_in + G.s_out);",
     [f"{T_DIF}::test_half_plane_pec_matches_the_textbook_form"]),
    ("diffraction_spreading", CPP,
     "const double geo = lam / (4.0 * kPi * std::sqrt(G.s_in * G.s_out * (G.s_in + G.s_out)));",
     "const double geo = lam / (4.0 * kPi * (G.s_in + G.s_out));",
     [f"{T_DIF}::test_half_plane_pec_matches_the_textbook_form"]),
    ("face_n_incidence_angle", CPP, "c1 = G.sinb * std::sin(W.nw * kPi - G.phi_out);",
     "c1 = G.sinb * std::sin(G.phi_out);", [f"{T_DIF}::test_grazing_face_material_drops_out"]),
    ("face_0_incidence_angle", CPP, "const double c0 = G.sinb * std::sin(G.phi_in),",
     "const double c0 = G.sinb * std::sin(G.phi_out),",
     [f"{T_DIF}::test_grazing_face_material_drops_out"]),
    ("diffraction_visibility_unchecked", CPP, "      if (h.hit) vis = false;", "      (void)h;",
     [f"{T_DIF}::test_diffraction_point_must_see_tx_and_rx"]),
    ("transition_asymptote_sign", CPP, "term *= -(2.0 * n - 1.0) / (cd(0.0, 2.0 * x));",
     "term *= (2.0 * n - 1.0) / (cd(0.0, 2.0 * x));", [T_DIF]),
    ("exterior_angle_sign", CPP, "W.nw = 2.0 - std::acos", "W.nw = 2.0 + std::acos",
     [f"{T_DIF}::test_exterior_angle_closed_forms"]),
    ("transition_index_floored", CPP,
     "const double N = std::round((beta + sgn * kPi) / (2.0 * kPi * nw));",
     "const double N = std::floor((beta + sgn * kPi) / (2.0 * kPi * nw));", [T_DIF]),
    # Eq. 2 SDF (ablation)
    ("sdf_sign", CPP, "sf += w * dot(S->N[i], v);", "sf -= w * dot(S->N[i], v);",
     [f"{T_SDF}::test_single_point_gives_its_tangent_plane"]),
    ("sdf_label_of_the_farthest_point", CPP, "if (dd < dmin || (dd == dmin && i < lab)) {",
     "if (dd > dmin || dmin == kInf) {", [f"{T_SDF}::test_label_is_the_nearest_points"]),
    ("sdf_kernel_width", CPP, "inv2s2 = 1.0 / (2.0 * sigma * sigma);", "inv2s2 = 1.0 / (sigma * sigma);",
     [f"{T_SDF}::test_planar_faces_are_hit_exactly"]),
    ("sdf_defined_region", CPP, "const double wmin = std::exp(-2.0),",
     "const double wmin = std::exp(-4.0),", [f"{T_SDF}::test_single_point_gives_its_tangent_plane"]),
    # CFR and Eq. 5 (Python)
    ("cfr_phase_sign", "cfr.py", "np.exp(-2j * np.pi * tau[m, None] * f[None, :])",
     "np.exp(2j * np.pi * tau[m, None] * f[None, :])", [T_CFR]),
    ("cfr_frequency_step", "cfr.py", "return fc + k * (bandwidth / (n - 1))",
     "return fc + k * (bandwidth / n)", [f"{T_CFR}::test_frequency_grid"]),
    ("eq5_normalised_by_the_estimate", "cfr.py", "/ np.sum(np.abs(T) ** 2, axis=-1)",
     "/ np.sum(np.abs(H) ** 2, axis=-1)", [T_CFR]),
    ("eq5_gradient_factor", "cfr.py", "w = 2.0 * np.asarray(rx_weight, np.float64)[rx] / D[rx]",
     "w = 1.0 * np.asarray(rx_weight, np.float64)[rx] / D[rx]", [T_CFR]),
    ("eq5_gradient_phase", "cfr.py", "np.exp(2j * np.pi * tau[:, None] * np.asarray(f)[None, :])",
     "np.exp(-2j * np.pi * tau[:, None] * np.asarray(f)[None, :])", [T_CFR]),
    ("cir_forward_transform", "cfr.py", "return np.fft.ifft(np.asarray(H), axis=-1)",
     "return np.fft.fft(np.asarray(H), axis=-1)",
     [f"{T_CFR}::test_cir_of_one_path_is_a_delayed_impulse"]),
    # proposal network (Python)
    ("splitmix_shift", "mlp.py", "z = (z ^ (z >> np.uint64(30))) * _M1",
     "z = (z ^ (z >> np.uint64(31))) * _M1", [f"{T_MLP}::test_splitmix64_published_outputs"]),
    ("counter_off_by_one", "mlp.py", "(idx + np.uint64(1)) * GAMMA", "idx * GAMMA",
     [f"{T_MLP}::test_counter_uniform_and_gumbel_moments"]),
    ("gumbel_sign", "mlp.py", "return -np.log(-np.log(counter_uniform(seed, idx)))",
     "return np.log(-np.log(counter_uniform(seed, idx)))",
     [f"{T_MLP}::test_counter_uniform_and_gumbel_moments"]),
    ("feature_octave", "mlp.py", "a = np.pi * (2.0 ** k) * v[:, c]",
     "a = np.pi * (2.0 ** (k + 1)) * v[:, c]", [f"{T_MLP}::test_features_closed_forms"]),
    ("bf16_ties_away", "mlp.py", "r = ((b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)",
     "r = ((b + np.uint64(0x8000)) >> np.uint64(16)) << np.uint64(16)",
     [f"{T_MLP}::test_bf16_matches_torch_cast"]),
    ("relu_mask_dropped", "mlp.py", "dZ2 = r((dZ3 @ W3) * (A[\"H2\"] > 0))", "dZ2 = r(dZ3 @ W3)",
     [f"{T_MLP}::test_forward_and_gradients_match_torch_autograd"]),
    ("bce_positive_weight_dropped", "mlp.py",
     "dz = (s * (pos_weight * y + 1.0 - y) - pos_weight * y) / B", "dz = (s - y) / B",
     [f"{T_MLP}::test_forward_and_gradients_match_torch_autograd"]),
    ("adam_bias_correction_dropped", "mlp.py", "mh = m / (1.0 - b1 ** t)", "mh = m",
     [f"{T_MLP}::test_adam_matches_torch_optim"]),
    ("top_k_one_short", "mlp.py", "    k_top = min(k_top, n)", "    k_top = min(k_top, n - 1)",
     [f"{T_MLP}::test_select_structure"]),
    ("adam_epsilon_inside_the_root", "mlp.py",
     "return theta - lr * mh / (np.sqrt(vh) + eps), m, v",
     "return theta - lr * mh / np.sqrt(vh + eps), m, v", [f"{T_MLP}::test_adam_matches_torch_optim"]),
    ("selection_ties_larger_index", "mlp.py",
     "order = np.lexsort((np.arange(n), -key.astype(np.float64)))",
     "order = np.lexsort((-np.arange(n), -key.astype(np.float64)))",
     [f"{T_MLP}::test_select_structure"]),
    ("strata_reuse_the_top_k_counters", "mlp.py", "u = counter_uniform(seed, n + s)",
     "u = counter_uniform(seed, s)",
     [f"{T_MLP}::test_strata_draws_are_independent_of_the_gumbel_noise"]),
]

CONTROL_NODES = [f"{T_GEO}::test_gaussian_weight_closed_form", f"{T_CFR}::test_frequency_grid",
                 f"{T_MLP}::test_splitmix64_published_outputs"]

# Registers the oracle package from a given directory before pytest starts,
# so that every `import oracle` in the pins resolves to the copy.
_BOOT = (
    "import importlib.util, sys\n"
    "d = sys.argv[1]\n"
    "spec = importlib.util.spec_from_file_location('oracle', d + '/__init__.py',\n"
    "                                              submodule_search_locations=[d])\n"
    "m = importlib.util.module_from_spec(spec)\n"
    "sys.modules['oracle'] = m\n"
    "spec.loader.exec_module(m)\n"
    "import pytest\n"
    "sys.exit(pytest.main(sys.argv[2:]))\n")


def _run(entry, tmp, good_lib):
    name, fname, old, new, nodes = entry
    d = os.path.join(tmp, name, "oracle")
    shutil.copytree(ORACLE_DIR, d, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    path = os.path.join(d, fname)
    src = open(path).read()
    if old:
        if src.count(old) != 1:
            return -1, f"the original text occurs {src.count(old)} times in {fname}"
        open(path, "w").write(src.replace(old, new))
    lib = good_lib
    if fname == CPP and old:
        lib = os.path.join(d, "mutant.so")
        r = subprocess.run(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-fopenmp",
                            "-ffp-contract=off", "-o", lib, path], capture_output=True, text=True)
        if r.returncode:
            return -1, "compile error:\n" + r.stderr[-2000:]
    env = dict(os.environ, NRT_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-c", _BOOT, d, "-x", "-q", "-p", "no:cacheprovider",
                        "--tb=line", *nodes], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    return r.returncode, r.stdout[-3000:] + r.stderr[-1000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("mutants"))
    good = oracle.build()
    entries = MUTANTS + [("control", CPP, "", "", CONTROL_NODES)]
    with cf.ThreadPoolExecutor(max(1, (os.cpu_count() or 2) // 2)) as ex:
        futs = {e[0]: ex.submit(_run, e, tmp, good) for e in entries}
        return {k: f.result() for k, f in futs.items()}


def test_mutant_names_unique():
    names = [m[0] for m in MUTANTS]
    assert len(names) == len(set(names))


def test_unplanted_copy_passes_the_pins(outcomes):
    rc, out = outcomes["control"]
    assert rc == 0, out


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(outcomes, name):
    rc, out = outcomes[name]
    # pytest exit status 1: the pins ran and at least one failed
    assert rc == 1, out
