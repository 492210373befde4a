"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake (a dropped term, a wrong sign, a wrong index or
coefficient) in a copy of the oracle's C source, builds it in a temporary
directory and runs the pin that should catch it against that copy, in a child
process.  The pin must fail.  The real oracle is never modified.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "celeris_oracle.c")

_FS = ("fs = dd * dxd * Qy / 6.0 + dd * dyd * Qx / 6.0 + B3 * dd * dd * Qxy;\n"
       "                gs = dd * dyd * Px / 6.0 + dd * dxd * Py / 6.0 + B3 * dd * dd * Pxy;")
_ETA = ("Bd * g * dd * dd * (dxd * (2.0 * exx + eyy) + dyd * exy);\n"
        "                gg += Bd * g * dd * dd * dd * (eyyy + exxy) +\n"
        "                      Bd * g * dd * dd * (dyd * (2.0 * eyy + exx) + dxd * exy);")
_CORNER = ("        for (int i = -2; i < nx + 2; i++)\n"
           "            for (int k = 0; k < 2; k++) {\n"
           "                int gj")

MUTANTS = [
    # (name, original text, mutated text, pin that must fail)
    ("drop_Fstar", "fs = dd * dxd * Qy / 6.0 + dd * dyd * Qx / 6.0 + B3 * dd * dd * Qxy;",
     "fs = dd * dxd * Qy / 6.0 + dd * dyd * Qx / 6.0;", "test_dispersion_relation_2d_oblique"),
    ("sign_exyy", "Bd * g * dd * dd * dd * (exxx + exyy)", "Bd * g * dd * dd * dd * (exxx - exyy)",
     "test_dispersion_relation_2d_oblique"),
    ("drop_exxx", "Bd * g * dd * dd * dd * (exxx + exyy)", "Bd * g * dd * dd * dd * (exyy)",
     "test_dispersion_relation_1d"),
    ("bed_slope_sign", "g * hb * (Bx(o, i + 1, j) - Bx(o, i, j)) / dx;",
     "g * hb * (Bx(o, i, j) - Bx(o, i + 1, j)) / dx;", "test_lake_at_rest_submerged"),
    ("ab3_coef", "(23.0 * o->E[0][c] - 16.0 * o->E[1][c] + 5.0 * o->E[2][c])",
     "(23.0 * o->E[0][c] - 15.0 * o->E[1][c] + 5.0 * o->E[2][c])", "test_dispersion_relation_1d"),
    ("ab3_U_coef", "(23.0 * o->F[0][c] - 16.0 * o->F[1][c] + 5.0 * o->F[2][c])",
     "(23.0 * o->F[0][c] - 16.0 * o->F[1][c] + 4.0 * o->F[2][c])", "test_friction_quadratic_order"),
    ("am4_U_coef", "(9.0 * o->Fc[c] + 19.0 * o->F[0][c] - 5.0 * o->F[1][c] + o->F[2][c])",
     "(9.0 * o->Fc[c] + 18.0 * o->F[0][c] - 5.0 * o->F[1][c] + o->F[2][c])",
     "test_time_stepping_formulas_step_by_step"),
    ("wall_no_negate", "P[gc] = -P[sc];", "P[gc] = P[sc];", "test_mass_soliton_channel"),
    ("positivity_high_branch", "lo[0] = 2.0 * w[c] - Bhi;", "lo[0] = w[c];", "test_symmetry_mirror_x_wet_dry"),
    ("positivity_low_branch", "hi[0] = 2.0 * w[c] - Blo;", "hi[0] = w[c];", "test_symmetry_mirror_x_wet_dry"),
    ("sponge_skips_Q", "o->Q1[c] *= gam;", ";", "test_symmetry_transpose_with_sponges"),
    ("sponge_to_zero_level", "o->w1[c] = o->p.ws + gam * (o->w1[c] - o->p.ws);", "o->w1[c] = gam * o->w1[c];",
     "test_lake_at_rest_with_sponges_off_zero_level"),
    ("sine_discharge_sign", "*Pg += c * cs * em;", "*Pg -= c * cs * em;", "test_sine_maker_progressive_wave"),
    ("sine_celerity", "orc_real c = om / k;", "orc_real c = k / om;", "test_sine_maker_progressive_wave"),
    ("sine_corrector_time", "fill_ghosts(o, o->w1, o->P1, o->Q1, t1);", "fill_ghosts(o, o->w1, o->P1, o->Q1, t0);",
     "test_sine_maker_progressive_wave"),
    ("sine_predictor_time", "fill_ghosts(o, o->w, o->P, o->Q, t0);", "fill_ghosts(o, o->w, o->P, o->Q, t1);",
     "test_sine_maker_progressive_wave"),
    ("sine_line_rows_time", "solve_lines(o, 0, o->U1, o->P1, t1);", "solve_lines(o, 0, o->U1, o->P1, t0);",
     "test_sine_maker_progressive_wave"),
    ("sine_y_discharge_sign", "*Qg += c * sn * em;", "*Qg -= c * sn * em;", "test_symmetry_transpose_sine_makers"),
    ("sine_y_line_rows_time", "solve_lines(o, 1, o->V1, o->Q1, t1);", "solve_lines(o, 1, o->V1, o->Q1, t0);",
     "test_symmetry_transpose_sine_makers"),
    ("desing_sqrt2", "return sqrt(2.0) * h / sqrt(h4 + fmax(h4, eps));", "return h / sqrt(h4 + fmax(h4, eps));",
     "test_soliton_speed"),
    ("eq23_sign_s", "*a = s - r;", "*a = -s - r;", "test_symmetry_mirror_x"),
    ("eta_depth_gradient_terms", "Bd * g * dd * dd * (dxd * (2.0 * exx + eyy) + dyd * exy);", "0.0;",
     "test_linear_shoaling_on_a_slope"),
    ("depth_gradient_sign", "(o->d[IX(o, i + 1, j)] - o->d[IX(o, i - 1, j)]) / (2.0 * o->p.dx)",
     "(o->d[IX(o, i - 1, j)] - o->d[IX(o, i + 1, j)]) / (2.0 * o->p.dx)", "test_linear_shoaling_on_a_slope"),
    ("eq23_depth_gradient_dropped", "orc_real s = dd * dda / (6.0 * h);", "orc_real s = 0.0;",
     "test_linear_shoaling_on_a_slope"),
    ("tridiag_B", "*b = 1.0 + 2.0 * r;", "*b = 1.0 + r;", "test_dispersion_relation_1d"),
    ("hydrostatic_half", "FL1 = qnL * uL + 0.5 * g * hL * hL", "FL1 = qnL * uL + g * hL * hL",
     "test_lake_at_rest_submerged"),
    ("tangential_flux_side", "FL2 = qnL * vL;", "FL2 = qnL * vR;", "test_central_upwind_consistency"),
    ("flux_mass_diffusion_sign", "ap * am * (wR - wL)", "ap * am * (wL - wR)", "test_ritter_dam_break"),
    ("friction_h_power", "f -= fc * P[c] * mag * hinv * hinv;", "f -= fc * P[c] * mag * hinv;",
     "test_friction_manning_ode"),
    ("soliton_y_discharge_sign", "o->Q[c] += cs * es * st;", "o->Q[c] -= cs * es * st;",
     "test_symmetry_transpose_solitons"),
    ("soliton_ks", "sqrt(3.0 * fabs(H) / (4.0 * ds * ds * ds))", "sqrt(3.0 * fabs(H) / (2.0 * ds * ds * ds))",
     "test_soliton_speed"),
    ("eckart", "return k0 * sqrt(1.0 / tanh(k0 * d));", "return k0 * (1.0 / tanh(k0 * d));",
     "test_eckart_vs_exact_dispersion"),
    ("transpose_y_solve", "coef23(o->p.Bd, o->p.dy, o->d[c], o->ddy[c], &a, &b, &cc);",
     "coef23(o->p.Bd, o->p.dy, o->d[c], o->ddx[c], &a, &b, &cc);", "test_lake_at_rest_submerged"),
    ("runup_keeps_last", "else if (wet && o->w[c] > o->maxw[k]) o->maxw[k] = o->w[c];",
     "else if (wet) o->maxw[k] = o->w[c];", "test_runup_tracking_standing_mode"),
    ("runup_threshold_inclusive", "int wet = o->w[c] - o->Bbar[c] > o->delta;", "int wet = o->w[c] - o->Bbar[c] >= o->delta;",
     "test_runup_tracking_threshold_and_dry_land"),
    ("runup_no_threshold", "int wet = o->w[c] - o->Bbar[c] > o->delta;", "int wet = 1;",
     "test_runup_tracking_threshold_and_dry_land"),
    # depth-gradient terms that vanish in 1-D (F*, G* of Eq. 12-13; the
    # cross terms of Eq. 10-11), changed alike in both momentum equations
    # so that the transpose symmetry still holds: the isotropy pin
    ("Fstar_dxQy_dyPx_dropped", _FS, _FS.replace("dd * dxd * Qy / 6.0 + ", "").replace("dd * dyd * Px / 6.0 + ", ""),
     "test_isotropy_over_a_round_shoal"),
    ("Fstar_dyQx_dxPy_dropped", _FS, _FS.replace(" + dd * dyd * Qx / 6.0", "").replace(" + dd * dxd * Py / 6.0", ""),
     "test_isotropy_over_a_round_shoal"),
    ("Fstar_sixth_as_third", _FS, _FS.replace("/ 6.0", "/ 3.0"), "test_isotropy_over_a_round_shoal"),
    ("Fstar_dxd_dyd_swapped", "fs = dd * dxd * Qy / 6.0 + dd * dyd * Qx / 6.0",
     "fs = dd * dyd * Qy / 6.0 + dd * dxd * Qx / 6.0", "test_isotropy_over_a_round_shoal"),
    ("eta_dx_eyy_dropped", _ETA, _ETA.replace("(2.0 * exx + eyy)", "(2.0 * exx)").replace("(2.0 * eyy + exx)",
                                                                                        "(2.0 * eyy)"),
     "test_isotropy_over_a_round_shoal"),
    ("eta_dy_exy_dropped", _ETA, _ETA.replace(" + dyd * exy)", ")").replace(" + dxd * exy)", ")"),
     "test_isotropy_over_a_round_shoal"),
    # corner ghosts (Reading A-B5): the y-sides filled over interior columns
    # only, so the corner ghosts keep stale values
    ("corner_ghosts_stale_two_makers", _CORNER, _CORNER.replace("int i = -2; i < nx + 2;", "int i = 0; i < nx;"),
     "test_corner_ghosts_where_two_makers_meet"),
    ("corner_ghosts_stale_beside_wall", _CORNER, _CORNER.replace("int i = -2; i < nx + 2;", "int i = 0; i < nx;"),
     "test_corner_ghost_of_a_maker_beside_a_wall_by_embedding"),
    # time stepping (Sec. 2.3, Eq. 15-20)
    ("am4_E_coef", "(9.0 * o->Ec[c] + 19.0 * o->E[0][c] - 5.0 * o->E[1][c] + o->E[2][c])",
     "(9.0 * o->Ec[c] + 19.0 * o->E[0][c] - 5.0 * o->E[1][c] - o->E[2][c])",
     "test_dispersion_relation_1d_with_corrector"),
    ("am4_E_coef_oblique", "(9.0 * o->Ec[c] + 19.0 * o->E[0][c] - 5.0 * o->E[1][c] + o->E[2][c])",
     "(9.0 * o->Ec[c] + 19.0 * o->E[0][c] - 5.0 * o->E[1][c] - o->E[2][c])",
     "test_standing_mode_started_from_its_discharges"),
    ("euler_Fstar_increment", "(o->Fs[0][c] - o->Fs[1][c]);", "(o->Fs[0][c]);",
     "test_standing_mode_started_from_its_discharges"),
    ("euler_Gstar_increment", "(o->Gs[0][c] - o->Gs[1][c]);", "(o->Gs[0][c]);",
     "test_standing_mode_started_from_its_discharges"),
    ("ab3_Fstar_first_order", "2.0 * o->Fs[0][c] - 3.0 * o->Fs[1][c] + o->Fs[2][c]", "o->Fs[0][c] - o->Fs[1][c]",
     "test_isotropy_over_a_round_shoal"),
    ("am4_Fstar_increment", "o->Fsc[c] - o->Fs[0][c];", "o->Fsc[c] - o->Fs[1][c];",
     "test_dispersion_relation_2d_oblique"),
    # pieces: limiter, local speeds, friction law, sponge, Thomas
    ("minmod_drop_central", "return fmin(a, fmin(b, c));", "return fmin(a, c);", "test_minmod_cases"),
    ("minmod_theta_ignored", "orc_real a = theta * (q0 - qm), b = 0.5 * (qp - qm), c = theta * (qp - q0);",
     "orc_real a = (q0 - qm), b = 0.5 * (qp - qm), c = (qp - q0);", "test_minmod_cases"),
    ("wave_speed_am_side", "orc_real am = fmin(fmin(uL - sL, uR - sR), 0.0);",
     "orc_real am = fmin(fmin(uL - sL, uL - sR), 0.0);", "test_central_upwind_mirror_symmetry"),
    ("wave_speed_ap_side", "orc_real ap = fmax(fmax(uL + sL, uR + sR), 0.0);",
     "orc_real ap = fmax(fmax(uL + sL, uR + sL), 0.0);", "test_central_upwind_mirror_symmetry"),
    ("manning_cube_root", "cbrt(hinv)", "hinv", "test_friction_manning_ode"),
    ("sponge_cos_sign", "return 0.5 * (1.0 + cos(ORC_PI * (Ls - D) / Ls));",
     "return 0.5 * (1.0 - cos(ORC_PI * (Ls - D) / Ls));", "test_sponge_gamma"),
    ("thomas_back_sub_sign", "x[i] = dp[i] - cp[i] * x[i + 1];", "x[i] = dp[i] + cp[i] * x[i + 1];",
     "test_thomas_vs_dense"),
    ("friction_y_without_depth", "gg -= fc * Q[c] * mag * hinv * hinv;", "gg -= fc * Q[c] * mag * hinv / hinv;",
     "test_friction_quadratic_oblique_flow"),
    ("friction_speed_from_P_only", "orc_real mag = sqrt(P[c] * P[c] + Q[c] * Q[c]);", "orc_real mag = fabs(P[c]);",
     "test_friction_quadratic_oblique_flow"),
    # dry cells (Reading A-D1) and gauges
    ("dry_zero_strict", "if (w[c] - o->Bbar[c] <= 0.0) {", "if (w[c] - o->Bbar[c] < 0.0) {",
     "test_dry_land_holds_no_water_and_no_discharge"),
    ("clamp_to_zero_level", "                w[c] = o->Bbar[c];\n", "                w[c] = 0.0;\n",
     "test_dry_land_holds_no_water_and_no_discharge"),
    ("clamp_mass_every_stage", "if (count) o->clamp_mass +=", "o->clamp_mass +=",
     "test_dry_land_holds_no_water_and_no_discharge"),
    ("sponge_relaxes_land", "if (o->d[c] > 0.0) o->w1[c] = o->p.ws + gam * (o->w1[c] - o->p.ws);",
     "o->w1[c] = o->p.ws + gam * (o->w1[c] - o->p.ws);", "test_sponge_leaves_dry_land_at_its_bed"),
    ("soliton_sech_not_sech2", "orc_real es = H * sh * sh;", "orc_real es = H * sh;", "test_soliton_speed"),
    ("east_maker_depth_cell", "orc_real dadj = o->d[IX(o, side == ORC_W ? 0 : nx - 1, j)];",
     "orc_real dadj = o->d[IX(o, side == ORC_W ? 0 : nx + 1, j)];", "test_symmetry_mirror_sine_makers"),
    ("north_maker_depth_cell", "orc_real dadj = o->d[IX(o, ic, side == ORC_S ? 0 : ny - 1)];",
     "orc_real dadj = o->d[IX(o, ic, side == ORC_S ? 0 : ny + 1)];", "test_symmetry_mirror_sine_makers"),
    ("west_sponge_width_in_cells_over_dx", "L = bc->width * o->p.dx; }", "L = bc->width / o->p.dx; }",
     "test_sponge_profile_in_metres"),
    ("west_sponge_distance_over_dx", "if (s == ORC_W) { D = (i + 0.5) * o->p.dx;", "if (s == ORC_W) { D = (i + 0.5) / o->p.dx;",
     "test_symmetry_transpose_with_sponges"),
    ("y_face_low_bed_of_south_cell", "recon_cell(th, w, P, Q, IX(o, i, gq - 1), ex, By(o, i, gq - 1), By(o, i, gq), loS, hiS);",
     "recon_cell(th, w, P, Q, IX(o, i, gq - 1), ex, By(o, i, gq + 1), By(o, i, gq), loS, hiS);",
     "test_symmetry_transpose_wet_dry"),
    ("y_face_high_bed_of_north_cell", "recon_cell(th, w, P, Q, IX(o, i, gq), ex, By(o, i, gq), By(o, i, gq + 1), loN, hiN);",
     "recon_cell(th, w, P, Q, IX(o, i, gq), ex, By(o, i, gq), By(o, i, gq - 1), loN, hiN);",
     "test_symmetry_transpose_wet_dry"),
    ("maker_beside_dry_cell", "if (!(dadj > 0.0)) return;", "if (!(dadj >= 0.0)) return;", "test_sine_maker_beside_dry_land"),
    ("soliton_crest_orientation", "orc_real xi = ((i + 0.5) * o->p.dx - x0) * ct + ((j + 0.5) * o->p.dy - y0) * st;",
     "orc_real xi = ((i + 0.5) * o->p.dx - x0) * ct - ((j + 0.5) * o->p.dy - y0) * st;",
     "test_solitary_wave_heading_and_depth"),
    ("soliton_width_depth_power", "orc_real ks = sqrt(3.0 * fabs(H) / (4.0 * ds * ds * ds));",
     "orc_real ks = sqrt(3.0 * fabs(H) / (4.0 * ds / ds * ds));", "test_solitary_wave_heading_and_depth"),
    ("accepts_zero_eps", "!(p->dt > 0) || p->K < 0 || !(p->eps > 0))", "!(p->dt > 0) || p->K < 0 || !(p->eps >= 0))",
     "test_oracle_refuses_invalid_parameters"),
    ("accepts_zero_dx", "p->nx < 2 || p->ny < 2 || !(p->dx > 0)", "p->nx < 2 || p->ny < 2 || !(p->dx >= 0)",
     "test_oracle_refuses_invalid_parameters"),
    ("gauge_records_w", "o->grec[(size_t)slot * o->ng + gk] = o->w[IX(o, i, j)] - o->p.ws;",
     "o->grec[(size_t)slot * o->ng + gk] = o->w[IX(o, i, j)];", "test_gauges_record_eta_about_the_still_water_level"),
]


@pytest.mark.parametrize("name,orig,mut,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_mutant(tmp_path, name, orig, mut, pin):
    src = open(SRC).read()
    assert src.count(orig) >= 1, f"mutation site for {name} not found"
    mdir = tmp_path / "oracle_mutant"
    mdir.mkdir()
    (mdir / "celeris_oracle.c").write_text(src.replace(orig, mut, 1))
    hdr = os.path.join(ROOT, "oracle", "celeris_oracle.h")
    (mdir / "celeris_oracle.h").write_text(open(hdr).read())
    so = mdir / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fPIC",
                    "-shared", "-o", str(so), str(mdir / "celeris_oracle.c"), "-lm"], check=True)
    env = dict(os.environ, ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-k", pin],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"pin {pin} did not catch mutant {name}:\n{r.stdout[-2000:]}"


RENDER_SRC = os.path.join(ROOT, "oracle", "render_oracle.c")
RENDER_MUTANTS = [
    ("fresnel_index_side", "float rs = (cos_i - kN2 * cos_t) / (cos_i + kN2 * cos_t);",
     "float rs = (kN2 * cos_i - cos_t) / (kN2 * cos_i + cos_t);", "test_fresnel_closed_forms"),
    ("grid_off_by_one", "floorf((float)(i + 1) * dx / p->grid) != floorf((float)i * dx / p->grid)",
     "floorf((float)(i + 2) * dx / p->grid) != floorf((float)(i + 1) * dx / p->grid)", "test_grid_lines"),
    ("normal_gradient_sign", "float n[3] = {-(p->exaggeration * gx), -(p->exaggeration * gy), 1.0f};",
     "float n[3] = {(p->exaggeration * gx), -(p->exaggeration * gy), 1.0f};", "test_tilted_plane_oblique_view"),
    ("refraction_weight", "float a = 1.0f / (1.0f + p->absorb * h);", "float a = 1.0f / (1.0f + p->absorb);",
     "test_flat_lake_from_above"),
    ("speed_uses_P_twice", "v = sqrtf(u * u + vv * vv);", "v = sqrtf(u * u + u * u);",
     "test_speed_and_velocity_components"),
    ("velocity_depth_floor", "float hd = h > p->h_min ? h : p->h_min;", "float hd = h;",
     "test_speed_and_velocity_components"),
    ("hillshade_unclamped", "float shade = 0.35f + 0.65f * (d > 0.0f ? d : 0.0f);", "float shade = 0.35f + 0.65f * d;",
     "test_flat_land_hillshade"),
    ("north_neighbour_index", "jn = j < ny - 1 ? j + 1 : j;", "jn = j < ny - 1 ? j - 1 : j;",
     "test_tilted_plane_both_directions_grazing_view"),
    ("y_span_over_dy", "spany = (float)(jn - js) * dy;", "spany = (float)(jn - js) / dy;",
     "test_tilted_plane_both_directions_grazing_view"),
    ("west_neighbour_eta_sign", "float eW = AT(w, iw, j) - AT(Bbar, iw, j) > p->dry_h ? AT(w, iw, j) - ws : ec;",
     "float eW = AT(w, iw, j) - AT(Bbar, iw, j) > p->dry_h ? AT(w, iw, j) + ws : ec;",
     "test_tilted_plane_both_directions_grazing_view"),
    ("dry_neighbour_level", "const float ec = wc - ws;", "const float ec = wc + ws;", "test_lake_shore_is_level"),
    ("incidence_dot_sign", "float idn = I[0] * n[0] + I[1] * n[1] + I[2] * n[2];",
     "float idn = I[0] * n[0] - I[1] * n[1] + I[2] * n[2];", "test_tilted_plane_both_directions_grazing_view"),
    ("reflected_height", "float rz = I[2] - 2.0f * idn * n[2];", "float rz = I[2] - 2.0f * idn / n[2];",
     "test_tilted_plane_both_directions_grazing_view"),
    ("normalise_y", "    v[1] = v[1] / n;\n", "    v[1] = v[1] * n;\n", "test_tilted_plane_both_directions_grazing_view"),
    ("value_range", "return (v - lo) / (hi - lo);", "return (v - lo) / (hi + lo);", "test_colormap_range_of_the_value"),
    ("colormap_quarters", "float s = t * 4.0f;", "float s = t / 4.0f;", "test_colormap_control_points_and_linearity"),
    ("grid_rows_off_by_one", "int ly = floorf((float)(j + 1) * dy / p->grid)", "int ly = floorf((float)(j - 1) * dy / p->grid)",
     "test_grid_lines"),
    ("hillshade_y_term", "float d = nb[0] * L[0] + nb[1] * L[1] + nb[2] * L[2];",
     "float d = nb[0] * L[0] - nb[1] * L[1] + nb[2] * L[2];", "test_hillshade_of_a_plane_in_both_directions"),
    ("dry_threshold_inclusive", "const int wet = h > p->dry_h;", "const int wet = h >= p->dry_h;",
     "test_depth_equal_to_dry_h_is_land"),
    ("east_neighbour_threshold", "float eE = AT(w, ie, j) - AT(Bbar, ie, j) > p->dry_h",
     "float eE = AT(w, ie, j) - AT(Bbar, ie, j) >= p->dry_h", "test_depth_equal_to_dry_h_is_land"),
    ("land_span_guard", "float gx = spanx > 0.0f ? (AT(Bbar, ie, j) - AT(Bbar, iw, j)) / spanx : 0.0f;",
     "float gx = spanx >= 0.0f ? (AT(Bbar, ie, j) - AT(Bbar, iw, j)) / spanx : 0.0f;",
     "test_one_cell_wide_strips_see_a_level_surface"),
]


@pytest.mark.parametrize("name,orig,mut,pin", RENDER_MUTANTS, ids=[m[0] for m in RENDER_MUTANTS])
def test_render_pin_catches_mutant(tmp_path, name, orig, mut, pin):
    src = open(RENDER_SRC).read()
    assert src.count(orig) == 1, f"mutation site for {name} not found"
    mdir = tmp_path / "render_mutant"
    mdir.mkdir()
    (mdir / "render_oracle.c").write_text(src.replace(orig, mut, 1))
    (mdir / "render_oracle.h").write_text(open(os.path.join(ROOT, "oracle", "render_oracle.h")).read())
    so = mdir / "librender_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                    str(mdir / "render_oracle.c"), "-lm"], check=True)
    env = dict(os.environ, RENDER_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_render_oracle_pins.py"), "-k", pin],
                       cwd=ROOT, env=env, capture_output=True, text=True)
    assert r.returncode != 0, f"pin {pin} did not catch mutant {name}:\n{r.stdout[-2000:]}"


# The tangent-linear oracle's dual-number arithmetic (oracle/celeris_tlm.cpp):
# a wrong derivative rule must break the match with central differences.
TLM_SRC = os.path.join(ROOT, "oracle", "celeris_tlm.cpp")
TLM_MUTANTS = [
    ("product_rule", "static inline orc_dual operator*(orc_dual a, orc_dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }",
     "static inline orc_dual operator*(orc_dual a, orc_dual b) { return {a.v * b.v, a.d * b.v}; }"),
    ("quotient_rule", "return {q, (a.d - q * b.d) / b.v};", "return {q, (a.d + q * b.d) / b.v};"),
    ("sqrt_rule", "return {s, s > 0.0 ? a.d / (2.0 * s) : 0.0};", "return {s, s > 0.0 ? a.d / s : 0.0};"),
    ("cbrt_rule", "return {c, c != 0.0 ? a.d / (3.0 * c * c) : 0.0};", "return {c, c != 0.0 ? a.d / (3.0 * c) : 0.0};"),
    ("tanh_rule", "return {t, (1.0 - t * t) * a.d};", "return {t, (1.0 + t * t) * a.d};"),
    ("sin_rule", "return {::sin(a.v), ::cos(a.v) * a.d};", "return {::sin(a.v), -::cos(a.v) * a.d};"),
    ("difference_rule", "static inline orc_dual operator-(orc_dual a, orc_dual b) { return {a.v - b.v, a.d - b.d}; }",
     "static inline orc_dual operator-(orc_dual a, orc_dual b) { return {a.v - b.v, a.d + b.d}; }"),
    ("scaling_in_place", "        d = d * b.v + v * b.d;\n", "        d = d + v * b.d;\n"),
]


@pytest.mark.parametrize("name,orig,mut", TLM_MUTANTS, ids=[m[0] for m in TLM_MUTANTS])
def test_tangent_pin_catches_mutant(tmp_path, name, orig, mut):
    src = open(TLM_SRC).read()
    assert src.count(orig) == 1, f"mutation site for {name} not found"
    mdir = tmp_path / "tlm_mutant"
    mdir.mkdir()
    (mdir / "celeris_tlm.cpp").write_text(src.replace(orig, mut, 1))
    for f in ("celeris_oracle.c", "celeris_oracle.h"):
        (mdir / f).write_text(open(os.path.join(ROOT, "oracle", f)).read())
    so = mdir / "libtlm_mutant.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                    str(mdir / "celeris_tlm.cpp")], check=True)
    env = dict(os.environ, TLM_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_tlm_oracle.py"), "-k", "central_differences or manning_paths"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"the central-difference pin did not catch mutant {name}:\n{r.stdout[-2000:]}"
