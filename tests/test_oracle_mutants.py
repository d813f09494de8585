"""Planted mistakes in the oracle, and the pins that catch them.

Every parity claim rests on the oracle, and the oracle rests on its pins.
This file checks the pins themselves.  Each case below copies
oracle/qed_oracle.c, plants one plausible mistake: a dropped term, a wrong
sign, a transposed operand or index, a wrong constant or Bessel order.  It
builds the copy into a library of its own with the oracle's compiler flags,
then runs the listed pins against it in a subprocess, with QED_ORACLE_LIB
naming the copy.  Every pin set must fail on its mutant, and pass on an
unmodified copy built the same way.  The CUDA library is not involved.
"""
import concurrent.futures as cf
import os
import subprocess
import sys
from pathlib import Path

import pytest

from oracle import oracle as o

ROOT = Path(__file__).resolve().parent.parent

# (name, text in qed_oracle.c, its replacement, occurrences, pins that must fail)
MUTANTS = [
    # synchrotron functions (Sec. IV.E): the Bessel orders of F1 and F2
    ("F1 from K_1/3", "cosh(5.0 * u / 3.0) / cosh(u)", "cosh(1.0 * u / 3.0) / cosh(u)", 1,
     ["tests/test_oracle_special.py::test_F_against_scipy", "tests/test_oracle_golden.py"]),
    ("F2 from K_1/3", "double t2 = e * cosh(2.0 * u / 3.0);", "double t2 = e * cosh(1.0 * u / 3.0);", 1,
     ["tests/test_oracle_special.py::test_F_against_scipy"]),
    ("F1, F2: the u = 0 term at full weight", "double s1 = 0.5 * e0, s2 = 0.5 * e0;", "double s1 = e0, s2 = e0;", 1,
     ["tests/test_oracle_special.py::test_F_against_scipy"]),
    ("F1 without its factor x", "    *f1 = x * h * s1;", "    *f1 = h * s1;", 1,
     ["tests/test_oracle_special.py::test_F_against_scipy"]),
    # emission density, Eq. (24), and the modified generator, Eq. (25)
    ("G: F2 term with the wrong sign", "(f1 + 1.5 * delta * chi * zq * f2)", "(f1 - 1.5 * delta * chi * zq * f2)", 1,
     ["tests/test_oracle_rates.py::test_G_against_scipy"]),
    ("G: F2 term dropped", "(f1 + 1.5 * delta * chi * zq * f2)", "(f1)", 1,
     ["tests/test_oracle_rates.py::test_G_against_scipy", "tests/test_oracle_golden.py"]),
    ("G: z_q with delta and 1 - delta transposed", "double zq = (2.0 / 3.0) / chi * delta / (1.0 - delta);",
     "double zq = (2.0 / 3.0) / chi * (1.0 - delta) / delta;", 1,
     ["tests/test_oracle_rates.py::test_G_against_scipy"]),
    ("P without 1/gamma", "return OR_ALPHA * dt * or_G(delta, chi) / gamma;", "return OR_ALPHA * dt * or_G(delta, chi);", 1,
     ["tests/test_oracle_golden.py", "tests/test_oracle_rates.py::test_small_delta_asymptote"]),
    ("P_m with the Jacobian 2 r1^2", "return 3.0 * r1 * r1 * or_P(delta, chi, gamma, dt);",
     "return 2.0 * r1 * r1 * or_P(delta, chi, gamma, dt);", 1,
     ["tests/test_oracle_golden.py", "tests/test_oracle_generator.py::test_frozen_spectrum_gamma100_chi1"]),
    # pair density, Eq. (30)
    ("P_p: F2 term with the wrong sign", "(f1 - 1.5 * chig * zp * f2)", "(f1 + 1.5 * chig * zp * f2)", 1,
     ["tests/test_oracle_rates.py::test_pair_rate_known_values"]),
    ("P_p: chi_g eps_g for chi_g / eps_g", "chig / epsg * (de - 1.0) * de", "chig * epsg * (de - 1.0) * de", 1,
     ["tests/test_oracle_rates.py::test_pair_rate_erber_limit", "tests/test_oracle_golden.py"]),
    # chi and the effective fields, Eqs. (3)-(4), (31)-(32)
    ("chi: p x B with the wrong sign", "double ax = g * E[0] + (p[1] * B[2] - p[2] * B[1]);",
     "double ax = g * E[0] - (p[1] * B[2] - p[2] * B[1]);", 1,
     ["tests/test_oracle_rates.py::test_chi_definitions"]),
    ("H_eff without (p_hat . E)^2", "double pe = pm > 0.0 ? (p[0] * E[0] + p[1] * E[1] + p[2] * E[2]) / pm : 0.0;",
     "double pe = 0.0;", 1, ["tests/test_oracle_rates.py::test_longitudinal_field_terms"]),
    ("photon H_eff without (k_hat . E)^2", "double ke = nx * E[0] + ny * E[1] + nz * E[2];", "double ke = 0.0;", 1,
     ["tests/test_oracle_rates.py::test_longitudinal_field_terms"]),
    ("Esirkepov: current with the wrong sign", "acc -= qw * d[0] / (dt * dV) * W;", "acc += qw * d[0] / (dt * dV) * W;", 1,
     ["tests/test_oracle_grid.py::test_esirkepov_continuity"]),
    # sub-interval bounds, Eqs. (28) and (33), and their count (Sec. IV.H)
    ("dt_q: 173 for 137", "return kappa * 137.0 * (a < b ? a : b);", "return kappa * 173.0 * (a < b ? a : b);", 1,
     ["tests/test_oracle_golden.py"]),
    ("dt_q: H^(-1/3) for H^(-2/3)", "double a = 0.67 * cbrt(gamma) * pow(1.0 / heff, 2.0 / 3.0);",
     "double a = 0.67 * cbrt(gamma) * pow(1.0 / heff, 1.0 / 3.0);", 1, ["tests/test_oracle_golden.py"]),
    ("dt_q of photons without lambda_C / c = 2 pi", "return kappa * 130.0 * 2.0 * OR_PI / heff_g;",
     "return kappa * 130.0 / heff_g;", 1, ["tests/test_oracle_golden.py::test_time_step_bounds_match_the_rates"]),
    ("sub-intervals longer than dt_q", "double n = ceil(ratio);", "double n = floor(ratio);", 1,
     ["tests/test_oracle_rates.py::test_time_step_bounds"]),
    # Boris push (Appendix A)
    ("Boris: rotation operands transposed", "double up[3] = {um[0] + (um[1] * t[2] - um[2] * t[1]),",
     "double up[3] = {um[0] + (um[2] * t[1] - um[1] * t[2]),", 1,
     ["tests/test_oracle_push.py::test_uniform_B_rotation_exact"]),
    ("Boris: s = 2t without 1/(1 + t^2)",
     "double s[3] = {2.0 * t[0] / (1.0 + t2), 2.0 * t[1] / (1.0 + t2), 2.0 * t[2] / (1.0 + t2)};",
     "double s[3] = {2.0 * t[0], 2.0 * t[1], 2.0 * t[2]};", 1,
     ["tests/test_oracle_push.py::test_uniform_B_rotation_exact"]),
    ("Boris: second rotation with the wrong sign", "double uq[3] = {um[0] + (up[1] * s[2] - up[2] * s[1]),",
     "double uq[3] = {um[0] - (up[1] * s[2] - up[2] * s[1]),", 1,
     ["tests/test_oracle_push.py::test_uniform_B_rotation_exact"]),
    ("Boris: a whole E step on each side", "double a = 0.5 * q * h;", "double a = q * h;", 1,
     ["tests/test_oracle_push.py::test_uniform_E_acceleration_exact"]),
    # events (Sec. IV.G, V.A): momentum shares
    ("photon takes r1^2", "double delta = a1 * a1 * a1;", "double delta = a1 * a1;", 1,
     ["tests/test_oracle_step.py::test_momentum_conservation_uniform_E"]),
    ("no recoil of the emitting lepton",
     "for (int c = 0; c < 3; ++c) q->p[c] = (1.0 - delta) * p0[c];\n                C->D->emissions++;\n                double k[3]",
     "for (int c = 0; c < 3; ++c) q->p[c] = p0[c];\n                C->D->emissions++;\n                double k[3]", 1,
     ["tests/test_oracle_step.py::test_momentum_conservation_uniform_E"]),
    ("positron takes r1 too", "po.p[c] = (1.0 - a1) * q->p[c];", "po.p[c] = a1 * q->p[c];", 1,
     ["tests/test_oracle_step.py::test_momentum_conservation_uniform_E"]),
    # the generators of Sec. IV.F through the particle step
    ("alternative generator: delta from r2", "delta = r1;                          /* r2 < P(r1), delta = r1 */",
     "delta = r2;                          /* r2 < P(r1), delta = r1 */", 1,
     ["tests/test_oracle_generators.py::test_step_emits_the_generator_densities"]),
    ("standard generator: fires on r2", "fire = r1 < pe;\n                    delta = fire ? or_delta_std(chi, r2)",
     "fire = r2 < pe;\n                    delta = fire ? or_delta_std(chi, r2)", 1,
     ["tests/test_oracle_generators.py::test_step_emits_the_generator_densities"]),
    ("standard generator: W without the Jacobian 3 s^2", "acc += or_gl8_w[k] * 3.0 * s * s * or_G(s * s * s, chi);",
     "acc += or_gl8_w[k] * or_G(s * s * s, chi);", 1,
     ["tests/test_oracle_generators.py::test_standard_total_and_cdf_against_scipy"]),
    ("Gauss-Legendre: recurrence with 2n + 1", "double p2 = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;",
     "double p2 = ((2.0 * n + 1.0) * x * p1 - (n - 1.0) * p0) / n;", 1,
     ["tests/test_oracle_generators.py::test_gauss_legendre_rule_of_the_standard_generator"]),
    ("Gauss-Legendre: weights with 1 + x^2", "or_gl8_w[7 - i] = or_gl8_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);",
     "or_gl8_w[7 - i] = or_gl8_w[i] = 2.0 / ((1.0 + x * x) * dp * dp);", 1,
     ["tests/test_oracle_generators.py::test_gauss_legendre_rule_of_the_standard_generator"]),
    ("standard generator: delta = s^2", "    double sr = 0.5 * (a + b);\n    return sr * sr * sr;",
     "    double sr = 0.5 * (a + b);\n    return sr * sr;", 1,
     ["tests/test_oracle_generators.py::test_standard_energy_is_the_inverse_cdf"]),
    ("sub-interval cap ignored", "    if (n > (double)nmax) { *capped = 1; return nmax; }",
     "    if (0) { *capped = 1; return nmax; }", 1, ["tests/test_oracle_rates.py::test_time_step_bounds"]),
    ("uniforms without the half offset (0 can occur)", "return (k + 0.5) * (1.0 / 4503599627370496.0);",
     "return k * (1.0 / 4503599627370496.0);", 1, ["tests/test_oracle_generator.py::test_u52_range_edges"]),
    # the focused pulse of the collision (a paraxial Gaussian beam)
    ("pulse: Rayleigh length k w0^2", "double zr = 0.5 * w * w0 * w0;", "double zr = w * w0 * w0;", 1,
     ["tests/test_oracle_step.py::test_gaussian_pulse_solves_the_wave_equation"]),
    ("pulse: Gouy phase with the wrong sign", "double phase = w * eta - 0.5 * w * r2 * invR + gouy + fp[8];",
     "double phase = w * eta - 0.5 * w * r2 * invR - gouy + fp[8];", 1,
     ["tests/test_oracle_step.py::test_gaussian_pulse_solves_the_wave_equation"]),
    # mesh (Appendix C): FDTD, CIC, Esirkepov
    ("FDTD: current term with the wrong sign", "E[c][q] += dt * (tmp[c][q] - 4.0 * OR_PI * OR_ALPHA * J[c][q]);",
     "E[c][q] += dt * (tmp[c][q] + 4.0 * OR_PI * OR_ALPHA * J[c][q]);", 1,
     ["tests/test_oracle_grid.py::test_gauss_law_kept_by_the_field_update"]),
    ("FDTD: whole B steps", "B[c][q] -= 0.5 * dt * tmp[c][q];", "B[c][q] -= dt * tmp[c][q];", 2,
     ["tests/test_oracle_grid.py::test_plane_wave_dispersion"]),
    ("CIC: Ex and Ey staggers transposed", "{{0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5},",
     "{{0, 0.5, 0}, {0.5, 0, 0}, {0, 0, 0.5},", 1, ["tests/test_oracle_grid.py::test_cic_linear_exact"]),
    ("Esirkepov: 1/2 for 1/3 in the Jx weight", "dS[1][j] * dS[2][k] / 3.0", "dS[1][j] * dS[2][k] / 2.0", 1,
     ["tests/test_oracle_grid.py::test_esirkepov_continuity"]),
    # particle motion, ensembles, weights and placement
    ("position update without the mass", "for (int c = 0; c < 3; ++c) q->x[c] += q->p[c] / (m * g) * h;",
     "for (int c = 0; c < 3; ++c) q->x[c] += q->p[c] / g * h;", 1,
     ["tests/test_oracle_step.py::test_free_streaming_velocity"]),
    ("ensemble table: Bx and By swapped", "B[0] = q[6]; B[1] = q[7]; B[2] = q[8];",
     "B[0] = q[7]; B[1] = q[6]; B[2] = q[8];", 1,
     ["tests/test_oracle_sec6.py::test_one_ensemble_is_the_uniform_mode"]),
    ("spectrum counts photons, not weights", "if (a >= 0.0 && a < P->nbins) C->D->spectrum[(long)a] += w;",
     "if (a >= 0.0 && a < P->nbins) C->D->spectrum[(long)a] += 1.0;", 1,
     ["tests/test_oracle_sec6.py::test_spectra_are_weighted"]),
    ("pair products without 1/N_g", "el.w = po.w = q->w * (fg / (double)ng);", "el.w = po.w = q->w * fg;", 1,
     ["tests/test_oracle_sec6.py::test_pair_factor_keeps_lepton_yield"]),
    ("vacuum pair offsets: y from the x draw", "el.x[1] = po.x[1] = P->x0[1] + ((double)j + uy) * P->d[1];",
     "el.x[1] = po.x[1] = P->x0[1] + ((double)j + ux) * P->d[1];", 1,
     ["tests/test_oracle_schwinger.py::test_pairs_at_rest_colocated_uniform_in_cells"]),
    ("step deposits without the charge", "or_deposit(P->n, P->d, P->x0, C->J, xs, q->x, P->charge[sp] * q->w, C->dt);",
     "or_deposit(P->n, P->d, P->x0, C->J, xs, q->x, q->w, C->dt);", 1,
     ["tests/test_oracle_grid.py::test_step_current_is_continuous"]),
    # vacuum pairs (Sec. V.B), thinning (Sec. VI), Philox
    ("Schwinger rate exp(-1/E)", "exp(-OR_PI / Em)", "exp(-1.0 / Em)", 1,
     ["tests/test_oracle_schwinger.py::test_pair_count_matches_the_si_rate"]),
    ("thinning factor N/L instead of the weight ratio", "w = w * (wall[g] / wsurv[g]);",
     "w = w * ((double)count[g] / (double)L);", 1,
     ["tests/test_oracle_sec6.py::test_thinning_conserves_group_weight_and_is_binomial"]),
    # photons in the step (Sec. V.A, Eqs. (31)-(33))
    ("photon flies at |k| instead of c", "for (int c = 0; c < 3; ++c) q->x[c] += q->p[c] / eps * h;",
     "for (int c = 0; c < 3; ++c) q->x[c] += q->p[c] * h;", 1,
     ["tests/test_oracle_step.py::test_boundaries_open_and_periodic"]),
    ("chi_gamma without the photon energy", "double chig = eps * hg;", "double chig = hg;", 1,
     ["tests/test_oracle_step.py::test_pair_step_converts_at_the_rate_and_splits_by_its_density"]),
    ("pair draw over the whole step", "double pp = or_Pp(r1, chig, eps, h);", "double pp = or_Pp(r1, chig, eps, t_span);", 1,
     ["tests/test_oracle_step.py::test_pair_step_converts_at_the_rate_and_splits_by_its_density"]),
    ("P_p: z_p without 1 - delta_e", "double zp = (2.0 / 3.0) / (chig * (1.0 - de) * de);",
     "double zp = (2.0 / 3.0) / (chig * de);", 1,
     ["tests/test_oracle_rates.py::test_pair_rate_known_values",
      "tests/test_oracle_step.py::test_pair_step_converts_at_the_rate_and_splits_by_its_density"]),
    ("photon sub-intervals from chi_gamma", "n = or_nsub(t_span, or_dtq_photon(hg, P->kappa), P->nsub_max, &capped);",
     "n = or_nsub(t_span, or_dtq_photon(chig, P->kappa), P->nsub_max, &capped);", 1,
     ["tests/test_oracle_step.py::test_pair_products_evolve_for_the_rest_of_the_step"]),
    ("pair defect: positron takes r1", "ke[c] = r1 * q->p[c]; kp[c] = (1.0 - r1) * q->p[c];",
     "ke[c] = r1 * q->p[c]; kp[c] = r1 * q->p[c];", 1,
     ["tests/test_oracle_step.py::test_energy_conservation_uniform_B"]),
    # products of a step evolve for its rest (reading of Sec. IV.H)
    ("photon product flies one sub-interval too long",
     "                or_emit_child(C, OR_PHOTON, &ph, (double)(n - 1 - s) * h, E, B);\n            }\n            if (r2 < pm)",
     "                or_emit_child(C, OR_PHOTON, &ph, (double)(n - s) * h, E, B);\n            }\n            if (r2 < pm)", 1,
     ["tests/test_oracle_step.py::test_children_modes"]),
    ("pair products move one sub-interval too long", "double t_rem = (double)(n - 1 - s) * h;",
     "double t_rem = (double)(n - s) * h;", 1,
     ["tests/test_oracle_step.py::test_pair_products_evolve_for_the_rest_of_the_step"]),
    # the lepton's time-step bound and effective field
    ("dt_q: the larger of the two branches", "return kappa * 137.0 * (a < b ? a : b);",
     "return kappa * 137.0 * (a > b ? a : b);", 1, ["tests/test_oracle_rates.py::test_time_step_bounds"]),
    ("H_eff: p x B for v x B", "double vx = p[0] / g, vy = p[1] / g, vz = p[2] / g;",
     "double vx = p[0], vy = p[1], vz = p[2];", 1, ["tests/test_oracle_rates.py::test_chi_definitions"]),
    # the generators of Sec. IV.F
    ("alternative generator: P at r2", "pe = or_P(r1, chi, g, h);", "pe = or_P(r2, chi, g, h);", 1,
     ["tests/test_oracle_generators.py::test_step_emits_the_generator_densities"]),
    ("standard generator: W(1) without 1/gamma", "return OR_ALPHA * dt / gamma * or_Wnorm(1.0, chi);",
     "return OR_ALPHA * dt * or_Wnorm(1.0, chi);", 1,
     ["tests/test_oracle_generators.py::test_three_generators_frozen_spectra"]),
    # analytic fields
    ("rotating E: cos and sin swapped", "E[0] = fp[0] * cos(fp[1] * t);\n        E[1] = fp[0] * sin(fp[1] * t);",
     "E[0] = fp[0] * sin(fp[1] * t);\n        E[1] = fp[0] * cos(fp[1] * t);", 1,
     ["tests/test_oracle_sec6.py::test_one_ensemble_is_the_rotating_mode"]),
    ("standing wave: B_z with the wrong sign", "B[2] = -fp[0] * cos(fp[1] * x[0]) * sin(fp[1] * t);",
     "B[2] = fp[0] * cos(fp[1] * x[0]) * sin(fp[1] * t);", 1,
     ["tests/test_oracle_step.py::test_standing_wave_field"]),
    ("pulse: envelope ln 2 for 2 ln 2", "double env = exp(-2.0 * log(2.0) * eta * eta / (tau * tau));",
     "double env = exp(-log(2.0) * eta * eta / (tau * tau));", 1,
     ["tests/test_oracle_step.py::test_gaussian_pulse_properties"]),
    ("pulse: B along +E", "        B[2] = -E[1];\n    } else if (mode == OR_FIELD_ROTATING_E)",
     "        B[2] = E[1];\n    } else if (mode == OR_FIELD_ROTATING_E)", 1,
     ["tests/test_oracle_step.py::test_gaussian_pulse_properties"]),
    ("ensemble: rotating E_x by sin", "E[0] = q[3] + q[0] * cos(ph);", "E[0] = q[3] + q[0] * sin(ph);", 1,
     ["tests/test_oracle_sec6.py::test_rotating_field_closed_form_orbit"]),
    # boundaries
    ("open box: lower faces keep particles", "} else if (q->x[c] < lo || q->x[c] >= lo + L) {",
     "} else if (q->x[c] >= lo + L) {", 1, ["tests/test_oracle_step.py::test_boundaries_open_and_periodic"]),
    ("periodic wrap the wrong way", "q->x[c] -= u * L;", "q->x[c] += u * L;", 1,
     ["tests/test_oracle_step.py::test_boundaries_open_and_periodic"]),
    # mesh: curls, CIC, charge density, Esirkepov
    ("curl B: (curl B)_z with dy for dx", "out[2][c] = (B[1][c] - B[1][or_idx(n, i - 1, j, k)]) / d[0]",
     "out[2][c] = (B[1][c] - B[1][or_idx(n, i - 1, j, k)]) / d[1]", 1,
     ["tests/test_oracle_grid.py::test_plane_wave_dispersion"]),
    ("curl E: backward difference", "out[0][c] = (E[2][or_idx(n, i, j + 1, k)] - E[2][c]) / d[1]",
     "out[0][c] = (E[2][c] - E[2][or_idx(n, i, j - 1, k)]) / d[1]", 1,
     ["tests/test_oracle_grid.py::test_plane_wave_dispersion"]),
    ("CIC: fraction from the node above", "        fr[c] = v[c] - (double)b[c];\n    }\n    double acc",
     "        fr[c] = (double)b[c] + 1.0 - v[c];\n    }\n    double acc", 1,
     ["tests/test_oracle_grid.py::test_cic_linear_exact"]),
    ("charge density: x weights transposed",
     "                    double wgt = (di ? fr[0] : 1.0 - fr[0]) * (dj ? fr[1] : 1.0 - fr[1])",
     "                    double wgt = (di ? 1.0 - fr[0] : fr[0]) * (dj ? fr[1] : 1.0 - fr[1])", 1,
     ["tests/test_oracle_grid.py::test_esirkepov_continuity"]),
    ("Esirkepov: 1/2 for 1/3 in the Jz weight", "dS[0][i] * dS[1][j] / 3.0", "dS[0][i] * dS[1][j] / 2.0", 1,
     ["tests/test_oracle_grid.py::test_esirkepov_continuity"]),
    ("Esirkepov: Jy scaled by dx", "acc -= qw * d[1] / (dt * dV) * W;", "acc -= qw * d[0] / (dt * dV) * W;", 1,
     ["tests/test_oracle_grid.py::test_esirkepov_continuity"]),
    # ensembles, thinning, weights (Sec. VI)
    ("products leave their parent's ensemble", "return (parent & hi) | (mix & ~hi);", "return mix;", 1,
     ["tests/test_oracle_sec6.py::test_ensembles_together_equal_ensembles_alone"]),
    ("ensemble guard one row too lenient", "if (!P->ens || e >= (uint32_t)P->n_ens) return;",
     "if (!P->ens || e > (uint32_t)P->n_ens) return;", 1,
     ["tests/test_oracle_sec6.py::test_an_ensemble_without_a_row_sees_no_field"]),
    ("thinning keeps the complement", "if (u < (double)L / (double)count[g]) wsurv[g] += s->w[i];",
     "if (u >= (double)L / (double)count[g]) wsurv[g] += s->w[i];", 1,
     ["tests/test_oracle_sec6.py::test_thinning_conserves_group_weight_and_is_binomial"]),
    ("thinning limit without the ensemble's scale", "if (sc > 0.0) L = (int64_t)floor((double)L * sc);",
     "if (sc > 0.0) L = L;", 1, ["tests/test_oracle_sec6.py::test_thinning_conserves_group_weight_and_is_binomial"]),
    ("pair products at weight w N_g", "el.w = po.w = q->w * (fg / (double)ng);", "el.w = po.w = q->w * fg * (double)ng;", 1,
     ["tests/test_oracle_sec6.py::test_pair_factor_keeps_lepton_yield"]),
    # vacuum pairs (Sec. V.B)
    ("Schwinger rate over 4 pi^2", "(4.0 * OR_PI * OR_PI * OR_PI)", "(4.0 * OR_PI * OR_PI)", 1,
     ["tests/test_oracle_schwinger.py::test_pair_count_matches_the_si_rate"]),
    ("Schwinger rate with E for E^2", "double ps = Em * Em * exp(", "double ps = Em * exp(", 1,
     ["tests/test_oracle_schwinger.py::test_pair_count_matches_the_si_rate"]),
    ("Philox: nine rounds", "for (int r = 0; r < 10; ++r) {", "for (int r = 0; r < 9; ++r) {", 1,
     ["tests/test_philox_pin.py::test_oracle_philox_matches_aten"]),
    ("Philox: low words of the products swapped", "c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;",
     "c[0] = n0; c[1] = lo0; c[2] = n2; c[3] = lo1;", 1, ["tests/test_philox_pin.py::test_oracle_philox_matches_aten"]),
    # more of the push, the rates and the mesh
    ("Boris: gamma without 1/m^2", "double gm = sqrt(1.0 + (um[0] * um[0] + um[1] * um[1] + um[2] * um[2]) / (m * m));",
     "double gm = sqrt(1.0 + (um[0] * um[0] + um[1] * um[1] + um[2] * um[2]));", 1,
     ["tests/test_oracle_push.py::test_uniform_B_rotation_exact"]),
    ("Boris: rotation vector without 1/m", "double f = a / (m * gm);", "double f = a / gm;", 1,
     ["tests/test_oracle_push.py::test_uniform_B_rotation_exact"]),
    ("photon H_eff: k x B with the wrong sign", "double ax = E[0] + (ny * B[2] - nz * B[1]);",
     "double ax = E[0] - (ny * B[2] - nz * B[1]);", 1, ["tests/test_oracle_rates.py::test_chi_definitions"]),
    ("G without the factor 1 - delta", "return sqrt(3.0) / (2.0 * OR_PI) * chi * (1.0 - delta) / delta",
     "return sqrt(3.0) / (2.0 * OR_PI) * chi / delta", 1, ["tests/test_oracle_rates.py::test_G_against_scipy"]),
    ("spectrum binned in ln delta", "double a = (log10(delta) - P->lg_lo) / span * P->nbins;",
     "double a = (log(delta) - P->lg_lo) / span * P->nbins;", 1,
     ["tests/test_oracle_martingale.py::test_sampled_spectrum_matches_its_expectation_along_the_trajectories"]),
    ("CIC: Bz staggered in z too", "{0, 0.5, 0.5}, {0.5, 0, 0.5}, {0.5, 0.5, 0}};",
     "{0, 0.5, 0.5}, {0.5, 0, 0.5}, {0.5, 0.5, 0.5}};", 1, ["tests/test_oracle_grid.py::test_cic_linear_exact"]),
    ("Esirkepov: stencil one node up", "base[c] = (long)floor(ua[c]) - 1;", "base[c] = (long)floor(ua[c]);", 1,
     ["tests/test_oracle_grid.py::test_esirkepov_continuity"]),
    ("ions emit", "int qed = (sp != OR_ION) && P->emission_on;", "int qed = P->emission_on;", 1,
     ["tests/test_oracle_step.py::test_ions_never_emit"]),
    ("vacuum pairs: field at the cell's corner", "double xc[3] = {P->x0[0] + (i + 0.5) * P->d[0],",
     "double xc[3] = {P->x0[0] + (i + 0.0) * P->d[0],", 1,
     ["tests/test_oracle_schwinger.py::test_mesh_field_taken_at_the_cell_centre"]),
    # ensembles and the generator factors (Sec. VI)
    ("ensemble: phase dropped", "double ph = q[1] * t + q[2];", "double ph = q[1] * t;", 1,
     ["tests/test_oracle_sec6.py::test_rotating_field_closed_form_orbit"]),
    ("ensemble from one bit too few", "return P->ens_bits > 0 ? (uint32_t)(id >> (64 - P->ens_bits)) : 0u;",
     "return P->ens_bits > 0 ? (uint32_t)(id >> (63 - P->ens_bits)) : 0u;", 1,
     ["tests/test_oracle_sec6.py::test_ensembles_together_equal_ensembles_alone"]),
    ("thinning factor inverted", "if (u < (double)L / (double)count[g]) w = w * (wall[g] / wsurv[g]);",
     "if (u < (double)L / (double)count[g]) w = w * (wsurv[g] / wall[g]);", 1,
     ["tests/test_oracle_sec6.py::test_thinning_conserves_group_weight_and_is_binomial"]),
    ("products kept with probability f_g", "return u < 1.0 / fg;", "return u < fg;", 1,
     ["tests/test_oracle_sec6.py::test_emission_factor_fg_keeps_yields"]),
    ("photon products without 1/N_g", "ph.w = q->w * (fg / (double)ng);", "ph.w = q->w * fg;", 1,
     ["tests/test_oracle_sec6.py::test_emission_factor_ng_keeps_yields"]),
    ("energy spectrum binned by delta", "double b = (log10(eps) - P->lg_lo) / span * P->nbins;",
     "double b = (log10(delta) - P->lg_lo) / span * P->nbins;", 1,
     ["tests/test_oracle_step.py::test_energy_spectrum_is_the_photons_energies"]),
    ("pulse: intensity waist for the field's", "double amp = E0 * (w0 / wz) * exp(-r2 / (wz * wz)) * env;",
     "double amp = E0 * (w0 / wz) * exp(-2.0 * r2 / (wz * wz)) * env;", 1,
     ["tests/test_oracle_step.py::test_gaussian_pulse_properties"]),
    ("pulse: no w0/w(z) amplitude", "double amp = E0 * (w0 / wz) * exp(-r2 / (wz * wz)) * env;",
     "double amp = E0 * exp(-r2 / (wz * wz)) * env;", 1,
     ["tests/test_oracle_step.py::test_gaussian_pulse_solves_the_wave_equation"]),
    ("pulse: wave-front curvature 1/zeta", "double invR = zeta / (zeta * zeta + zr * zr);",
     "double invR = 1.0 / zeta;", 1, ["tests/test_oracle_step.py::test_gaussian_pulse_solves_the_wave_equation"]),
    ("standing wave: cos(kx) for sin(kx)", "E[1] = fp[0] * sin(fp[1] * x[0]) * cos(fp[1] * t);",
     "E[1] = fp[0] * cos(fp[1] * x[0]) * cos(fp[1] * t);", 1, ["tests/test_oracle_step.py::test_standing_wave_field"]),
    ("uniform mode: Bx and By swapped", "B[0] = fp[3]; B[1] = fp[4]; B[2] = fp[5];",
     "B[0] = fp[4]; B[1] = fp[3]; B[2] = fp[5];", 1,
     ["tests/test_oracle_sec6.py::test_one_ensemble_is_the_uniform_mode"]),
    ("boundary: periodic and open swapped", "if (P->periodic[c]) {", "if (!P->periodic[c]) {", 1,
     ["tests/test_oracle_step.py::test_boundaries_open_and_periodic"]),
    ("Philox: a Weyl constant off by one", "k[1] += 0xBB67AE85u;", "k[1] += 0xBB67AE86u;", 1,
     ["tests/test_philox_pin.py::test_oracle_philox_matches_aten"]),
]


def build_copy(tmp: Path, name: str, text: str) -> Path:
    d = tmp / name
    d.mkdir()
    src, out = d / "qed_oracle.c", d / "libqed_oracle.so"
    src.write_text(text)
    o.compile_library(str(src), str(out))
    return out


def run_pins(lib: Path, pins) -> subprocess.CompletedProcess:
    env = dict(os.environ, QED_ORACLE_LIB=str(lib), PYTHONPATH=str(ROOT))
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *pins],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


def test_every_mutant_is_caught(tmp_path):
    source = Path(o.SRC).read_text()
    # the pins pass on an unmodified copy built the same way
    union = sorted({p for m in MUTANTS for p in m[4]})
    base = run_pins(build_copy(tmp_path, "unmodified", source), union)
    assert base.returncode == 0, base.stdout[-3000:]

    def one(k, m):
        name, old, new, count, pins = m
        assert source.count(old) == count, (name, source.count(old))
        lib = build_copy(tmp_path, f"mutant{k}", source.replace(old, new))
        r = run_pins(lib, pins)
        # 1: tests ran and failed (not a collection error or a crash)
        return name, r.returncode, r.stdout[-1500:]

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda km: one(*km), enumerate(MUTANTS)))
    survivors = [(name, rc, out) for name, rc, out in results if rc != 1]
    assert not survivors, "\n\n".join(f"{name}: exit {rc}\n{out}" for name, rc, out in survivors)


@pytest.mark.parametrize("m", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_text_is_in_the_source(m):
    # a planted mistake must name text the oracle holds, so that an edit of
    # the oracle cannot silently turn a case into a copy of the original
    name, old, new, count, pins = m
    assert Path(o.SRC).read_text().count(old) == count and old != new
