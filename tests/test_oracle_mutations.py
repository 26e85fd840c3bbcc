"""The oracle's pins are sensitive: each plausible mistake, planted in a copy
of the oracle source and compiled on the CPU, makes at least one pin fail.

The mutants never touch the real oracle build; they are compiled into a
temporary directory and swapped in only for the duration of one check.
"""
import numpy as np
import pytest

import oracle
import test_oracle_hlbm as H
import test_oracle_open as O
import test_oracle_diss as DS
import test_oracle_diss3d as D3
import test_oracle_pins as P
import test_oracle_powell as W
import test_oracle_resistive as R

IDEAL_PINS = [
    lambda o: P.test_lattice_quadrature(o, 5),
    lambda o: P.test_lattice_quadrature(o, 7),
    lambda o: P.test_flux_jacobian_eigenvalues_are_mhd_wave_speeds(o, 1),
    lambda o: P.test_flux_jacobian_eigenvalues_are_mhd_wave_speeds(o, 2),
    lambda o: P.test_equilibrium_moments_return_state_and_flux(o, 2),
    lambda o: P.test_equilibrium_moments_return_state_and_flux(o, 3),
    lambda o: P.test_exact_conservation_periodic(o, 2, 0.9),
    lambda o: P.test_centred_divB_stays_zero_with_tau_B_one(o, 3),
    lambda o: P.test_linear_wave_speed_and_decay(o, "sound"),
    lambda o: P.test_linear_wave_speed_and_decay(o, "oblique"),
    lambda o: P.test_direct_source_injection_adds_S_per_cell_per_step(o),
    lambda o: P.test_update_is_covariant_under_the_rotations_of_the_lattice(o, 2),
    lambda o: P.test_update_is_covariant_under_the_rotations_of_the_lattice(o, 3),
    lambda o: P.test_linearised_update_operator_predicts_the_run(o),
    lambda o: P.test_linearised_d3q7_operator_predicts_the_3d_run(o),
    lambda o: P.test_linearised_operator_has_the_mhd_speeds_and_decay(o),
]
RES_PINS = [
    lambda o: R.test_mass_exact_and_force_adds_F_per_cell(o),
    lambda o: R.test_shear_wave_decay_gives_viscosity(o),
    lambda o: R.test_magnetic_diffusion_gives_eta(o),
    lambda o: R.test_poiseuille_profile(o),
    lambda o: R.test_hartmann_profile(o, 5.0),
    lambda o: R.test_channel_update_is_symmetric_under_the_mirror_between_its_walls(o),
    lambda o: R.test_channel_update_is_covariant_under_the_quarter_turn_about_y(o),
]

POWELL_PINS = [
    lambda o: W.test_trace_flux_is_the_trace_of_the_gradient_tensor_flux(),
    lambda o: W.test_solenoidal_field_keeps_D_zero_and_matches_the_ideal_scheme((6, 8, 10)),
    lambda o: W.test_D_relaxes_to_tau_m_times_the_divergence(),
    lambda o: W.test_powell_source_cancels_the_monopole_force(),
    lambda o: W.test_mass_is_conserved_exactly(),
    lambda o: W.test_uniform_state_D_decays_geometrically_and_first_step_momentum(),
    lambda o: W.test_one_uniform_step_moves_every_field_by_the_divergence_times_its_factor(),
]

HLBM_PINS = [
    lambda o: H.test_porosity_of_the_signed_distance(),
    lambda o: H.test_blended_state_of_one_cell(0.25),
    lambda o: H.test_update_is_covariant_under_the_rotations_of_the_lattice(3),
    lambda o: H.test_fluid_everywhere_is_the_ideal_scheme((4, 6, 5)),
    lambda o: H.test_uniform_solid_cell_relaxes_to_the_solid_state(),
    lambda o: H.test_mass_is_conserved_exactly(),
    lambda o: H.test_channel_between_homogenised_walls_is_parabolic_with_walls_at_d_half(),
    lambda o: H.test_uniform_cell_pressure_follows_the_relaxation_of_the_blend(0.6),
]

OPEN_PINS = [
    lambda o: O.test_uniform_state_is_a_fixed_point(
        (12, 16), [(O.ALL, O.BG), (0, None), (0b10110, O.BG), (0b01001, O.BG)]),
    lambda o: O.test_open_run_equals_the_periodic_run_inside_the_light_cone(
        (40, 40), [(O.ALL, O.BG), (0, None), (0b10110, O.BG), (0b01001, O.BG)], 12),
    lambda o: O.test_supersonic_inflow_flushes_the_domain_to_the_inflow_state(),
    lambda o: O.test_zero_gradient_faces_let_a_pulse_leave(),
    lambda o: O.test_oracle_matches_numpy_restatement((5, 6, 7)),
    lambda o: O.test_update_is_symmetric_under_the_mirror_that_swaps_the_x_faces(),
]

DISS_PINS = [
    lambda o: DS.test_gradient_lattices_relax_to_tau_m_times_the_gradients(),
    lambda o: DS.test_shear_wave_decays_at_nu_plus_the_lattice_diffusion(0.01),
    lambda o: DS.test_magnetic_sheet_diffuses_at_eta_plus_the_lattice_diffusion(0.01),
    lambda o: DS.test_current_dependent_resistivity_projects_onto_the_mode(),
    lambda o: DS.test_conserved_fields_are_conserved_exactly(),
    lambda o: DS.test_heat_appears_where_the_dissipation_is("viscous"),
    lambda o: DS.test_heat_appears_where_the_dissipation_is("ohmic"),
    lambda o: DS.test_uniform_step_with_the_powell_source_and_relaxing_gradients(),
    lambda o: DS.test_oracle_matches_numpy_restatement(True),
    lambda o: DS.test_update_is_covariant_under_the_quarter_turn_of_the_lattice(True),
]

DISS3_PINS = [
    lambda o: D3.test_without_dissipation_the_mhd_fields_follow_the_ideal_scheme(),
    lambda o: D3.test_update_is_covariant_under_the_cyclic_rotation_of_the_axes(True),
    lambda o: D3.test_shear_wave_along_z_decays_at_nu_plus_the_lattice_diffusion(0.01),
    lambda o: D3.test_magnetic_sheet_along_z_diffuses_at_eta_plus_the_lattice_diffusion(0.01),
    lambda o: D3.test_z_gradient_lattices_relax_to_tau_m_times_the_gradients(),
    lambda o: D3.test_uniform_step_with_the_powell_source_and_relaxing_gradients(),
    lambda o: D3.test_conserved_fields_are_conserved_exactly(),
]

# (name, original text, planted mistake, which pin family must catch it)
MUTANTS = [
    ("induction flux transposed", "phi[3 * (5 + b) + a] = u[a] * B[b] - B[a] * u[b];",
     "phi[3 * (5 + b) + a] = u[b] * B[a] - B[b] * u[a];", IDEAL_PINS),
    ("energy flux misses B(u.B)", "phi[3 * 4 + a] = (e + ptot) * u[a] - B[a] * uB;",
     "phi[3 * 4 + a] = (e + ptot) * u[a];", IDEAL_PINS),
    ("total pressure misses B^2/2", "double ptot = p + 0.5 * B2;", "double ptot = p;",
     IDEAL_PINS),
    ("EOS misses magnetic energy", "(e - 0.5 * rho * u2 - 0.5 * B2); /* Eq. 9 */",
     "(e - 0.5 * rho * u2); /* Eq. 9 */", IDEAL_PINS),
    ("Maxwell stress sign", "+ ptot * delta - B[a] * B[b];", "+ ptot * delta + B[a] * B[b];",
     IDEAL_PINS),
    ("Maxwell stress from B_x on every axis", "+ ptot * delta - B[a] * B[b];", "+ ptot * delta - B[0] * B[b];",
     IDEAL_PINS),
    ("D2Q5 rest weight", "set_dir(L, 0, 0, 0, 0, 1.0 / 3.0);\n        set_dir(L, 1, 1, 0, 0, 1.0 / 6.0);",
     "set_dir(L, 0, 0, 0, 0, 0.3);\n        set_dir(L, 1, 1, 0, 0, 1.0 / 6.0);", IDEAL_PINS),
    ("equilibrium drops 1/cs^2", "feq[k][i] = L->w[i] * (Q[k] + cphi / L->cs2);",
     "feq[k][i] = L->w[i] * (Q[k] + cphi);", IDEAL_PINS),
    ("BGK relaxes the wrong way", "double out = f + (feq[k][i] - f) / tau[k];",
     "double out = f + (f - feq[k][i]) / tau[k];", IDEAL_PINS),
    ("BGK takes the first lattice's tau", "double out = f + (feq[k][i] - f) / tau[k];",
     "double out = f + (feq[k][i] - f) / tau[0];", IDEAL_PINS),
    ("streams against c_i", "long dst = neighbour(x, y, z, L.c[i], nx, ny, nz);\n            for (int k = 0;",
     "long dst = neighbour(x, y, z, L.c[L.opp[i]], nx, ny, nz);\n            for (int k = 0;",
     IDEAL_PINS),
    ("source injected without weight", "if (src) out += L->w[i] * src[k];",
     "if (src) out += src[k];", IDEAL_PINS),
    ("bounce-back keeps direction", "fout[(long)L19.opp[i] * N + cell] = fs[i];",
     "fout[(long)i * N + cell] = fs[i];", RES_PINS),
    ("bounce-back at the bottom wall only", "if (is_wall(dy, ny, walls_y))",
     "if (is_wall(dy, ny, walls_y) && dy == 0)", RES_PINS),
    ("Guo force half-step factor", "double guo = (1.0 - 0.5 / tau_f) * L19->w[i] *",
     "double guo = L19->w[i] *", RES_PINS),
    ("magnetic flux transposed", "for (int a = 0; a < 3; ++a) phi[a] = u[a] * B[b] - B[a] * u[b];",
     "for (int a = 0; a < 3; ++a) phi[a] = u[b] * B[a] - B[b] * u[a];", RES_PINS),
    ("Maxwell stress missing in flow", "(a == b ? 0.5 * B2 : 0.0) - B[a] * B[b];",
     "(a == b ? 0.5 * B2 : 0.0);", RES_PINS),
    ("trace flux adds B", "phi[3 * 8 + a] = Q[8] * (Q[1 + a] / rho) - Q[5 + a];",
     "phi[3 * 8 + a] = Q[8] * (Q[1 + a] / rho) + Q[5 + a];", POWELL_PINS),
    ("trace flux misses D u", "phi[3 * 8 + a] = Q[8] * (Q[1 + a] / rho) - Q[5 + a];",
     "phi[3 * 8 + a] = -Q[5 + a];", POWELL_PINS),
    ("divergence scaled by tau_M", "double divB = Q[8] / tau_m;", "double divB = Q[8] * tau_m;",
     POWELL_PINS),
    ("momentum source along u", "S[1 + b] = -divB * B[b];", "S[1 + b] = -divB * u[b];", POWELL_PINS),
    ("induction source along B", "S[5 + b] = -divB * u[b];", "S[5 + b] = -divB * B[b];", POWELL_PINS),
    ("energy source sign", "S[4] = -divB * uB;", "S[4] = divB * uB;", POWELL_PINS),
    ("mass source", "S[0] = 0.0;", "S[0] = -divB;", POWELL_PINS),
    ("trace relaxation sign", "S[8] = -Q[8] / tau_m;", "S[8] = Q[8] / tau_m;", POWELL_PINS),
    ("Powell step streams against c_i", "long to = neighbour(x, y, z, L.c[i], nx, ny, nz);",
     "long to = neighbour(x, y, z, L.c[L.opp[i]], nx, ny, nz);", POWELL_PINS),
    ("Powell equilibrium drops 1/cs^2", "double moving = cphi / L->cs2;", "double moving = cphi;",
     POWELL_PINS),
    ("porosity blend reversed", "uh[a] = d * u[a] + (1.0 - d) * uB[a];",
     "uh[a] = (1.0 - d) * u[a] + d * uB[a];", HLBM_PINS),
    ("field blended with the solid velocity", "Bh[a] = d * B[a] + (1.0 - d) * BB[a];",
     "Bh[a] = d * B[a] + (1.0 - d) * uB[a];", HLBM_PINS),
    ("porosity without the 1/2 offset", "return phi / eps_h + 0.5;", "return phi / eps_h;", HLBM_PINS),
    ("blended density", "Qhat[0] = rho;", "Qhat[0] = d * rho + (1.0 - d);", HLBM_PINS),
    ("HLBM step streams against c_i", "long target = neighbour(x, y, z, L.c[i], nx, ny, nz);",
     "long target = neighbour(x, y, z, L.c[L.opp[i]], nx, ny, nz);", HLBM_PINS),
    ("blended energy keeps the cell's e", "Qhat[4] = p / (gamma - 1.0) + 0.5 * rho * uh2 + 0.5 * Bh2;",
     "Qhat[4] = Q[4];", HLBM_PINS),
    ("blended energy misses the field energy", "Qhat[4] = p / (gamma - 1.0) + 0.5 * rho * uh2 + 0.5 * Bh2;",
     "Qhat[4] = p / (gamma - 1.0) + 0.5 * rho * uh2;", HLBM_PINS),
    ("boundary fills the leaving direction", "inward[a] = (face % 2 == 0) ? 1 : -1;",
     "inward[a] = (face % 2 == 0) ? -1 : 1;", OPEN_PINS),
    ("Dirichlet and Neumann swapped",
     "Qb[k] = ((mask[face] >> k) & 1u) ? vals[ORC_NVAR_IDEAL * face + k] : Qn[k];",
     "Qb[k] = ((mask[face] >> k) & 1u) ? Qn[k] : vals[ORC_NVAR_IDEAL * face + k];", OPEN_PINS),
    ("Neumann copies the boundary cell itself",
     "long nb = (long)(x + normal[0]) + (long)nx * ((long)(y + normal[1]) + (long)ny * (long)(z + normal[2]));",
     "long nb = cell;", OPEN_PINS),
    ("every face takes face 0's values",
     "Qb[k] = ((mask[face] >> k) & 1u) ? vals[ORC_NVAR_IDEAL * face + k] : Qn[k];",
     "Qb[k] = ((mask[face] >> k) & 1u) ? vals[k] : Qn[k];", OPEN_PINS),
    ("boundary state from the pre-stream state", "Qn[k] += fout[(long)(k * q + i) * N + nb]; /* Eq. 4 */",
     "Qn[k] += fin[(long)(k * q + i) * N + nb]; /* Eq. 4 */", OPEN_PINS),
    ("viscous stress sign", "- B[c] * B[b] - visc[c][b];", "- B[c] * B[b] + visc[c][b];", DISS_PINS),
    ("viscous stress without the transpose", "rho * nu * (du[a][b] + du[b][a])", "rho * nu * (du[a][b] + du[a][b])",
     DISS_PINS),
    ("resistivity linear in j", "j2 / (j_c * j_c)", "sqrt(j2) / j_c", DISS_PINS),
    ("induction diffusion sign", "- eta * dB[c][b];", "+ eta * dB[c][b];", DISS_PINS),
    ("induction diffusion transposed", "- eta * dB[c][b];", "- eta * dB[b][c];", DISS_PINS),
    ("ohmic energy flux sign", "- u_visc + eta * jxB[c];", "- u_visc - eta * jxB[c];", DISS_PINS),
    ("viscous work sign", "- u_visc + eta * jxB[c];", "+ u_visc + eta * jxB[c];", DISS_PINS),
    ("gradient flux on the wrong axis", "phi[3 * (8 + 3 * a + b) + c] = Q[8 + 3 * a + b] * u[c] - (a == c ? B[b] : 0.0);",
     "phi[3 * (8 + 3 * a + b) + c] = Q[8 + 3 * a + b] * u[c] - (b == c ? B[a] : 0.0);", DISS_PINS),
    ("velocity gradient fed by B", "phi[3 * (w0 + 3 * a + b) + c] = Q[w0 + 3 * a + b] * u[c] - (a == c ? u[b] : 0.0);",
     "phi[3 * (w0 + 3 * a + b) + c] = Q[w0 + 3 * a + b] * u[c] - (a == c ? B[b] : 0.0);", DISS_PINS),
    ("divergence from G_xy", "trace += Q[8 + 4 * a]; /* G_aa */", "trace += Q[8 + a]; /* G_aa */", DISS_PINS),
    ("gradient relaxation sign", "for (int k = 8; k < nvar; ++k) S[k] = -Q[k] / tau_m;",
     "for (int k = 8; k < nvar; ++k) S[k] = Q[k] / tau_m;", DISS_PINS),
    ("current without the minus of the curl", "dB[0][1] - dB[1][0]", "dB[0][1] + dB[1][0]", DISS_PINS),
    ("3-D gradients read two rows", "dB[a][b] = a < dim ? Q[8 + 3 * a + b] / tau_m : 0.0;",
     "dB[a][b] = a < 2 ? Q[8 + 3 * a + b] / tau_m : 0.0;", DISS3_PINS),
    ("3-D velocity gradients read two rows", "du[a][b] = a < dim ? Q[w0 + 3 * a + b] / tau_m : 0.0;",
     "du[a][b] = a < 2 ? Q[w0 + 3 * a + b] / tau_m : 0.0;", DISS3_PINS),
    ("3-D Powell divergence misses G_zz", "for (int a = 0; a < dim; ++a) trace += Q[8 + 4 * a];",
     "for (int a = 0; a < 2; ++a) trace += Q[8 + 4 * a];", DISS3_PINS),
    ("3-D W fluxes at the 2-D offset", "    const int w0 = 8 + 3 * dim;\n    double rho = Q[0];",
     "    const int w0 = 14;\n    double rho = Q[0];", DISS3_PINS),
    ("3-D gradient fluxes stop at the y row", "        for (int a = 0; a < dim; ++a)\n            for (int b = 0; b < 3; ++b) {\n                phi[3 * (8",
     "        for (int a = 0; a < 2; ++a)\n            for (int b = 0; b < 3; ++b) {\n                phi[3 * (8", DISS3_PINS),
    ("Powell source without weight", "fout[k * L->q + i] = f + (feq[k][i] - f) / tau[k] + L->w[i] * sk;",
     "fout[k * L->q + i] = f + (feq[k][i] - f) / tau[k] + sk;", POWELL_PINS),
]


@pytest.mark.parametrize("name,orig,planted,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, orig, planted, pins):
    src = oracle.source_text()
    assert src.count(orig) == 1, "mutation anchor not unique: " + name
    so = oracle.compile_variant(src.replace(orig, planted), str(tmp_path / "mutant.so"))
    caught = []
    with oracle.use_library(so):
        for pin in pins:
            try:
                with np.errstate(all="ignore"):
                    pin(oracle)
            except Exception as exc:  # an assertion or a numerical failure
                caught.append(type(exc).__name__)
    assert caught, "no pin caught the planted mistake: " + name
