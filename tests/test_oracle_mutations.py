"""Each oracle pin must catch a plausible mistake planted in the oracle.

A mutation rewrites one expression of a temporary copy of ``oracle/sph_oracle.c``
(a dropped term, a wrong sign, a transposed operand, a wrong constant); the copy
is compiled and the named pin is run against it in a subprocess: the pin must
fail.  The unmutated oracle passes the same pins (the other test files).

Not listed: the sign of the Christoffel term of the shear equation, which is identically
zero for the transverse components evolved in boost-invariant 2+1D (an equivalent mutant); and
Gamma^tau_{eta eta}, which ideal flow feeds only into the energy balance (the Milne work
integral), pinned by the second-law and energy-balance test.
"""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sph_oracle.c")

# (name, original text, mutated text, pin that must fail)
MUTATIONS = [
    ("kernel_norm", "return 10.0 / (7.0 * M_PI * h * h);", "return 10.0 / (7.0 * h * h);",
     "test_oracle_kernel_neighbors.py::test_kernel_normalisation"),
    ("kernel_grad_coef", "return sd / h * (-3.0 * q + 2.25 * q * q);", "return sd / h * (-3.0 * q + 2.5 * q * q);",
     "test_oracle_kernel_neighbors.py::test_kernel_shape_and_gradient"),
    ("support_inclusive", "if (r2_of(dim, x, n, a, b) < supp2) {", "if (r2_of(dim, x, n, a, b) <= supp2) {",
     "test_oracle_kernel_neighbors.py::test_boundary_cases"),
    ("morton_axis_swap", "<< (dim * b + d);", "<< (dim * b + (dim - 1 - d));",
     "test_oracle_kernel_neighbors.py::test_morton_keys_by_hand"),
    ("rest_frame_gamma", "double vol = u0 * G.sqrtg;", "double vol = G.sqrtg;",
     "test_oracle_physics.py::test_gubser_ideal_against_closed_form"),
    ("eos_drop_fprime", "sn[0] = 4.0 * T * T * T * f + T * T * T * T * fp + T * cm2;",
     "sn[0] = 4.0 * T * T * T * f + T * cm2;", "test_oracle_eos.py::test_analytic_thermodynamic_identities"),
    ("eos_jacobian_transposed", "for (int j = 0; j < m; ++j) A[i * m + j] = H[act[j] * 4 + act[i]];",
     "for (int j = 0; j < m; ++j) A[i * m + j] = H[act[i] * 4 + act[j]];",
     "test_oracle_eos.py::test_eos_derivatives_by_finite_difference"),
    ("table_weight_index", "w[k] = bit[k] ? t[k] : 1.0 - t[k];", "w[k] = bit[k] ? 1.0 - t[k] : t[k];",
     "test_oracle_eos.py::test_table_nodes_and_jacobian"),
    ("bulk_sign", "R->dBv = -(q->Pi + q->zeta * theta)", "R->dBv = -(q->Pi - q->zeta * theta)",
     "test_oracle_physics.py::test_bjorken_viscous_against_ode"),
    ("shear_drop_theta_term", " - 4.0 / 3.0 * q->taupi * q->pi[i][j] * theta) / q->taupi;", ") / q->taupi;",
     "test_oracle_physics.py::test_bjorken_viscous_against_ode"),
    ("entropy_drop_bulk", "R->dS = (-q->Pi * theta + pisig + q->uI)", "R->dS = (pisig + q->uI)",
     "test_oracle_physics.py::test_bjorken_viscous_against_ode"),
    ("shear_drop_accel_coupling", "double dpi = (rhs - chr - coup) / u0;", "double dpi = (rhs - chr) / u0;",
     "test_oracle_physics.py::test_viscous_gubser_against_ode"),
    ("momentum_drop_pi0i", "R->dP[i] = (u[i] / q->sigma) * dw + (w / q->sigma) * a[i] - (w * u[i] / (q->sigma * q->sigma)) * dsig + dpi0;",
     "R->dP[i] = (u[i] / q->sigma) * dw + (w / q->sigma) * a[i] - (w * u[i] / (q->sigma * q->sigma)) * dsig;",
     "test_oracle_physics.py::test_viscous_second_law_and_energy_balance"),
    ("force_sign", "grad[(dim * dim + i) * n + a] = -G.sqrtg * F[i];", "grad[(dim * dim + i) * n + a] = G.sqrtg * F[i];",
     "test_oracle_physics.py::test_gubser_ideal_against_closed_form"),
    ("heun_drop_slope", "y[i] = 0.5 * ((y[i] + y1[i]) + dtau * k[i]);", "y[i] = 0.5 * (y[i] + y1[i]);",
     "test_oracle_physics.py::test_gubser_ideal_against_closed_form"),
    ("work_missing_sqrtg", "wr += G.sqrtg * src / aux[0 * n + a];", "wr += src / aux[0 * n + a];",
     "test_oracle_physics.py::test_viscous_second_law_and_energy_balance"),
    ("transversality_sign", "pi[0][i] = pi[i][0] = -acc / ul[0];", "pi[0][i] = pi[i][0] = acc / ul[0];",
     "test_oracle_physics.py::test_shear_reconstruction_properties"),
    ("enthalpy_drop_dw", "R->dP[i] = (u[i] / q->sigma) * dw +", "R->dP[i] = 0.0 * dw +",
     "test_oracle_physics.py::test_gubser_ideal_against_closed_form"),
    ("fo_advection_sign", "double N[4] = {-((e - eprev[a]) / dtau - adv), 0.0, 0.0, 0.0};",
     "double N[4] = {-((e - eprev[a]) / dtau + adv), 0.0, 0.0, 0.0};",
     "test_oracle_freezeout.py::test_normals_follow_the_gubser_isotherm"),
    ("fo_gradient_sign", "de[d] += eb * dWdr * (y[d * n + a] - y[d * n + b]) / r;",
     "de[d] += eb * dWdr * (y[d * n + b] - y[d * n + a]) / r;",
     "test_oracle_freezeout.py::test_normals_follow_the_gubser_isotherm"),
    ("fo_dsigma_lab_density", "double dsig = 1.0 / (aux[16 * n + a] * fabs(un));",
     "double dsig = 1.0 / (aux[0 * n + a] * fabs(un));",
     "test_oracle_freezeout.py::test_dsigma_is_inverse_sigma_u_dot_n"),
    ("fo_drop_eta_advection", "for (int i = 0; i < dim; ++i) adv += (u[1 + i] / u[0]) * de[i];",
     "for (int i = 0; i < 2; ++i) adv += (u[1 + i] / u[0]) * de[i];",
     "test_oracle_freezeout.py::test_3d_normals_with_longitudinal_flow"),
    ("fo_norm_covariant_metric", "NN += N[mu] * N[mu] / G.g[mu];", "NN += N[mu] * N[mu] * G.g[mu];",
     "test_oracle_freezeout.py::test_3d_elements_satisfy_their_definition"),
    ("src_drop_momentum", "for (int i = 0; i < dim; ++i) F[1 + i] += G.sqrtg * I[1 + i] / aux[0 * n + a];", "",
     "test_oracle_sources.py::test_track_deposits_its_energy_and_momentum"),
    ("src_drop_heat", "for (int mu = 0; mu < 4; ++mu) q.uI += G.g[mu] * q.u[mu] * I[mu];", "",
     "test_oracle_sources.py::test_track_deposits_its_energy_and_momentum"),
    ("src_gaussian_norm", "pow(2.0 * M_PI, 1.5)", "pow(M_PI, 1.5)",
     "test_oracle_sources.py::test_track_deposits_its_energy_and_momentum"),
    ("inv_weight_swap", "w *= bit ? t[a] : 1.0 - t[a];", "w *= bit ? 1.0 - t[a] : t[a];",
     "test_oracle_offline_inverter.py::test_interpolant_converges_to_the_online_inversion"),
    ("inv_node_spacing", "double s = P->inv_p10[i / K] * (1.0 + 9.0 * (double)(i % K) / K);",
     "double s = P->inv_p10[i / K] * (1.0 + 9.5 * (double)(i % K) / K);",
     "test_oracle_offline_inverter.py::test_nodes_reproduce_the_online_inversion"),
    ("pi3_slot_swap", "static const int PI3[5][2] = {{1, 1}, {1, 2}, {1, 3}, {2, 2}, {2, 3}};",
     "static const int PI3[5][2] = {{1, 1}, {1, 2}, {2, 2}, {1, 3}, {2, 3}};",
     "test_oracle_physics.py::test_viscous_gubser_in_3p1_milne"),
    ("milne_drop_gamma_eta_tau_eta", "G->G[3][0][3] = 1.0 / tau;", "G->G[3][0][3] = 0.0;",
     "test_oracle_physics.py::test_shifted_gubser_3p1_against_closed_form"),
    ("milne_du0_drop_metric_rate", "acc += 2.0 * G->g[i] * u[i] * a[i] + u[i] * u[i] * G->dg[i];",
     "acc += 2.0 * G->g[i] * u[i] * a[i];", "test_oracle_physics.py::test_shifted_gubser_3p1_against_closed_form"),
    ("milne_norm_flat_metric", "uu += -G.g[1 + i] * ui * ui;", "uu += ui * ui;",
     "test_oracle_physics.py::test_shifted_gubser_3p1_against_closed_form"),
    ("dnmr_drop_tau_pipi", "dpp * q->pi[i][j] * theta - tpp * Ppis[i][j] +", "dpp * q->pi[i][j] * theta +",
     "test_oracle_physics.py::test_bjorken_dnmr_against_ode"),
    ("dnmr_phi7_sign", "ph7 * Ppipi[i][j] + lpP * q->Pi * sig[i][j])", "-ph7 * Ppipi[i][j] + lpP * q->Pi * sig[i][j])",
     "test_oracle_physics.py::test_bjorken_dnmr_against_ode"),
    ("dnmr_drop_lambda_piPi", "ph7 * Ppipi[i][j] + lpP * q->Pi * sig[i][j])", "ph7 * Ppipi[i][j])",
     "test_oracle_physics.py::test_bjorken_dnmr_against_ode"),
    ("dnmr_lambda_Pipi_sign", "dPP * q->Pi * theta + lPp * pisig) / q->tauPi;",
     "dPP * q->Pi * theta - lPp * pisig) / q->tauPi;", "test_oracle_physics.py::test_bjorken_dnmr_against_ode"),
    ("dnmr_projector_trace", "Ppis[m][nu] = pa - Du_up * trA / 3.0;", "Ppis[m][nu] = pa - Du_up * trA / 2.0;",
     "test_oracle_physics.py::test_bjorken_dnmr_against_ode"),
    ("parton_drop_sqrtg", "const double f = P->parton_norm * oc_W(sqrt(r2), P->parton_h, dim) / (sqrtg * P->parton_dt);",
     "const double f = P->parton_norm * oc_W(sqrt(r2), P->parton_h, dim) / P->parton_dt;",
     "test_oracle_sources.py::test_partons_in_milne_coordinates"),
    ("parton_kernel_dim", "const double f = P->parton_norm * oc_W(sqrt(r2), P->parton_h, dim) / (sqrtg * P->parton_dt);",
     "const double f = P->parton_norm * oc_W(sqrt(r2), P->parton_h, 2) / (sqrtg * P->parton_dt);",
     "test_oracle_sources.py::test_partons_deposit_their_four_momentum"),
    ("parton_window_open_end", "if (!(q[0] > t - P->parton_dt && q[0] <= t)) continue;",
     "if (!(q[0] > t - 2.0 * P->parton_dt && q[0] <= t)) continue;",
     "test_oracle_sources.py::test_partons_deposit_their_four_momentum"),
    ("charge_drop_entropy_term", "for (int c = 0; c < 3; ++c) q.uI -= q.mu[c] * Iq[c];", "",
     "test_oracle_sources.py::test_charge_deposit_changes_entropy_by_minus_mu_over_T"),
    ("charge_rate_drop_sqrtg", "q.dN[c] = G.sqrtg * Iq[c] / aux[0 * n + a];",
     "q.dN[c] = Iq[c] / aux[0 * n + a];", "test_oracle_sources.py::test_parton_charges_are_deposited"),
    ("charge_drop_enthalpy_term", "((q->n[c] / q->sigma) * dsig + q->sigma * dNq[c]);", "((q->n[c] / q->sigma) * dsig);",
     "test_oracle_sources.py::test_charge_deposit_into_moving_fluid_keeps_energy_and_momentum"),
    ("backup_ps_factor", "out[6] = out[0] / 3.0;", "out[6] = out[0] / 4.0;",
     "test_oracle_eos.py::test_backup_eos_inverts_what_the_closed_form_cannot"),
    ("backup_mu_inversion", "out[1 + q] = cbrt(n[q] * m0 * m0 * m0 * m0 / (4.0 * A0));",
     "out[1 + q] = cbrt(n[q] * m0 * m0 * m0 * m0 / (3.0 * A0));",
     "test_oracle_eos.py::test_backup_eos_inverts_what_the_closed_form_cannot"),
    ("enthalpy_drop_bulk_rate", "double dw = (q->T + q->ps) * ds + dPi;", "double dw = (q->T + q->ps) * ds;",
     "test_oracle_bulk_flow.py::test_bulk_sound_wave_in_moving_fluid"),
    ("stress_drop_bulk", "double X = -(p + Pi) * (j == i", "double X = -(p) * (j == i",
     "test_oracle_bulk_flow.py::test_bulk_sound_wave_in_moving_fluid"),
    ("diffusion_density_drop_J0", "aux[(2 + c) * n + a] = (nn[c] / G.sqrtg - j0_of(&G, dim, u, J)) / u0;",
     "aux[(2 + c) * n + a] = (nn[c] / G.sqrtg) / u0;", "test_oracle_diffusion.py::test_charge_waves_against_linear_diffusion"),
    ("diffusion_flux_drop_vJ0", "Fls[9 * a + 3 * c + k] = (J[1 + k] - (u[1 + k] / u[0]) * J[0]) / (sstar * sstar);",
     "Fls[9 * a + 3 * c + k] = (J[1 + k]) / (sstar * sstar);",
     "test_oracle_diffusion.py::test_charge_waves_against_linear_diffusion"),
    ("diffusion_projection_drop_Dalpha",
     "src += q->kap[c][c2] * (G->gi[i] * q->ga[c2][i] - u[i] * Dal_in[c2]);",
     "src += q->kap[c][c2] * (G->gi[i] * q->ga[c2][i]);",
     "test_oracle_diffusion.py::test_charge_waves_against_linear_diffusion"),
    ("diffusion_kappa_transposed", "q.kap[c][c2] = P->kappaT2[3 * c + c2] * T * T;",
     "q.kap[c][c2] = P->kappaT2[3 * c2 + c] * T * T;",
     "test_oracle_diffusion.py::test_charge_waves_against_linear_diffusion"),
    ("diffusion_drop_u0", "const double dJ = (DJ - chr) / u[0];", "const double dJ = (DJ - chr);",
     "test_oracle_diffusion.py::test_charge_waves_against_linear_diffusion"),
    ("diffusion_flux_sign", "dNt[3 * a + c] = -G.sqrtg * dv[c];", "dNt[3 * a + c] = G.sqrtg * dv[c];",
     "test_oracle_diffusion.py::test_charge_waves_against_linear_diffusion"),
    ("diffusion_source_sign", "const double DJ = (-q->Jc[c][i] + src) / q->tJ[c] - u[i] * jDu;",
     "const double DJ = (-q->Jc[c][i] - src) / q->tJ[c] - u[i] * jDu;",
     "test_oracle_diffusion.py::test_charge_waves_against_linear_diffusion"),
    ("diffusion_flux_not_antisymmetric", "dv[c] += (Fls[9 * a + 3 * c + kk] + Fls[9 * b + 3 * c + kk]) * gw[kk];",
     "dv[c] += (2.0 * Fls[9 * b + 3 * c + kk]) * gw[kk];", "test_oracle_diffusion.py::test_lab_charge_conserved_exactly"),
    ("dnmr_bulk_drop_volume_rate", "R->dBv = (DPi + q->Pi * theta) / (u0 * q->sigma);",
     "R->dBv = DPi / (u0 * q->sigma);", "test_oracle_physics.py::test_bjorken_dnmr_against_ode"),
    ("stop_rule_inverted", "(P->T_stop_GeV > 0.0 && aux[5 * n + a] * HBARC < P->T_stop_GeV)",
     "(P->T_stop_GeV > 0.0 && aux[5 * n + a] * HBARC > P->T_stop_GeV)",
     "test_oracle_physics.py::test_stop_temperature_freezes_cold_particles"),
    ("stop_rule_frozen_at_rest", "for (int i = 0; i < dim; ++i) dydt[i * n + a] = y[(dim + i) * n + a] / u0;",
     "for (int i = 0; i < dim; ++i) dydt[i * n + a] = 0.0 * u0;",
     "test_oracle_physics.py::test_stop_temperature_freezes_cold_particles"),
]


def _spec(m):
    return m.values if hasattr(m, "values") else m


def _run_mutant(workdir, name, orig, mut, pin):
    src = open(SRC).read()
    if src.count(orig) != 1:
        return ("anchor", f"mutation anchor not unique/absent: {orig}")
    cfile = os.path.join(workdir, f"{name}.c")
    sofile = os.path.join(workdir, f"{name}.so")
    open(cfile, "w").write(src.replace(orig, mut))
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fopenmp", "-fPIC",
                           "-shared", "-o", sofile, cfile, "-lm"])
    env = dict(os.environ, SPH_ORACLE_LIB=sofile, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pin)], env=env, capture_output=True, text=True, cwd=ROOT,
                       timeout=900)
    return (r.returncode, r.stdout[-2000:])


@pytest.fixture(scope="module")
def results():
    """All mutants compiled and run concurrently (each pin in its own process)."""
    with tempfile.TemporaryDirectory() as d:
        workers = max(2, (os.cpu_count() or 4) // 2)
        with cf.ThreadPoolExecutor(max_workers=workers) as ex:
            futs = {_spec(m)[0]: ex.submit(_run_mutant, d, *_spec(m)) for m in MUTATIONS}
            yield {k: f.result() for k, f in futs.items()}


@pytest.mark.parametrize("name,orig,mut,pin", MUTATIONS,
                         ids=[m[0] if isinstance(m, tuple) else None for m in MUTATIONS])
def test_pin_catches_planted_mistake(results, name, orig, mut, pin):
    code, out = results[name]
    assert code != "anchor", out
    assert code != 0, f"pin {pin} did not catch mutation {name}:\n{out}"
