"""The oracle pins must fail when a plausible mistake is planted in the oracle.

Each case compiles a copy of oracle/phb_oracle.cpp with one textual mistake
(on the CPU, in a temporary directory) and runs the pins that should catch it
against that copy.  A mutation that no pin catches fails this test.
"""
import os
import subprocess
import tempfile

import pytest

import oracle
from oracle import build as obuild

import test_oracle_adapt as tadapt
import test_oracle_fit as tfit
import test_oracle_levels as tlev
import test_oracle_neighbors as tnb
import test_oracle_rhs as trhs
import test_oracle_step as tstep

MUTATIONS = {
    "hessian_diag_factor": ("hess[f][0] = T(2.0) * C[3 * NF + f] * il2;",
                            "hess[f][0] = C[3 * NF + f] * il2;"),
    "weight_power": ("(T(1.0) - s2);  // sqrt of", "(T(1.0) - s2) * (T(1.0) - s2);  // sqrt of"),
    "not_centred": ("sw * (U[f * n + j] - U[f * n + i])", "sw * (U[f * n + j])"),
    "lorentz_sign": ("J[1] * B[2] - J[2] * B[1]", "J[2] * B[1] - J[1] * B[2]"),
    "curl_sign": ("g[6][1] - g[5][2]", "g[6][1] + g[5][2]"),
    "no_pressure": ("T(-(gamma - 1.0)) * g[7][a]", "T(0.0) * g[7][a]"),
    "zeta_sign": ("/ rho + zeta * gdivV[a]", "/ rho - zeta * gdivV[a]"),
    "no_heating": ("+ rho * zeta * divV * divV", "+ T(0.0) * divV"),
    "eta_dropped": ("+ eta * gdivB[a]", "+ T(0.0) * gdivB[a]"),
    "induction_compression": ("- B[a] * divV", "+ B[a] * divV"),
    "not_strict": ("return d2 < r * r;", "return d2 <= r * r;"),
    "no_min_image": ("if (periodic) d = d - len", "if (periodic < 0) d = d - len"),
    "euler_corrector": ("U[f * n + i] += 0.5 * dt * (F0[f * n + i] + F1[f * n + i]);",
                        "U[f * n + i] += dt * F0[f * n + i];"),
    "frozen_ignored": ("auto moving = [&](int64_t i) { return !(prm->frozen && prm->frozen[i]); };",
                       "auto moving = [&](int64_t i) { return i >= 0; };"),
    "law_abs_divv": ("if (val(divV) < 0.0) zeta = zeta - T(prm.c_zeta_a) * l * l * divV;",
                     "zeta = zeta + T(prm.c_zeta_a) * l * l * (val(divV) < 0.0 ? -divV : divV);"),
    "law_speed_without_field": ("const T c = sqrt((T(prm.gamma) * P + u[4] * u[4] + u[5] * u[5] + u[6] * u[6]) / u[0]);",
                                "const T c = sqrt((T(prm.gamma) * P) / u[0]);"),
    "law_lambda_once": ("zeta = zeta - T(prm.c_zeta_a) * l * l * divV;", "zeta = zeta - T(prm.c_zeta_a) * l * divV;"),
    "adapt_region_rf": ("if (!((ox * ox + oy * oy) + oz * oz < rin * rin)) continue;",
                        "if (!((ox * ox + oy * oy) + oz * oz < r * r)) continue;"),
    "adapt_clump_order": ("if (j < i && dd < dc * dc) cl = 1;", "if (j > i && dd < dc * dc) cl = 1;"),
    "adapt_grid_step": ("const double h = r * 0.25;", "const double h = r * 0.2;"),
    "adapt_best_first": ("if (mind > bclear) {", "if (mind >= bclear) {"),
    "basis_xyz_missing": ("p[13] = x * y * z;", "p[13] = x * y;"),
    "lambda_scale": ("grad[f][0] = C[0 * NF + f] * il;", "grad[f][0] = C[0 * NF + f] * il * il;"),
    "level_off_by_one": ("    int32_t L = 0;\n    while (L < max_level", "    int32_t L = 1;\n    while (L < max_level"),
    "limiter_two_levels": ("if (L0[i] - 1 > levels[j]) levels[j] = L0[i] - 1;",
                           "if (L0[i] - 2 > levels[j]) levels[j] = L0[i] - 2;"),
    "limiter_gathers": ("if (L0[i] - 1 > levels[j]) levels[j] = L0[i] - 1;",
                        "if (L0[j] - 1 > levels[i]) levels[i] = L0[j] - 1;"),
    "speed_with_bulk_velocity": ("const double c2 = (gamma * P + B2) / rho;",
                                 "const double c2 = (gamma * P + B2) / rho + U[n + i] * U[n + i];"),
    "speed_without_field": ("const double c2 = (gamma * P + B2) / rho;",
                            "const double c2 = (gamma * P) / rho;"),
}

PINS = [
    lambda: tadapt.test_isolated_particle_counts_the_shell(oracle),
    lambda: tadapt.test_lattice_has_no_voids_or_clumps(oracle),
    lambda: tadapt.test_hole_in_a_lattice(oracle),
    lambda: tadapt.test_clump_marks_the_larger_index(oracle),
    lambda: tnb.test_golden_ties_strict_periodic_nonmutual(oracle),
    lambda: tnb.test_exact_rational_bruteforce_tiny(oracle),
    lambda: tfit.test_cubic_reproduction(oracle, 0),
    lambda: tfit.test_matches_library_lstsq(oracle),
    lambda: tfit.test_rotation_equivariance(oracle),
    lambda: trhs.test_uniform_state_is_exactly_steady(oracle),
    lambda: trhs.test_circular_alfven_exact_solution_third_order(oracle),
    lambda: trhs.test_linear_wave_eigenmode_third_order(oracle, "fast"),
    lambda: trhs.test_damped_sound_wave_bulk_viscosity(oracle),
    lambda: trhs.test_divb_diffusion(oracle),
    lambda: trhs.test_viscous_heating_linear_flow(oracle),
    lambda: trhs.test_viscosity_laws_linear_flow(oracle, -1.0),
    lambda: trhs.test_viscosity_laws_linear_flow(oracle, 1.0),
    lambda: trhs.test_divb_diffusion_law(oracle),
    lambda: tstep.test_heun_is_second_order_in_time(oracle),
    lambda: tstep.test_frozen_particles_in_uniform_flow(oracle),
    lambda: tlev.test_golden_line(),
    lambda: tlev.test_power_of_two_rounding_against_the_courant_step(),
    lambda: tlev.test_bulk_velocity_does_not_change_levels(),
    lambda: tlev.test_limiter_guarantee_and_minimality(),
]


def _compile(src_text, out):
    with open(out + ".cpp", "w") as f:
        f.write(src_text)
    subprocess.run([os.environ.get("CXX", "g++"), *obuild.FLAGS, out + ".cpp", "-o", out],
                   check=True)


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, tmp_path):
    src = open(obuild.SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor not unique/found: {old!r}"
    lib = str(tmp_path / f"mut_{name}.so")
    _compile(src.replace(old, new), lib)
    caught = []
    with oracle.using(lib):
        for i, pin in enumerate(PINS):
            try:
                pin()
            except AssertionError:
                caught.append(i)
                break
    assert caught, f"no pin caught mutation {name}"


# Mistakes planted in the numpy part of the oracle (particle deletion and
# creation): each must fail one of the adaptivity pins.
APPLY_MUTATIONS = {
    "apply_new_beyond_walls": ("inside &= (cand[ax] >= lo[ax]) & (cand[ax] < lo[ax] + length[ax])",
                               "inside &= cand[ax] == cand[ax]"),
    "apply_hessian_factor": ("Unew[f] += 0.5 * hess[", "Unew[f] += 1.0 * hess["),
    "apply_no_gradient": ("Unew[f] += grad[f, a, parents] * o[a]", "Unew[f] += 0.0 * o[a]"),
    "apply_keeps_clumps": ("keep = clump == 0", "keep = clump == clump"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(APPLY_MUTATIONS))
def test_apply_mutation_is_caught(name, monkeypatch):
    import inspect
    import types
    from oracle import oracle as omod
    src = inspect.getsource(omod.adapt_apply)
    old, new = APPLY_MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor not unique/found: {old!r}"
    ns = dict(vars(omod))
    exec(compile(src.replace(old, new), "<mutated adapt_apply>", "exec"), ns)
    mutated = types.SimpleNamespace(**{k: getattr(oracle, k) for k in dir(oracle)
                                       if not k.startswith("_")})
    mutated.adapt_apply = ns["adapt_apply"]
    caught = False
    for pin in (tadapt.test_apply_fills_the_hole_with_exact_states,
                tadapt.test_apply_deletes_the_larger_index_of_a_pair):
        try:
            pin(mutated)
        except AssertionError:
            caught = True
            break
    assert caught, f"no pin caught mutation {name}"


# Mistakes planted in the numpy block-step integrator: each must fail one of
# its pins.
BLOCK_MUTATIONS = {
    # inactive neighbours held at their anchor state instead of predicted
    "block_no_prediction": ("tau = ((k + 1) - s) * delta",
                            "tau = np.where((k + 1) % m == 0, ((k + 1) - s) * delta, 0.0)"),
    # corrector with one substep instead of the particle's own step
    "block_wrong_step": ("half = 0.5 * (m[A] * delta)", "half = 0.5 * delta"),
    # explicit Euler instead of the trapezoidal corrector
    "block_euler": ("ua = u0[:, A] + half * (f0[:, A] + F)", "ua = u0[:, A] + 2.0 * half * f0[:, A]"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(BLOCK_MUTATIONS))
def test_block_mutation_is_caught(name):
    import inspect
    import types
    from oracle import oracle as omod
    import test_oracle_step as tstep
    src = inspect.getsource(omod.block_step)
    old, new = BLOCK_MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor not unique/found: {old!r}"
    ns = dict(vars(omod))
    exec(compile(src.replace(old, new), "<mutated block_step>", "exec"), ns)
    mutated = types.SimpleNamespace(**{k: getattr(oracle, k) for k in dir(oracle)
                                       if not k.startswith("_")})
    mutated.block_step = ns["block_step"]
    caught = False
    for pin in (tstep.test_block_step_one_level_is_heun, tstep.test_block_step_uniform_flow_is_exact,
                tstep.test_block_step_two_levels_second_order):
        try:
            pin(mutated)
        except AssertionError:
            caught = True
            break
    assert caught, f"no pin caught mutation {name}"
