"""Pins against planted mistakes: each mutation below changes one sign,
factor, weight, index or stored value of the oracle (a copy of lbmo.c built
into a temporary library), and the pin named beside it must then fail.  An
unmutated build passes the same pins.  The mutated oracles never leave the
test: they are loaded by child processes through LBMO_LIBRARY."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbmo.c")

# name: (first occurrence in lbmo.c, its replacement, pin that must fail)
MUTATIONS = {
    # collision of the flow populations (Sec. 2.3) and the closure
    "velocity_force_half": ("c->u[i] = J[i] / (c->rho * CS2) + c->F[i] / (2.0 * c->rho);",
                            "c->u[i] = J[i] / (c->rho * CS2) + c->F[i] / c->rho;",
                            "test_oracle_collision.py::test_moment_identities"),
    "xi_drops_force": ("Xi[a] = CS2 * (G - L->w[a]) * cmu_grho + cmu_F * G;",
                       "Xi[a] = CS2 * (G - L->w[a]) * cmu_grho;",
                       "test_oracle_collision.py::test_moment_identities"),
    "omega_offset": ("1.0 / (c->nu / CS2 + 0.5);", "1.0 / (c->nu / CS2 + 0.25);",
                     "test_oracle_collision.py::test_moment_identities"),
    "mu_laplacian_sign": ("(2.0 * phi - 1.0) - d->kappa * lap;", "(2.0 * phi - 1.0) + d->kappa * lap;",
                          "test_oracle_collision.py::test_moment_identities"),
    "body_force_sign": ("c->F[s->vert] -= (c->rho", "c->F[s->vert] += (c->rho",
                        "test_oracle_collision.py::test_moment_identities"),
    "trace_equilibrium": ("T -= ob * (T - 3.0 * CS2);", "T -= ob * (T - 3.0);",
                          "test_oracle_collision.py::test_unit_rates_give_product_equilibrium"),
    "shear_split_index": ("K[KI(0, 0, 2)] = (T + d1 - 2.0 * d2) / 3.0;", "K[KI(0, 0, 2)] = (T - 2.0 * d1 + d2) / 3.0;",
                          "test_oracle_collision.py::test_shear_rate_on_second_order_only"),
    "cumulant4_factor": ("K[KI(2, 2, 0)] = k[KI(2, 2, 0)] - (k200 * k020 + 2.0 * k110 * k110);",
                         "K[KI(2, 2, 0)] = k[KI(2, 2, 0)] - (k200 * k020 + 1.0 * k110 * k110);",
                         "test_oracle_cumulants.py::test_forward_cumulants_match_partition_formula"),
    "cumulant6_cubic_factor": ("double cub = 16.0 * k110 * k101 * k011", "double cub = 8.0 * k110 * k101 * k011",
                               "test_oracle_cumulants.py::test_forward_cumulants_match_partition_formula"),
    # phase field (Sec. 2.2)
    "sharpening_sign": ("+ d->lambda_phi * Lg->w[a] * cn * X + corr;", "- d->lambda_phi * Lg->w[a] * cn * X + corr;",
                        "test_oracle_collision.py::test_phase_field_collision_moments"),
    "tau_phi_offset": ("o->tau_phi = o->M / cs2g + 0.5;", "o->tau_phi = o->M / cs2g + 1.0;",
                       "test_oracle_lattice.py::test_derived_closure"),
    # reduced phase lattice (Sec. 2.2 alternative, readings P1-P3)
    "reduced_equilibrium_sign": ("geq = Lg->w[a] * phi * (1.0 + cu / Lg->cs2);",
                                 "geq = Lg->w[a] * phi * (1.0 - cu / Lg->cs2);",
                                 "test_oracle_phase_reduced.py::test_reduced_collision_moments"),
    "correction_factor": ("corr = d->lambda_phi * Lg->w[a] * cd / Lg->cs2;", "corr = Lg->w[a] * cd / Lg->cs2;",
                          "test_oracle_phase_reduced.py::test_reduced_collision_moments"),
    "face_weight": ("L->w[L->Q] = moving ? 1.0 / 8.0 : 1.0 / 4.0;", "L->w[L->Q] = moving ? 1.0 / 6.0 : 0.0;",
                    "test_oracle_phase_reduced.py::test_reduced_lattice"),
    "phase_lattice_cs2": ("const double cs2g = ((p->flags & LBMO_FLAG_PHASE_REDUCED) && D == 3) ? 0.25 : CS2;",
                          "const double cs2g = CS2;",
                          "test_oracle_phase_reduced.py::test_reduced_relaxation_time"),
    "stored_phi_u": ("for (int k = 0; k < 3; ++k) s->phiu_prev[(size_t)k * N + i] = diag[14 + k];",
                     "for (int k = 0; k < 3; ++k) s->phiu_prev[(size_t)k * N + i] = 0.0;",
                     "test_oracle_phase_reduced.py::test_reduced_interface_galilean_invariance"),
    # symmetry axis of the 2-D splash (Sec. 3.4, reading A28)
    "symmetry_bounces_back": ("                p = xyz[k];\n                flip[k] = mirrored = 1;",
                              "                wall = 1;",
                              "test_oracle_symmetry.py::test_half_domain_equals_half_of_the_symmetric_full_domain"),
    "symmetry_keeps_direction": ("const int b = mirrored ? mirror_dir(Lx, a, flip) : a;", "const int b = a;",
                                 "test_oracle_symmetry.py::test_half_domain_equals_half_of_the_symmetric_full_domain"),
    "symmetry_ghost_wraps": ("    if (periodic == 1) return ((y % n) + n) % n;", "    if (periodic) return ((y % n) + n) % n;",
                             "test_oracle_symmetry.py::test_half_domain_equals_half_of_the_symmetric_full_domain"),
    "drop_axis_ignored": ("double c0 = (k == v) ? zc : (nargs > 4 ? A[4] : (double)(s->n[k] / 2));",
                          "double c0 = (k == v) ? zc : (double)(s->n[k] / 2);",
                          "test_oracle_symmetry.py::test_half_domain_equals_half_of_the_symmetric_full_domain"),
    # observables and initial states
    "kinetic_energy_half": ("ke_c[i] = 0.5 * m.rho * uu;", "ke_c[i] = m.rho * uu;",
                            "test_oracle_observables.py::test_kinetic_energy_closed_forms"),
    "kinetic_energy_density": ("ke_c[i] = 0.5 * m.rho * uu;", "ke_c[i] = 0.5 * uu;",
                               "test_oracle_observables.py::test_kinetic_energy_closed_forms"),
    "max_speed_squared": ("um_c[i] = sqrt(uu);", "um_c[i] = uu;",
                          "test_oracle_observables.py::test_max_speed_closed_forms"),
    "spike_tip_weight": ("o->tip_spike = k - (pk - 0.5) / (pk - pm);", "o->tip_spike = k - (pk - 0.5) / (pk + pm);",
                         "test_oracle_observables.py::test_tip_interpolation_exact_on_linear_columns"),
    "bubble_tip_index": ("o->tip_bubble = k + (0.5 - pk) / (pp - pk);",
                         "o->tip_bubble = k + 1 + (0.5 - pk) / (pp - pk);",
                         "test_oracle_observables.py::test_tip_interpolation_exact_on_linear_columns"),
    "drop_centre_offset": ("double zc = sheet + 0.5 * Dd + 2.0 * d->W;", "double zc = sheet + 0.5 * Dd + d->W;",
                           "test_oracle_observables.py::test_drop_sheet_start_geometry"),
    "drop_radius": ("double d_drop = 0.5 * Dd - sqrt(r2);", "double d_drop = Dd - sqrt(r2);",
                    "test_oracle_observables.py::test_drop_sheet_start_geometry"),
    "drop_sheet_union": ("phi = tanh_profile(fmax(d_drop, d_sheet), d->W);",
                         "phi = tanh_profile(fmin(d_drop, d_sheet), d->W);",
                         "test_oracle_observables.py::test_drop_sheet_start_geometry"),
    "hydrostatic_factor": ("p = -d->g_accel * (d->rho_h - d->rho_l) * 0.25 * d->W * lncosh;",
                           "p = -d->g_accel * (d->rho_h - d->rho_l) * 0.5 * d->W * lncosh;",
                           "test_oracle_observables.py::test_rt_hydrostatic_start"),
    "hydrostatic_sign": ("p = -d->g_accel * (d->rho_h - d->rho_l) * 0.25 * d->W * lncosh;",
                         "p = d->g_accel * (d->rho_h - d->rho_l) * 0.25 * d->W * lncosh;",
                         "test_oracle_observables.py::test_rt_hydrostatic_start"),
    "rt_perturbation_y": ("if (D == 3) h += A[1] * cos(2.0 * PI * y / s->n[1]);",
                          "if (D == 3) h += A[1] * sin(2.0 * PI * y / s->n[1]);",
                          "test_oracle_observables.py::test_rt_start_interface_and_tips"),
    # divergence term (reading V1)
    "wall_ghost_sign": ("if ((v < 0 || v >= s->n[k]) && s->per[k] == 0) sign = -1;",
                        "if ((v < 0 || v >= s->n[k]) && s->per[k] == 0) sign = 1;",
                        "test_oracle_divu.py::test_divergence_wall_ghost_closed_form"),
    "divergence_factor": ("Xi[a] += L->w[a] * CS2 * c.rho * divu;", "Xi[a] += 0.5 * L->w[a] * CS2 * c.rho * divu;",
                          "test_oracle_divu.py::test_divergence_term_moments"),
    "previous_velocity_reset": ("s->u_prev[(size_t)k * N + i] = c.u[k];", "s->u_prev[(size_t)k * N + i] = 0.0;",
                                "test_oracle_divu.py::test_divergence_step_matches_cellwise"),
}


def _build(source, out):
    subprocess.run(["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", "-I", os.path.join(ROOT, "oracle"),
                    "-o", out, source, "-lm"], check=True)


def _pin_passes(lib, pin):
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", pin), "-q", "-x",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=dict(os.environ, LBMO_LIBRARY=lib),
                       capture_output=True, text=True, timeout=600)
    return r.returncode == 0


def test_unmutated_copy_passes_the_pins(tmp_path):
    lib = str(tmp_path / "liblbmo_ref.so")
    _build(SRC, lib)
    for pin in sorted({m[2] for m in MUTATIONS.values()}):
        assert _pin_passes(lib, pin), pin


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new, pin = MUTATIONS[name]
    text = open(SRC).read()
    assert old in text, f"{name}: anchor not found in lbmo.c"
    src = tmp_path / "lbmo.c"
    src.write_text(text.replace(old, new, 1))
    lib = str(tmp_path / "liblbmo_mut.so")
    _build(str(src), lib)
    assert not _pin_passes(lib, pin), f"{name} went unnoticed by {pin}"
