"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a temporary copy of oracle/apbf_oracle.c,
compiles it on the CPU, points the oracle wrapper at the mutant and runs the
pin that should catch it, which must then fail.
"""
import os
import subprocess

import pytest

import oracle as O
from oracle import build as B
import tests.test_oracle_dtvs_pins as dtvs
import tests.test_oracle_obstacle_pins as obst
import tests.test_oracle_pins as pins

MUTATIONS = [
    ("self term dropped from the density",
     "double rho = m * orc_poly6(0.0, h);", "double rho = 0.0;",
     lambda: pins.test_interior_lattice_particle_at_rest_density(O.rest_density(0.1, 1.0, 0.05))),
    ("grad_i C_i dropped from the lambda denominator",
     "    sum_sq += gi[0] * gi[0] + gi[1] * gi[1] + gi[2] * gi[2];\n", "\n",
     pins.test_lambda_zeroes_the_linearised_constraint),
    ("lambda_j replaced by lambda_i in Eq. 7",
     "double s = lam[i] + lam[j] +", "double s = lam[i] + lam[i] +",
     pins.test_delta_p_equals_eq3_summed_over_constraints),
    ("spiky gradient with the wrong sign",
     "double c = -45.0 /", "double c = 45.0 /",
     pins.test_spiky_gradient_matches_finite_differences),
    ("neighbour search skips the +x cells",
     "for (int dx = -1; dx <= 1; ++dx)", "for (int dx = -1; dx <= 0; ++dx)",
     lambda: pins.test_neighbors_equal_brute_force(0)),
    ("LOD levels reversed (near gets n_min)",
     "level[i] = p->n_max - b;", "level[i] = p->n_min + b;",
     pins.test_lod_levels_bins),
    ("counting sort not stable",
     "order[cell_start[k] + fill[k]] = i;", "order[cell_start[k + 1] - 1 - fill[k]] = i;",
     pins.test_counting_sort_is_stable_argsort),
    ("XSPH with the relative velocity reversed",
     "acc[a] += mr * (v[3 * j + a] - v[3 * i + a]) * W;", "acc[a] += mr * (v[3 * i + a] - v[3 * j + a]) * W;",
     pins.test_xsph_invariants),
    ("prediction uses the velocity before the forces",
     "float xp = x[3 * i + a] + p->dt * vv;", "float xp = x[3 * i + a] + p->dt * v[3 * i + a];",
     pins.test_isolated_particle_free_fall),
    ("finished particles keep moving for one more iteration",
     "            if (lvl[s] >= l) {\n                xs[3 * s + 0] += dp[3 * s + 0];",
     "            if (lvl[s] + 1 >= l) {\n                xs[3 * s + 0] += dp[3 * s + 0];",
     lambda: pins.test_active_sets_nested_and_finished_particles_fixed(O.rest_density(0.1, 1.0, 0.05))),
    ("DTVS depth at the sphere's exit instead of its entry",
     "float t = b - sqrtf(disc);", "float t = b + sqrtf(disc);",
     lambda: dtvs.test_depth_of_one_sphere_is_the_closed_form(0)),
    ("DTVS image rows counted from the bottom",
     "float sy = (1.0f - (float)(2 * py + 1) / (float)v->height) * ay;",
     "float sy = ((float)(2 * py + 1) / (float)v->height - 1.0f) * ay;",
     dtvs.test_pixel_rays_are_pinhole_rays),
    ("DTVS depth keeps the last sphere drawn, not the nearest",
     "if (t < *dp)", "if (t == t)",
     dtvs.test_depth_keeps_the_nearest_sphere_in_any_order),
    ("DTVS distance measured from the centre instead of the front surface",
     "float front = sqrtf(dot3(rel, rel)) - v->radius;", "float front = sqrtf(dot3(rel, rel));",
     dtvs.test_distance_to_the_visible_surface_along_a_ray),
    ("DTVS particles outside the view enter the automatic range",
     "            if (d[i] < 0.0f)\n                continue; /* DTVS: outside the view */\n", "",
     dtvs.test_dtvs_levels_of_a_wall_with_particles_behind_it),
    ("DTVS cull box without its one-pixel margin",
     "x0 = (int32_t)floorf(fmaxf(fx_lo, -1.0f)) - 1;", "x0 = (int32_t)floorf(fmaxf(fx_lo, -1.0f)) + 1;",
     lambda: dtvs.test_bounding_box_cull_equals_every_pixel(0)),
    ("DTVS outside level ignored (unseen particles always at n_min)",
     "level[i] = p->view.outside_level ? p->view.outside_level : p->n_min;", "level[i] = p->n_min;",
     dtvs.test_outside_level_option_changes_only_the_particles_outside_the_view),
    ("pre-stabilisation moves only the current position",
     "                x0d[3 * s + a] = q[a];\n                xs[3 * s + a] += d;\n",
     "                x0d[3 * s + a] = q[a];\n                (void)d;\n",
     obst.test_prestabilisation_keeps_the_particles_own_velocity),
    ("pre-stabilisation applied to the levels at or above S",
     "if (!(lvl[s] < p->stabil_s))", "if (!(lvl[s] >= p->stabil_s))",
     obst.test_only_levels_below_S_are_prestabilised),
    ("cone projection along a wrongly oriented normal",
     "double rho2 = rho - g * H / L, z2 = z - g * R / L;", "double rho2 = rho - g * R / L, z2 = z - g * H / L;",
     lambda: obst.test_projection_is_the_nearest_surface_point(obst.CONE)),
    ("block contacts ignore the upper faces",
     "            if (dh < best) {", "            if (0 && dh < best) {",
     lambda: obst.test_projection_is_the_nearest_surface_point(obst.BLOCK)),
    ("finished neighbours enter Eq. 7 with lambda = 0 instead of their last lambda",
     "                if (p->lambda_mode == ORC_LAMBDA_ZERO)\n                    lam[s] = 0.0;",
     "                lam[s] = 0.0;",
     lambda: pins.test_finished_neighbour_enters_with_its_last_lambda(O.ORC_LAMBDA_STALE, "stale")),
    ("lambda recomputed for finished particles too",
     "if (active || p->lambda_mode == ORC_LAMBDA_RECOMPUTE) {", "if (1) {",
     lambda: pins.test_finished_neighbour_enters_with_its_last_lambda(O.ORC_LAMBDA_STALE, "stale")),
    ("contact response left out of the solver's position update",
     "                contact_obstacles(p, xs + 3 * s);\n                clamp_box(p, xs + 3 * s);",
     "                clamp_box(p, xs + 3 * s);",
     obst.test_no_particle_ends_inside_an_obstacle_after_a_pbf_step),
]


@pytest.mark.parametrize("name,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pin_catches_mutation(tmp_path, name, old, new, pin):
    src = open(B.SRC).read()
    assert src.count(old) == 1, name
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", *B.CFLAGS, "-I", os.path.dirname(B.SRC), str(mutant), "-o", str(lib), "-lm"],
                   check=True)
    good = O.lib()
    try:
        O._lib = None
        orig_build = B.build
        B.build = lambda force=False: str(lib)
        O.lib()
        with pytest.raises((AssertionError, O.OracleError)):
            pin()
    finally:
        B.build = orig_build
        O._lib = good
    # the genuine oracle still passes the same pin
    pin()
