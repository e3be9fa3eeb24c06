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
