"""Seeded synthetic inputs for the implicit sea-ice momentum step.

This module is shared by the CPU oracle and the CUDA path.  It produces
input arrays only (ice thickness, concentration, wind, ocean current,
previous velocity) and holds none of the solver's arithmetic.

Layouts (the same as the C-ABI):
  * cell fields ``h``, ``A``: shape (N, N), index [j, i] (j = y, slowest);
  * node fields ``wind``, ``ocean``, ``v_old``: shape (N+1, N+1, 2),
    index [j, i, k] with k = 0 (x) / 1 (y), node (i, j) at (i*dx, j*dx).
"""
from .fields import (Constants, Problem, gaussian_random_field, ice_fields,
                     rankine_vortex, ocean_gyre, make_problem, make_problem_q2, config,
                     translating_centre, vortex_centre, problem_one, problem_two,
                     problem_two_wind, problem_two_ocean, CONFIG_NAMES)

__all__ = ["Constants", "Problem", "gaussian_random_field", "ice_fields",
           "rankine_vortex", "ocean_gyre", "make_problem", "make_problem_q2", "config",
           "translating_centre", "vortex_centre", "problem_one", "problem_two",
           "problem_two_wind", "problem_two_ocean", "CONFIG_NAMES"]
