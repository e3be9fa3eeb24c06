"""Metrics reported by the benchmark.

improvement() is the performance-improvement figure of Table 1 (Sec. 7.4):
the plain-PBF time at the maximum iteration count divided by the adaptive
time, minus one.
"""
from __future__ import annotations

import numpy as np


def improvement(t_pbf_nmax: float, t_apbf: float) -> float:
    """T_PBF(N_max) / T_APBF - 1 (Table 1)."""
    return float(t_pbf_nmax) / float(t_apbf) - 1.0


def percentile(values, q: float) -> float:
    """q-th percentile (0..100) with linear interpolation."""
    a = np.asarray(values, np.float64)
    if a.size == 0:
        return float("nan")
    return float(np.percentile(a, q))


def particle_iterations(levels) -> int:
    """Solver work of one step: the sum of per-particle iteration counts N_i."""
    return int(np.asarray(levels, np.int64).sum())
