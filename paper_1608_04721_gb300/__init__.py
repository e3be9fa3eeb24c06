"""GB300-native (sm_103a) Adaptive Position-Based Fluids step.

The simulation runs in libapbf.so (C ABI: include/apbf.h); `apbf` is its thin
ctypes binding, `scenes` the seeded synthetic inputs, `metrics` the reported
figures.
"""
from . import metrics, scenes  # noqa: F401

__all__ = ["apbf", "metrics", "scenes"]
