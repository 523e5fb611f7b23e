"""GB300 (sm_103a) implementation of the Continuous Simulation Extension hot path.

Yang, Thompson & Sklar, "Guarantees for Comprehensive Simulation Assessment of
Statistical Methods" (arXiv 2212.10042).  The compute lives in the CUDA library
built from csrc/ (C ABI in include/cse.h); `binding` is its ctypes binding and
`workloads` builds seeded synthetic designs and tile sets.
"""
from . import workloads  # noqa: F401


def __getattr__(name):
    # the CUDA binding imports torch; load it on first use only
    if name in ("binding",):
        import importlib
        return importlib.import_module(".binding", __name__)
    raise AttributeError(name)
