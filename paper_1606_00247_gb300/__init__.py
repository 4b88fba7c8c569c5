"""GB300-native tetrahedral FMM for the micromagnetic demagnetisation potential
(Palmesi et al., arXiv:1606.00247).  The compute path is libdemag.so (CUDA,
sm_103a) behind the C ABI of include/demag.h; this package holds its build
script, the ctypes binding and a thin Plan wrapper."""
from .build import build  # noqa: F401


def __getattr__(name):
    if name == "Plan":
        from .api import Plan

        return Plan
    raise AttributeError(name)
