"""GPU (sm_103a) fast multipole method for the reaction field of the electric
dyadic Green's function of Maxwell's equations in layered media
(arXiv 2507.18491).  The compute path is the CUDA library built from
``csrc/`` and reached through the C ABI in ``include/lmfmm.h``; ``lmfmm`` is
its Python binding."""
from . import lmfmm, workloads  # noqa: F401
from .lmfmm import Operator  # noqa: F401
