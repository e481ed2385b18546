"""GB300-native (sm_103a) online evaluation of thermomechanical direct deep
material networks (arXiv 2109.14403): a C-ABI CUDA library (``include/dmn.h``)
and a thin Python binding."""
from .dmn import DMN, OUT_WORDS, PT_NONFINITE, PT_NOT_CONVERGED, PT_OK, load  # noqa: F401
