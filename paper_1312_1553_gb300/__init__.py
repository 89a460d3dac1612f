"""GB300-native (sm_103a) DACG-Newton eigensolver with a BFGS-updated IC
preconditioner (Bergamaschi & Martinez, arXiv:1312.1553).

The compute path is the CUDA library ``libnle.so`` (C ABI in include/nle.h);
``nle`` is its thin Python binding.
"""
from . import nle  # noqa: F401
from .nle import Eigensolver, NLEError, load_library  # noqa: F401
