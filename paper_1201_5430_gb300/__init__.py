"""GB300 Lamb-Helmholtz vortex FMM: v and s = (w . grad) v of N vortex elements.

The computation lives in ``liblhv.so`` (CUDA for sm_103a, C ABI in
``include/lhv.h``); ``LHV`` is a thin binding that passes torch CUDA tensors to
it.  Build with ``paper_1201_5430_gb300.build.build()``."""
from .api import LHV  # noqa: F401
from ._lib import LHVError, load  # noqa: F401
