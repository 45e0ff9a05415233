"""GB300-native contraction of the independent-set tensor network
(arXiv:2501.00227): a C-ABI CUDA library (include/tn.h, built from csrc/) and
its Python binding (``tn``).  Import is cheap: the shared library is loaded on
first use."""
from . import tn  # noqa: F401
from .tn import Plan, TNError  # noqa: F401
