"""GB300-native curvature matrices (G, OPG, exact Hessian, OPG eigenpairs) for
dense MLPs with softmax cross-entropy, behind the C ABI in include/hessmlp.h."""

from ._lib import EXPORTS, HessError, load, last_error  # noqa: F401
from .api import (  # noqa: F401
    HessBatch,
    HessMLP,
    HessServer,
    autotune,
    autotune_entries,
    autotune_load,
    autotune_save,
    param_permutation,
)
