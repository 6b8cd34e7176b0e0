"""GB300-native preconditioned nonlinear conjugate gradient micromagnetic
minimiser (arXiv:1801.03690): a CUDA library behind the C-ABI of
include/mmncg.h, with a thin Python binding."""
from .api import (Magnet, Params, MMError, Batch, batch_plan, amg_host_apply, k32_host_apply, coercive_field, MLP,
                  warmstart_features, warmstart_apply)

__all__ = ["Magnet", "Params", "MMError", "Batch", "batch_plan", "amg_host_apply", "k32_host_apply", "coercive_field", "MLP",
           "warmstart_features", "warmstart_apply"]
