"""GB300-native e-ph hot path of the Perturbo method (arXiv 2002.02045).

The compute lives in ``libpertgb.so`` (CUDA, sm_103a) behind the C ABI of
``include/pertgb.h``; ``native`` is its thin ctypes binding.
"""
from .native import (  # noqa: F401
    ABI_SYMBOLS,
    Batch,
    PGB_EINVAL,
    PGB_ENOMEM,
    PGB_ETIMEOUT,
    PGB_FP32,
    PGB_FP64,
    PGB_G2_FULL,
    PGB_G_ABS,
    PGB_Q_CAUCHY,
    PGB_Q_UNIFORM,
    PGB_TC_BF16X3,
    PGB_TC_TF32X3,
    PRECISIONS,
    Context,
    PgbError,
    load,
)
