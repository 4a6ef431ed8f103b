"""GB300-native batched negacyclic NTT (arxiv 2410.05934, Sec. II-D / V).

The compute path is the sm_103a library built from ``csrc/`` (C ABI in
``include/ntt_gb300.h``); this package only marshals arguments to it.
"""
from .ntt import (NTT_BATCH_GRAPH, NTT_BATCH_GROUPED, NTT_FLAG_CHECK, NTT_FLAG_HOST_ONLY, NTT_FLAG_NATURAL_ORDER, NTT_FLAG_OTF_TWIDDLES, NTT_FLAG_WORD32, Batch, BConv, Plan, ntt_forward,  # noqa: F401
                  forward_inverse, ntt_inverse, ntt_plan, poly_mul_pointwise, schedule_count, schedule_name)
from ._native import NttError  # noqa: F401

__version__ = "0.1.0"
