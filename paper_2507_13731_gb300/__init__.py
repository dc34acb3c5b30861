"""GB300 (sm_103a) pass-efficient randomized quaternion low-rank approximation.

The compute lives in the C-ABI library libqlr.so (include/qlr.h); `qlr` is its thin ctypes
binding with the same entry-point names.
"""
from .qlr import *  # noqa: F401,F403
from .qlr import (Context, QlrError, cholqr, empty_thin, lib, qblock_krylov, qchol, qgram, qmat,  # noqa: F401
                  qrangefinder, qsketch, qsvd_lowrank, qsvd_lowrank_batched, qtsvd, residual_norm, to_thin,
                  workspace_size)
