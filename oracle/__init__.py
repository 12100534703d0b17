"""Plain FP64 CPU oracle of the incremental-SVD method (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package. It shares no code with the CUDA path and never imports it.
"""
from .isvd import (COL, ENTRY, POLICY_ADAPTIVE_RANK, POLICY_ANGLE, POLICY_ERROR, POLICY_NOVELTY_RANK,  # noqa: F401
                   POLICY_RANK_SHRINK,
                   POLICY_NONE, POLICY_PERIODIC, ROW, Metrics, OracleISVD, Policy,
                   col_append_update, rank_one_update, rank_one_update_exact, row_append_update,
                   theta_max, truncate, truncated_svd)
