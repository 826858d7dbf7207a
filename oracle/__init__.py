"""FP64 CPU oracle for the circular-geometry PAT/TAT operators A and A*.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``, never by the product package.
"""
from .tat_oracle import (OraclePlan, adjoint, forward, hybrid_rule, inverse, inverse_direct, kwave_truth,
                         poisson_truth, smooth_ceil)

__all__ = ["OraclePlan", "forward", "adjoint", "inverse", "inverse_direct", "hybrid_rule", "kwave_truth",
           "poisson_truth", "smooth_ceil"]
