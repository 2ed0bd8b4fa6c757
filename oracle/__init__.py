"""FP64 CPU oracle of the TPO hot path — TEST INFRASTRUCTURE ONLY.

Written from the paper (arXiv 2405.11922, Algorithms 1-3 and Eqs. 1-23) as a
plain, slow, checkable restatement. It is imported only by ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline / reference arm;
the CUDA library neither imports nor links anything here, and nothing here
imports the CUDA library.

Parity status: every function is pinned by a ``-m "not gpu"`` test against
something other than itself (published generator vectors, brute force on
explicit n x n matrices, closed forms, invariants the paper states, the
paper's worked example, library SVD). See ``tests/test_oracle_*.py``.
"""
from . import bruteforce, metrics, philox, tpo  # noqa: F401
