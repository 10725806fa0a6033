"""FP64 CPU oracle for the t-product hot path (test infrastructure only).

Only `tests/`, `__graft_entry__.smoke()` and `bench.py`'s CPU-baseline legs may
import this package; the CUDA library never does.
"""
from . import tproduct  # noqa: F401
