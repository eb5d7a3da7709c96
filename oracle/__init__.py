"""FP64 CPU oracle (test infrastructure only; see sw_lagmean.py)."""
from .sw_lagmean import SWOracle, rel_l2, LM_FIELDS  # noqa: F401
