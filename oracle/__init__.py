"""FP64 CPU oracle: test infrastructure only (tests, smoke check, bench CPU baseline)."""
from . import fdas_oracle  # noqa: F401
