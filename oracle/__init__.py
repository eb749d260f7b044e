"""CPU FP64 oracle (test infrastructure; never imported by the product path)."""
from . import mf_oracle  # noqa: F401
