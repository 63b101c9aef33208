"""CPU FP64 oracle (test infrastructure only; see csl_oracle)."""
from .csl_oracle import *  # noqa: F401,F403
