"""FP64 CPU oracle (test infrastructure only; see ns_oracle.py)."""
from .ns_oracle import *  # noqa: F401,F403
from . import ns_oracle  # noqa: F401
