"""FP64 CPU oracle (test infrastructure only; see sfrd_oracle's header)."""
from .sfrd_oracle import *  # noqa: F401,F403
