"""FP64 CPU oracle (test infrastructure only; see gp_oracle's header)."""
from .gp_oracle import *  # noqa: F401,F403
from .gp_oracle import GAUSSIAN, MATERN32  # noqa: F401
