"""FP64 CPU oracle of the Shield-MPPI hot path (test infrastructure only)."""
from .oracle import *  # noqa: F401,F403
from .oracle import build, lib, Model  # noqa: F401
