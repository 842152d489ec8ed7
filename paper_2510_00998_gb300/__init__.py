"""GB300-native matrix-free SIPG hp-multigrid (arXiv 2510.00998): libdgmg + binding."""
from .dgmg import Context, DGMGError, load  # noqa: F401
