"""Oracle package: CPU complex128 reference simulator (test infrastructure only)."""
from .oracle import *  # noqa: F401,F403
from .oracle import build  # noqa: F401
