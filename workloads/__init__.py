"""Seeded synthetic input generators shared by the oracle and the GPU tests."""
from .circuits import *  # noqa: F401,F403
