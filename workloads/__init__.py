"""Seeded synthetic input generators shared by the oracle and the CUDA path."""
from . import hashrng, configs  # noqa: F401
