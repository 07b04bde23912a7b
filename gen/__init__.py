"""Seeded synthetic input generators shared by the tests, the benchmark and
the selector training; they hold none of the method's arithmetic."""
from .synth import *  # noqa: F401,F403
from .synth import CSR  # noqa: F401
