"""Seeded synthetic workloads (plants, transitions, track, user input).

This package holds the inputs both the oracle-side tests and the CUDA path
consume; it contains none of the controller's arithmetic.
"""
from . import plants, data  # noqa: F401
