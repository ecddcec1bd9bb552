"""Seeded synthetic workloads shared by the oracle tests and the GPU path.

This package holds parameters and random draws only -- none of the
reconstruction arithmetic.  Both sides take their inputs from here so that
they see byte-identical data.
"""
from .presets import GEOMETRIES, geometry, angles_rad  # noqa: F401
from . import generators  # noqa: F401
