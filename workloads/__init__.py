"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

Geometry and bookkeeping only; the method's arithmetic lives in the CUDA
library (product) and, independently, in ``oracle/`` (tests).
"""
from . import configs, geometry  # noqa: F401
from .configs import System  # noqa: F401
