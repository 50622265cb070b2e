"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle's checks.

Holds only input generators (body templates, initial placements, parameter
sets); none of the gDC method's arithmetic lives here.
"""
from . import shapes, workloads  # noqa: F401
from .workloads import Workload  # noqa: F401
