"""Seeded synthetic catalogs shared by the oracle, the tests and the bench.

This package only draws point positions (and, for the continuous-field
path, random maps on a grid). It holds none of the correlation
method's arithmetic (no gridding, no kernels, no sums), so that the oracle
and the CUDA path can both consume its output without sharing any of the
computation they are compared on.
"""
from .catalogs import (  # noqa: F401
    Catalog,
    GridSpec,
    SurveyMask,
    lattice_catalog,
    neyman_scott_box,
    neyman_scott_survey,
    uniform_box,
    uniform_survey,
    workload,
    WORKLOADS,
    batch_workload,
    continuous_maps,
)
