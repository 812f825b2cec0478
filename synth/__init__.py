"""Seeded synthetic inputs shaped like the paper's workloads.

This package holds input definitions only (meshes, potential fields, atoms,
projector functions, trial vectors) and none of the method's arithmetic: no
quadrature, no basis functions, no Jacobians, no operator.  Both the CUDA path's
tests / benchmark and the CPU oracle draw their inputs from here.
"""
from .workloads import *  # noqa: F401,F403
