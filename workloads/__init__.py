"""Seeded synthetic inputs for nonlinear eigenvalue problems T(z) = sum_k f_k(z) A_k.

This package only draws random numbers and lays out problems, regions and probe
blocks. It contains none of the contour-integral arithmetic, so both the CPU
oracle and the GPU path can read the same inputs without sharing method code.
"""
from .gen import *  # noqa: F401,F403
