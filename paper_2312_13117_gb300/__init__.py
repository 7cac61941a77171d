"""GB300 (sm_103a) implementation of the pmCIMb hot path (Xi & Sun, parallel
multi-step contour integral methods for nonlinear eigenvalue problems).

The compute path is libpmcim.so (C ABI in include/pmcim.h); ``pmcim`` is its
ctypes binding. ``build.build()`` compiles the library in-tree.
"""
from . import pmcim  # noqa: F401
from .pmcim import Problem, options, load  # noqa: F401
