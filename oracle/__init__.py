"""CPU oracle for the pmCIMb hot path (test infrastructure only).

A plain, slow, FP64 restatement of the paper's method, written to be checked
against the paper by eye: trapezoid nodes on circles (Eq. 3.2-3.3), dense LU
solves at every node (Eq. 2.4), the ratio spectral indicator (Eq. 3.1),
Beyn's extraction by SVD and a small eigenproblem (Eq. 2.8, pmCIMb step 2),
the square filter (step 2.f) and verification by the smallest singular value
of T(lambda) (step 3); and the Nystrom matrix of the double-layer operator of
the scattering-pole problem (Sec. 4.2).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package. The GPU library never calls it and shares no code with
it; both read the same inputs from the separate ``workloads`` package.
"""
from .pmcim_ref import *  # noqa: F401,F403
from .lu_ref import lu_factor_pp, lu_solve_pp  # noqa: F401
from .bie_ref import log_weights, dlp_matrix  # noqa: F401
