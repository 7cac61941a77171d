"""The node-solve entry point that allocates no device memory.

It serves callers that cannot allocate while they run (their own pool owns the
device memory, or cudaFree's device-wide synchronisation is not acceptable).
Each solution must equal the CPU oracle's LAPACK solve at the same point within
the backward-error bound of two LU solves, and the solutions summed with the
trapezoid weights must equal the moments that the regular entry point
pmcim_moments returns for the same disk, within the bound the other parity
tests use; checked on two calls in a row, so the second call runs on the array
the first one left behind.
"""
import ctypes

import numpy as np
import pytest

import oracle as o
import workloads as w
from tests.test_gpu_parity import _moment_bound

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


def _solve_bound(prob, zj, V, c=4.0):
    """c u (n kappa_1(T(z_j)) + 4) ||X_j||, kappa from LAPACK's condition estimate."""
    import scipy.linalg as sla
    from scipy.linalg.lapack import zgecon
    T = o.assemble_T(prob, zj)
    lu, piv = sla.lu_factor(T)
    X = sla.lu_solve((lu, piv), V)
    rcond, _ = zgecon(lu, np.max(np.sum(np.abs(T), axis=0)), norm="1")
    return c * U64 * (prob.n / max(rcond, 1e-300) + 4) * np.linalg.norm(X)


def _call_noalloc(pm, prob, z, V):
    import torch
    lib = pm.load()
    n = prob.n
    K = len(prob.terms)
    ft = (pm.pmcim_fterm * K)()
    dense = (ctypes.c_uint8 * K)()
    mats = []
    for k, (A, kind, deg, tau) in enumerate(prob.terms):
        ft[k].kind, ft[k].degree, ft[k].tau = kind, deg, tau
        if np.isscalar(A):
            ft[k].id_re, ft[k].id_im = complex(A).real, complex(A).imag
        else:
            dense[k] = 1
            mats.append(np.asarray(A, np.complex128).T)        # row-major of A^T = column-major of A
    A_d = torch.from_numpy(np.ascontiguousarray(np.stack(mats))).cuda()
    z_d = torch.from_numpy(np.ascontiguousarray(z.astype(np.complex128))).cuda()
    V_d = torch.from_numpy(np.ascontiguousarray(V.T)).cuda()
    m, l = len(z), V.shape[1]
    X_d = torch.full((m, l, n), complex("nan"), dtype=torch.complex128, device="cuda")
    info_d = torch.full((m,), -7, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    rc = lib.pmcim_solve_points_noalloc(n, K, ft, dense, A_d.data_ptr(), m, z_d.data_ptr(), l, V_d.data_ptr(),
                                        X_d.data_ptr(), info_d.data_ptr(), None)
    assert rc == 0, rc
    assert (info_d.cpu().numpy() == 0).all()
    return X_d.cpu().numpy().transpose(0, 2, 1)                  # m x n x l


def test_noalloc_matches_moments_two_calls():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2312_13117_gb300 import build, pmcim
    build.build()
    pmcim.load()
    W = w.quadratic_small(seed=3, n=96, l=8, N=16)
    P = pmcim.Problem(W.problem.n, W.problem.terms)
    for reg in (W.regions[5], W.regions[10]):
        C0, C1, _, _ = P.moments([reg], W.V)
        z, wts = o.nodes_weights(reg.c, reg.r, reg.N)
        X = _call_noalloc(pmcim, W.problem, z, W.V)
        Xo = o.solve_nodes(W.problem, z, W.V)
        for j in range(reg.N):
            assert np.linalg.norm(X[j] - Xo[j]) <= _solve_bound(W.problem, z[j], W.V), j
        C0_na = np.einsum("j,jnl->nl", wts, X)
        C1_na = np.einsum("j,jnl->nl", wts * z, X)
        b0, b1, _ = _moment_bound(W.problem, reg, W.V)
        assert np.linalg.norm(C0_na - C0[0]) <= b0
        assert np.linalg.norm(C1_na - C1[0]) <= b1
    P.close()


def test_noalloc_rejects_oversized_problem():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2312_13117_gb300 import pmcim
    lib = pmcim.load()
    ft = (pmcim.pmcim_fterm * 1)()
    ft[0].kind, ft[0].degree, ft[0].id_re = 0, 1, 1.0
    dense = (ctypes.c_uint8 * 1)()
    n, l = 2048, 16                                              # 2048 x 2064 x 16 B > 32 MiB
    rc = lib.pmcim_solve_points_noalloc(n, 1, ft, dense, None, 1, 1, l, 1, 1, None, None)
    assert rc == -6                                              # PMCIM_ENOTSUP
