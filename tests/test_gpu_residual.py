"""The refinement residual on the tensor cores (pmcim_residual) against an exact reference.

R_j = V - T(z_j) X_j is formed by the library from exact BF16 digits of the
coefficients and of f_k(z_j) X_j (7 digits of 7 bits per number, digit products
accumulated exactly in FP32, recombined in FP64). The reference here is the same
sum evaluated in NumPy with compensated dot products (TwoProduct by Veltkamp
splitting and TwoSum, the Dot2 algorithm of Ogita, Rump and Oishi, SIAM J. Sci.
Comput. 26, 2005), which is as accurate as if computed in twice the working
precision. The bound tested, 2^-44 of sum_j |T_ij| |X_jc| per element, is a few
times the splitting's own 2^-47 and below the componentwise error bound of an FP64
product of n terms, n u / (1 - n u) with u = 2^-53 (the plain FP64 product's
error is measured beside it and reported on failure).
"""
import math

import numpy as np
import pytest

import oracle as o
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2312_13117_gb300 import build, pmcim
    build.build()
    pmcim.load()
    return pmcim


_SPLIT = 134217729.0  # 2^27 + 1


def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _two_prod(a, b):
    p = a * b
    ca, cb = _SPLIT * a, _SPLIT * b
    ah, bh = ca - (ca - a), cb - (cb - b)
    al, bl = a - ah, b - bh
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def _dot2_matmul(A, B):
    """A @ B for real A (m x k) and B (k x c), compensated (Dot2)."""
    s = np.zeros((A.shape[0], B.shape[1]))
    comp = np.zeros_like(s)
    for j in range(A.shape[1]):
        p, e = _two_prod(A[:, j][:, None], B[j, :][None, :])
        s, t = _two_sum(s, p)
        comp += t + e
    return s + comp


def _exact_residual(prob, z, V, X):
    """V - T(z) X with the matrix product by compensated dot products."""
    T = o.assemble_T(prob, z)
    Tr, Ti, Xr, Xi = T.real, T.imag, X.real, X.imag
    re = _dot2_matmul(np.hstack([Tr, -Ti]), np.vstack([Xr, Xi]))
    im = _dot2_matmul(np.hstack([Tr, Ti]), np.vstack([Xi, Xr]))
    return V - (re + 1j * im), np.abs(T) @ np.abs(X)


@pytest.mark.parametrize("n,l", [(300, 5), (160, 20), (1024, 16)])
def test_residual_digits_match_exact_product(pm, n, l):
    """Delay-type T(z) (two dense terms and an identity term) at points around a disk; n and l
    give ragged row blocks (128), inner chunks (32) and column blocks (16). Solution columns are
    scaled over six orders of magnitude."""
    W = w.delay_large(seed=5, n=n, l=l, N=8, nx=4, ny=12)
    rng = np.random.default_rng(n + l)
    z = np.array([W.regions[7].c + W.regions[7].r * np.exp(2j * np.pi * k / 3) for k in range(3)])
    scale = 10.0 ** rng.uniform(-3, 3, l)
    X = w.complex_gaussian(rng, (len(z), n, l)) * scale[None, None, :]
    P = pm.Problem(n, W.problem.terms)
    R = P.residual(z, W.V, X, opt=pm.options(precision=pm.PREC_FP32_IR))
    worst, worst64 = 0.0, 0.0
    for j in range(len(z)):
        ref, mag = _exact_residual(W.problem, z[j], W.V, X[j])
        err = np.abs(R[j] - ref) / mag
        worst = max(worst, float(err.max()))
        R64 = W.V - o.assemble_T(W.problem, z[j]) @ X[j]
        worst64 = max(worst64, float((np.abs(R64 - ref) / mag).max()))
    # within the componentwise FP64 bound n u / (1 - n u) of an n-term product, with room to spare
    assert worst <= 2.0 ** -44, (worst, worst64)
    P.close()


def test_residual_of_an_exact_solution_is_small(pm):
    """At X = T(z)^-1 V from LAPACK the residual is at rounding level of ||T|| ||X||, as in FP64."""
    W = w.quadratic_small(seed=11, n=96, l=6, N=8)
    z = np.array([0.3 + 0.4j])
    T = o.assemble_T(W.problem, z[0])
    X = np.linalg.solve(T, W.V)
    P = pm.Problem(W.problem.n, W.problem.terms)
    R = P.residual(z, W.V, X)
    assert np.linalg.norm(R) <= 64 * 2.0 ** -53 * np.linalg.norm(T) * np.linalg.norm(X) * math.sqrt(96)
    P.close()
