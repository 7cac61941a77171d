"""Independent ground truth for pinning the oracle (no oracle code is used here).

* eigenvalues of quadratic T(z) = A0 + z A1 + z^2 A2 by the 2n x 2n companion
  pencil solved with QZ (brute force);
* roots of scalar delay functions -z + alpha + beta e^{-tau z} through every
  branch of the Lambert W function;
* eigenvalue counts inside a circle by the argument principle,
  (1/2 pi i) \\oint tr(T(z)^{-1} T'(z)) dz on a fine trapezoid rule.
"""
import numpy as np
import scipy.linalg as sla
from scipy.special import lambertw


def companion_eigs(A0, A1, A2):
    n = A0.shape[0]
    I = np.eye(n)
    Z = np.zeros((n, n))
    L0 = np.block([[Z, I], [-A0, -A1]])
    L1 = np.block([[I, Z], [Z, A2]])
    return sla.eigvals(L0, L1)


def delay_roots(alpha, beta, tau, branches=range(-40, 41)):
    """All roots z of -z + alpha + beta exp(-tau z) over the given W branches."""
    x = tau * beta * np.exp(-tau * alpha)
    return np.array([alpha + lambertw(x, k) / tau for k in branches])


def dense_T_and_dT(terms, n, z):
    """T(z) and T'(z) for terms (A or scalar*I, kind, degree, tau), written independently."""
    T = np.zeros((n, n), complex)
    dT = np.zeros((n, n), complex)
    for (A, kind, deg, tau) in terms:
        M = complex(A) * np.eye(n) if np.isscalar(A) else np.asarray(A, complex)
        if kind == 0:
            f = z ** deg
            df = deg * z ** (deg - 1) if deg > 0 else 0.0
        else:
            f = np.exp(-tau * z)
            df = -tau * f
        T += f * M
        dT += df * M
    return T, dT


def argument_principle_count(terms, n, c, r, N=512):
    th = 2 * np.pi * np.arange(N) / N
    s = 0j
    for t in th:
        z = c + r * np.exp(1j * t)
        T, dT = dense_T_and_dT(terms, n, z)
        s += np.trace(np.linalg.solve(T, dT)) * r * np.exp(1j * t)
    return s / N
