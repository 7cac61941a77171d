"""Nystrom matrix of the 2-D Helmholtz double-layer operator (oracle, test infrastructure).

The paper's second experiment (Sec. 4.2) asks for the scattering poles of a
sound-soft disk: the kappa with Im kappa < 0 at which (I + K(kappa)) / 2 is
singular, K the double-layer operator with the factor 2 of its definition and
Phi(x, y) = (i/4) H_0^(1)(kappa |x - y|). The paper says only that K is
discretised by "Nystrom's method"; the rule and the number of points are not
given. Reading: Kress's Nystrom rule for operators with a logarithmic
singularity (R. Kress, Linear Integral Equations, Sec. 12.3; D. Colton and
R. Kress, Inverse Acoustic and Electromagnetic Scattering Theory, Sec. 3.5) on
n = 2 n' equally spaced parameter points t_j = pi j / n'. For a curve x(t),
counter-clockwise, with n(t) = (x2'(t), -x1'(t)) and r = |x(t) - x(tau)|:

  (K psi)(t) = int_0^{2 pi} L(t, tau) psi(tau) dtau,
  L  = (i kappa / 2) n(tau).(x(t) - x(tau)) H_1^(1)(kappa r) / r,
  L1 = (kappa / (2 pi)) n(tau).(x(tau) - x(t)) J_1(kappa r) / r,
  L2 = L - L1 log(4 sin^2((t - tau) / 2)),
  L1(t, t) = 0,  L2(t, t) = n(t).x''(t) / (2 pi |x'(t)|^2),

and the two parts are integrated by the weights R_j of the logarithm and by
the trapezoid rule pi / n':

  (K_n psi)_i = sum_j [ R_{(i - j) mod n} L1(t_i, t_j) + (pi / n') L2(t_i, t_j) ] psi_j,
  R_m = -(2 pi / n') sum_{k=1}^{n'-1} cos(k m pi / n') / k - (pi / n'^2) cos(m pi).

Bessel and Hankel functions come from SciPy (AMOS), one library call per
array; nothing here is fused or reordered.
"""
from __future__ import annotations

import numpy as np
from scipy import special

__all__ = ["HELMHOLTZ_DLP", "log_weights", "dlp_matrix"]

HELMHOLTZ_DLP = 2


def log_weights(n: int) -> np.ndarray:
    """R_m, m = 0..n-1: int_0^{2 pi} log(4 sin^2((t - tau)/2)) f(tau) dtau ~ sum_j R_{(i-j) mod n} f(t_j)."""
    if n < 4 or n % 2:
        raise ValueError("n must be even and at least 4")
    h = n // 2
    m = np.arange(n)
    R = np.zeros(n)
    for k in range(1, h):
        R -= (2.0 * np.pi / h) * np.cos(k * m * np.pi / h) / k
    R -= (np.pi / h ** 2) * np.cos(m * np.pi)
    return R


def dlp_matrix(samples: np.ndarray, kappa: complex) -> np.ndarray:
    """K_n(kappa) for the curve sampled at t_j = 2 pi j / n (rows x1, x2, x1', x2', x1'', x2'')."""
    x1, x2, d1, d2, dd1, dd2 = (np.asarray(r, dtype=np.float64) for r in samples)
    n = x1.size
    h = n // 2
    kappa = complex(kappa)
    R = log_weights(n)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")  # row i (point t_i), column j (t_j)
    off = i != j
    ex = x1[i] - x1[j]
    ey = x2[i] - x2[j]
    r = np.hypot(ex, ey)
    q = d2[j] * ex - d1[j] * ey  # n(t_j) . (x(t_i) - x(t_j))
    L = np.zeros((n, n), dtype=np.complex128)
    L1 = np.zeros((n, n), dtype=np.complex128)
    kr = kappa * r[off]
    L[off] = (0.5j * kappa) * q[off] * special.hankel1(1, kr) / r[off]
    L1[off] = (kappa / (2.0 * np.pi)) * (-q[off]) * special.jv(1, kr) / r[off]
    lg = np.zeros((n, n))
    lg[off] = np.log(4.0 * np.sin(np.pi * (i[off] - j[off]) / n) ** 2)
    L2 = L - L1 * lg
    diag = (d2 * dd1 - d1 * dd2) / (2.0 * np.pi * (d1 ** 2 + d2 ** 2))  # n(t).x''(t) / (2 pi |x'(t)|^2)
    L2[np.arange(n), np.arange(n)] = diag
    return R[(i - j) % n] * L1 + (np.pi / h) * L2
