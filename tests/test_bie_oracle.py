"""Pins of the oracle's double-layer Nystrom matrix and of pmCIMb on the
scattering-pole problem of Sec. 4.2 (CPU only).

Each pin is fixed independently of the code it checks:
  * the logarithm's quadrature weights integrate trigonometric polynomials
    exactly: int_0^{2 pi} log(4 sin^2(tau/2)) e^{i m tau} dtau = -2 pi / |m|
    for m != 0 and 0 for m = 0;
  * on the unit circle the Fourier modes e^{i m t} diagonalise (I + K)/2 with
    eigenvalue (i pi kappa / 2) J_m'(kappa) H_m^(1)(kappa) (interior and exterior
    expansions of the double-layer potential joined by its jump relation and the
    Wronskian J_m H_m' - J_m' H_m = 2i / (pi kappa));
  * Gauss's identity: for kappa -> 0 the double layer of a constant density is
    -1 on any smooth closed curve (here an ellipse, so that |x'| varies);
  * the paper's own check: the poles pmCIMb computes are the zeros of the
    Hankel functions H_m^(1) in Omega (found here by Newton's method).
Mutation tests plant mistakes in the oracle and check that a pin catches each.
"""
import numpy as np
import pytest
from scipy import special

import oracle as o
import oracle.bie_ref as bie
import workloads as w

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _mode_error(n, kappas, mmax=12):
    """max over kappa and |m| <= mmax of ||T e_m - mu_m e_m||_inf on the unit circle."""
    C = w.circle_curve(n)
    t = 2.0 * np.pi * np.arange(n) / n
    err = 0.0
    for kappa in kappas:
        T = 0.5 * np.eye(n) + 0.5 * o.dlp_matrix(C.samples, kappa)
        for m in range(-mmax, mmax + 1):
            e = np.exp(1j * m * t)
            mu = (0.5j * np.pi * kappa) * special.jvp(m, kappa) * special.hankel1(m, kappa)
            err = max(err, float(np.max(np.abs(T @ e - mu * e))))
    return err


KAPPAS = [1.3 - 0.7j, 2.2 - 1.9j, 0.4 - 2.6j, 3.0 - 0.2j, 1.1 + 0.3j]


def _weights_error(ns=(8, 16, 64)):
    """max error of the weights on e^{i m t}, |m| < n', and on cos(n' t) (the interpolant of the
    alternating samples), whose integral against the logarithm is -2 pi / n' cos(n' t)."""
    err = 0.0
    for n in ns:
        R = o.log_weights(n)
        t = 2.0 * np.pi * np.arange(n) / n
        h = n // 2
        for m in range(-(h - 1), h + 1):
            f = np.cos(h * t) if m == h else np.exp(1j * m * t)
            # sum_j R_{(i - j) mod n} f(t_j) at every t_i
            lhs = np.array([np.sum(R[(i - np.arange(n)) % n] * f) for i in range(n)])
            rhs = (0.0 if m == 0 else -2.0 * np.pi / abs(m)) * f
            err = max(err, float(np.max(np.abs(lhs - rhs))))
    return err


def test_log_weights_exact_on_trig_polynomials():
    assert _weights_error() < 1e-12


def test_circle_modes_are_eigenvectors_with_closed_form_eigenvalues():
    assert _mode_error(64, KAPPAS) < 1e-12


def test_gauss_identity_on_an_ellipse():
    E = w.ellipse_curve(128, 1.5, 0.8)
    K = o.dlp_matrix(E.samples, 1e-6)
    one = np.ones(128)
    assert np.max(np.abs(one + K @ one)) < 1e-9
    # the same on the circle, where the diagonal term is -1/(2 pi)
    C = w.circle_curve(64)
    K = o.dlp_matrix(C.samples, 1e-6)
    assert np.max(np.abs(np.ones(64) + K @ np.ones(64))) < 1e-9


def hankel_zeros_in(omega, mmax=12):
    """Zeros of H_m^(1), 0 <= m <= mmax, inside the rectangle, by Newton from a grid of starts."""
    x0, x1, y0, y1 = omega
    out = []
    for m in range(mmax + 1):
        for a in np.linspace(0.05, x1 + 1.0, 24):
            for b in np.linspace(y0 - 1.0, -0.02, 24):
                z = complex(a, b)
                for _ in range(60):
                    f, d = special.hankel1(m, z), special.h1vp(m, z)
                    if not (np.isfinite(f) and np.isfinite(d)) or d == 0:
                        break
                    dz = f / d
                    z -= dz
                    if abs(dz) < 1e-15 * max(1.0, abs(z)):
                        if x0 <= z.real <= x1 and y0 <= z.imag <= y1 and all(abs(z - q) > 1e-8 for _, q in out
                                                                            if _ == m):
                            out.append((m, z))
                        break
    return out


def test_scattering_poles_are_hankel_zeros():
    """pmCIMb (oracle) on the disks that hold a zero of some H_m^(1): every pole it keeps is such a
    zero, within 1e-10, and each zero of order m >= 1 appears twice (the modes m and -m)."""
    W = w.scattering_disk(n=48)
    zeros = hankel_zeros_in(W.omega)
    assert len(zeros) == 6  # the paper reports 5 poles in Omega; the zeros of H_m^(1) there are 6
    disks = [g for g in W.regions
             if any(abs(complex(g.c) - z) < g.r for _, z in zeros)]
    res = o.pmcimb(W.problem, disks, W.V, W.tol_ind, W.tol_svd, W.tol_verify)
    lam = list(res.lam)
    want = sorted([z for m, z in zeros for _ in range(2 if m else 1)], key=lambda z: (z.real, z.imag))
    # a disk may see a zero of its neighbour's square; the square filter keeps each in one square
    assert len(lam) == len(want)
    for z in want:
        k = int(np.argmin([abs(q - z) for q in lam]))
        assert abs(lam[k] - z) <= 1e-10 * max(1.0, abs(z))
        lam.pop(k)
    assert np.all(res.sigma_min < 1e-10)


class _Mutant:
    def __init__(self, **over):
        self.over = over

    def __getattr__(self, name):
        return self.over.get(name, getattr(special, name))


@pytest.mark.parametrize("mutation", ["l1_sign", "hankel2", "log_weight_tail", "normal_flip"])
def test_mutations_fail_a_pin(monkeypatch, mutation):
    if mutation == "l1_sign":
        monkeypatch.setattr(bie, "special", _Mutant(jv=lambda v, z: -special.jv(v, z)))
    elif mutation == "hankel2":
        monkeypatch.setattr(bie, "special", _Mutant(hankel1=special.hankel2))
    elif mutation == "log_weight_tail":
        plain = bie.log_weights

        def no_tail(n):
            h = n // 2
            return plain(n) + (np.pi / h ** 2) * np.cos(np.arange(n) * np.pi)
        monkeypatch.setattr(bie, "log_weights", no_tail)
        monkeypatch.setattr(o, "log_weights", no_tail)
    elif mutation == "normal_flip":
        plain = bie.dlp_matrix

        def flipped(samples, kappa):
            s = np.array(samples, dtype=np.float64)
            s = s[:, ::-1].copy()  # clockwise traversal: the normal points inwards
            s[2:4] *= -1.0
            return plain(s, kappa)[::-1, ::-1]
        monkeypatch.setattr(bie, "dlp_matrix", flipped)
        monkeypatch.setattr(o, "dlp_matrix", flipped)
    assert _mode_error(32, KAPPAS[:3], mmax=6) > 1e-6 or _weights_error((8, 16)) > 1e-6


def test_scattering_two_pass_and_pmcima():
    """The oracle's two-pass schedule (indicator on 16 of the 64 nodes) keeps the one-pass poles, and its
    pmCIMa (Sec. 3.1) places each pole it finds within tol_eps of a zero of some H_m^(1)."""
    W = w.scattering_disk(n=40, l=4)
    zeros = [z for _, z in hankel_zeros_in(W.omega)]
    disks = [g for g in W.regions if any(abs(complex(g.c) - z) < g.r for z in zeros)]
    one = o.pmcimb(W.problem, disks, W.V, W.tol_ind, W.tol_svd, W.tol_verify)
    two = o.pmcimb(W.problem, disks, W.V, W.tol_ind, W.tol_svd, W.tol_verify, indicator_N=16)
    assert len(one.lam) == len(two.lam) == 12  # the 6 zeros (of H_2 .. H_5), each twice
    assert np.max(np.abs(np.sort_complex(one.lam) - np.sort_complex(two.lam))) < 1e-12
    regs16 = [w.Region(g.c, g.r, 16) for g in disks[:2]]
    res = o.pmcima(W.problem, regs16, W.V, tol_eps=1e-6)
    assert len(res.lam) >= 1
    for lam in res.lam:
        assert min(abs(lam - z) for z in zeros) <= 1e-6
