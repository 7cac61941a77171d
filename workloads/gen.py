"""Seeded input generators (NumPy PCG64 ``default_rng``).

A problem is ``Problem(n, terms)`` where every term is ``(A, kind, degree, tau)``:
``A`` is a dense complex128 n x n matrix (column-major), or a Python complex
scalar ``s`` standing for the matrix ``s * I`` (never stored densely);
``kind`` is ``MONOMIAL`` (f(z) = z**degree) or ``EXP_NEG`` (f(z) = exp(-tau z)).
This is the problem class T(z) = sum_k f_k(z) A_k of Sec. 1 with the fixed
scalar-function set of the hot path. A term of kind ``HELMHOLTZ_DLP`` instead
carries a ``BoundaryCurve`` in place of ``A``: the term is ``scale * K_n(z)``,
the Nystrom matrix of the 2-D Helmholtz double-layer operator on that closed
curve at wave number z (the scattering-pole problem of Sec. 4.2).

Regions are disks circumscribing the squares of a uniform grid over a
rectangle Omega (Sec. 3, circumscribed-disk cover): centre c, radius
r = s / sqrt(2) for square side s, and N trapezoid nodes.

Complex Gaussian entries are (N(0,1) + i N(0,1)) / sqrt(2).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

MONOMIAL = 0
EXP_NEG = 1
HELMHOLTZ_DLP = 2

__all__ = [
    "MONOMIAL", "EXP_NEG", "HELMHOLTZ_DLP", "BoundaryCurve", "Problem", "Region", "Workload",
    "complex_gaussian", "probe_block", "grid_regions",
    "quadratic_small", "paper_quadratic", "delay_large", "batched_quadratics", "mass_spring",
    "diagonal_linear", "similarity_linear", "diagonal_delay", "paper_n4_example",
    "diagonal_quadratic", "screen_trace_problems", "config_trace_problems",
    "circle_curve", "ellipse_curve", "scattering_disk",
]


@dataclasses.dataclass
class BoundaryCurve:
    """A smooth closed curve x(t), t in [0, 2 pi), counter-clockwise, sampled at
    t_j = 2 pi j / n: ``samples`` is a 6 x n float64 array of the rows
    x1, x2, x1', x2', x1'', x2'' (derivatives with respect to t). ``scale`` is
    the complex factor the term multiplies its operator by."""
    samples: np.ndarray
    scale: complex = 0.5


@dataclasses.dataclass
class Problem:
    n: int
    terms: List[Tuple[Optional[np.ndarray], int, int, float]]

    def term_arrays(self):
        """(matrices-or-None, kinds, degrees, taus) as parallel lists."""
        return ([t[0] for t in self.terms], [t[1] for t in self.terms],
                [t[2] for t in self.terms], [t[3] for t in self.terms])


@dataclasses.dataclass
class Region:
    c: complex
    r: float
    N: int


@dataclasses.dataclass
class Workload:
    name: str
    problem: Problem
    regions: List[Region]
    V: np.ndarray              # n x l complex128, unit-norm columns
    tol_ind: float = 0.1
    tol_svd: float = 1e-6
    tol_verify: float = 1e-6
    omega: Tuple[float, float, float, float] = (0.0, 0.0, 0.0, 0.0)  # xmin, xmax, ymin, ymax


def complex_gaussian(rng: np.random.Generator, shape) -> np.ndarray:
    g = rng.standard_normal(tuple(shape) + (2,))
    return (g[..., 0] + 1j * g[..., 1]) / math.sqrt(2.0)


def probe_block(rng: np.random.Generator, n: int, l: int) -> np.ndarray:
    """n x l complex Gaussian probe block with unit-norm columns, column-major order."""
    V = complex_gaussian(rng, (n, l))
    V /= np.linalg.norm(V, axis=0, keepdims=True)
    return np.asfortranarray(V)


def grid_regions(xmin: float, xmax: float, ymin: float, ymax: float,
                 nx: int, ny: int, N: int) -> List[Region]:
    """Disks circumscribing an nx x ny grid of equal squares over [xmin,xmax]x[ymin,ymax].

    Squares must be square: (xmax-xmin)/nx == (ymax-ymin)/ny. Ordered x-major
    like the paper's test driver (Appendix, test.m).
    """
    sx = (xmax - xmin) / nx
    sy = (ymax - ymin) / ny
    if abs(sx - sy) > 1e-12 * max(sx, sy):
        raise ValueError("grid cells are not square")
    r = sx / math.sqrt(2.0)
    out = []
    for i in range(nx):
        for j in range(ny):
            out.append(Region(complex(xmin + (i + 0.5) * sx, ymin + (j + 0.5) * sy), r, N))
    return out


# ----------------------------------------------------------------------------
# The five workload shapes
# ----------------------------------------------------------------------------

def quadratic_small(seed: int = 0, n: int = 64, l: int = 8, N: int = 32) -> Workload:
    """Quadratic T(z) = A0 + z A1 + z^2 A2, A_k complex Gaussian / sqrt(n).

    Omega = [-2,2]^2 split 4x4; N nodes per circle; l probes.
    """
    rng = np.random.default_rng(seed)
    A = [complex_gaussian(rng, (n, n)) / math.sqrt(n) for _ in range(3)]
    V = probe_block(rng, n, l)
    prob = Problem(n, [(np.asfortranarray(A[d]), MONOMIAL, d, 0.0) for d in range(3)])
    return Workload("quadratic_n%d" % n, prob, grid_regions(-2, 2, -2, 2, 4, 4, N), V,
                    omega=(-2, 2, -2, 2))


def paper_quadratic(seed: int = 0, n: int = 100, m: int = 15, l: int = 10, N: int = 64) -> Workload:
    """The paper's quadratic experiment (Sec. 4.1) with seeded inputs: T(z) = T0 + z T1 + z^2 T2
    with real T_j of uniform [0, 1) entries (the shape and distribution of MATLAB rand),
    n = 100, Omega = [-0.5, 0.5]^2 split m x m = 15 x 15, N = 64 nodes for Beyn, l = 10 probes
    (the Appendix listing's numEig)."""
    rng = np.random.default_rng(seed)
    T = [np.asfortranarray(rng.random((n, n)).astype(np.complex128)) for _ in range(3)]
    V = probe_block(rng, n, l)
    prob = Problem(n, [(T[d], MONOMIAL, d, 0.0) for d in range(3)])
    return Workload("paper_quadratic_n%d" % n, prob, grid_regions(-0.5, 0.5, -0.5, 0.5, m, m, N), V,
                    omega=(-0.5, 0.5, -0.5, 0.5))


def delay_large(seed: int = 0, n: int = 1024, l: int = 16, N: int = 64,
                nx: int = 16, ny: int = 48) -> Workload:
    """Delay-type T(z) = -z I + A0 + A1 exp(-z).

    A0 = Q D Q^-1 with D's n eigenvalues uniform in the disk |z| <= 4 and
    Q = U1 diag(s) U2^H (U from QR of complex Gaussians, s ~ U[1,2], so
    cond(Q) <= 2); Q^-1 = U2 diag(1/s) U1^H is formed from the factors.
    A1 complex Gaussian scaled 0.5/sqrt(n). Omega = [-3,1] x [-6,6] split nx x ny.
    """
    rng = np.random.default_rng(seed)
    rad = 4.0 * np.sqrt(rng.random(n))
    ang = 2.0 * np.pi * rng.random(n)
    d = rad * np.exp(1j * ang)
    U1, _ = np.linalg.qr(complex_gaussian(rng, (n, n)))
    U2, _ = np.linalg.qr(complex_gaussian(rng, (n, n)))
    s = rng.uniform(1.0, 2.0, n)
    Q = (U1 * s) @ U2.conj().T
    Qinv = (U2 * (1.0 / s)) @ U1.conj().T
    A0 = (Q * d) @ Qinv
    A1 = complex_gaussian(rng, (n, n)) * (0.5 / math.sqrt(n))
    V = probe_block(rng, n, l)
    prob = Problem(n, [(-1.0 + 0j, MONOMIAL, 1, 0.0),
                       (np.asfortranarray(A0), MONOMIAL, 0, 0.0),
                       (np.asfortranarray(A1), EXP_NEG, 0, 1.0)])
    return Workload("delay_n%d" % n, prob, grid_regions(-3, 1, -6, 6, nx, ny, N), V,
                    omega=(-3, 1, -6, 6))


def batched_quadratics(seeds: Sequence[int] = range(1, 513), l: int = 8,
                       n_lo: int = 32, n_hi: int = 768) -> List[Workload]:
    """Independent quadratic problems of uneven size, one per seed.

    Per seed: n ~ U{n_lo..n_hi}; A_k complex Gaussian / sqrt(n); a square Omega
    of side ~ U[2,6] centred at 0 split m x m with m ~ U{2..8};
    N ~ choice{16,32,64}; l probes.
    """
    out = []
    for sd in seeds:
        rng = np.random.default_rng(sd)
        n = int(rng.integers(n_lo, n_hi + 1))
        A = [complex_gaussian(rng, (n, n)) / math.sqrt(n) for _ in range(3)]
        side = float(rng.uniform(2.0, 6.0))
        m = int(rng.integers(2, 9))
        N = int(rng.choice([16, 32, 64]))
        V = probe_block(rng, n, l)
        prob = Problem(n, [(np.asfortranarray(A[d]), MONOMIAL, d, 0.0) for d in range(3)])
        h = side / 2
        out.append(Workload("batched_seed%d_n%d" % (sd, n), prob,
                            grid_regions(-h, h, -h, h, m, m, N), V, omega=(-h, h, -h, h)))
    return out


def mass_spring(seed: int = 0, n: int = 2048, l: int = 48, N: int = 64,
                nx: int = 32, ny: int = 256) -> Workload:
    """Damped mass-spring T(z) = z^2 I + z C + K.

    K tridiagonal from n+1 springs k ~ lognormal(0, 0.5), fixed-fixed ends;
    C = 0.02 K + sum of 8 grounded dashpots at distinct seeded DOFs with
    gains ~ U[0,1]. Omega = [-1,0] x [0,8] split nx x ny.
    """
    rng = np.random.default_rng(seed)
    k = rng.lognormal(0.0, 0.5, n + 1)
    K = np.zeros((n, n))
    idx = np.arange(n)
    K[idx, idx] = k[:-1] + k[1:]
    K[idx[:-1], idx[:-1] + 1] = -k[1:-1]
    K[idx[:-1] + 1, idx[:-1]] = -k[1:-1]
    dofs = rng.choice(n, 8, replace=False)
    g = rng.random(8)
    C = 0.02 * K
    C[dofs, dofs] += g
    V = probe_block(rng, n, l)
    prob = Problem(n, [(1.0 + 0j, MONOMIAL, 2, 0.0),
                       (np.asfortranarray(C.astype(np.complex128)), MONOMIAL, 1, 0.0),
                       (np.asfortranarray(K.astype(np.complex128)), MONOMIAL, 0, 0.0)])
    return Workload("mass_spring_n%d" % n, prob, grid_regions(-1, 0, 0, 8, nx, ny, N), V,
                    omega=(-1, 0, 0, 8))


def circle_curve(n: int, radius: float = 1.0) -> BoundaryCurve:
    """The circle of the given radius about 0, n samples."""
    t = 2.0 * np.pi * np.arange(n) / n
    c, s = np.cos(t), np.sin(t)
    return BoundaryCurve(np.array([radius * c, radius * s, -radius * s, radius * c,
                                   -radius * c, -radius * s], dtype=np.float64))


def ellipse_curve(n: int, a: float, b: float) -> BoundaryCurve:
    """The ellipse x = (a cos t, b sin t), n samples."""
    t = 2.0 * np.pi * np.arange(n) / n
    c, s = np.cos(t), np.sin(t)
    return BoundaryCurve(np.array([a * c, b * s, -a * s, b * c, -a * c, -b * s], dtype=np.float64))


def scattering_disk(seed: int = 0, n: int = 256, l: int = 8, N: int = 64, m: int = 10,
                    radius: float = 1.0, omega=(0.2, 3.2, -3.2, -0.2)) -> Workload:
    """Scattering poles of a sound-soft disk (Sec. 4.2): T(kappa) = (I + K_n(kappa)) / 2,
    K_n the Nystrom matrix of the double-layer operator on n boundary points.
    Omega = [0.2, 3.2] x [-3.2, -0.2] split m x m = 10 x 10 (the paper's 100 squares),
    N nodes per circle, l probes."""
    rng = np.random.default_rng(seed)
    V = probe_block(rng, n, l)
    prob = Problem(n, [(0.5 + 0j, MONOMIAL, 0, 0.0),
                       (circle_curve(n, radius), HELMHOLTZ_DLP, 0, 0.0)])
    x0, x1, y0, y1 = omega
    return Workload("scattering_disk_n%d" % n, prob, grid_regions(x0, x1, y0, y1, m, m, N), V,
                    omega=tuple(omega))


# ----------------------------------------------------------------------------
# Closed-form families (used to pin the oracle)
# ----------------------------------------------------------------------------

def diagonal_linear(mu: np.ndarray) -> Problem:
    """T(z) = diag(z - mu_i) = -diag(mu) * 1 + z I  (terms: diag(-mu) z^0, I z^1)."""
    n = len(mu)
    return Problem(n, [(np.asfortranarray(np.diag(-np.asarray(mu, dtype=np.complex128))), MONOMIAL, 0, 0.0),
                       (1.0 + 0j, MONOMIAL, 1, 0.0)])


def similarity_linear(mu: np.ndarray, seed: int = 0) -> Tuple[Problem, np.ndarray]:
    """T(z) = A - z I with A = Q diag(mu) Q^-1, Q complex Gaussian. Returns (problem, Q)."""
    rng = np.random.default_rng(seed)
    n = len(mu)
    Q = complex_gaussian(rng, (n, n)) + 2.0 * np.eye(n)
    A = Q @ np.diag(mu) @ np.linalg.inv(Q)
    return Problem(n, [(np.asfortranarray(A), MONOMIAL, 0, 0.0),
                       (-1.0 + 0j, MONOMIAL, 1, 0.0)]), Q


def diagonal_quadratic(mu1: np.ndarray, mu2: np.ndarray, lead: np.ndarray) -> Problem:
    """T(z) = diag(lead_i (z - mu1_i)(z - mu2_i)) as A0 + z A1 + z^2 A2."""
    lead = np.asarray(lead, dtype=np.complex128)
    a0 = lead * mu1 * mu2
    a1 = -lead * (mu1 + mu2)
    return Problem(len(lead), [(np.asfortranarray(np.diag(a0)), MONOMIAL, 0, 0.0),
                               (np.asfortranarray(np.diag(a1)), MONOMIAL, 1, 0.0),
                               (np.asfortranarray(np.diag(lead)), MONOMIAL, 2, 0.0)])


def diagonal_delay(alpha: np.ndarray, beta: np.ndarray, tau: float = 1.0) -> Problem:
    """T(z) = diag(-z + alpha_i + beta_i exp(-tau z))."""
    return Problem(len(alpha), [(-1.0 + 0j, MONOMIAL, 1, 0.0),
                                (np.asfortranarray(np.diag(np.asarray(alpha, np.complex128))), MONOMIAL, 0, 0.0),
                                (np.asfortranarray(np.diag(np.asarray(beta, np.complex128))), EXP_NEG, 0, float(tau))])


def paper_n4_example(path: str) -> Problem:
    """The 4x4 quadratic printed in the paper's appendix (generateT), read from a text fixture."""
    mats = {}
    cur = None
    with open(path) as fh:
        for line in fh:
            s = line.strip()
            if not s or s.startswith("#"):
                continue
            if s.endswith(":"):
                cur = s[:-1]
                mats[cur] = []
                continue
            mats[cur].append([float(x) for x in s.split()])
    T0, T1, T2 = (np.asfortranarray(np.array(mats[k], dtype=np.complex128)) for k in ("T0", "T1", "T2"))
    return Problem(4, [(T0, MONOMIAL, 0, 0.0), (T1, MONOMIAL, 1, 0.0), (T2, MONOMIAL, 2, 0.0)])


def screen_trace_problems(seeds: Sequence[int], n_choices=(16, 24, 32), disks: int = 48, N: int = 64,
                          l: int = 1):
    """Small delay-type and quadratic problems with randomly placed disks, for screen traces.

    Even seeds give -zI + A0 + A1 exp(-z) (A0 from a spectrum uniform in |z| <= 2,
    A1 Gaussian * 0.5/sqrt(n)); odd seeds give A0 + z A1 + z^2 A2 (Gaussian / sqrt(n)).
    Disk centres are uniform in [-3,3] x [-3,3], radii log-uniform in [0.01, 1].
    """
    out = []
    for sd in seeds:
        rng = np.random.default_rng(10_000 + sd)
        n = int(rng.choice(n_choices))
        if sd % 2 == 0:
            d = 2.0 * np.sqrt(rng.random(n)) * np.exp(2j * np.pi * rng.random(n))
            Q = complex_gaussian(rng, (n, n)) + 2.0 * np.eye(n)
            A0 = Q @ np.diag(d) @ np.linalg.inv(Q)
            A1 = complex_gaussian(rng, (n, n)) * (0.5 / math.sqrt(n))
            prob = Problem(n, [(-1.0 + 0j, MONOMIAL, 1, 0.0), (np.asfortranarray(A0), MONOMIAL, 0, 0.0),
                               (np.asfortranarray(A1), EXP_NEG, 0, 1.0)])
        else:
            A = [complex_gaussian(rng, (n, n)) / math.sqrt(n) for _ in range(3)]
            prob = Problem(n, [(np.asfortranarray(A[k]), MONOMIAL, k, 0.0) for k in range(3)])
        c = rng.uniform(-3, 3, disks) + 1j * rng.uniform(-3, 3, disks)
        r = 10.0 ** rng.uniform(-2, 0, disks)
        regs = [Region(complex(c[i]), float(r[i]), N) for i in range(disks)]
        out.append((prob, regs, probe_block(rng, n, l)))
    return out


def config_trace_problems(delay_seeds: Sequence[int], batched_seeds: Sequence[int],
                          delay_n=(64, 96, 128), delay_grids=(8, 16, 32), batched_n_hi: int = 128):
    """Screen traces from the delay and batched workloads, by other seeds of their own generators
    at smaller n (one probe column each), yielded one problem at a time.

    Delay: delay_large(seed, n, N = 64) on Omega = [-3,1] x [-6,6] split g x 3g, with n and g
    cycling through delay_n and delay_grids. Batched: batched_quadratics(seeds) with
    n ~ U{32..batched_n_hi}, a random square Omega split m x m and N in {16, 32, 64}."""
    for k, sd in enumerate(delay_seeds):
        n = delay_n[k % len(delay_n)]
        g = delay_grids[(k // len(delay_n)) % len(delay_grids)]
        Wd = delay_large(seed=sd, n=n, l=1, N=64, nx=g, ny=3 * g)
        yield Wd.problem, Wd.regions, Wd.V
    for sd in batched_seeds:
        Wb = batched_quadratics([sd], l=1, n_lo=32, n_hi=batched_n_hi)[0]
        yield Wb.problem, Wb.regions, Wb.V
