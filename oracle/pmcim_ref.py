"""Plain FP64 restatement of pmCIMb's hot path (oracle, test infrastructure).

Every function follows one passage of the paper, in the paper's order and
notation, with NumPy/SciPy library calls as single steps (dense LU through
LAPACK, SVD, eig). Nothing here is blocked, fused or reordered.

Readings of passages the paper leaves open (listed again in the design notes):
  * nodes theta_j = 2 pi j / N, j = 0..N-1 (Appendix, the node vector drops
    the endpoint 2 pi of an equally spaced grid starting at 0);
  * weights w_j = (r/N) e^{i theta_j}: Eq. 3.2 after cancelling i/(iN); the
    appendix's extra factor 1/i is a common unit-modulus factor that leaves
    sigma, p and eig(D) unchanged, so it is dropped;
  * C1 uses z_j = c + r e^{i theta_j} (Eq. 3.3 prints z + r theta_j, a typo;
    the appendix multiplies by the node itself);
  * the N/2 rule of Eq. 3.1 uses the 1-based even nodes x_2, x_4, ..., x_N,
    i.e. the 0-based odd nodes, each with weight 2 w_j;
  * one probe block V (n x l, unit columns) serves every region and node, and
    the indicator's random vector is f = V[:, 0] (pmCIMb steps 1.a and 2.a);
  * candidate <=> I > tol_ind, strict (pmCIMb step 1.c);
  * P f = 0 when a disk holds no eigenvalue (Sec. 2.1), so Eq. 3.1 is 0/0
    there; in floating point P f|_N then sits at rounding level. When
    ||P f|_N|| <= 1e-10 * || sum_j |w_j| |x_j| || the indicator is taken as 0;
    componentwise, a component whose |P f|_{N/2}| is at or below that level
    (an exact zero included) has no determined ratio, and I is the root mean
    square of the other components' ratios (Eq. 3.1's norm over sqrt(n) when
    none is left out);
  * tol_svd is absolute (Sec. 3.2) and p counts sigma_i > tol_svd;
  * a region is saturated when p reaches min(n, l) (all probe directions
    used); it is then split into four children with the pmCIMa geometry and
    re-run, up to a fixed depth (the paper's remedy "use smaller subregions",
    Sec. 3.2 parameter list);
  * the square filter keeps c - s/2 <= Re, Im < c + s/2 with s/2 = r/sqrt(2)
    (step 2.f, half-open so each point lies in exactly one square);
  * verification uses the smallest singular value of T(lambda) and accepts
    sigma_min <= tol_verify * max(1, ||T(lambda)||_F / sqrt(n)) (step 3);
  * eigenvectors have unit 2-norm with their largest-modulus entry real and
    positive.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np
import scipy.linalg as sla

from .bie_ref import HELMHOLTZ_DLP, dlp_matrix

__all__ = [
    "MONOMIAL", "EXP_NEG", "HELMHOLTZ_DLP", "scalar_f", "assemble_T", "nodes_weights", "solve_nodes",
    "Moments", "moments", "indicator_value", "indicator", "BeynResult", "beyn_extract",
    "square_filter", "normalise_vectors", "sigma_min", "verify", "split4",
    "hankel_moments", "beyn_extract_hankel", "pmcimb", "PmcimbResult", "pmcima", "PmcimaResult", "pmcima_levels", "merge_centres",
]

MONOMIAL = 0
EXP_NEG = 1


# ---------------------------------------------------------------------------
# The problem T(z) = sum_k f_k(z) A_k  (Sec. 1; the user routine generateT of
# the Appendix, restricted to monomials and exp(-tau z))
# ---------------------------------------------------------------------------

def scalar_f(kind: int, degree: int, tau: float, z: complex) -> complex:
    """f_k(z): z**degree for a monomial term, exp(-tau z) for a delay term."""
    if kind == MONOMIAL:
        return complex(z) ** int(degree)
    if kind == EXP_NEG:
        return complex(np.exp(-tau * complex(z)))
    raise ValueError("unknown scalar function kind %r" % kind)


def assemble_T(problem, z: complex) -> np.ndarray:
    """Dense T(z) = sum_k f_k(z) A_k; a scalar A_k stands for A_k * I. A term of
    kind HELMHOLTZ_DLP carries a boundary curve instead and adds scale * K_n(z),
    the double-layer Nystrom matrix of Sec. 4.2 (bie_ref.dlp_matrix)."""
    n = problem.n
    T = np.zeros((n, n), dtype=np.complex128)
    for (A, kind, deg, tau) in problem.terms:
        if kind == HELMHOLTZ_DLP:
            T += complex(A.scale) * dlp_matrix(A.samples, z)
            continue
        fz = scalar_f(kind, deg, tau, z)
        if np.isscalar(A):
            T[np.arange(n), np.arange(n)] += fz * complex(A)
        else:
            T += fz * np.asarray(A, dtype=np.complex128)
    return T


# ---------------------------------------------------------------------------
# Trapezoid rule on a circle (Eq. 3.2-3.3; Appendix, indicator/ContourSVD)
# ---------------------------------------------------------------------------

def nodes_weights(c: complex, r: float, N: int):
    """z_j = c + r e^{i theta_j}, w_j = (r/N) e^{i theta_j}, theta_j = 2 pi j / N."""
    j = np.arange(N)
    e = np.exp(1j * 2.0 * np.pi * j / N)
    return complex(c) + r * e, (r / N) * e


def solve_nodes(problem, z: np.ndarray, V: np.ndarray) -> np.ndarray:
    """X_j = T(z_j)^{-1} V for every node (Eq. 2.4), dense LU with partial pivoting."""
    out = np.empty((len(z), problem.n, V.shape[1]), dtype=np.complex128)
    for j, zj in enumerate(z):
        lu, piv = sla.lu_factor(assemble_T(problem, zj), check_finite=True)
        out[j] = sla.lu_solve((lu, piv), V)
    return out


@dataclasses.dataclass
class Moments:
    C0: np.ndarray       # n x l: sum_j w_j X_j          (Eq. 3.2)
    C1: np.ndarray       # n x l: sum_j w_j z_j X_j      (Eq. 3.3)
    pf_N: np.ndarray     # n:     sum_j w_j x_j, f = V[:,0]          (P f |_N)
    pf_half: np.ndarray  # n:     sum_{j odd} 2 w_j x_j              (P f |_{N/2})
    pf_abs: np.ndarray = None  # n: sum_j |w_j| |x_j|, the size of the terms of P f |_N


def moments(problem, c: complex, r: float, N: int, V: np.ndarray) -> Moments:
    """Quadrature sums of one disk: Beyn's C_{0,N}, C_{1,N} and the two P f approximations."""
    if N % 2:
        raise ValueError("the ratio indicator needs an even N")
    z, w = nodes_weights(c, r, N)
    X = solve_nodes(problem, z, V)
    n, l = problem.n, V.shape[1]
    C0 = np.zeros((n, l), dtype=np.complex128)
    C1 = np.zeros((n, l), dtype=np.complex128)
    pf_N = np.zeros(n, dtype=np.complex128)
    pf_half = np.zeros(n, dtype=np.complex128)
    pf_abs = np.zeros(n)
    for j in range(N):
        C0 += w[j] * X[j]
        C1 += w[j] * z[j] * X[j]
        pf_N += w[j] * X[j][:, 0]
        pf_abs += abs(w[j]) * np.abs(X[j][:, 0])
        if j % 2 == 1:                       # 1-based even nodes x_2, x_4, ..., x_N
            pf_half += 2.0 * w[j] * X[j][:, 0]
    return Moments(C0, C1, pf_N, pf_half, pf_abs)


PF_FLOOR = 1e-10


def indicator_value(pf_N: np.ndarray, pf_half: np.ndarray, pf_abs: np.ndarray = None) -> float:
    """I = || P f|_N ./ P f|_{N/2} ||_2 / sqrt(n)   (Eq. 3.1); 0 when P f|_N is at rounding level.

    That is the root mean square of the componentwise ratios |a_i| / |b_i| with a = P f|_N,
    b = P f|_{N/2}. With pf_abs given, a component whose |b_i| is at or below the same rounding
    level (PF_FLOOR times || sum_j |w_j| |x_j| ||, an exact zero included) has no determined
    ratio: the mean runs over the other components."""
    if pf_abs is not None and np.linalg.norm(pf_N) <= PF_FLOOR * np.linalg.norm(pf_abs):
        return 0.0
    num = pf_N.real ** 2 + pf_N.imag ** 2
    den = pf_half.real ** 2 + pf_half.imag ** 2
    floor2 = (PF_FLOOR * np.linalg.norm(pf_abs)) ** 2 if pf_abs is not None else 0.0
    keep = den > floor2
    if not np.any(keep):
        return 0.0
    return float(math.sqrt(float(np.sum(num[keep] / den[keep])) / int(np.sum(keep))))


def indicator(problem, regions: Sequence, V: np.ndarray, tol_ind: float = 0.1):
    """pmCIMb step 1: indicators of all disks, candidate <=> I > tol_ind."""
    I = np.array([indicator_value(*_pf(moments(problem, g.c, g.r, g.N, V))) for g in regions])
    return I, I > tol_ind


def _pf(m: Moments):
    return m.pf_N, m.pf_half, m.pf_abs


# ---------------------------------------------------------------------------
# Beyn's extraction (Eq. 2.8; pmCIMb steps 2.c-2.e)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class BeynResult:
    sigma: np.ndarray    # singular values of C0, descending
    p: int               # number of sigma_i > tol_svd
    saturated: bool      # p == min(n, l)
    lam: np.ndarray      # eigenvalues of D (p,)
    vecs: np.ndarray     # n x p eigenvectors V0 s, normalised


def normalise_vectors(Vc: np.ndarray) -> np.ndarray:
    """Unit 2-norm columns, each rotated so its largest-modulus entry is real positive."""
    out = np.array(Vc, dtype=np.complex128, copy=True)
    for k in range(out.shape[1]):
        v = out[:, k]
        v = v / np.linalg.norm(v)
        i = int(np.argmax(np.abs(v)))
        v = v * (abs(v[i]) / v[i])
        out[:, k] = v
    return out


def beyn_extract(C0: np.ndarray, C1: np.ndarray, tol_svd: float = 1e-6) -> BeynResult:
    """SVD C0 = V Sigma W^H, keep sigma > tol_svd, D = V0^H C1 W0 Sigma0^{-1}, eig(D)."""
    n, l = C0.shape
    Vs, s, Wh = np.linalg.svd(C0, full_matrices=False)
    p = int(np.sum(s > tol_svd))
    saturated = p >= min(n, l)
    if p == 0:
        return BeynResult(s, 0, False, np.zeros(0, np.complex128), np.zeros((n, 0), np.complex128))
    V0 = Vs[:, :p]
    W0 = Wh.conj().T[:, :p]
    D = V0.conj().T @ C1 @ W0 @ np.diag(1.0 / s[:p])
    lam, S = np.linalg.eig(D)
    return BeynResult(s, p, saturated, lam, normalise_vectors(V0 @ S))


def hankel_moments(problem, c: complex, r: float, N: int, V: np.ndarray, K: int):
    """Scaled moments M_p = sum_j w_j ((z_j - c)/r)^p X_j, p = 0..2K-1, of one disk.

    The higher moments of Beyn's method (the pointer to Beyn's Remark 3.5 in
    Sec. 2.2) in the variable (z - c)/r, whose powers on the nodes are the unit
    phases e^{i p theta_j}: the contour integrals of z^p T^{-1} V would grow like
    |c|^p instead."""
    z, w = nodes_weights(c, r, N)
    X = solve_nodes(problem, z, V)
    zeta = np.exp(1j * 2.0 * np.pi * np.arange(N) / N)
    return [sum(w[j] * zeta[j] ** p * X[j] for j in range(N)) for p in range(2 * K)]


def beyn_extract_hankel(M, c: complex, r: float, tol_svd: float = 1e-6) -> BeynResult:
    """Beyn's extraction from the block Hankel matrices of the scaled moments.

    B0 = [M_{i+j}] and B1 = [M_{i+j+1}] (i, j < K; K n x K l). SVD B0 = V Sigma W^H,
    keep sigma > tol_svd, D = V0^H B1 W0 Sigma0^{-1}, eig(D) = mu, lambda = c + r mu.
    B0's left factor has block rows v, v mu, ..., v mu^{K-1}, so an eigenvector is
    the first n-block of V0 s. With K = 1 this is Eq. 2.8 in the variable (z - c)/r."""
    K = len(M) // 2
    n, l = M[0].shape
    B0 = np.block([[M[i + j] for j in range(K)] for i in range(K)])
    B1 = np.block([[M[i + j + 1] for j in range(K)] for i in range(K)])
    Vs, s, Wh = np.linalg.svd(B0, full_matrices=False)
    p = int(np.sum(s > tol_svd))
    saturated = p >= min(K * n, K * l)
    if p == 0:
        return BeynResult(s, 0, False, np.zeros(0, np.complex128), np.zeros((n, 0), np.complex128))
    V0 = Vs[:, :p]
    W0 = Wh.conj().T[:, :p]
    D = V0.conj().T @ B1 @ W0 @ np.diag(1.0 / s[:p])
    mu, S = np.linalg.eig(D)
    return BeynResult(s, p, saturated, c + r * mu, normalise_vectors((V0 @ S)[:n]))


def square_filter(lam: np.ndarray, c: complex, r: float) -> np.ndarray:
    """Step 2.f: keep lambda inside the square inscribed in the disk (half-open)."""
    h = r / math.sqrt(2.0)
    re_ok = (lam.real >= c.real - h) & (lam.real < c.real + h)
    im_ok = (lam.imag >= c.imag - h) & (lam.imag < c.imag + h)
    return re_ok & im_ok


# ---------------------------------------------------------------------------
# Verification (pmCIMb step 3)
# ---------------------------------------------------------------------------

def sigma_min(problem, lam: complex):
    """(smallest singular value of T(lambda), ||T(lambda)||_F)."""
    T = assemble_T(problem, lam)
    return float(sla.svdvals(T)[-1]), float(np.linalg.norm(T))


def verify(problem, lams: Sequence[complex], tol_verify: float = 1e-6):
    sig = np.zeros(len(lams))
    acc = np.zeros(len(lams), dtype=bool)
    for i, lam in enumerate(lams):
        s, fro = sigma_min(problem, lam)
        sig[i] = s
        acc[i] = s <= tol_verify * max(1.0, fro / math.sqrt(problem.n))
    return sig, acc


# ---------------------------------------------------------------------------
# Region split (pmCIMa's quadrisection geometry) and the pmCIMb driver
# ---------------------------------------------------------------------------

def split4(c: complex, r: float):
    """Four child disks of radius r/2 centred at c + (+-1 +- i) (r/2)/sqrt(2)."""
    rc = r / 2.0
    d = rc / math.sqrt(2.0)
    return [(complex(c.real + sx * d, c.imag + sy * d), rc)
            for (sx, sy) in ((1, 1), (-1, 1), (1, -1), (-1, -1))]


@dataclasses.dataclass
class RegionRecord:
    c: complex
    r: float
    N: int
    depth: int
    I: float
    candidate: bool
    p: int = -1
    saturated: bool = False
    split: bool = False
    lam: np.ndarray = None        # eigenvalues of D before the square filter
    kept: np.ndarray = None       # mask after the square filter
    sigma: np.ndarray = None


@dataclasses.dataclass
class PmcimbResult:
    lam: np.ndarray               # verified eigenvalues, sorted by (Re, Im)
    vecs: np.ndarray              # n x m, matching lam
    sigma_min: np.ndarray         # per verified eigenvalue
    cand_lam: np.ndarray          # all filtered candidates before verification, sorted
    cand_sigma: np.ndarray
    cand_accept: np.ndarray
    records: List[RegionRecord]


def pmcimb(problem, regions: Sequence, V: np.ndarray, tol_ind: float = 0.1,
           tol_svd: float = 1e-6, tol_verify: float = 1e-6, max_depth: int = 8,
           indicator_N: int = 0, beyn_K: int = 1) -> PmcimbResult:
    """pmCIMb steps 1-3 over the given disks, with saturated disks split and re-run.

    indicator_N = 0: one N per disk serves both the indicator and Beyn's moments.
    indicator_N > 0: the paper's two-pass schedule (Appendix, pmCIMb driver; Sec. 3.2
    remark that N = 16 suffices for the indicator and N = 64 for Beyn): step 1
    screens each disk with the indicator on an indicator_N-node rule, step 2 runs
    Beyn with the disk's N on the candidates. Split children go through both steps
    again. Each disk's N must be a multiple of indicator_N.
    beyn_K > 1: Beyn's step uses the block Hankel matrices of 2 beyn_K scaled
    moments (beyn_extract_hankel); a disk is saturated, and split, only when
    p reaches min(K n, K l).
    """
    n = problem.n
    records: List[RegionRecord] = []
    lam_list, vec_list = [], []
    level = [(complex(g.c), float(g.r), int(g.N), 0) for g in regions]
    while level:
        nxt = []
        for (c, r, N, depth) in level:
            if indicator_N:
                if N % indicator_N:
                    raise ValueError("N = %d is not a multiple of indicator_N = %d" % (N, indicator_N))
                mi = moments(problem, c, r, indicator_N, V)
                I = indicator_value(mi.pf_N, mi.pf_half, mi.pf_abs)
                m = moments(problem, c, r, N, V) if I > tol_ind else None
            else:
                m = moments(problem, c, r, N, V)
                I = indicator_value(m.pf_N, m.pf_half, m.pf_abs)
            rec = RegionRecord(c, r, N, depth, I, I > tol_ind)
            if rec.candidate:
                if beyn_K > 1:
                    b = beyn_extract_hankel(hankel_moments(problem, c, r, N, V, beyn_K), c, r, tol_svd)
                else:
                    b = beyn_extract(m.C0, m.C1, tol_svd)
                rec.p, rec.saturated, rec.sigma, rec.lam = b.p, b.saturated, b.sigma, b.lam
                if b.saturated and depth < max_depth:
                    rec.split = True
                    nxt += [(cc, rr, N, depth + 1) for (cc, rr) in split4(c, r)]
                else:
                    keep = square_filter(b.lam, c, r)
                    rec.kept = keep
                    lam_list += list(b.lam[keep])
                    vec_list += [b.vecs[:, k] for k in np.flatnonzero(keep)]
            records.append(rec)
        level = nxt
    lam = np.array(lam_list, dtype=np.complex128)
    vecs = np.array(vec_list, dtype=np.complex128).T.reshape(n, len(lam_list))
    sig, acc = verify(problem, lam, tol_verify)
    order = np.lexsort((lam.imag, lam.real))
    lam, vecs, sig, acc = lam[order], vecs[:, order], sig[order], acc[order]
    return PmcimbResult(lam[acc], vecs[:, acc], sig[acc], lam, sig, acc, records)


# ---------------------------------------------------------------------------
# pmCIMa (Sec. 3.1): the indicator alone, level by level, then one linear
# eigenproblem per value
# ---------------------------------------------------------------------------

def pmcima_levels(r: float, tol_eps: float) -> int:
    """Levels of pmCIMa for a disk of radius r: ceil(log2(r / tol_eps)) + 2.

    Step 1.a gives ceil(log2(r / tol_eps)); the Appendix listing adds 2, which makes
    the last disks' radius r / 2^(L-1) at most tol_eps / 2, so that neighbouring
    final squares around one eigenvalue have centres within tol_eps of each other
    and the merge of the remark after the algorithm joins them. Taken as written in
    the listing."""
    return max(1, int(math.ceil(math.log2(r / tol_eps))) + 2)


def merge_centres(z: np.ndarray, tol_eps: float) -> np.ndarray:
    """The merge of the remark after pmCIMa: in order, each not yet merged centre
    takes every not yet merged centre within tol_eps of it (itself included, once)
    and is replaced by their mean."""
    z = np.asarray(z, dtype=np.complex128)
    used = np.zeros(len(z), dtype=bool)
    out = []
    for i in range(len(z)):
        if used[i]:
            continue
        grp = [j for j in range(len(z)) if not used[j] and abs(z[i] - z[j]) < tol_eps]
        used[grp] = True
        out.append(np.mean(z[grp]))
    return np.array(out, dtype=np.complex128)


@dataclasses.dataclass
class PmcimaResult:
    lam: np.ndarray      # merged approximate eigenvalues, sorted by (Re, Im)
    vecs: np.ndarray     # n x m: right singular vector of T(lam) for sigma_min (unit norm)
    sigma: np.ndarray    # sigma_min(T(lam))
    centres: np.ndarray  # the last level's candidate centres, before the merge
    regions: int         # indicator evaluations over all levels


def pmcima(problem, regions: Sequence, V: np.ndarray, tol_ind: float = 0.1,
           tol_eps: float = 1e-6) -> PmcimaResult:
    """pmCIMa. Step 1: each level computes the indicator (Eq. 3.1, the disk's N
    nodes, probe column f = V[:, 0]) of every disk; candidates (I > tol_ind) are
    quadrisected (split4) until the disk's level count is reached, and the last
    level's candidate centres approximate the eigenvalues (1.c), merged as in the
    remark. Step 2: for each value, the eigenvector of T(lambda) is taken as the
    right singular vector of its smallest singular value (the reading used for
    verification in pmCIMb)."""
    f = np.asarray(V)[:, :1]
    centres = []
    evaluated = 0
    level = [(complex(g.c), float(g.r), int(g.N), pmcima_levels(float(g.r), tol_eps), 0) for g in regions]
    while level:
        nxt = []
        for (c, r, N, L, depth) in level:
            m = moments(problem, c, r, N, f)
            evaluated += 1
            if indicator_value(m.pf_N, m.pf_half, m.pf_abs) <= tol_ind:
                continue
            if depth + 1 < L:
                nxt += [(cc, rr, N, L, depth + 1) for (cc, rr) in split4(c, r)]
            else:
                centres.append(c)
        level = nxt
    centres = np.array(centres, dtype=np.complex128)
    lam = merge_centres(centres, tol_eps)
    lam = lam[np.lexsort((lam.imag, lam.real))] if len(lam) else lam
    vecs = np.zeros((problem.n, len(lam)), dtype=np.complex128)
    sig = np.zeros(len(lam))
    for i, z in enumerate(lam):
        _, s, vh = np.linalg.svd(assemble_T(problem, z))
        sig[i] = s[-1]
        vecs[:, i] = vh[-1].conj()
    return PmcimaResult(lam, vecs, sig, centres, evaluated)
