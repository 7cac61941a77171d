"""Pins of the CPU oracle against facts fixed by mathematics or by the paper.

None of these compares the oracle with itself: each pin is a closed form
derived independently (exact discrete sums of the trapezoid rule for simple
poles), a brute-force eigen-solve (companion pencil, Lambert W roots), an
invariant (argument-principle counts, Beyn's similarity), or the paper's own
worked example. The mutation tests at the end plant plausible mistakes in the
oracle and check that a pin catches each one.
"""
import math

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

import oracle as o
import workloads as w
from tests import _truth as tr

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _poles(rng, c, r, n_in, n_out, rin=(0.2, 0.8), rout=(1.3, 3.0)):
    """Poles mu = c + r a with |a| in the given annuli (inside / outside the circle)."""
    ain = rng.uniform(*rin, n_in) * np.exp(2j * np.pi * rng.random(n_in))
    aout = rng.uniform(*rout, n_out) * np.exp(2j * np.pi * rng.random(n_out))
    a = np.concatenate([ain, aout])
    return c + r * a, a


# ---------------------------------------------------------------------------
# P1: exact discrete sums.  For T(z) = z - mu and a = (mu - c)/r with a^N != 1,
# (r/N) sum_j e^{i th_j} / (z_j - mu) = 1/(1 - a^N)       (|a| < 1 and |a| > 1),
# the rotated N/2 rule on the odd nodes gives 1/(1 + a^{N/2}), and
# (r/N) sum_j e^{i th_j} z_j / (z_j - mu) = mu / (1 - a^N) for N >= 2.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N", [8, 16, 32])
def test_diagonal_linear_moments_exact(N):
    rng = np.random.default_rng(11)
    c, r = 0.3 - 0.2j, 0.7
    mu, a = _poles(rng, c, r, 5, 7)
    P = w.diagonal_linear(mu)
    V = w.probe_block(rng, len(mu), 3)
    m = o.moments(P, c, r, N, V)
    q = 1.0 / (1.0 - a ** N)
    assert _rel(m.C0, q[:, None] * V) < 1e-12
    assert _rel(m.C1, (mu * q)[:, None] * V) < 1e-12
    assert _rel(m.pf_N, q * V[:, 0]) < 1e-12
    assert _rel(m.pf_half, V[:, 0] / (1.0 + a ** (N // 2))) < 1e-12
    I_exact = np.linalg.norm(1.0 / (1.0 - a ** (N // 2))) / math.sqrt(len(mu))
    assert abs(o.indicator_value(m.pf_N, m.pf_half) - I_exact) < 1e-12 * I_exact


def test_similarity_linear_moments_exact():
    """T(z) = A - z I, A = Q diag(mu) Q^-1:  C0 = -Q diag(q) Q^-1 V, C1 = -Q diag(mu q) Q^-1 V."""
    rng = np.random.default_rng(12)
    c, r, N = -0.1 + 0.4j, 0.5, 32
    mu, a = _poles(rng, c, r, 4, 8)
    P, Q = w.similarity_linear(mu, seed=3)
    V = w.probe_block(rng, len(mu), 4)
    m = o.moments(P, c, r, N, V)
    q = 1.0 / (1.0 - a ** N)
    Qi_V = np.linalg.solve(Q, V)
    assert _rel(m.C0, -Q @ (q[:, None] * Qi_V)) < 1e-11
    assert _rel(m.C1, -Q @ ((mu * q)[:, None] * Qi_V)) < 1e-11


def test_diagonal_quadratic_partial_fractions():
    """t(z) = g (z - m1)(z - m2): 1/t = [1/(z-m1) - 1/(z-m2)] / (g (m1 - m2))."""
    rng = np.random.default_rng(13)
    c, r, N = 0.0, 1.0, 32
    m1, a1 = _poles(rng, c, r, 3, 3)
    m2, a2 = _poles(rng, c, r, 2, 4)
    g = rng.uniform(0.5, 2.0, 6) + 0.3j
    P = w.diagonal_quadratic(m1, m2, g)
    V = w.probe_block(rng, 6, 2)
    m = o.moments(P, c, r, N, V)
    q1, q2 = 1.0 / (1.0 - a1 ** N), 1.0 / (1.0 - a2 ** N)
    k0 = (q1 - q2) / (g * (m1 - m2))
    k1 = (m1 * q1 - m2 * q2) / (g * (m1 - m2))
    assert _rel(m.C0, k0[:, None] * V) < 1e-12
    assert _rel(m.C1, k1[:, None] * V) < 1e-12


def test_indicator_is_one_inside_and_small_outside():
    """Eq. 3.1: I ~ 1 with eigenvalues inside, I ~ |a|^{-N/2} without (decay in N/2)."""
    rng = np.random.default_rng(14)
    c, r, N = 1.0 + 1.0j, 0.5, 16
    mu_in, _ = _poles(rng, c, r, 6, 0, rin=(0.1, 0.3))
    V = w.probe_block(rng, 6, 1)
    I_in = o.indicator_value(*_pf(o.moments(w.diagonal_linear(mu_in), c, r, N, V)))
    assert abs(I_in - 1.0) < 1e-3
    mu_out = c + r * 2.0 * np.exp(2j * np.pi * rng.random(6))
    I_out = o.indicator_value(*_pf(o.moments(w.diagonal_linear(mu_out), c, r, N, V)))
    assert I_out == pytest.approx(2.0 ** (-N // 2), rel=1e-2)
    assert I_out < 0.1 < I_in


def _pf(m):
    return m.pf_N, m.pf_half


# ---------------------------------------------------------------------------
# P2: Beyn's extraction.  With n <= l, C0 = diag(q) V with V of full row rank,
# so D = V0^H diag(mu) V0 is similar to diag(mu): eig(D) = mu wherever mu is.
# ---------------------------------------------------------------------------

def test_beyn_square_case_recovers_all_poles():
    rng = np.random.default_rng(21)
    c, r, N = 0.0, 1.0, 16
    mu, a = _poles(rng, c, r, 3, 3, rout=(1.05, 1.1))
    P = w.diagonal_linear(mu)
    V = w.probe_block(rng, 6, 8)
    m = o.moments(P, c, r, N, V)
    b = o.beyn_extract(m.C0, m.C1, tol_svd=1e-13)
    assert b.p == 6 and b.saturated
    ri, ci = linear_sum_assignment(np.abs(mu[:, None] - b.lam[None, :]))
    assert np.max(np.abs(mu[ri] - b.lam[ci])) < 1e-10


def test_beyn_rank_equals_count_with_gap():
    """n > l, inside |a| <= 0.5, outside |a| >= 1.65 at N = 32: p = #inside, lambda ~ mu_in."""
    rng = np.random.default_rng(22)
    c, r, N = 0.5j, 0.8, 32
    mu, a = _poles(rng, c, r, 3, 20, rin=(0.05, 0.5), rout=(1.65, 4.0))
    P = w.diagonal_linear(mu)
    V = w.probe_block(rng, len(mu), 6)
    m = o.moments(P, c, r, N, V)
    b = o.beyn_extract(m.C0, m.C1, tol_svd=1e-6)
    assert b.p == 3 and not b.saturated
    ri, ci = linear_sum_assignment(np.abs(mu[:3, None] - b.lam[None, :]))
    err = np.max(np.abs(mu[:3][ri] - b.lam[ci]))
    assert err < 1e-9 * r
    # eigenvectors of a diagonal T are coordinate vectors
    for k in range(3):
        idx = int(np.argmin(np.abs(mu - b.lam[k])))
        assert abs(abs(b.vecs[idx, k]) - 1.0) < 1e-9


# ---------------------------------------------------------------------------
# P3/P4: brute-force eigenvalues, end to end through pmCIMb
# ---------------------------------------------------------------------------

def _match(truth, got, median=False):
    ri, ci = linear_sum_assignment(np.abs(truth[:, None] - got[None, :]))
    d = np.abs(truth[ri] - got[ci])
    if median:
        return len(ri), (np.max(d) if len(ri) else 0.0), (np.median(d) if len(ri) else 0.0)
    return len(ri), np.max(d) if len(ri) else 0.0


def _in_box(ev, box):
    x0, x1, y0, y1 = box
    return ev[(ev.real >= x0) & (ev.real < x1) & (ev.imag >= y0) & (ev.imag < y1)]


def test_paper_example_all_eigenvalues():
    """Appendix example (generateT, test.m grid): all 8 companion eigenvalues, none spurious."""
    P = w.paper_n4_example(_golden("paper_n4_example.txt"))
    s, M = 6.0, 9
    h = s / M
    regs = [w.Region(complex(-3 + (i + 0.5) * h, -3 + (j + 0.5) * h), math.sqrt(2) * s / M / 2, 64)
            for i in range(M) for j in range(M)]
    V = w.probe_block(np.random.default_rng(0), 4, 10)
    res = o.pmcimb(P, regs, V, tol_svd=1e-6)
    truth = _in_box(tr.companion_eigs(*[t[0] for t in P.terms]), (-3, 3, -3, 3))
    assert len(truth) == 8 and len(res.lam) == 8
    k, err = _match(truth, res.lam)
    assert k == 8 and err < 1e-10


def test_random_quadratic_matches_companion():
    rng = np.random.default_rng(31)
    n = 10
    A = [w.complex_gaussian(rng, (n, n)) / math.sqrt(n) for _ in range(3)]
    P = w.Problem(n, [(A[d], w.MONOMIAL, d, 0.0) for d in range(3)])
    regs = w.grid_regions(-1.6, 1.6, -1.6, 1.6, 4, 4, 64)
    V = w.probe_block(rng, n, 6)
    res = o.pmcimb(P, regs, V)
    truth = _in_box(tr.companion_eigs(*A), (-1.6, 1.6, -1.6, 1.6))
    k, err, med = _match(truth, res.lam, median=True)
    assert k == len(truth) == len(res.lam)
    # worst case is an eigenvalue just outside a circle (quadrature error |a|^-N);
    # the paper's eigenvalue precision tol_eps = 1e-6 bounds it, most are exact
    assert err < 1e-6 and med < 1e-7


def test_diagonal_delay_matches_lambert_w():
    alpha = np.array([-0.5 + 0.3j, 0.2 - 0.1j, -1.0 + 2.0j])
    beta = np.array([0.4, -0.3 + 0.2j, 0.25j])
    P = w.diagonal_delay(alpha, beta, tau=1.0)
    box = (-4.0, 1.0, -8.0, 8.0)
    regs = w.grid_regions(*box, 5, 16, 64)
    V = w.probe_block(np.random.default_rng(5), 3, 4)
    res = o.pmcimb(P, regs, V)
    roots = np.concatenate([tr.delay_roots(a, b, 1.0) for a, b in zip(alpha, beta)])
    truth = _in_box(roots, box)
    assert len(truth) >= 8
    k, err, med = _match(truth, res.lam, median=True)
    assert k == len(truth) == len(res.lam)
    assert err < 1e-6 and med < 1e-9


def test_rank_matches_argument_principle_count():
    """P5: the count inside each disk is an integer equal to the brute-force count, and
    p equals it wherever the gap condition of Beyn's rank test holds
    (max |a_in|^N < 1/2 and max |a_out|^-N below tol_svd / 10)."""
    W = w.quadratic_small(seed=0, n=12, l=8, N=64)
    terms = W.problem.terms
    ev = tr.companion_eigs(*[t[0] for t in terms])
    checked = counted = 0
    for g in W.regions:
        a = np.abs(ev - g.c) / g.r
        if np.min(np.abs(a - 1.0)) < 0.05:    # the fine rule needs the contour clear of eigenvalues
            continue
        cnt = tr.argument_principle_count(terms, W.problem.n, g.c, g.r)
        assert abs(cnt.imag) < 1e-6 and abs(cnt.real - round(cnt.real)) < 1e-6
        truth = int(np.sum(a < 1.0))
        assert round(cnt.real) == truth
        counted += 1
        a_in = a[a < 1.0]
        a_out = a[a > 1.0]
        gap = (a_in.size == 0 or np.max(a_in) ** g.N < 0.5) and np.min(a_out) ** (-g.N) < 1e-7
        if 0 < truth < 8 and gap:
            m = o.moments(W.problem, g.c, g.r, g.N, W.V)
            assert o.beyn_extract(m.C0, m.C1).p == truth
            checked += 1
    assert counted >= 8 and checked >= 2


# ---------------------------------------------------------------------------
# P6: verification quantity
# ---------------------------------------------------------------------------

def test_sigma_min_diagonal_and_at_eigenvalue():
    rng = np.random.default_rng(41)
    mu = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    P = w.diagonal_linear(mu)
    z = 0.3 + 0.1j
    s, fro = o.sigma_min(P, z)
    assert s == pytest.approx(np.min(np.abs(z - mu)), rel=1e-14)
    assert fro == pytest.approx(np.linalg.norm(z - mu), rel=1e-14)
    s0, _ = o.sigma_min(P, mu[3])
    assert s0 <= 1e-15
    sig, acc = o.verify(P, [mu[2], mu[2] + 1e-3], 1e-6)
    assert acc[0] and not acc[1]


# ---------------------------------------------------------------------------
# P7: the hand-written LU (pivot rule |Re| + |Im|, first index on ties)
# ---------------------------------------------------------------------------

def test_hand_lu_matches_lapack_pivots_and_solves():
    import scipy.linalg as sla
    rng = np.random.default_rng(51)
    for n in (1, 2, 5, 33, 64):
        T = w.complex_gaussian(rng, (n, n))
        LU, piv = o.lu_factor_pp(T)
        _, piv_l = sla.lu_factor(T)
        assert np.array_equal(piv, piv_l)
        L = np.tril(LU, -1) + np.eye(n)
        U = np.triu(LU)
        PT = T.copy()
        for k in range(n):
            PT[[k, piv[k]], :] = PT[[piv[k], k], :]
        assert _rel(L @ U, PT) < 1e-14 * n
        B = w.complex_gaussian(rng, (n, 3))
        X = o.lu_solve_pp(LU, piv, B)
        assert np.linalg.norm(T @ X - B) <= 1e-13 * n * np.linalg.norm(T) * np.linalg.norm(X)


def test_hand_lu_tie_goes_to_lowest_row():
    T = np.array([[1.0, 2.0], [1j, 3.0]], dtype=complex)     # |1| and |i| tie in column 0
    _, piv = o.lu_factor_pp(T)
    assert piv[0] == 0


# ---------------------------------------------------------------------------
# Geometry
# ---------------------------------------------------------------------------

def test_square_filter_half_open_and_split_geometry():
    c, r = 1.0 + 1.0j, math.sqrt(2.0)                     # square [0,2) x [0,2)
    lam = np.array([0.0 + 0.0j, 2.0 + 1.0j, 1.0 + 1.999j, 1.0 - 1e-12j, 1.5 + 0.5j])
    assert list(o.square_filter(lam, c, r)) == [True, False, True, False, True]
    kids = o.split4(c, r)
    assert sorted((k[0].real, k[0].imag) for k in kids) == [(0.5, 0.5), (0.5, 1.5), (1.5, 0.5), (1.5, 1.5)]
    assert all(k[1] == pytest.approx(r / 2) for k in kids)


def _golden(name):
    import os
    return os.path.join(os.path.dirname(__file__), "golden", name)


# ---------------------------------------------------------------------------
# Mutation tests: plausible mistakes planted in the oracle are caught by a pin
# ---------------------------------------------------------------------------

def _diag_case():
    rng = np.random.default_rng(61)
    c, r, N = 0.2, 0.9, 16
    mu, a = _poles(rng, c, r, 3, 3)
    return w.diagonal_linear(mu), w.probe_block(rng, 6, 2), c, r, N, mu, a


def test_pin_catches_wrong_half_rule(monkeypatch):
    P, V, c, r, N, mu, a = _diag_case()
    real = o.nodes_weights

    def rotated(cc, rr, NN):                  # starts at theta_1 instead of theta_0: swaps odd/even
        z, ww = real(cc, rr, NN)
        return np.roll(z, -1), np.roll(ww, -1)
    monkeypatch.setattr(o.pmcim_ref, "nodes_weights", rotated)
    m = o.moments(P, c, r, N, V)
    assert _rel(m.pf_half, V[:, 0] / (1.0 + a ** (N // 2))) > 1e-3


def test_pin_catches_c1_without_node(monkeypatch):
    P, V, c, r, N, mu, a = _diag_case()
    real = o.nodes_weights

    def plain_theta(cc, rr, NN):              # the printed Eq. 3.3 typo z + r theta_j
        z, ww = real(cc, rr, NN)
        return cc + rr * (2 * np.pi * np.arange(NN) / NN), ww
    monkeypatch.setattr(o.pmcim_ref, "nodes_weights", plain_theta)
    m = o.moments(P, c, r, N, V)
    q = 1.0 / (1.0 - a ** N)
    assert _rel(m.C1, (mu * q)[:, None] * V) > 1e-3


def test_pin_catches_transpose_instead_of_adjoint(monkeypatch):
    rng = np.random.default_rng(21)
    c, r, N = 0.0, 1.0, 16
    mu, a = _poles(rng, c, r, 3, 3, rout=(1.05, 1.1))
    V = w.probe_block(rng, 6, 8)
    m = o.moments(w.diagonal_linear(mu), c, r, N, V)
    real_svd = np.linalg.svd

    def svd_conj(A, full_matrices=True):      # returns V conj'd: a missing conjugation in V0^H
        U, s, Wh = real_svd(A, full_matrices=full_matrices)
        return U.conj(), s, Wh
    monkeypatch.setattr(o.pmcim_ref.np.linalg, "svd", svd_conj)
    b = o.beyn_extract(m.C0, m.C1, tol_svd=1e-13)
    ri, ci = linear_sum_assignment(np.abs(mu[:, None] - b.lam[None, :]))
    assert np.max(np.abs(mu[ri] - b.lam[ci])) > 1e-3


def test_indicator_is_zero_when_pf_is_at_rounding_level():
    """Sec. 2.1: P = 0 without eigenvalues inside, so P f = 0. With every pole at |a| = 5 and
    N = 64 the exact indicator is 5^-32 ~ 2e-23, and P f|_N is rounding noise; the oracle
    returns 0 there, within 1e-12 of the exact value, and is unchanged with poles inside."""
    rng = np.random.default_rng(71)
    c, r, N = 0.0, 1.0, 64
    far = c + r * 5.0 * np.exp(2j * np.pi * rng.random(10))
    V = w.probe_block(rng, 10, 2)
    m = o.moments(w.diagonal_linear(far), c, r, N, V)
    I = o.indicator_value(m.pf_N, m.pf_half, m.pf_abs)
    assert I == 0.0 and abs(I - 5.0 ** -32) < 1e-12
    # poles inside and just outside (|a| <= 1.8 at N = 32 keeps every component of P f resolved)
    N = 32
    mu, a = _poles(rng, c, r, 3, 7, rout=(1.3, 1.8))
    m = o.moments(w.diagonal_linear(mu), c, r, N, w.probe_block(rng, 10, 2))
    I_exact = np.linalg.norm(1.0 / (1.0 - a ** (N // 2))) / math.sqrt(10)
    assert o.indicator_value(m.pf_N, m.pf_half, m.pf_abs) == pytest.approx(I_exact, rel=1e-12)


# ---------------------------------------------------------------------------
# Two-pass schedule (Appendix pmCIMb driver: the indicator on 16 nodes, Beyn on
# 64 nodes of the candidates).  For T = diag(z - mu) and f with no zero entry,
# P f|_N ./ P f|_{N/2} has entries (1 + a^{N/2}) / (1 - a^N) = 1 / (1 - a^{N/2}),
# so the coarse indicator is || 1 / (1 - a^{Ni/2}) ||_2 / sqrt(n) with Ni the
# indicator's node count (P1's sums).
# ---------------------------------------------------------------------------

def test_two_pass_schedule_decisions_and_eigenvalues():
    # 3 x 3 squares of side 1 on [-1.5, 1.5]^2, circumscribed disks, N = 64, indicator on 16 nodes
    regs = w.grid_regions(-1.5, 1.5, -1.5, 1.5, 3, 3, 64)
    mu = np.array([-1.0 + 0.9j, -0.8 + 1.1j, 0.1 - 0.05j, 1.05 - 1.0j,    # inside squares
                   -1.0 - 1.0j + 1.2 * 0.7071 * np.exp(0.3j),                 # |a| = 1.2 from the (-1,-1) disk
                   3.5 + 0.2j, -0.3 - 3.0j])                                  # outside the grid
    P = w.diagonal_linear(mu)
    V = w.probe_block(np.random.default_rng(41), len(mu), 4)
    Ni, tol = 16, 0.1
    res2 = o.pmcimb(P, regs, V, indicator_N=Ni)
    res1 = o.pmcimb(P, regs, V)
    tops = [rec for rec in res2.records if rec.depth == 0]
    assert len(tops) == len(regs)
    coarse_only = 0
    for rec in tops:
        a = (mu - rec.c) / rec.r
        q = 1.0 / (1.0 - a ** (Ni // 2))
        I_exact = np.linalg.norm(q) / math.sqrt(len(mu))
        assert rec.candidate == (I_exact > tol)
        if np.max(np.abs(q)) > 1e-3:
            assert rec.I == pytest.approx(I_exact, rel=1e-8)
        fine = np.linalg.norm(1.0 / (1.0 - a ** 32)) / math.sqrt(len(mu))
        coarse_only += int(rec.candidate and not fine > tol)
    assert coarse_only >= 1   # the |a| = 1.2 pole: a candidate on 16 nodes, not on 64
    inside = mu[(np.abs(mu.real) < 1.5) & (np.abs(mu.imag) < 1.5)]
    for lam in (res2.lam, res1.lam):
        assert len(lam) == len(inside)
        k, err = _match(inside, lam)
        assert k == len(inside) and err < 1e-10


# ---------------------------------------------------------------------------
# pmCIMa (Sec. 3.1): T(z) = A - zI with a prescribed spectrum (A = Q diag(mu) Q^-1, so
# every component of P f carries each pole's residue). The merged last-level centres
# must be the eigenvalues inside Omega, one each, within tol_eps; the vectors are unit
# null vectors of T(lambda) to sigma_min.
# ---------------------------------------------------------------------------

def test_pmcima_finds_prescribed_eigenvalues():
    mu = np.array([0.12 + 0.31j, -0.27 - 0.05j, 0.33 - 0.38j, 0.9 + 0.9j, -0.8 + 0.6j, 1.3 - 0.2j])
    P, _ = w.similarity_linear(mu, seed=4)
    V = w.probe_block(np.random.default_rng(3), len(mu), 2)
    regs = w.grid_regions(-0.5, 0.5, -0.5, 0.5, 2, 2, 16)
    tol_eps = 1e-6
    L = o.pmcima_levels(regs[0].r, tol_eps)
    assert regs[0].r / 2 ** (L - 1) <= tol_eps / 2      # the last disks are below the merge radius
    res = o.pmcima(P, regs, V, tol_eps=tol_eps)
    inside = mu[(np.abs(mu.real) < 0.5) & (np.abs(mu.imag) < 0.5)]
    assert len(res.lam) == len(inside) == 3
    k, err = _match(inside, res.lam)
    assert k == 3 and err < tol_eps
    T = [o.assemble_T(P, z) for z in res.lam]
    for i in range(len(res.lam)):
        v = res.vecs[:, i]
        assert abs(np.linalg.norm(v) - 1.0) < 1e-12
        assert np.linalg.norm(T[i] @ v) == pytest.approx(res.sigma[i], rel=1e-6)
        assert res.sigma[i] < 10 * tol_eps * np.linalg.norm(T[i], 2)


def test_merge_centres_groups_within_tol():
    z = np.array([0.0, 0.4e-6, 0.9e-6, 5e-6, 5.3e-6, 1.0])
    m = o.merge_centres(z, 1e-6)
    # the first centre takes the two within 1e-6 of it; the next free one takes its neighbour
    assert np.allclose(m, [np.mean(z[:3]), np.mean(z[3:5]), 1.0], atol=1e-15)


# ---------------------------------------------------------------------------
# Higher moments (block Hankel Beyn).  For T = diag(z - mu) the scaled moments are
# M_p = diag(a^p / (1 - a^N)) V (P1's sums with the extra phase e^{i p theta_j}), so
# B0 factors as [a^{i} ...] blocks and eig(D) returns every pole inside once K l
# reaches their number, with no split.
# ---------------------------------------------------------------------------

def test_hankel_moments_exact_sums():
    rng = np.random.default_rng(51)
    c, r, N, K = 0.2 - 0.1j, 0.8, 32, 3
    mu, a = _poles(rng, c, r, 4, 3)
    V = w.probe_block(rng, 7, 2)
    M = o.hankel_moments(w.diagonal_linear(mu), c, r, N, V, K)
    for p in range(2 * K):
        assert _rel(M[p], (a ** p / (1.0 - a ** N))[:, None] * V) < 1e-12


def test_hankel_beyn_resolves_more_poles_than_probes():
    rng = np.random.default_rng(52)
    c, r, N = 0.0, 1.0, 64
    mu, a = _poles(rng, c, r, 10, 5, rin=(0.1, 0.7), rout=(1.5, 3.0))
    P = w.diagonal_linear(mu)
    V = w.probe_block(rng, 15, 3)
    m = o.moments(P, c, r, N, V)
    b1 = o.beyn_extract(m.C0, m.C1, tol_svd=1e-10)
    assert b1.p == 3 and b1.saturated                       # l = 3 probes cannot hold 10 poles
    b4 = o.beyn_extract_hankel(o.hankel_moments(P, c, r, N, V, 4), c, r, tol_svd=1e-10)
    assert b4.p == 10 and not b4.saturated                  # K l = 12 >= 10
    k, err = _match(mu[:10], b4.lam)
    assert k == 10 and err < 1e-10
    for i in range(10):                                     # eigenvectors: e_i up to phase
        j = int(np.argmin(np.abs(b4.lam - mu[i])))
        assert abs(abs(b4.vecs[i, j]) - 1.0) < 1e-8


def test_hankel_with_one_moment_pair_is_beyn():
    rng = np.random.default_rng(53)
    W = w.quadratic_small(seed=5, n=12, l=6, N=32)
    reg = W.regions[5]
    m = o.moments(W.problem, reg.c, reg.r, reg.N, W.V)
    b = o.beyn_extract(m.C0, m.C1, tol_svd=1e-8)
    h = o.beyn_extract_hankel(o.hankel_moments(W.problem, reg.c, reg.r, reg.N, W.V, 1), reg.c, reg.r, tol_svd=1e-8)
    assert b.p == h.p > 0
    k, err = _match(b.lam, h.lam)
    assert k == b.p and err < 1e-9


# ---------------------------------------------------------------------------
# Eigenvector normalisation: unit 2-norm, largest-modulus entry real and
# positive. The rule fixes a vector's free complex factor, so any s e^{i phi}
# multiple of a vector must map to one and the same output.
# ---------------------------------------------------------------------------

def _phase_rule_holds(fn):
    rng = np.random.default_rng(93)
    n, k = 7, 3
    base = w.complex_gaussian(rng, (n, k))
    imax = [2, 5, 0]
    for j, i in enumerate(imax):                  # a unique largest entry, real positive
        base[:, j] *= 0.5 / np.max(np.abs(base[:, j]))
        base[i, j] = 1.0
    want = base / np.linalg.norm(base, axis=0, keepdims=True)
    ok = True
    for phi in (0.0, 0.7, 2.9, -1.4):
        for s in (1e-3, 1.0, 40.0):
            got = fn(s * np.exp(1j * phi) * base)
            ok &= bool(np.allclose(got, want, rtol=0, atol=1e-14))
    return ok


def test_normalise_vectors_phase_rule():
    """Every s e^{i phi} multiple of a vector whose largest entry is real positive maps back to
    that unit vector; on a diagonal problem Beyn's eigenvector of pole mu_i is e_i itself."""
    assert _phase_rule_holds(o.normalise_vectors)
    rng = np.random.default_rng(94)
    mu, a = _poles(rng, 0.0, 1.0, 3, 2, rout=(1.6, 2.5))
    V = w.probe_block(rng, 5, 4)
    m = o.moments(w.diagonal_linear(mu), 0.0, 1.0, 64, V)
    b = o.beyn_extract(m.C0, m.C1, tol_svd=1e-9)
    assert b.p == 3
    for k in range(b.p):
        i = int(np.argmin(np.abs(mu - b.lam[k])))
        e = np.zeros(5, np.complex128)
        e[i] = 1.0
        assert np.max(np.abs(b.vecs[:, k] - e)) < 1e-9


@pytest.mark.parametrize("mistake", ["no_rotation", "conjugate_rotation", "no_scaling"])
def test_pin_catches_wrong_phase_rule(mistake):
    def broken(Vc):
        out = np.array(Vc, dtype=np.complex128, copy=True)
        for k in range(out.shape[1]):
            v = out[:, k]
            if mistake != "no_scaling":
                v = v / np.linalg.norm(v)
            i = int(np.argmax(np.abs(v)))
            if mistake == "conjugate_rotation":
                v = v * (v[i] / abs(v[i]))
            elif mistake == "no_scaling":
                v = v * (abs(v[i]) / v[i])
            out[:, k] = v
        return out
    assert not _phase_rule_holds(broken)


def test_indicator_leaves_out_components_at_rounding_level():
    """Eq. 3.1 componentwise: with pf_abs given, a component whose |P f|_{N/2}| is at or below
    PF_FLOOR ||pf_abs|| (an exact zero included) has no determined ratio, and I is the root mean
    square of the other ratios (Eq. 3.1 exactly when none is left out)."""
    a = np.array([0.5 + 0.5j, 1e-3 + 0j, 2.0 - 1j])
    b = np.array([0.5 + 0.0j, 1e-3 + 0j, 1.0 + 0j])
    pa = np.array([1.0, 1.0, 1.0])
    full = np.linalg.norm(a / b) / np.sqrt(3)
    assert o.indicator_value(a, b) == pytest.approx(full, rel=1e-15)
    assert o.indicator_value(a, b, pa) == pytest.approx(full, rel=1e-15)
    rest = np.linalg.norm((a / b)[1:]) / np.sqrt(2)              # RMS over the two determined ratios
    for tiny in (0.0, 1e-300, 1e-11):
        b2 = np.array([tiny + 0j, b[1], b[2]])
        assert o.indicator_value(a, b2, pa) == pytest.approx(rest, rel=1e-15), tiny
    b3 = np.array([1e-9 + 0j, b[1], b[2]])                      # above the floor: counted
    assert o.indicator_value(a, b3, pa) > 1e8
