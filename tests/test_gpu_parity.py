"""GPU path (through the C ABI) against the CPU oracle, element by element.

Tolerances:
  * moments C0, C1, P f|_{N/2}: the difference of two backward-stable LU solves
    at node j is bounded by c n u kappa(T(z_j)) ||X_j|| (u = 2^-53), and the
    weighted N-term sum adds at most c (N + 4) u |w_j| ||X_j||; summed over the
    nodes this gives the bound of `_moment_bound`, c = 4;
  * eigenvalues: |d lambda| / max(1, |lambda|) <= 1e-10;
  * indicator values: relative 1e-6 where P f is resolved above rounding
    noise (||P f|_N|| > 1e-6 * pf_scale); decisions must then be equal unless
    |I - tol_ind| <= 1e-6 * tol_ind (a threshold tie). Where P f is below that
    level both indicators are ratios of rounding noise and only the final
    eigenvalue sets are compared.
"""
import math

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

import oracle as o
import workloads as w

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
LAM_TOL = 1e-10


@pytest.fixture(scope="module")
def pm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2312_13117_gb300 import build, pmcim
    build.build()
    pmcim.load()
    return pmcim


def _moment_bound(problem, reg, V, c=4.0):
    """Sum over nodes of |w_j| c u (n kappa_1(T(z_j)) + N + 4) ||X_j|| (LAPACK condition estimate)."""
    import scipy.linalg as sla
    from scipy.linalg.lapack import zgecon
    z, wts = o.nodes_weights(reg.c, reg.r, reg.N)
    n = problem.n
    b0 = b1 = bh = 0.0
    for j in range(reg.N):
        T = o.assemble_T(problem, z[j])
        lu, piv = sla.lu_factor(T)
        X = sla.lu_solve((lu, piv), V)
        anorm = np.max(np.sum(np.abs(T), axis=0))
        rcond, info = zgecon(lu, anorm, norm="1")
        kap = 1.0 / max(rcond, 1e-300)
        e = c * U64 * (n * kap + reg.N + 4)
        b0 += abs(wts[j]) * e * np.linalg.norm(X)
        b1 += abs(wts[j] * z[j]) * e * np.linalg.norm(X)
        if j % 2 == 1:
            bh += 2 * abs(wts[j]) * e * np.linalg.norm(X[:, 0])
    return b0, b1, bh


def _check_moments(pm, problem, regions, V, opt=None):
    P = pm.Problem(problem.n, problem.terms)
    C0, C1, ph, pa = P.moments(regions, V, opt=opt)
    for g, reg in enumerate(regions):
        m = o.moments(problem, reg.c, reg.r, reg.N, V)
        b0, b1, bh = _moment_bound(problem, reg, V)
        assert np.linalg.norm(C0[g] - m.C0) <= b0 + 1e-300, (g, np.linalg.norm(C0[g] - m.C0), b0)
        assert np.linalg.norm(C1[g] - m.C1) <= b1 + 1e-300, (g, np.linalg.norm(C1[g] - m.C1), b1)
        assert np.linalg.norm(ph[g] - m.pf_half) <= bh + 1e-300, g
    P.close()


def _match_lam(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    assert len(a) == len(b), (len(a), len(b))
    if len(a) == 0:
        return 0.0
    cost = np.abs(a[:, None] - b[None, :])
    ri, ci = linear_sum_assignment(cost)
    return float(np.max(np.abs(a[ri] - b[ci]) / np.maximum(1.0, np.abs(b[ci]))))


# ---------------------------------------------------------------------------
# a1-a6: moments
# ---------------------------------------------------------------------------

def test_moments_quadratic_n64(pm):
    W = w.quadratic_small()
    _check_moments(pm, W.problem, W.regions, W.V)


@pytest.mark.parametrize("n,l,N", [(1, 1, 2), (2, 3, 4), (3, 1, 8), (17, 4, 16), (33, 8, 16),
                                   (65, 5, 8), (130, 2, 4), (200, 16, 6)])
def test_moments_ragged_sizes(pm, n, l, N):
    """Sizes below, at and across the 32-column panel and 64-row tile edges."""
    rng = np.random.default_rng(100 + n)
    A = [w.complex_gaussian(rng, (n, n)) / math.sqrt(n) for _ in range(3)]
    prob = w.Problem(n, [(A[d], w.MONOMIAL, d, 0.0) for d in range(3)])
    V = w.probe_block(rng, n, l)
    regs = [w.Region(complex(0.3, -0.2), 0.9, N), w.Region(complex(-1.1, 0.8), 0.45, N)]
    _check_moments(pm, prob, regs, V)


@pytest.mark.parametrize("n,l,N", [(33, 8, 16), (65, 5, 8), (100, 10, 8), (130, 2, 4), (200, 16, 6)])
def test_moments_fp64_tile32(pm, n, l, N):
    """The FP64 node kernel with 32 x 32 trailing tiles (option fp64_tile, the autotuner's
    other FP64 candidate up to n = 256): the same bound against the oracle, across the
    32-row tile and panel edges."""
    rng = np.random.default_rng(300 + n)
    A = [w.complex_gaussian(rng, (n, n)) / math.sqrt(n) for _ in range(3)]
    prob = w.Problem(n, [(A[d], w.MONOMIAL, d, 0.0) for d in range(3)])
    V = w.probe_block(rng, n, l)
    regs = [w.Region(complex(0.3, -0.2), 0.9, N), w.Region(complex(-1.1, 0.8), 0.45, N)]
    _check_moments(pm, prob, regs, V, opt=pm.options(precision=pm.PREC_FP64, fp64_tile=32))


def test_solve_fp64_tile32_quadratic_n64(pm):
    W = w.quadratic_small()
    P = pm.Problem(W.problem.n, W.problem.terms)
    res = P.solve(W.regions, W.V, opt=pm.options(precision=pm.PREC_FP64, fp64_tile=32))
    ref = o.pmcimb(W.problem, W.regions, W.V)
    assert _match_lam(res["lam"], ref.lam) <= LAM_TOL
    P.close()


def test_moments_delay_and_identity_terms(pm):
    W = w.delay_large(n=96, l=4, N=16, nx=4, ny=12)
    _check_moments(pm, W.problem, W.regions[::9], W.V)


def test_moments_closed_form_diagonal(pm):
    """The GPU moments also satisfy the exact discrete sums of a diagonal T."""
    rng = np.random.default_rng(3)
    c, r, N = 0.2 + 0.1j, 0.8, 16
    a = np.concatenate([rng.uniform(0.2, 0.8, 4), rng.uniform(1.3, 2.5, 4)]) * np.exp(2j * np.pi * rng.random(8))
    mu = c + r * a
    P = pm.Problem(8, w.diagonal_linear(mu).terms)
    V = w.probe_block(rng, 8, 3)
    C0, C1, ph, _ = P.moments([w.Region(c, r, N)], V)
    q = 1.0 / (1.0 - a ** N)
    assert np.linalg.norm(C0[0] - q[:, None] * V) <= 1e-13 * np.linalg.norm(q[:, None] * V)
    assert np.linalg.norm(C1[0] - (mu * q)[:, None] * V) <= 1e-13 * np.linalg.norm((mu * q)[:, None] * V)
    assert np.linalg.norm(ph[0] - V[:, 0] / (1 + a ** (N // 2))) <= 1e-13 * np.linalg.norm(V[:, 0])


# ---------------------------------------------------------------------------
# a7: indicator and decisions
# ---------------------------------------------------------------------------

def _check_decisions(pm, W, regions):
    """Indicator decisions against the oracle's on every disk, the oracle's rounding-level
    floor (P f|_N at or below 1e-10 of sum_j |w_j||x_j| gives I = 0) included; only a threshold
    tie |I - tol_ind| <= 1e-6 tol_ind is exempt. Values are compared where P f|_N is resolved
    well above rounding noise."""
    P = pm.Problem(W.problem.n, W.problem.terms)
    ind, cand, pn, ps = P.indicator(regions, W.V)
    for g, reg in enumerate(regions):
        m = o.moments(W.problem, reg.c, reg.r, reg.N, W.V)
        I = o.indicator_value(m.pf_N, m.pf_half, m.pf_abs)
        assert pn[g] == pytest.approx(np.linalg.norm(m.pf_N), rel=1e-8, abs=1e-13 * ps[g])
        if abs(I - W.tol_ind) > 1e-6 * W.tol_ind:
            assert bool(cand[g]) == (I > W.tol_ind), (g, I, ind[g])
        if pn[g] > 1e-6 * ps[g]:
            assert ind[g] == pytest.approx(I, rel=1e-6)
    P.close()


def test_indicator_and_decisions(pm):
    W = w.quadratic_small()
    _check_decisions(pm, W, W.regions)


def test_indicator_decisions_delay_n1024_sampled(pm):
    """Six disks spread over the benchmark's n = 1024 delay grid (corners and interior)."""
    W = w.delay_large()
    _check_decisions(pm, W, [W.regions[g] for g in (300, 517, 0, 47, 401, 767)])


def test_device_pointers_through_the_abi(pm):
    """Inputs and outputs given as CUDA device buffers (torch tensors)."""
    import ctypes
    import torch
    W = w.quadratic_small(n=32, l=4, N=16)
    P = pm.Problem(W.problem.n, W.problem.terms)
    ind_h, cand_h, _, _ = P.indicator(W.regions, W.V)
    Vt = torch.from_numpy(np.ascontiguousarray(W.V.T)).cuda()  # column-major n x l
    R = len(W.regions)
    ind_d = torch.zeros(R, dtype=torch.float64, device="cuda")
    cand_d = torch.zeros(R, dtype=torch.uint8, device="cuda")
    opt = pm.options()
    lib = pm.load()
    rc = lib.pmcim_indicator(P.handle, ctypes.byref(opt), R, pm.regions_array(W.regions), W.V.shape[1],
                             Vt.data_ptr(), ind_d.data_ptr(), None, None, cand_d.data_ptr())
    assert rc == 0
    assert np.array_equal(ind_d.cpu().numpy(), ind_h)
    assert np.array_equal(cand_d.cpu().numpy().astype(bool), cand_h)
    P.close()


# ---------------------------------------------------------------------------
# a8-a10: Beyn's extraction with splitting and the square filter
# ---------------------------------------------------------------------------

def _oracle_beyn_levels(problem, regions, V, tol_ind=0.1, tol_svd=1e-6, max_depth=8):
    """pmcim_beyn's contract in oracle steps: no gate on the given disks, gate on children."""
    lam = []
    level = [(complex(g.c), g.r, g.N, 0) for g in regions]
    while level:
        nxt = []
        for (c, r, N, d) in level:
            m = o.moments(problem, c, r, N, V)
            if d > 0 and not o.indicator_value(m.pf_N, m.pf_half) > tol_ind:
                continue
            b = o.beyn_extract(m.C0, m.C1, tol_svd)
            if b.saturated and d < max_depth:
                nxt += [(cc, rr, N, d + 1) for (cc, rr) in o.split4(c, r)]
            else:
                lam += list(b.lam[o.square_filter(b.lam, c, r)])
        level = nxt
    return np.array(lam)


def test_beyn_on_regions(pm):
    W = w.quadratic_small()
    regs = W.regions[4:8]
    P = pm.Problem(W.problem.n, W.problem.terms)
    lam, vecs, rof, st = P.beyn(regs, W.V)
    ref = _oracle_beyn_levels(W.problem, regs, W.V)
    # only values that verify are unique; spurious ones come from rounding-level directions
    sg, acc = o.verify(W.problem, ref)
    sg2, acc2 = o.verify(W.problem, lam)
    assert _match_lam(lam[acc2], ref[acc]) <= LAM_TOL
    for k in np.flatnonzero(acc2):
        v = vecs[:, k]
        assert abs(np.linalg.norm(v) - 1.0) < 1e-12
        i = int(np.argmax(np.abs(v)))
        assert abs(v[i].imag) < 1e-14 and v[i].real > 0
        T = o.assemble_T(W.problem, lam[k])
        assert np.linalg.norm(T @ v) <= 1e-7 * np.linalg.norm(T)
    P.close()


def test_beyn_square_case_all_poles(pm):
    """n <= l: eig(D) returns every pole; the square filter keeps those in the square."""
    rng = np.random.default_rng(21)
    c, r, N = 0.0, 1.0, 16
    a = np.concatenate([rng.uniform(0.2, 0.6, 3), rng.uniform(1.05, 1.1, 3)]) * np.exp(2j * np.pi * rng.random(6))
    mu = c + r * a
    P = pm.Problem(6, w.diagonal_linear(mu).terms)
    V = w.probe_block(rng, 6, 8)
    lam, _, _, st = P.beyn([w.Region(c, r, N)], V, opt=pm.options(tol_svd=1e-13, max_split_depth=0))
    assert st[0] & pm.RS_SATURATED and not st[0] & pm.RS_SPLIT
    keep = o.square_filter(mu, c, r)
    assert _match_lam(lam, mu[keep]) <= 1e-9
    P.close()


# ---------------------------------------------------------------------------
# a11: verification
# ---------------------------------------------------------------------------

def test_verify_sigma_min(pm):
    W = w.quadratic_small(n=48, l=4, N=16)
    res = o.pmcimb(W.problem, W.regions[:4], W.V)
    rng = np.random.default_rng(9)
    lam = np.concatenate([res.lam, rng.standard_normal(6) + 1j * rng.standard_normal(6)])
    P = pm.Problem(W.problem.n, W.problem.terms)
    sig, acc = P.verify(lam)
    for i, z in enumerate(lam):
        s_ref, fro = o.sigma_min(W.problem, z)
        assert abs(sig[i] - s_ref) <= max(1e-8 * s_ref, 1e-13 * fro), (i, sig[i], s_ref)
    sg_ref, acc_ref = o.verify(W.problem, lam)
    assert np.array_equal(acc, acc_ref)
    P.close()


# ---------------------------------------------------------------------------
# whole pmCIMb
# ---------------------------------------------------------------------------

def _solve_and_compare(pm, problem, regions, V, **kw):
    P = pm.Problem(problem.n, problem.terms)
    res = P.solve(regions, V, opt=pm.options(**kw))
    ref = o.pmcimb(problem, regions, V, **{k: v for k, v in kw.items() if k in ("tol_ind", "tol_svd", "tol_verify")})
    assert _match_lam(res["lam"], ref.lam) <= LAM_TOL
    P.close()
    return res, ref


def test_solve_quadratic_n64_all_eigenvalues(pm):
    W = w.quadratic_small()
    res, ref = _solve_and_compare(pm, W.problem, W.regions, W.V)
    assert len(res["lam"]) == 114
    assert res["stats"]["splits"] == sum(r.split for r in ref.records)
    assert res["stats"]["regions"] == len(ref.records)
    assert res["stats"]["certified"] + res["stats"]["unverified"] >= 1
    for k in range(len(res["lam"])):
        v = res["vecs"][:, k]
        T = o.assemble_T(W.problem, res["lam"][k])
        assert np.linalg.norm(T @ v) <= 1e-6 * np.linalg.norm(T)
        # the reported value is sigma_min or a certificate ||T v|| >= sigma_min, below the threshold
        s_ref, fro = o.sigma_min(W.problem, res["lam"][k])
        assert res["sigma_min"][k] >= s_ref - 1e-14 * fro
        assert res["sigma_min"][k] <= 1e-6 * max(1.0, fro / math.sqrt(W.problem.n))


def test_solve_paper_example(pm):
    import os
    P4 = w.paper_n4_example(os.path.join(os.path.dirname(__file__), "golden", "paper_n4_example.txt"))
    s, M = 6.0, 9
    h = s / M
    regs = [w.Region(complex(-3 + (i + 0.5) * h, -3 + (j + 0.5) * h), math.sqrt(2) * s / M / 2, 64)
            for i in range(M) for j in range(M)]
    V = w.probe_block(np.random.default_rng(0), 4, 10)
    res, ref = _solve_and_compare(pm, P4, regs, V)
    assert len(res["lam"]) == 8


def test_solve_delay_small(pm):
    W = w.delay_large(n=64, l=8, N=32, nx=4, ny=12)
    _solve_and_compare(pm, W.problem, W.regions, W.V)


def test_singular_node_is_reported_not_fatal(pm):
    """An eigenvalue exactly on node 0 makes T(z_0) singular: status bit, no failure."""
    c, r = 0.25, 0.5
    mu = np.array([c + r, 0.1 + 0.05j, -0.6 + 0.3j])
    P = pm.Problem(3, w.diagonal_linear(mu).terms)
    V = w.probe_block(np.random.default_rng(1), 3, 2)
    res = P.solve([w.Region(complex(c), r, 8)], V)
    assert res["status"][0] & pm.RS_SINGULAR_NODE
    assert res["stats"]["singular_nodes"] == 1
    P.close()


def test_full_size_delay_sampled_regions(pm):
    """n = 1024 delay problem in the benchmark's launch configuration, two sampled disks."""
    W = w.delay_large()
    regs = [W.regions[300], W.regions[517]]
    _check_moments(pm, W.problem, regs, W.V)


# ---------------------------------------------------------------------------
# a5: precision form (FP32 LU + FP64 refinement) against the FP64 oracle
# ---------------------------------------------------------------------------

MIXED_FORMS = ["fp32ir", "tf32x3", "bf16x3"]


def _mixed_opt(pm, form="fp32ir", **kw):
    prec = {"fp32ir": pm.PREC_FP32_IR, "tf32x3": pm.PREC_TF32X3_IR, "bf16x3": pm.PREC_BF16X3_IR}[form]
    return pm.options(precision=prec, **kw)


@pytest.mark.parametrize("form", MIXED_FORMS)
def test_mixed_moments_close_to_oracle(pm, form):
    """Refined solutions: |dX| <= 1e-9 |X| per node is the contract of the refinement stop."""
    W = w.quadratic_small(seed=2, n=72, l=6, N=16)
    P = pm.Problem(W.problem.n, W.problem.terms)
    C0, C1, _, _ = P.moments(W.regions[:6], W.V, opt=_mixed_opt(pm, form))
    for g, reg in enumerate(W.regions[:6]):
        m = o.moments(W.problem, reg.c, reg.r, reg.N, W.V)
        z, wts = o.nodes_weights(reg.c, reg.r, reg.N)
        X = o.solve_nodes(W.problem, z, W.V)
        scale = sum(abs(wts[j]) * np.linalg.norm(X[j]) for j in range(reg.N))
        b0, b1, _ = _moment_bound(W.problem, reg, W.V)
        assert np.linalg.norm(C0[g] - m.C0) <= b0 + 1e-9 * scale
        assert np.linalg.norm(C1[g] - m.C1) <= b1 + 1e-9 * scale * (abs(reg.c) + reg.r)
    P.close()


@pytest.mark.parametrize("form", MIXED_FORMS)
def test_mixed_moments_one_column_fp64_residual(pm, form):
    """One probe column (l = 1) with the residuals on the FP64 pipe, which then run as a
    matrix-vector product: n = 1100 spans two row blocks of 1024 and a ragged tail."""
    W = w.quadratic_small(seed=5, n=1100, l=1, N=16)
    P = pm.Problem(W.problem.n, W.problem.terms)
    C0, C1, _, _ = P.moments(W.regions[:2], W.V, opt=_mixed_opt(pm, form, residual_fp64=True))
    for g, reg in enumerate(W.regions[:2]):
        m = o.moments(W.problem, reg.c, reg.r, reg.N, W.V)
        z, wts = o.nodes_weights(reg.c, reg.r, reg.N)
        X = o.solve_nodes(W.problem, z, W.V)
        scale = sum(abs(wts[j]) * np.linalg.norm(X[j]) for j in range(reg.N))
        b0, b1, _ = _moment_bound(W.problem, reg, W.V)
        assert np.linalg.norm(C0[g] - m.C0) <= b0 + 1e-9 * scale
        assert np.linalg.norm(C1[g] - m.C1) <= b1 + 1e-9 * scale * (abs(reg.c) + reg.r)
    P.close()


@pytest.mark.parametrize("form", MIXED_FORMS)
def test_mixed_solve_quadratic_n64(pm, form):
    W = w.quadratic_small()
    P = pm.Problem(W.problem.n, W.problem.terms)
    res = P.solve(W.regions, W.V, opt=_mixed_opt(pm, form))
    ref = o.pmcimb(W.problem, W.regions, W.V)
    assert _match_lam(res["lam"], ref.lam) <= LAM_TOL
    assert res["stats"]["ir_sweeps"] >= res["stats"]["solves"]
    assert res["stats"]["tc_timeouts"] == 0
    P.close()


@pytest.mark.parametrize("form", MIXED_FORMS)
def test_mixed_solve_delay_small(pm, form):
    W = w.delay_large(n=64, l=8, N=32, nx=4, ny=12)
    P = pm.Problem(W.problem.n, W.problem.terms)
    res = P.solve(W.regions, W.V, opt=_mixed_opt(pm, form))
    ref = o.pmcimb(W.problem, W.regions, W.V)
    assert _match_lam(res["lam"], ref.lam) <= LAM_TOL
    P.close()


@pytest.mark.parametrize("form", ["tf32x3", "bf16x3"])
def test_tc_moments_ragged_tiles(pm, form):
    """Tensor-core trailing updates over several 128-row and 32-column tiles with ragged
    edges (n = 291: 3 row tiles at the first panel, the last one 35 rows; n + l = 296
    columns). T(z) = A - zI with a prescribed spectrum: 3 + 2 eigenvalues inside the two
    disks, the rest at |z| >= 3, so every node is well conditioned and the refinement must
    converge without the FP64 fallback. Moments and eigenvalues against the oracle."""
    rng = np.random.default_rng(31)
    n, l, N = 291, 5, 16
    regs = [w.Region(0.3 + 0.2j, 0.4, N), w.Region(-1.1 - 0.5j, 0.6, N)]
    inside = [0.3 + 0.2j + 0.2 * np.exp(2j * np.pi * k / 3) for k in range(3)]
    inside += [-1.1 - 0.5j + 0.25 * np.exp(2j * np.pi * k / 2 + 0.4j) for k in range(2)]
    far = (3.0 + 2.0 * rng.random(n - 5)) * np.exp(2j * np.pi * rng.random(n - 5))
    prob, _ = w.similarity_linear(np.concatenate([inside, far]), seed=8)
    V = w.probe_block(rng, n, l)
    P = pm.Problem(n, prob.terms)
    opt = _mixed_opt(pm, form)
    C0, C1, _, _ = P.moments(regs, V, opt=opt)
    for g, reg in enumerate(regs):
        m = o.moments(prob, reg.c, reg.r, reg.N, V)
        z, wts = o.nodes_weights(reg.c, reg.r, reg.N)
        X = o.solve_nodes(prob, z, V)
        scale = sum(abs(wts[j]) * np.linalg.norm(X[j]) for j in range(reg.N))
        b0, b1, _ = _moment_bound(prob, reg, V)
        assert np.linalg.norm(C0[g] - m.C0) <= b0 + 1e-9 * scale
        assert np.linalg.norm(C1[g] - m.C1) <= b1 + 1e-9 * scale * (abs(reg.c) + reg.r)
    res = P.solve(regs, V, opt=opt)
    ref = o.pmcimb(prob, regs, V)
    assert len(ref.lam) == 5
    assert _match_lam(res["lam"], ref.lam) <= LAM_TOL
    assert res["stats"]["ir_fallbacks"] == 0
    assert res["stats"]["tc_timeouts"] == 0
    P.close()


@pytest.mark.parametrize("form", MIXED_FORMS)
def test_mixed_fallback_path(pm, form):
    """An eigenvalue 1e-7 from node 0 makes T(z_0) too ill-conditioned for FP32 (kappa u32 ~ 1):
    refinement cannot converge there, so that node is re-solved in FP64 and flagged; the
    moments still agree with the FP64 form."""
    rng = np.random.default_rng(77)
    c, r, N, n = 0.0, 1.0, 16, 40          # n > 32: the precision-form kernel (smaller n use the warp kernel)
    a = np.concatenate([rng.uniform(0.2, 0.7, 8), rng.uniform(1.4, 3.0, n - 9)]) * np.exp(2j * np.pi * rng.random(n - 1))
    mu = np.concatenate([[c + r * (1.0 + 1e-7)], c + r * a])   # node 0 is z_0 = c + r
    prob, _ = w.similarity_linear(mu, seed=5)
    V = w.probe_block(rng, n, 4)
    reg = [w.Region(c, r, N)]
    P = pm.Problem(n, prob.terms)
    res = P.solve(reg, V, opt=_mixed_opt(pm, form))
    assert res["stats"]["ir_fallbacks"] >= 1
    assert res["status"][0] & pm.RS_IR_FALLBACK
    Cm0, Cm1, _, _ = P.moments(reg, V, opt=_mixed_opt(pm, form))
    Cd0, Cd1, _, _ = P.moments(reg, V)
    z, wts = o.nodes_weights(c, r, N)
    X = o.solve_nodes(prob, z, V)
    scale = sum(abs(wts[j]) * np.linalg.norm(X[j]) for j in range(1, N))
    assert np.linalg.norm(Cm0[0] - Cd0[0]) <= 1e-9 * scale
    assert np.linalg.norm(Cm1[0] - Cd1[0]) <= 1e-9 * scale * 2.0
    P.close()


@pytest.mark.parametrize("form", MIXED_FORMS)
def test_mixed_full_size_delay_sampled(pm, form):
    """n = 1024 delay problem: eigenvalues of two disks through the precision forms."""
    W = w.delay_large()
    regs = [W.regions[300], W.regions[517]]
    P = pm.Problem(W.problem.n, W.problem.terms)
    res = P.solve(regs, W.V, opt=_mixed_opt(pm, form))
    ref = o.pmcimb(W.problem, regs, W.V)
    assert len(ref.lam) >= 2
    assert _match_lam(res["lam"], ref.lam) <= LAM_TOL
    assert res["stats"]["ir_fallbacks"] == 0
    assert res["stats"]["tc_timeouts"] == 0
    P.close()


# ---------------------------------------------------------------------------
# a12: many problems of uneven size in one call
# ---------------------------------------------------------------------------

def _small_batch(count=6, seed0=1000):
    out = []
    for s in range(seed0, seed0 + count):
        rng = np.random.default_rng(s)
        n = int(rng.choice([17, 24, 40, 64, 100, 130]))
        A = [w.complex_gaussian(rng, (n, n)) / math.sqrt(n) for _ in range(3)]
        prob = w.Problem(n, [(A[d], w.MONOMIAL, d, 0.0) for d in range(3)])
        side = float(rng.uniform(1.0, 2.5))
        m = int(rng.integers(1, 4))
        N = int(rng.choice([16, 32]))
        regs = w.grid_regions(-side / 2, side / 2, -side / 2, side / 2, m, m, N)
        V = w.probe_block(rng, n, 6)
        out.append((prob, regs, V))
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32ir", "tf32x3", "auto"])
def test_batch_matches_oracle_per_problem(pm, precision):
    prec = {"fp64": pm.PREC_FP64, "fp32ir": pm.PREC_FP32_IR, "tf32x3": pm.PREC_TF32X3_IR,
            "auto": pm.PREC_AUTO}[precision]
    batch = _small_batch()
    handles = [pm.Problem(p.n, p.terms) for (p, _, _) in batch]
    res = pm.batch_solve(handles, [r for (_, r, _) in batch], [V for (_, _, V) in batch],
                         opt=pm.options(precision=prec))
    assert res["stats"]["graphs"] >= 1
    if precision == "auto":
        st = res["stats"]
        assert st["tuned_fp64"] + st["tuned_mixed"] + st["tuned_tc"] == len(batch)
    for q, (prob, regs, V) in enumerate(batch):
        ref = o.pmcimb(prob, regs, V)
        got = res["lam"][res["problem_of"] == q]
        assert _match_lam(got, ref.lam) <= LAM_TOL, q
    for h in handles:
        h.close()


def _config_batch():
    """Problems of the batched quadratic workload itself (seeds 427, 1, 25, 23: n = 765, 380,
    403, 58), one disk each: the first of the grid whose circle lies outside |z| = 0.9
    (inside it the eigenvalues are dense and the disks split eight levels deep)."""
    out = []
    for W in w.batched_quadratics([427, 1, 25, 23]):
        g = next((i for i, r in enumerate(W.regions) if abs(r.c) - r.r > 0.9), len(W.regions) - 1)
        out.append((W.problem, [W.regions[g]], W.V))
    return out


@pytest.fixture(scope="module")
def config_batch_oracle():
    batch = _config_batch()
    return batch, [o.pmcimb(prob, regs, V) for (prob, regs, V) in batch]


@pytest.mark.parametrize("precision", ["tf32x3", "auto"])
def test_batch_config_sizes_match_oracle(pm, precision, config_batch_oracle):
    """pmcim_batch_solve on problems of the batched workload up to n = 765 (ragged sizes in
    one launch): each problem's eigenvalues equal the oracle's, and so do its split and
    candidate counts."""
    batch, refs = config_batch_oracle
    prec = {"tf32x3": pm.PREC_TF32X3_IR, "auto": pm.PREC_AUTO}[precision]
    handles = [pm.Problem(p.n, p.terms) for (p, _, _) in batch]
    try:
        res = pm.batch_solve(handles, [r for (_, r, _) in batch], [V for (_, _, V) in batch],
                             opt=pm.options(precision=prec))
    finally:
        for h in handles:
            h.close()
    assert res["stats"]["splits"] == sum(sum(1 for r in ref.records if r.split) for ref in refs)
    for q, ref in enumerate(refs):
        got = res["lam"][res["problem_of"] == q]
        assert len(got) == len(ref.lam), q
        assert _match_lam(got, ref.lam) <= LAM_TOL, q


def test_batch_equals_single_calls(pm):
    """The batched path gives each problem the same eigenvalues as a call of its own."""
    batch = _small_batch(count=4, seed0=2000)
    handles = [pm.Problem(p.n, p.terms) for (p, _, _) in batch]
    res = pm.batch_solve(handles, [r for (_, r, _) in batch], [V for (_, _, V) in batch])
    for q, (prob, regs, V) in enumerate(batch):
        single = handles[q].solve(regs, V)
        got = res["lam"][res["problem_of"] == q]
        assert _match_lam(got, single["lam"]) <= 1e-13
    for h in handles:
        h.close()


# ---------------------------------------------------------------------------
# two-pass schedule (indicator on a coarse rule, Beyn on candidates, solves reused)
# ---------------------------------------------------------------------------

def _two_pass_diagonal():
    regs = w.grid_regions(-1.5, 1.5, -1.5, 1.5, 3, 3, 64)
    mu = np.array([-1.0 + 0.9j, -0.8 + 1.1j, 0.1 - 0.05j, 1.05 - 1.0j,
                   -1.0 - 1.0j + 1.2 * 0.7071 * np.exp(0.3j), 3.5 + 0.2j, -0.3 - 3.0j])
    V = w.probe_block(np.random.default_rng(41), len(mu), 4)
    return w.diagonal_linear(mu), regs, V, mu


@pytest.mark.parametrize("precision", ["fp64", "fp32ir", "tf32x3"])
def test_two_pass_decisions_solves_and_eigenvalues(pm, precision):
    """Closed-form coarse indicator (16 of 64 nodes): the candidate set matches it, the solve
    count is 16 per disk + 48 per candidate (the 16 indicator solves are reused), and the
    eigenvalues are the poles inside the squares."""
    prob, regs, V, mu = _two_pass_diagonal()
    prec = {"fp64": pm.PREC_FP64, "fp32ir": pm.PREC_FP32_IR, "tf32x3": pm.PREC_TF32X3_IR}[precision]
    P = pm.Problem(prob.n, prob.terms)
    res = P.solve(regs, V, opt=pm.options(precision=prec, indicator_N=16))
    ref = o.pmcimb(prob, regs, V, indicator_N=16)
    tops = [rec for rec in ref.records if rec.depth == 0]
    cand = np.array([bool(st & pm.RS_CANDIDATE) for st in res["status"]])
    assert list(cand) == [rec.candidate for rec in tops]
    for g, reg in enumerate(regs):
        a = (mu - reg.c) / reg.r
        I_exact = np.linalg.norm(1.0 / (1.0 - a ** 8)) / np.sqrt(len(mu))
        assert cand[g] == (I_exact > 0.1)
    assert not any(rec.split for rec in ref.records)
    assert res["stats"]["solves"] == 16 * len(regs) + 48 * int(cand.sum())
    inside = mu[(np.abs(mu.real) < 1.5) & (np.abs(mu.imag) < 1.5)]
    assert _match_lam(res["lam"], inside) <= LAM_TOL
    assert _match_lam(res["lam"], ref.lam) <= LAM_TOL
    P.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32ir"])
def test_two_pass_quadratic_matches_oracle(pm, precision):
    """n = 64 quadratic, N = 32, indicator on 8 nodes: the oracle's two-pass eigenvalues,
    with splitting (the spectrum covers the grid, so nearly every disk is a candidate and the
    schedule saves few solves here; the reuse itself is checked exactly above)."""
    W = w.quadratic_small()
    prec = {"fp64": pm.PREC_FP64, "fp32ir": pm.PREC_FP32_IR}[precision]
    P = pm.Problem(W.problem.n, W.problem.terms)
    two = P.solve(W.regions, W.V, opt=pm.options(precision=prec, indicator_N=8))
    one = P.solve(W.regions, W.V, opt=pm.options(precision=prec))
    ref = o.pmcimb(W.problem, W.regions, W.V, indicator_N=8)
    assert _match_lam(two["lam"], ref.lam) <= LAM_TOL
    assert _match_lam(two["lam"], one["lam"]) <= LAM_TOL
    assert two["stats"]["solves"] <= one["stats"]["solves"]
    P.close()


def test_two_pass_rejects_bad_indicator_rule(pm):
    W = w.quadratic_small()
    P = pm.Problem(W.problem.n, W.problem.terms)
    with pytest.raises(RuntimeError):
        P.solve(W.regions[:2], W.V, opt=pm.options(indicator_N=12))   # 32 is not a multiple of 12
    with pytest.raises(RuntimeError):
        P.solve(W.regions[:2], W.V, opt=pm.options(indicator_N=7))    # odd
    P.close()


# ---------------------------------------------------------------------------
# pmCIMa: levels of indicators with quadrisection, merge, sigma_min vectors
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "fp32ir"])
def test_pmcima_matches_oracle(pm, precision):
    """Prescribed spectrum (A = Q diag(mu) Q^-1): the GPU's merged values equal the oracle's
    (same decisions at every level, same merge) to rounding, are within tol_eps of the
    eigenvalues inside Omega, and come with unit vectors v with ||T(lambda) v|| = sigma_min."""
    mu = np.array([0.12 + 0.31j, -0.27 - 0.05j, 0.33 - 0.38j, 0.9 + 0.9j, -0.8 + 0.6j, 1.3 - 0.2j])
    prob, _ = w.similarity_linear(mu, seed=4)
    V = w.probe_block(np.random.default_rng(3), len(mu), 2)
    regs = w.grid_regions(-0.5, 0.5, -0.5, 0.5, 2, 2, 16)
    prec = {"fp64": pm.PREC_FP64, "fp32ir": pm.PREC_FP32_IR}[precision]
    P = pm.Problem(prob.n, prob.terms)
    res = P.pmcima(regs, V, tol_eps=1e-6, opt=pm.options(precision=prec))
    ref = o.pmcima(prob, regs, V, tol_eps=1e-6)
    assert len(res["lam"]) == len(ref.lam) == 3
    assert np.max(np.abs(res["lam"] - ref.lam)) <= 1e-12
    inside = mu[(np.abs(mu.real) < 0.5) & (np.abs(mu.imag) < 0.5)]
    assert _match_lam(res["lam"], inside) < 1e-6
    for i, lam in enumerate(res["lam"]):
        v = res["vecs"][:, i]
        T = o.assemble_T(prob, lam)
        assert abs(np.linalg.norm(v) - 1.0) < 1e-10
        assert np.linalg.norm(T @ v) == pytest.approx(res["sigma_min"][i], rel=1e-6)
        assert res["sigma_min"][i] == pytest.approx(ref.sigma[i], rel=1e-6)
    assert res["stats"]["solves"] == 16 * ref.regions
    P.close()


# ---------------------------------------------------------------------------
# Beyn's higher moments (block Hankel of 2K scaled moments)
# ---------------------------------------------------------------------------

def test_hankel_beyn_resolves_poles_without_split(pm):
    """10 poles in one disk, l = 3 probes: K = 1 must split the disk, K = 4 (K l = 12) returns
    all 10 from the disk itself, as the oracle does."""
    rng = np.random.default_rng(52)
    c, r, N = 0.0, 1.0, 64
    ain = rng.uniform(0.1, 0.6, 10) * np.exp(2j * np.pi * rng.random(10))
    aout = rng.uniform(1.5, 3.0, 5) * np.exp(2j * np.pi * rng.random(5))
    mu = c + r * np.concatenate([ain, aout])
    prob = w.diagonal_linear(mu)
    V = w.probe_block(rng, len(mu), 3)
    reg = [w.Region(c, r * np.sqrt(2.0), N)]      # the disk circumscribing the square of side 2
    P = pm.Problem(prob.n, prob.terms)
    k4 = P.solve(reg, V, opt=pm.options(beyn_K=4, tol_svd=1e-10))
    ref = o.pmcimb(prob, reg, V, tol_svd=1e-10, beyn_K=4)
    inside = mu[(np.abs(mu.real) < 1.0) & (np.abs(mu.imag) < 1.0)]
    assert k4["stats"]["splits"] == 0
    assert _match_lam(k4["lam"], inside) <= LAM_TOL
    assert _match_lam(k4["lam"], ref.lam) <= LAM_TOL
    k1 = P.solve(reg, V, opt=pm.options(tol_svd=1e-10))
    assert k1["stats"]["splits"] >= 1
    assert _match_lam(k1["lam"], inside) <= LAM_TOL
    P.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32ir"])
def test_hankel_quadratic_matches_oracle(pm, precision):
    """n = 64 quadratic (up to 31 eigenvalues per disk at l = 8): K = 2 halves the saturation
    of K = 1, so fewer disks split; eigenvalues equal the oracle's with the same K. Against
    K = 1 they agree to the quadrature's accuracy only: with fewer splits a value may come from
    a larger disk, where an eigenvalue near its circle carries a larger |a|^N error."""
    W = w.quadratic_small()
    prec = {"fp64": pm.PREC_FP64, "fp32ir": pm.PREC_FP32_IR}[precision]
    P = pm.Problem(W.problem.n, W.problem.terms)
    k2 = P.solve(W.regions, W.V, opt=pm.options(precision=prec, beyn_K=2))
    k1 = P.solve(W.regions, W.V, opt=pm.options(precision=prec))
    ref = o.pmcimb(W.problem, W.regions, W.V, beyn_K=2)
    assert _match_lam(k2["lam"], ref.lam) <= LAM_TOL
    assert _match_lam(k2["lam"], k1["lam"]) <= 1e-5
    assert k2["stats"]["splits"] < k1["stats"]["splits"]
    assert k2["stats"]["solves"] < k1["stats"]["solves"]
    P.close()


def test_hankel_rejects_too_many_columns(pm):
    W = w.quadratic_small()
    P = pm.Problem(W.problem.n, W.problem.terms)
    with pytest.raises(RuntimeError):
        P.solve(W.regions[:2], W.V, opt=pm.options(beyn_K=9))      # above 8
    with pytest.raises(RuntimeError):
        P.solve(W.regions[:2], np.hstack([W.V] * 3), opt=pm.options(beyn_K=3))   # K l = 72 > 64
    P.close()


def test_beyn_api_two_pass_and_hankel(pm):
    """pmcim_beyn runs Beyn on the given disks without the indicator gate; with the two-pass
    schedule only the split children are gated, on the coarse rule. The verified values equal
    those of the plain call; with beyn_K = 2 too, to the quadrature's accuracy."""
    W = w.quadratic_small()
    regs = W.regions[4:8]
    P = pm.Problem(W.problem.n, W.problem.terms)
    lam1, _, _, st1 = P.beyn(regs, W.V)
    lam2, _, _, st2 = P.beyn(regs, W.V, opt=pm.options(indicator_N=8))
    lam3, _, _, st3 = P.beyn(regs, W.V, opt=pm.options(indicator_N=8, beyn_K=2))
    acc = [o.verify(W.problem, lam)[1] for lam in (lam1, lam2, lam3)]
    assert _match_lam(lam2[acc[1]], lam1[acc[0]]) <= LAM_TOL
    assert _match_lam(lam3[acc[2]], lam1[acc[0]]) <= 1e-5
    P.close()


def test_paper_quadratic_two_pass_matches_oracle(pm):
    """The paper's quadratic experiment (n = 100, T_j uniform [0,1), 225 disks on [-0.5,0.5]^2)
    with the Appendix's schedule (indicator on 16 nodes, Beyn on 64, l = 10): the oracle's
    eigenvalues, all 34 in Omega by the companion pencil."""
    W = w.paper_quadratic()
    P = pm.Problem(W.problem.n, W.problem.terms)
    res = P.solve(W.regions, W.V, opt=pm.options(indicator_N=16))
    ref = o.pmcimb(W.problem, W.regions, W.V, indicator_N=16)
    assert len(ref.lam) == 34
    assert _match_lam(res["lam"], ref.lam) <= LAM_TOL
    P.close()


@pytest.mark.parametrize("form", MIXED_FORMS)
def test_mixed_residual_on_fp64_pipe(pm, form):
    """The precision forms with their refinement residuals on the FP64 pipe (option
    residual_fp64) instead of the tensor cores: the same eigenvalues as the oracle."""
    W = w.delay_large(n=64, l=8, N=32, nx=4, ny=12)
    P = pm.Problem(W.problem.n, W.problem.terms)
    res = P.solve(W.regions, W.V, opt=_mixed_opt(pm, form, residual_fp64=True))
    ref = o.pmcimb(W.problem, W.regions, W.V)
    assert _match_lam(res["lam"], ref.lam) <= LAM_TOL
    P.close()
