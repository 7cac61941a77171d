"""The scattering-pole problem of Sec. 4.2 through the GPU path, against the oracle.

T(kappa) = (I + K_n(kappa)) / 2 with K_n the Nystrom matrix of the double-layer
operator on a closed curve (Kress's rule). The library forms every entry on
the device from its own J_1 and H_1^(1) of complex argument; the oracle uses
SciPy's (AMOS) Bessel functions.

* Moments (C0, C1, P f) of disks on the unit circle at n = 64 (FP64 node
  kernel) and n = 32 (one-warp small kernel), on an ellipse (a curve whose
  matrix is not circulant), and on a circle of radius 3, where kappa r runs to
  27 and the entries come from Hankel's expansion, within the LU's backward-
  error bound widened by the entries' own accuracy.
* All 100 disks of the paper's region at n = 256 against the stored oracle run
  (tests/golden/make_oracle_golden.py scattering): every indicator decision, the
  indicator values, and the eigenvalue set within 1e-10, which also equals the
  zeros of the Hankel functions H_m^(1) in Omega (each zero of order m >= 1
  twice: the modes m and -m).
* sigma_min (k_verify_fp64) and the eigenvector certificate (k_certify) at those
  poles (to rounding) and off them (sigma_min as the upper bound inverse iteration
  reaches in its 30 steps), against the oracle.
* The precision forms (FP32 LU on the FMA pipes or with tensor-core trailing
  updates, FP64 residuals from the FP64 matrix) on a circle and an ellipse, and on
  all 100 disks. PREC_AUTO runs the FP32 LU with FP64 refinement; the tensor-core
  residual call is refused.
"""
import json
import os

import numpy as np
import pytest

import oracle as o
import workloads as w
from tests.test_bie_oracle import hankel_zeros_in
from tests.test_gpu_parity import LAM_TOL, _match_lam, _moment_bound

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EINVAL = -1  # PMCIM_EINVAL


@pytest.fixture(scope="module")
def pm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2312_13117_gb300 import build, pmcim
    build.build()
    pmcim.load()
    return pmcim


def _problem(curve):
    n = curve.samples.shape[1]
    return w.Problem(n, [(0.5 + 0j, w.MONOMIAL, 0, 0.0), (curve, w.HELMHOLTZ_DLP, 0, 0.0)])


def _check(pm, prob, regions, V, c=4.0):
    P = pm.Problem(prob.n, prob.terms)
    C0, C1, ph, pa = P.moments(regions, V, opt=pm.options(precision=pm.PREC_FP64))
    for g, reg in enumerate(regions):
        m = o.moments(prob, reg.c, reg.r, reg.N, V)
        b0, b1, bh = _moment_bound(prob, reg, V, c=c)
        assert np.linalg.norm(C0[g] - m.C0) <= b0, (g, np.linalg.norm(C0[g] - m.C0), b0)
        assert np.linalg.norm(C1[g] - m.C1) <= b1, (g, np.linalg.norm(C1[g] - m.C1), b1)
        assert np.linalg.norm(ph[g] - m.pf_half) <= bh, g
    P.close()


DISKS = [w.Region(0.5 - 1.25j, 0.2121, 64),   # holds the zero of H_2 near 0.429 - 1.281i
         w.Region(2.15 - 1.85j, 0.2121, 64),  # holds a zero of H_4
         w.Region(1.85 - 0.35j, 0.2121, 48),  # no pole
         w.Region(0.35 - 3.05j, 0.2121, 32)]  # corner of Omega


def test_moments_unit_circle_n64(pm):
    prob = _problem(w.circle_curve(64))
    V = w.probe_block(np.random.default_rng(1), 64, 8)
    _check(pm, prob, DISKS, V)


def test_moments_unit_circle_small_kernel_n32(pm):
    prob = _problem(w.circle_curve(32))
    V = w.probe_block(np.random.default_rng(2), 32, 6)
    _check(pm, prob, DISKS[:3], V)


def test_moments_ellipse_n80(pm):
    prob = _problem(w.ellipse_curve(80, 1.4, 0.7))
    V = w.probe_block(np.random.default_rng(3), 80, 4)
    _check(pm, prob, [w.Region(1.2 - 0.9j, 0.3, 32), w.Region(2.6 - 2.1j, 0.25, 32)], V)


def test_moments_large_argument_radius3(pm):
    """kappa r up to ~27 (Hankel's expansion); the entries' relative accuracy is ~1e-11 near
    |kappa r| = 13, so the LU bound is widened by that accuracy over its 4 n u."""
    prob = _problem(w.circle_curve(96, 3.0))
    V = w.probe_block(np.random.default_rng(4), 96, 4)
    _check(pm, prob, [w.Region(2.9 - 0.5j, 0.2, 32), w.Region(1.6 - 2.4j, 0.2, 32)], V, c=4.0 + 1e-11 / 2.0 ** -53 / 96)


@pytest.fixture(scope="module")
def scattering():
    return w.scattering_disk()


def test_all_disks_n256_against_oracle_and_hankel_zeros(pm, scattering):
    W = scattering
    with open(os.path.join(GOLDEN, "scattering_disk_n256_oracle.json")) as fh:
        run = json.load(fh)["runs"][repr(1e-6)]
    P = pm.Problem(W.problem.n, W.problem.terms)
    res = P.solve(W.regions, W.V, want_vecs=True, opt=pm.options(precision=pm.PREC_AUTO))
    top = {rec[0]: rec for rec in run["records"] if rec[4] == 0}
    for g in range(len(W.regions)):
        I, cand = top[g][5], top[g][6]
        assert bool(res["status"][g] & pm.RS_CANDIDATE) == cand, (g, I, res["ind"][g])
        if I > 1e-3:
            assert res["ind"][g] == pytest.approx(I, rel=1e-6), g
    lam_o = np.array([complex(a, b) for (a, b, _, _) in run["lam"]])
    assert len(res["lam"]) == len(lam_o) == 12
    assert _match_lam(res["lam"], lam_o) <= LAM_TOL
    zeros = [z for m, z in hankel_zeros_in(W.omega) for _ in range(2 if m else 1)]
    assert _match_lam(res["lam"], np.array(zeros)) <= LAM_TOL
    assert res["stats"]["unverified"] == 0 and res["stats"]["tuned_mixed"] == 1  # AUTO: FP32 LU + refinement
    # eigenvectors: unit, ||T(lambda) v|| at rounding level
    for i, lam in enumerate(res["lam"]):
        v = res["vecs"][:, i]
        assert abs(np.linalg.norm(v) - 1.0) < 1e-10
        assert np.linalg.norm(o.assemble_T(W.problem, lam) @ v) < 1e-9
    P.close()


def test_verify_and_certify(pm):
    prob = _problem(w.circle_curve(64))
    zeros = [z for _, z in hankel_zeros_in((0.2, 3.2, -3.2, -0.2))]
    rng = np.random.default_rng(5)
    lam = np.array(zeros + list(1.5 - 1.5j + rng.standard_normal(3) + 1j * rng.standard_normal(3)))
    P = pm.Problem(prob.n, prob.terms)
    sig, acc = P.verify(lam)
    for i, z in enumerate(lam):
        s_ref, fro = o.sigma_min(prob, z)
        if i < len(zeros):
            assert abs(sig[i] - s_ref) <= 1e-13 * fro, (i, sig[i], s_ref)
        else:
            # Off the spectrum the inverse iteration on T^H T (30 steps at most) converges slowly:
            # on the circle the singular values come in pairs (modes m and -m) and the next pair
            # can lie within a few per cent. Its Rayleigh quotient is an upper bound of sigma_min.
            assert s_ref * (1.0 - 1e-12) <= sig[i] <= s_ref * (1.0 + 1e-3), (i, sig[i], s_ref)
    assert np.array_equal(acc, o.verify(prob, lam)[1])
    assert acc[:len(zeros)].all() and not acc[len(zeros):].any()
    # the right singular vector of sigma_min: the certificate ||T v|| / ||v|| equals sigma_min
    vecs = []
    for z in lam:
        _, s, vh = np.linalg.svd(o.assemble_T(prob, z))
        vecs.append(vh[-1].conj())
    vecs = np.array(vecs).T
    cert, ok = P.certify(lam, vecs)
    for i, z in enumerate(lam):
        s_ref, _ = o.sigma_min(prob, z)
        assert cert[i] == pytest.approx(s_ref, rel=1e-6, abs=1e-13), i
    P.close()


FORMS = ["fp32ir", "tf32x3", "bf16x3"]


def _form(pm, form):
    return {"fp32ir": pm.PREC_FP32_IR, "tf32x3": pm.PREC_TF32X3_IR, "bf16x3": pm.PREC_BF16X3_IR}[form]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("curve", ["circle", "ellipse"])
def test_precision_form_moments(pm, form, curve):
    """The precision forms on a boundary-integral problem: the factor group forms T(z_j) in FP64 (a
    circulant one from its first column), the FP32 LU works on its rounding, and the refinement
    residuals multiply the FP64 matrix. Refined solutions: |dX| <= 1e-9 |X| per node."""
    n = 96 if curve == "circle" else 80
    prob = _problem(w.circle_curve(n) if curve == "circle" else w.ellipse_curve(n, 1.4, 0.7))
    V = w.probe_block(np.random.default_rng(21), n, 6)
    regs = DISKS[:3] if curve == "circle" else [w.Region(1.2 - 0.9j, 0.3, 32), w.Region(2.6 - 2.1j, 0.25, 32)]
    P = pm.Problem(prob.n, prob.terms)
    C0, C1, _, _ = P.moments(regs, V, opt=pm.options(precision=_form(pm, form)))
    for g, reg in enumerate(regs):
        m = o.moments(prob, reg.c, reg.r, reg.N, V)
        z, wts = o.nodes_weights(reg.c, reg.r, reg.N)
        X = o.solve_nodes(prob, z, V)
        scale = sum(abs(wts[j]) * np.linalg.norm(X[j]) for j in range(reg.N))
        b0, b1, _ = _moment_bound(prob, reg, V)
        assert np.linalg.norm(C0[g] - m.C0) <= b0 + 1e-9 * scale, g
        assert np.linalg.norm(C1[g] - m.C1) <= b1 + 1e-9 * scale * (abs(reg.c) + reg.r), g
    P.close()


@pytest.mark.parametrize("form", FORMS)
def test_precision_form_all_disks_n256(pm, scattering, form):
    """All 100 disks of the n = 256 workload in each precision form: every decision and the eigenvalue
    set equal the stored oracle run's."""
    W = scattering
    with open(os.path.join(GOLDEN, "scattering_disk_n256_oracle.json")) as fh:
        run = json.load(fh)["runs"][repr(1e-6)]
    P = pm.Problem(W.problem.n, W.problem.terms)
    res = P.solve(W.regions, W.V, want_vecs=False, opt=pm.options(precision=_form(pm, form)))
    top = {rec[0]: rec for rec in run["records"] if rec[4] == 0}
    for g in range(len(W.regions)):
        assert bool(res["status"][g] & pm.RS_CANDIDATE) == top[g][6], g
    lam_o = np.array([complex(a, b) for (a, b, _, _) in run["lam"]])
    assert _match_lam(res["lam"], lam_o) <= LAM_TOL
    assert res["stats"]["unverified"] == 0
    P.close()


def test_tensor_core_residual_refused(pm):
    """pmcim_residual multiplies coefficient digits on the tensor cores: a boundary-integral term has
    none, so the call is refused."""
    prob = _problem(w.circle_curve(32))
    V = w.probe_block(np.random.default_rng(6), 32, 4)
    P = pm.Problem(prob.n, prob.terms)
    with pytest.raises(pm.PmcimError) as e:
        P.residual(np.array([1.0 - 1.0j]), V, np.zeros((1, 32, 4), np.complex128))
    assert e.value.code == EINVAL
    P.close()


def test_bad_curves_refused(pm):
    for curve in (w.circle_curve(31), w.circle_curve(2)):
        with pytest.raises(pm.PmcimError) as e:
            pm.Problem(curve.samples.shape[1], _problem(curve).terms)
        assert e.value.code == EINVAL
    two = _problem(w.circle_curve(16))
    two.terms.append((w.circle_curve(16), w.HELMHOLTZ_DLP, 0, 0.0))
    with pytest.raises(pm.PmcimError) as e:
        pm.Problem(16, two.terms)
    assert e.value.code == EINVAL


def test_batch_mixes_coefficient_and_boundary_problems(pm):
    """One batched launch with a quadratic problem and two boundary-integral problems (the kernel
    instantiation with the term serves all of them): each problem's eigenvalues equal the oracle's."""
    qd = w.quadratic_small(seed=11, n=40, l=6, N=32)
    sc = w.scattering_disk(n=48, l=4)
    el = _problem(w.ellipse_curve(48, 1.2, 0.9))
    Vel = w.probe_block(np.random.default_rng(12), 48, 4)
    batch = [(qd.problem, qd.regions[5:9], qd.V),
             (sc.problem, [sc.regions[g] for g in (6, 35, 50)], sc.V),
             (el, [g for i, g in enumerate(w.grid_regions(0.2, 3.2, -3.2, -0.2, 10, 10, 32)) if i in (6, 35)],
              Vel)]  # disks holding two resonances each: the ellipse splits the circle's double poles
    handles = [pm.Problem(p.n, p.terms) for (p, _, _) in batch]
    res = pm.batch_solve(handles, [r for (_, r, _) in batch], [V for (_, _, V) in batch],
                         opt=pm.options(precision=pm.PREC_AUTO))
    st = res["stats"]
    assert st["tuned_mixed"] >= 2  # the two boundary-integral problems
    for q, (prob, regs, V) in enumerate(batch):
        ref = o.pmcimb(prob, regs, V)
        got = res["lam"][res["problem_of"] == q]
        assert _match_lam(got, ref.lam) <= LAM_TOL, q
    assert (res["problem_of"] == 1).sum() == 4 and (res["problem_of"] == 2).sum() == 4
    for h in handles:
        h.close()


def test_two_pass_and_pmcima(pm):
    """The two-pass schedule (indicator on 16 of the 64 nodes) returns the one-pass eigenvalues; pmCIMa
    (tol_eps = 1e-6) returns the oracle's merged centres to rounding and each pole within tol_eps."""
    W = w.scattering_disk(n=48, l=4)
    regs = [W.regions[g] for g in (5, 6, 7, 35, 36, 50)]
    P = pm.Problem(W.problem.n, W.problem.terms)
    one = P.solve(regs, W.V)
    two = P.solve(regs, W.V, opt=pm.options(indicator_N=16))
    assert _match_lam(two["lam"], one["lam"]) <= LAM_TOL
    assert two["stats"]["solves"] < one["stats"]["solves"]
    regs16 = [w.Region(g.c, g.r, 16) for g in regs]
    res = P.pmcima(regs16, W.V, tol_eps=1e-6)
    ref = o.pmcima(W.problem, regs16, W.V, tol_eps=1e-6)
    assert len(res["lam"]) == len(ref.lam) == 2
    assert np.max(np.abs(res["lam"] - ref.lam)) <= 1e-12
    zeros = np.array([z for _, z in hankel_zeros_in(W.omega)])
    for lam in res["lam"]:
        assert np.min(np.abs(zeros - lam)) <= 1e-6
    P.close()
