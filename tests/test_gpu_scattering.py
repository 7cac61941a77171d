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
* The precision forms and the tensor-core residual are refused with EINVAL;
  PREC_AUTO runs FP64.
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
    assert res["stats"]["unverified"] == 0 and res["stats"]["tuned_fp64"] == 1
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


def test_precision_forms_refused(pm):
    prob = _problem(w.circle_curve(32))
    V = w.probe_block(np.random.default_rng(6), 32, 4)
    P = pm.Problem(prob.n, prob.terms)
    for prec in (pm.PREC_FP32_IR, pm.PREC_TF32X3_IR, pm.PREC_BF16X3_IR):
        with pytest.raises(pm.PmcimError) as e:
            P.solve(DISKS[:1], V, opt=pm.options(precision=prec))
        assert e.value.code == EINVAL
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
