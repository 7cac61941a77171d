"""Certificates of approximate eigenpairs (pmCIMb step 3) through pmcim_certify.

sigma_min(T(lambda)) <= ||T(lambda) y|| / ||y|| for every y != 0, so every
certificate must be an upper bound of the oracle's sigma_min (up to the FP64
rounding of the two evaluations). At an eigenvalue, the bordered inverse step
must bring the certificate far below the acceptance threshold from a start
vector that is no eigenvector at all (seeded random). An inverse step through
an FP32 factorisation alone stops at the factorisation's backward error, which
at the n = 1024 delay workload's eigenvalues lies above the acceptance
threshold; the bordered step gets below it through its FP64-accurate residuals.

The step is y = T(lambda)^-H c with the certificate ||T^H y|| / ||y||
(sigma_min(T^H) = sigma_min(T)). From a start c close to the right singular
vector of sigma_min (Beyn's eigenvector in pmcim_solve) this comes within a
few digits of sigma_min; the test at the delay workload's largest-sigma_min
eigenvalues checks exactly that, with starts made by the oracle's own Beyn
step.

Cases: a prescribed spectrum (T(z) = A - z I, A = Q diag(mu) Q^-1) at n = 200
(precision-form node kernel) and n = 20 (warp-per-node FP64 kernel); the
oracle's eigenvalues of the n = 1024 delay workload (stored by
tests/golden/make_oracle_golden.py); values off the spectrum, which must stay
unaccepted with certificates above the oracle's sigma_min.
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as w
from oracle import pmcim_ref as ref

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL_VERIFY = 1e-6


@pytest.fixture(scope="module")
def pm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2312_13117_gb300 import build, pmcim
    build.build()
    pmcim.load()
    return pmcim


def _scale(problem, lam):
    """max(1, ||T(lambda)||_F / sqrt(n)), the factor of the acceptance threshold (step 3)."""
    return max(1.0, np.linalg.norm(ref.assemble_T(problem, lam)) / math.sqrt(problem.n))


def _random_starts(n, m, seed):
    rng = np.random.default_rng(seed)
    return w.complex_gaussian(rng, (n, m))


def _spectrum(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-2.0, 2.0, n) + 1j * rng.uniform(-2.0, 2.0, n)


@pytest.mark.parametrize("n", [200, 20])
def test_certify_prescribed_spectrum(pm, n):
    mu = _spectrum(n, seed=n)
    prob, _ = w.similarity_linear(mu, seed=n + 1)
    pick = np.arange(0, n, max(1, n // 16))
    lam = mu[pick]
    starts = _random_starts(n, len(lam), seed=7)
    h = pm.Problem(prob.n, prob.terms)
    try:
        cert, acc = h.certify(lam, starts, opt=pm.options(precision=pm.PREC_TF32X3_IR))
    finally:
        h.close()
    sig = np.array([ref.sigma_min(prob, z)[0] for z in lam])
    for i, z in enumerate(lam):
        sc = _scale(prob, z)
        # accepted, far below the threshold: a random start is no eigenvector, so
        # only the bordered step can give this
        assert acc[i], (z, cert[i])
        assert cert[i] <= 1e-9 * sc, (z, cert[i])
        # an upper bound of sigma_min, up to the rounding of both evaluations
        assert cert[i] >= sig[i] - 1e-13 * sc, (z, cert[i], sig[i])


def test_certify_start_eigenvector_needs_no_step(pm):
    """With an exact eigenvector as start, the first certificate ||T v|| / ||v|| accepts."""
    n = 200
    mu = _spectrum(n, seed=3)
    prob, Q = w.similarity_linear(mu, seed=4)
    lam = mu[:8]
    h = pm.Problem(prob.n, prob.terms)
    try:
        cert, acc = h.certify(lam, Q[:, :8], opt=pm.options(precision=pm.PREC_TF32X3_IR))
    finally:
        h.close()
    for i, z in enumerate(lam):
        v = Q[:, i] / np.linalg.norm(Q[:, i])
        direct = np.linalg.norm(ref.assemble_T(prob, z) @ v)
        assert acc[i]
        assert abs(cert[i] - direct) <= 1e-12 * _scale(prob, z) + 1e-6 * direct, (cert[i], direct)


def test_certify_off_spectrum_stays_above_sigma_min(pm):
    """Between eigenvalues T(lambda) is far from singular: no certificate may go below
    sigma_min, so none of these values is accepted."""
    n = 200
    mu = _spectrum(n, seed=5)
    prob, _ = w.similarity_linear(mu, seed=6)
    rng = np.random.default_rng(8)
    lam = rng.uniform(-2.5, 2.5, 8) + 1j * rng.uniform(-2.5, 2.5, 8)
    sig = np.array([ref.sigma_min(prob, z)[0] for z in lam])
    keep = sig > 1e-3  # away from every eigenvalue
    lam, sig = lam[keep], sig[keep]
    assert len(lam) >= 4
    h = pm.Problem(prob.n, prob.terms)
    try:
        cert, acc = h.certify(lam, _random_starts(n, len(lam), seed=9), opt=pm.options(precision=pm.PREC_FP32_IR))
    finally:
        h.close()
    for i, z in enumerate(lam):
        assert not acc[i], (z, cert[i], sig[i])
        assert cert[i] >= sig[i] * (1.0 - 1e-9), (z, cert[i], sig[i])


def test_certify_delay_n1024_oracle_eigenvalues(pm):
    """24 of the oracle's eigenvalues of the n = 1024 delay workload (spread over
    those whose sigma_min is at most 1e-9, half of them), random starts: every one
    accepted, with a certificate not below the oracle's sigma_min. A random start's
    inverse step overestimates sigma_min by about sqrt(n) (up to several hundred
    where a second singular value is close), which stays below the threshold
    (about 5e-6 here) for these values."""
    with open(os.path.join(GOLDEN, "delay_n1024_oracle.json")) as fh:
        gold = json.load(fh)
    lam_rec = [x for x in gold["runs"][repr(1e-6)]["lam"] if x[2] <= 1e-9]
    pick = np.linspace(0, len(lam_rec) - 1, 24).astype(int)
    lam = np.array([complex(lam_rec[k][0], lam_rec[k][1]) for k in pick])
    sig = np.array([lam_rec[k][2] for k in pick])
    W = w.delay_large()
    prob = W.problem
    h = pm.Problem(prob.n, prob.terms)
    try:
        cert, acc = h.certify(lam, _random_starts(prob.n, len(lam), seed=11),
                              opt=pm.options(precision=pm.PREC_TF32X3_IR))
    finally:
        h.close()
    for i, z in enumerate(lam):
        sc = _scale(prob, z)
        assert acc[i], (z, cert[i])
        assert cert[i] <= TOL_VERIFY * sc, (z, cert[i])
        assert cert[i] >= sig[i] - 1e-12 * sc, (z, cert[i], sig[i])


def test_certify_near_sigma_min_from_beyn_vectors(pm):
    """The six eigenvalues of the n = 1024 delay workload with the largest sigma_min
    (1.2e-6 to 2.3e-6, within a factor of 10 of the threshold), each with the
    eigenvector of the oracle's Beyn step on its disk as start: the first
    certificate ||T v|| rejects them all (1.7e-5 to 5.4e-5), a step with T itself
    would too; the step with T^H must give sigma_min to 1e-6 relative and accept."""
    with open(os.path.join(GOLDEN, "delay_n1024_oracle.json")) as fh:
        gold = json.load(fh)
    lam_rec = sorted(gold["runs"][repr(1e-6)]["lam"], key=lambda x: -x[2])[:6]
    W = w.delay_large()
    prob = W.problem
    lam, sig, starts, beyn = [], [], [], {}
    for re_, im_, s_, disk in lam_rec:
        z = complex(re_, im_)
        if disk not in beyn:
            reg = W.regions[disk]
            m = ref.moments(prob, reg.c, reg.r, reg.N, W.V)
            beyn[disk] = ref.beyn_extract(m.C0, m.C1, 1e-6)
        br = beyn[disk]
        j = int(np.argmin(np.abs(np.asarray(br.lam) - z)))
        assert abs(br.lam[j] - z) <= 1e-10 * max(1.0, abs(z))
        lam.append(z)
        sig.append(s_)
        starts.append(np.asarray(br.vecs)[:, j])
    lam, sig = np.array(lam), np.array(sig)
    h = pm.Problem(prob.n, prob.terms)
    try:
        cert, acc = h.certify(lam, np.stack(starts, axis=1), opt=pm.options(precision=pm.PREC_TF32X3_IR))
    finally:
        h.close()
    for i, z in enumerate(lam):
        assert acc[i], (z, cert[i], sig[i])
        # the exact step gives sigma_min to about 2e-9 relative here (numpy, FP64)
        assert sig[i] - 1e-12 <= cert[i] <= sig[i] * (1.0 + 1e-6), (z, cert[i], sig[i])


def test_certificate_threshold_uses_frobenius_norm(pm):
    """The acceptance threshold tol_verify * max(1, ||T(lambda)||_F / sqrt(n)), with the
    Frobenius norm formed from the coefficients' Gram data (two dense terms and an
    identity term here): with the right singular vector of sigma_min as start, the
    certificate is sigma_min itself, and a tol_verify 1e-7 above or below
    sigma_min / max(1, ||T||_F / sqrt(n)) (numpy) must accept or leave the value."""
    W = w.delay_large(seed=3, n=200, l=4, N=16, nx=1, ny=3)
    prob = W.problem
    lam = np.array([0.3 + 0.2j, -1.1 + 2.7j, -2.4 - 4.1j])
    vecs, thr = [], []
    for z in lam:
        T = ref.assemble_T(prob, z)
        _, sv, vh = np.linalg.svd(T)
        vecs.append(vh[-1].conj())
        thr.append(sv[-1] / max(1.0, np.linalg.norm(T) / math.sqrt(prob.n)))
    vecs, thr = np.stack(vecs, axis=1), np.array(thr)
    h = pm.Problem(prob.n, prob.terms)
    try:
        for i in range(len(lam)):
            hi = pm.options(precision=pm.PREC_TF32X3_IR, tol_verify=thr[i] * (1 + 1e-7))
            lo = pm.options(precision=pm.PREC_TF32X3_IR, tol_verify=thr[i] * (1 - 1e-7))
            _, acc_hi = h.certify(lam[i:i + 1], vecs[:, i:i + 1], opt=hi)
            _, acc_lo = h.certify(lam[i:i + 1], vecs[:, i:i + 1], opt=lo)
            assert acc_hi[0] and not acc_lo[0], (lam[i], thr[i])
    finally:
        h.close()
