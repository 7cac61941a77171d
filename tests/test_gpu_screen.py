"""Learned screen on the GPU: its training kernels against the NumPy oracle,
its features against the oracle's indicators, and its recall."""
import math

import numpy as np
import pytest

import oracle as o
import workloads as w
from oracle import screen_ref as sr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2312_13117_gb300 import build, pmcim
    build.build()
    pmcim.load()
    return pmcim


def test_gradient_and_forward_match_oracle(pm):
    rng = np.random.default_rng(4)
    params = sr.init_params(rng)
    X = (rng.standard_normal((500, 3)) * 2.0).astype(np.float32)
    y = (rng.random(500) < 0.3).astype(np.uint8)
    g, loss = pm.screen_gradient(X, y, params, pos_weight=4.0)
    loss_ref, g_ref = sr.loss_and_grad(params, X, y, 4.0)
    assert abs(loss - loss_ref) <= 1e-5 * abs(loss_ref)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    p = pm.screen_apply(X, params)
    assert np.max(np.abs(p - sr.probability(params, X))) <= 1e-5


def test_features_match_oracle_indicators(pm):
    W = w.quadratic_small(seed=5, n=24, l=1, N=64)
    regs = W.regions[:6]
    P = pm.Problem(W.problem.n, W.problem.terms)
    ind3, feats = P.screen_features(regs, W.V)
    for g, reg in enumerate(regs):
        for q, M in enumerate((8, 16, 64)):
            m = o.moments(W.problem, reg.c, reg.r, M, W.V)
            ref = o.indicator_value(m.pf_N, m.pf_half, m.pf_abs)
            if np.linalg.norm(m.pf_N) > 1e-6 * np.linalg.norm(m.pf_abs):
                assert ind3[g, q] == pytest.approx(ref, rel=1e-6), (g, M)
            if abs(ref - 0.1) > 1e-6:
                assert (ind3[g, q] > 0.1) == (ref > 0.1), (g, M)
        assert feats[g, 2] == pytest.approx(math.log10(reg.r), rel=1e-6)
    P.close()


def _traces(pm, seeds):
    F, Y = [], []
    for prob, regs, V in w.screen_trace_problems(seeds):
        P = pm.Problem(prob.n, prob.terms)
        ind3, feats = P.screen_features(regs, V)
        F.append(feats)
        Y.append(ind3[:, 2] > 0.1)          # label: the full rule's decision (step 1.c)
        P.close()
    return np.concatenate(F), np.concatenate(Y).astype(np.uint8)


def test_training_reaches_full_recall_on_held_out_traces(pm):
    F, Y = _traces(pm, range(0, 60))
    Ft, Yt = _traces(pm, range(1000, 1020))
    assert 0.1 < Y.mean() < 0.9
    p0 = sr.init_params(np.random.default_rng(0))
    params, loss = pm.screen_train(F, Y, p0, epochs=60, batch=256, lr=3e-3, pos_weight=8.0)
    assert loss[-1] < 0.6 * loss[0]
    prob = pm.screen_apply(F, params)
    thr = 0.5 * float(prob[Y == 1].min())           # calibrated: every training positive passes with margin
    pt = pm.screen_apply(Ft, params)
    recall = np.mean(pt[Yt == 1] >= thr)
    skipped = np.mean(pt < thr)
    assert recall == 1.0
    assert skipped > 0.2


def test_screened_solve_keeps_every_eigenvalue(pm):
    F, Y = _traces(pm, range(0, 60))
    params, _ = pm.screen_train(F, Y, sr.init_params(np.random.default_rng(0)), epochs=60, batch=256, lr=3e-3,
                                pos_weight=8.0)
    thr = 0.5 * float(pm.screen_apply(F, params)[Y == 1].min())
    W = w.quadratic_small(seed=9, n=24, l=8, N=64)
    regs = w.grid_regions(-3, 3, -3, 3, 8, 8, 64)
    P = pm.Problem(W.problem.n, W.problem.terms)
    plain = P.solve(regs, W.V)
    scr = P.solve(regs, W.V, opt=pm.options(screen_params=params, screen_threshold=thr))
    assert scr["stats"]["screened_out"] > 0
    assert scr["stats"]["screen_solves"] == 16 * len(regs)
    # what the network gains: the coarse one-column pass plus the full rule on the disks it keeps
    # costs fewer node solves than the full rule on every disk
    assert scr["stats"]["solves"] + scr["stats"]["screen_solves"] < plain["stats"]["solves"]
    got, exp = np.sort_complex(scr["lam"]), np.sort_complex(plain["lam"])
    assert len(got) == len(exp)
    assert np.max(np.abs(got - exp)) <= 1e-12 * max(1.0, np.max(np.abs(exp)))
    P.close()
