"""The precision-form node kernel's bounded waits, made to run out on purpose.

Every device wait of the kernel has a limit in SM clock cycles. These tests set
the limits to a few cycles through pmcim_debug_wait_limits, so that the waits
give up long before the work they wait for is done, and check what the
library promises then: a tensor-core wait that runs out leaves the node's
solution FP64-accurate (the LU is finished on the FMA pipes and refined, or the
node is solved again in FP64), and a hand-off wait between the kernel's two
thread groups that runs out ends the kernel and the call with PMCIM_ETIMEOUT,
after which the handle works normally. Nothing here faults or hangs the GPU:
each wait returns on its own, and the final wait for a tensor-core commit in
flight before the kernel frees its tensor memory keeps its default limit.
"""
import numpy as np
import pytest

import oracle as o
import workloads as w
from tests.test_gpu_parity import LAM_TOL, _match_lam

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2312_13117_gb300 import build, pmcim
    build.build()
    pmcim.load()
    yield pmcim
    pmcim.debug_wait_limits(0, 0)


def test_tensor_core_wait_timeout_keeps_fp64_accuracy(pm):
    """A 16-cycle limit on each tensor-core commit wait: the waits run out, the nodes are
    flagged (stats.tc_timeouts), and the eigenvalues still match the FP64 oracle."""
    W = w.delay_large(n=96, l=8, N=32, nx=4, ny=12)
    regs = W.regions[:12]
    P = pm.Problem(W.problem.n, W.problem.terms)
    try:
        pm.debug_wait_limits(16, 0)
        res = P.solve(regs, W.V, opt=pm.options(precision=pm.PREC_TF32X3_IR))
    finally:
        pm.debug_wait_limits(0, 0)
    assert res["stats"]["tc_timeouts"] > 0
    ref = o.pmcimb(W.problem, regs, W.V)
    assert len(ref.lam) > 0
    assert _match_lam(res["lam"], ref.lam) <= LAM_TOL
    # with the default limit the same call has no timeout and the same eigenvalues
    res2 = P.solve(regs, W.V, opt=pm.options(precision=pm.PREC_TF32X3_IR))
    assert res2["stats"]["tc_timeouts"] == 0
    assert _match_lam(res2["lam"], ref.lam) <= LAM_TOL
    P.close()


@pytest.mark.parametrize("form", ["fp32ir", "tf32x3"])
def test_handoff_wait_timeout_returns_etimeout(pm, form):
    """A 64-cycle limit on the waits between the factor and refine groups: the refine
    group gives up before the first node is factored, both groups end, and the call
    returns PMCIM_ETIMEOUT. With the default limit the next call on the same handle
    returns the oracle's moments."""
    prec = {"fp32ir": pm.PREC_FP32_IR, "tf32x3": pm.PREC_TF32X3_IR}[form]
    W = w.quadratic_small(seed=4, n=80, l=4, N=16)
    regs = W.regions[:3]
    P = pm.Problem(W.problem.n, W.problem.terms)
    try:
        pm.debug_wait_limits(0, 64)
        with pytest.raises(pm.PmcimError) as e:
            P.moments(regs, W.V, opt=pm.options(precision=prec))
        assert e.value.code == -4   # PMCIM_ETIMEOUT
    finally:
        pm.debug_wait_limits(0, 0)
    C0, _, _, _ = P.moments(regs, W.V, opt=pm.options(precision=prec))
    for g, reg in enumerate(regs):
        m = o.moments(W.problem, reg.c, reg.r, reg.N, W.V)
        assert np.linalg.norm(C0[g] - m.C0) <= 1e-9 * np.linalg.norm(m.C0)
    P.close()
