"""Pins of the screen network's oracle: gradient by finite differences, BF16
rounding against known bit patterns."""
import numpy as np

from oracle import screen_ref as sr


def test_bf16_rounding_known_values():
    x = np.array([1.0, 1.00390625, 1.005859375, 3.140625, -2.75, 65504.0], dtype=np.float32)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: ties go to the even mantissa (1.0)
    # 1 + 1.5 * 2^-8 rounds up to 1 + 2^-7
    exp = np.array([1.0, 1.0, 1.0078125, 3.140625, -2.75, 65536.0], dtype=np.float32)
    assert np.array_equal(sr.bf16_round(x), exp)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = sr.bf16_round(sr.init_params(rng)).astype(np.float64)  # on the BF16 grid, so rounding is identity
    X = rng.standard_normal((40, 3))
    y = (rng.random(40) < 0.3).astype(np.float64)
    # evaluate the FP64 functions directly on the unrounded FP64 parameters for the FD check
    def f(q):
        W1, b1, W2, b2, W3, b3 = sr.unpack(q)
        z1 = X @ W1.T + b1
        h1 = np.maximum(z1, 0)
        z2 = h1 @ W2.T + b2
        h2 = np.maximum(z2, 0)
        o = h2 @ W3 + b3
        wgt = np.where(y > 0, 3.0, 1.0)
        return np.mean(wgt * (np.logaddexp(0, o) - y * o))
    _, g = sr.loss_and_grad(p.astype(np.float32), X, y, 3.0)
    idx = rng.choice(sr.NPARAM, 60, replace=False)
    for i in idx:
        e = np.zeros(sr.NPARAM)
        e[i] = 1e-6
        fd = (f(p + e) - f(p - e)) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 + 1e-4 * abs(g[i]), (i, fd, g[i])
    assert sr.NPARAM == 4481
