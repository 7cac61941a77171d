"""CPU checks of bench.py's own helpers that the default benchmark line uses (no GPU):
the Hankel-zero search of the scattering leg, the library-LU comparison (run here on
CPU tensors), and the eigenvalue matching."""
import numpy as np
import pytest

import workloads as w


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def test_hankel_zeros_match_the_pin_search(bench):
    from tests.test_bie_oracle import hankel_zeros_in
    omega = (0.2, 3.2, -3.2, -0.2)
    a = sorted((m, z) for m, z in bench._hankel_zeros(omega))
    b = sorted((m, z) for m, z in hankel_zeros_in(omega))
    assert [m for m, _ in a] == [m for m, _ in b] == [2, 3, 4, 4, 5, 5]
    for (_, za), (_, zb) in zip(sorted(a, key=lambda t: (t[0], t[1].real)), sorted(b, key=lambda t: (t[0], t[1].real))):
        assert abs(za - zb) < 1e-12


def test_library_lu_leg_on_cpu(bench):
    W = w.quadratic_small(n=32, l=4, N=16)
    out = bench.library_lu_leg(W, 5, device="cpu", reps=1)
    assert "error" not in out, out.get("error")
    assert out["complex128"]["max_rel_residual"] < 1e-12
    assert out["complex64"]["max_rel_residual"] < 1e-3
    assert out["complex128"]["solves_per_s"] > 0


def test_library_lu_leg_reports_errors(bench):
    W = w.quadratic_small(n=32, l=4, N=16)
    out = bench.library_lu_leg(W, 5, device="no-such-device", reps=1)
    assert "error" in out


def test_max_rel_diff(bench):
    a = np.array([1.0 + 1.0j, 2.0 - 0.5j])
    assert bench._max_rel_diff(a, a[::-1]) == 0.0
    assert bench._max_rel_diff(a, a[:1]) is None
    assert bench._max_rel_diff(a, a * (1 + 1e-12)) <= 3e-12
