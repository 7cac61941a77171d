"""CPU checks of the device library's boundary-integral arithmetic (bie.cuh),
compiled for the host by the test harness tests/bie_host.cpp.

* J_1 and H_1^(1) of complex argument against SciPy's (AMOS) values, over
  |w| from 1e-3 to 40 and arguments in (-pi/2, pi/2), both branches of the
  evaluation (ascending series and Hankel's expansion) and the switch between.
* Whole matrices K_n(kappa) against the oracle's Nystrom matrix (which is built
  from SciPy's Bessel functions and its own weights), on a circle, an ellipse
  and a circle of radius 3 (so that |kappa r| exceeds the switch at 13).
* The geometry builder rejects odd n, coincident points and x' = 0, and marks a
  circle (whose matrix is circulant, so the node kernel forms only its first
  column) but not an ellipse or a shifted, rotated, rescaled circle sampled
  off its symmetry.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy import special

import oracle as o
import workloads as w

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not found")
    cuda_inc = None
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            cuda_inc = os.path.join(d, "include")
            break
    if cuda_inc is None:
        pytest.skip("CUDA headers not found")
    out = str(tmp_path_factory.mktemp("bie") / "bie_host.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I" + cuda_inc, "-o", out,
                    os.path.join(HERE, "bie_host.cpp")], check=True)
    L = C.CDLL(out)
    L.bie_host_j1_h1.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    L.bie_host_matrix.argtypes = [C.c_int32, C.c_void_p, C.c_double, C.c_double, C.c_void_p]
    L.bie_host_matrix.restype = C.c_int32
    L.bie_host_circulant.argtypes = [C.c_int32, C.c_void_p]
    L.bie_host_circulant.restype = C.c_int32
    return L


def _j1h1(lib, ws):
    ws = np.ascontiguousarray(ws, dtype=np.complex128)
    J = np.zeros_like(ws)
    H = np.zeros_like(ws)
    lib.bie_host_j1_h1(ws.size, ws.ctypes.data, J.ctypes.data, H.ctypes.data)
    return J, H


def _matrix(lib, samples, kappa):
    s = np.ascontiguousarray(np.asarray(samples, dtype=np.float64).ravel())
    n = s.size // 6
    K = np.zeros((n, n), dtype=np.complex128, order="F")
    rc = lib.bie_host_matrix(n, s.ctypes.data, kappa.real, kappa.imag, K.ctypes.data)
    return rc, K


def test_bessel_j1_h1_against_scipy(lib):
    mags = np.geomspace(1e-3, 40.0, 400)
    args = np.linspace(-np.pi / 2 + 0.02, np.pi / 2 - 0.02, 61)
    W = (mags[:, None] * np.exp(1j * args[None, :])).ravel()
    J, H = _j1h1(lib, W)
    ej = np.abs(J - special.jv(1, W)) / np.abs(special.jv(1, W))
    eh = np.abs(H - special.hankel1(1, W)) / np.abs(special.hankel1(1, W))
    low = W.imag <= 0.0
    assert ej[low].max() < 1e-11 and eh[low].max() < 1e-11
    mid = (W.imag > 0.0) & (W.imag <= 2.0)
    assert ej[mid].max() < 1e-11 and eh[mid].max() < 1e-10
    small = np.abs(W) <= 5.0
    assert ej[small].max() < 1e-13 and eh[small & low].max() < 1e-13


@pytest.mark.parametrize("curve,kappas", [
    (w.circle_curve(64), [1.3 - 0.7j, 3.1 - 2.2j, 0.3 - 0.2j]),
    (w.ellipse_curve(96, 1.5, 0.8), [1.3 - 0.7j, 3.1 - 2.2j, 2.0 + 0.5j]),
    (w.circle_curve(128, 3.0), [2.9 - 0.4j, 1.7 - 2.5j]),
])
def test_matrix_against_oracle(lib, curve, kappas):
    for kappa in kappas:
        rc, K = _matrix(lib, curve.samples, kappa)
        assert rc == 0
        B = o.dlp_matrix(curve.samples, kappa)
        assert np.abs(K - B).max() <= 1e-11 * np.abs(B).max(), kappa


def test_geometry_rejects_bad_curves(lib):
    good = w.circle_curve(16).samples
    assert _matrix(lib, good, 1.0 - 1.0j)[0] == 0
    odd = w.circle_curve(15).samples
    assert _matrix(lib, odd, 1.0 - 1.0j)[0] == -1
    dup = good.copy()
    dup[:, 5] = dup[:, 3]
    assert _matrix(lib, dup, 1.0 - 1.0j)[0] == -1
    flat = good.copy()
    flat[2:4, 7] = 0.0
    assert _matrix(lib, flat, 1.0 - 1.0j)[0] == -1
    nan = good.copy()
    nan[0, 2] = np.nan
    assert _matrix(lib, nan, 1.0 - 1.0j)[0] == -1


def _circ(lib, samples):
    s = np.ascontiguousarray(np.asarray(samples, dtype=np.float64).ravel())
    return lib.bie_host_circulant(s.size // 6, s.ctypes.data)


def test_circulant_detection(lib):
    C = w.circle_curve(64)
    assert _circ(lib, C.samples) == 1
    assert _circ(lib, w.circle_curve(96, 3.0).samples) == 1
    assert _circ(lib, w.ellipse_curve(64, 1.5, 0.8).samples) == 0
    # a circle translated by (0.3, -0.2): still shift-invariant
    s = C.samples.copy()
    s[0] += 0.3
    s[1] -= 0.2
    assert _circ(lib, s) == 1
    # one point moved off the circle: not
    s[0, 5] += 1e-6
    assert _circ(lib, s) == 0
    # the circulant reading holds for the circle's matrix: K_ij = K_{(i-j) mod n, 0}
    rc, K = _matrix(lib, C.samples, 1.7 - 0.9j)
    n = K.shape[0]
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    assert np.abs(K - K[(i - j) % n, 0]).max() <= 1e-13 * np.abs(K).max()
    assert _circ(lib, w.circle_curve(15).samples) == -1
