"""ctypes binding of libpmcim (the C ABI in include/pmcim.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels. Functions with the C names take raw pointers; the wrappers below take
NumPy arrays (host memory) or torch CUDA tensors (device memory) and return
NumPy arrays. Loading fails loudly when the library has not been built: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libpmcim.so")

PMCIM_OK = 0
STATUS = {0: "ok", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ECAPACITY", -6: "ENOTSUP"}

RS_CANDIDATE, RS_SATURATED, RS_SPLIT, RS_SINGULAR_NODE, RS_IR_FALLBACK, RS_NO_EIG, RS_SCREENED = 1, 2, 4, 8, 16, 32, 64
F_MONOMIAL, F_EXP_NEG, F_HELMHOLTZ_DLP = 0, 1, 2
PREC_FP64, PREC_FP32_IR, PREC_AUTO, PREC_TF32X3_IR, PREC_BF16X3_IR = 0, 1, 2, 3, 4

EXPORTS = ["pmcim_default_options", "pmcim_problem_create", "pmcim_problem_destroy", "pmcim_moments",
           "pmcim_indicator", "pmcim_beyn", "pmcim_verify", "pmcim_solve", "pmcim_status_string",
           "pmcim_last_error", "pmcim_profile_enable", "pmcim_profile_reset", "pmcim_profile_read",
           "pmcim_solve_points_noalloc", "pmcim_batch_solve", "pmcim_screen_features", "pmcim_screen_train",
           "pmcim_screen_apply", "pmcim_screen_gradient", "pmcim_pmcima", "pmcim_debug_wait_limits",
           "pmcim_residual", "pmcim_certify"]

KERNELS = ["factor_fp64", "reduce", "indicator", "beyn", "verify", "gather", "factor_fp32", "screen"]
SCREEN_PARAMS = 4481


class pmcim_fterm(C.Structure):
    _fields_ = [("kind", C.c_int32), ("degree", C.c_int32), ("tau", C.c_double),
                ("id_re", C.c_double), ("id_im", C.c_double)]


class pmcim_region(C.Structure):
    _fields_ = [("c_re", C.c_double), ("c_im", C.c_double), ("r", C.c_double),
                ("N", C.c_int32), ("depth", C.c_int32)]


class pmcim_options(C.Structure):
    _fields_ = [("tol_ind", C.c_double), ("tol_svd", C.c_double), ("tol_verify", C.c_double),
                ("precision", C.c_int32), ("max_ir_sweeps", C.c_int32), ("max_split_depth", C.c_int32),
                ("beyn_K", C.c_int32), ("cuda_stream", C.c_void_p), ("screen_params", C.c_void_p),
                ("screen_threshold", C.c_double), ("screen_N", C.c_int32), ("indicator_N", C.c_int32),
                ("tol_ir", C.c_double), ("residual_fp64", C.c_int32), ("fp64_tile", C.c_int32)]


class pmcim_batch_item(C.Structure):
    _fields_ = [("problem", C.c_void_p), ("R", C.c_int32), ("regions", C.c_void_p), ("l", C.c_int32),
                ("V", C.c_void_p)]


class pmcim_profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * 8), ("ms", C.c_double * 8), ("mixed_phase_cycles", C.c_double * 16)]


class pmcim_stats(C.Structure):
    _fields_ = [("solves", C.c_int64), ("regions", C.c_int32), ("candidates", C.c_int32),
                ("splits", C.c_int32), ("unverified", C.c_int32), ("ir_fallbacks", C.c_int32),
                ("singular_nodes", C.c_int32), ("ir_sweeps", C.c_int64), ("certified", C.c_int32),
                ("graphs", C.c_int32), ("tuned_fp64", C.c_int32), ("tuned_mixed", C.c_int32),
                ("screened_out", C.c_int32), ("screen_solves", C.c_int32), ("tuned_tc", C.c_int32),
                ("tc_timeouts", C.c_int32), ("node_ctas", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libpmcim.so (raises if it is missing: build it with paper_2312_13117_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libpmcim.so not found at %s; run paper_2312_13117_gb300.build.build()" % path)
    lib = C.CDLL(path)
    P, I32, D, VP = C.c_void_p, C.c_int32, C.c_double, C.c_void_p
    lib.pmcim_default_options.argtypes = [C.POINTER(pmcim_options)]
    lib.pmcim_default_options.restype = None
    lib.pmcim_problem_create.argtypes = [I32, I32, C.POINTER(C.c_void_p), C.POINTER(pmcim_fterm), C.POINTER(P)]
    lib.pmcim_problem_destroy.argtypes = [P]
    lib.pmcim_moments.argtypes = [P, C.POINTER(pmcim_options), I32, C.POINTER(pmcim_region), I32, VP, VP, VP, VP, VP]
    lib.pmcim_indicator.argtypes = [P, C.POINTER(pmcim_options), I32, C.POINTER(pmcim_region), I32, VP, VP, VP, VP, VP]
    lib.pmcim_beyn.argtypes = [P, C.POINTER(pmcim_options), I32, C.POINTER(pmcim_region), I32, VP, I32, VP, VP, VP,
                               VP, VP]
    lib.pmcim_verify.argtypes = [P, C.POINTER(pmcim_options), I32, VP, VP, VP]
    lib.pmcim_certify.argtypes = [P, C.POINTER(pmcim_options), I32, VP, VP, VP, VP]
    lib.pmcim_solve.argtypes = [P, C.POINTER(pmcim_options), I32, C.POINTER(pmcim_region), I32, VP, I32, VP, VP, VP,
                                VP, VP, VP, VP, C.POINTER(pmcim_stats)]
    lib.pmcim_status_string.argtypes = [C.c_int]
    lib.pmcim_status_string.restype = C.c_char_p
    lib.pmcim_last_error.argtypes = []
    lib.pmcim_last_error.restype = C.c_char_p
    lib.pmcim_profile_enable.argtypes = [C.c_int]
    lib.pmcim_profile_enable.restype = None
    lib.pmcim_profile_reset.argtypes = []
    lib.pmcim_profile_reset.restype = None
    lib.pmcim_profile_read.argtypes = [C.POINTER(pmcim_profile)]
    lib.pmcim_profile_read.restype = None
    lib.pmcim_debug_wait_limits.argtypes = [C.c_int64, C.c_int64]
    lib.pmcim_residual.argtypes = [P, C.POINTER(pmcim_options), I32, VP, I32, VP, VP, VP]
    lib.pmcim_solve_points_noalloc.argtypes = [I32, I32, C.POINTER(pmcim_fterm), C.POINTER(C.c_uint8), VP, I32,
                                               VP, I32, VP, VP, VP, VP]
    F = C.c_void_p
    lib.pmcim_screen_features.argtypes = [P, C.POINTER(pmcim_options), I32, C.POINTER(pmcim_region), I32, VP, VP, F]
    lib.pmcim_screen_train.argtypes = [I32, F, VP, I32, I32, D, D, F, VP, VP]
    lib.pmcim_screen_apply.argtypes = [I32, F, F, F, VP]
    lib.pmcim_screen_gradient.argtypes = [I32, F, VP, D, F, F, VP, VP]
    lib.pmcim_batch_solve.argtypes = [I32, C.POINTER(pmcim_batch_item), C.POINTER(pmcim_options), I32, VP, VP, VP,
                                      VP, VP, C.POINTER(pmcim_stats)]
    lib.pmcim_pmcima.argtypes = [P, C.POINTER(pmcim_options), I32, C.POINTER(pmcim_region), VP, D, I32, VP, VP, VP,
                                 VP, C.POINTER(pmcim_stats)]
    for name in ("pmcim_problem_create", "pmcim_problem_destroy", "pmcim_moments", "pmcim_indicator",
                 "pmcim_beyn", "pmcim_verify", "pmcim_solve", "pmcim_solve_points_noalloc", "pmcim_batch_solve",
                 "pmcim_screen_features", "pmcim_screen_train", "pmcim_screen_apply", "pmcim_screen_gradient",
                 "pmcim_pmcima", "pmcim_debug_wait_limits", "pmcim_residual", "pmcim_certify"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class PmcimError(RuntimeError):
    def __init__(self, code: int, where: str, count: int = 0):
        lib = load()
        msg = lib.pmcim_last_error().decode()
        super().__init__("%s failed: %s (%s) %s" % (where, STATUS.get(code, code), code, msg))
        self.code = code
        self.count = count


def _check(code: int, where: str, count=None):
    if code != PMCIM_OK:
        raise PmcimError(code, where, int(count[0]) if count is not None else 0)


# ---------------------------------------------------------------------------
# raw C names (pointers in, status out)
# ---------------------------------------------------------------------------

def pmcim_default_options() -> pmcim_options:
    o = pmcim_options()
    load().pmcim_default_options(C.byref(o))
    return o


def pmcim_problem_create(n, K, A_ptrs, fterms) -> int:
    h = C.c_void_p()
    arr = (C.c_void_p * K)(*A_ptrs)
    _check(load().pmcim_problem_create(n, K, arr, fterms, C.byref(h)), "pmcim_problem_create")
    return h.value


def pmcim_problem_destroy(h):
    _check(load().pmcim_problem_destroy(C.c_void_p(h)), "pmcim_problem_destroy")


def pmcim_profile_enable(on: bool):
    load().pmcim_profile_enable(1 if on else 0)


def pmcim_profile_reset():
    load().pmcim_profile_reset()


def debug_wait_limits(tc_wait_cycles: int = 0, handoff_wait_cycles: int = 0):
    """Limits of the precision-form kernel's bounded waits (0 = default); for tests."""
    _check(load().pmcim_debug_wait_limits(int(tc_wait_cycles), int(handoff_wait_cycles)), "pmcim_debug_wait_limits")


def pmcim_profile_read() -> dict:
    pr = pmcim_profile()
    load().pmcim_profile_read(C.byref(pr))
    out = {k: {"launches": int(pr.launches[i]), "ms": float(pr.ms[i])} for i, k in enumerate(KERNELS)}
    cyc = [float(x) for x in pr.mixed_phase_cycles]
    wall_ns = cyc[11]  # slot 11: CTA lifetimes in ns (globaltimer), not cycles
    cyc[11] = 0.0
    tot = sum(cyc)
    if tot > 0:
        # the node kernel runs two thread groups side by side: each phase is given
        # as a share of its own group's clock
        names = ["assemble", "lu_panel", "first_solve", "residual_fp64", "correction_solve", "fp64_fallback",
                 "node_setup", "lu_trsm", "lu_update", "factor_wait", "refine_wait", "cta_wall", "lu_swaps",
                 "unused13", "unused14", "unused15"]
        factor = {0, 1, 6, 7, 8, 9, 12}
        tot_f = sum(c for i, c in enumerate(cyc) if i in factor) or 1.0
        tot_r = sum(c for i, c in enumerate(cyc) if i not in factor) or 1.0
        share = {nm: c / (tot_f if i in factor else tot_r) for i, (nm, c) in enumerate(zip(names, cyc)) if c > 0}
        share["lu_fp32"] = sum(share.get(k, 0.0) for k in ("lu_panel", "lu_swaps", "lu_trsm", "lu_update"))
        out["factor_fp32"]["phase_share"] = share
        out["factor_fp32"]["phase_cycles"] = {nm: c for nm, c in zip(names, cyc) if c > 0}
        if wall_ns > 0:
            # SM cycles the refine group accounted for per ns of CTA lifetime: the
            # effective SM clock the node kernel ran at, in GHz
            out["factor_fp32"]["cta_wall_ns"] = wall_ns
            out["factor_fp32"]["effective_clock_ghz"] = tot_r / wall_ns
    return out


# ---------------------------------------------------------------------------
# array helpers
# ---------------------------------------------------------------------------

def _ptr(x) -> Optional[int]:
    """Address of a NumPy array or a torch tensor (host or CUDA), or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError("unsupported buffer type %r" % type(x))


def _colmajor_c128(A) -> np.ndarray:
    return np.asfortranarray(np.asarray(A, dtype=np.complex128))


def regions_array(regions: Sequence) -> C.Array:
    """Region objects with attributes (c, r, N) -> pmcim_region[R]."""
    R = len(regions)
    arr = (pmcim_region * max(R, 1))()
    for g, reg in enumerate(regions):
        arr[g].c_re = float(complex(reg.c).real)
        arr[g].c_im = float(complex(reg.c).imag)
        arr[g].r = float(reg.r)
        arr[g].N = int(reg.N)
        arr[g].depth = 0
    return arr


_screen_keep = []


def options(tol_ind=0.1, tol_svd=1e-6, tol_verify=1e-6, precision=PREC_FP64, max_ir_sweeps=6,
            max_split_depth=8, stream=None, screen_params=None, screen_threshold=0.0,
            screen_N=16, tol_ir=None, indicator_N=0, beyn_K=1, residual_fp64=False,
            fp64_tile=0) -> pmcim_options:
    o = pmcim_default_options()
    o.residual_fp64 = 1 if residual_fp64 else 0
    o.fp64_tile = int(fp64_tile)
    o.indicator_N = int(indicator_N)
    o.beyn_K = int(beyn_K)
    o.tol_ind, o.tol_svd, o.tol_verify = tol_ind, tol_svd, tol_verify
    if tol_ir is not None:
        o.tol_ir = float(tol_ir)
    o.precision, o.max_ir_sweeps, o.max_split_depth = precision, max_ir_sweeps, max_split_depth
    o.cuda_stream = stream
    if screen_params is not None:
        sp = np.ascontiguousarray(np.asarray(screen_params, dtype=np.float32))
        assert sp.size == SCREEN_PARAMS
        _screen_keep.append(sp)
        del _screen_keep[:-8]
        o.screen_params = sp.ctypes.data
        o.screen_threshold = float(screen_threshold)
        o.screen_N = int(screen_N)
    return o


# ---------------------------------------------------------------------------
# learned screen
# ---------------------------------------------------------------------------

def screen_train(feats, labels, params, epochs=30, batch=1024, lr=3e-3, pos_weight=4.0, stream=None):
    """Train the screen on the GPU; returns (trained params, per-epoch loss)."""
    lib = load()
    f = np.ascontiguousarray(np.asarray(feats, np.float32))
    y = np.ascontiguousarray(np.asarray(labels, np.uint8))
    p = np.ascontiguousarray(np.asarray(params, np.float32)).copy()
    el = np.zeros(max(epochs, 1))
    _check(lib.pmcim_screen_train(len(y), _ptr(f), _ptr(y), epochs, batch, lr, pos_weight, _ptr(p), _ptr(el),
                                  stream), "pmcim_screen_train")
    return p, el[:epochs]


def screen_apply(feats, params, stream=None):
    lib = load()
    f = np.ascontiguousarray(np.asarray(feats, np.float32))
    p = np.ascontiguousarray(np.asarray(params, np.float32))
    out = np.zeros(len(f), np.float32)
    _check(lib.pmcim_screen_apply(len(f), _ptr(f), _ptr(p), _ptr(out), stream), "pmcim_screen_apply")
    return out


def screen_gradient(feats, labels, params, pos_weight=4.0, stream=None):
    lib = load()
    f = np.ascontiguousarray(np.asarray(feats, np.float32))
    y = np.ascontiguousarray(np.asarray(labels, np.uint8))
    p = np.ascontiguousarray(np.asarray(params, np.float32))
    g = np.zeros(SCREEN_PARAMS, np.float32)
    loss = np.zeros(1)
    _check(lib.pmcim_screen_gradient(len(y), _ptr(f), _ptr(y), pos_weight, _ptr(p), _ptr(g), _ptr(loss), stream),
           "pmcim_screen_gradient")
    return g, float(loss[0])


class Problem:
    """Handle for T(z) = sum_k f_k(z) A_k built from ``(A, kind, degree, tau)`` terms.

    ``A`` is an n x n complex matrix (NumPy or torch, host or CUDA) or a complex
    scalar s meaning s * I; for kind PMCIM_F_HELMHOLTZ_DLP it is an object with a
    ``samples`` array (6 x n curve samples) and a complex ``scale``.
    """

    def __init__(self, n: int, terms):
        self.n = int(n)
        K = len(terms)
        ft = (pmcim_fterm * K)()
        keep, ptrs = [], []
        for k, (A, kind, deg, tau) in enumerate(terms):
            ft[k].kind, ft[k].degree, ft[k].tau = int(kind), int(deg), float(tau)
            if hasattr(A, "samples"):  # boundary-integral term: the curve's 6 x n samples, factor A.scale
                smp = np.ascontiguousarray(np.asarray(A.samples, dtype=np.float64))
                ft[k].id_re, ft[k].id_im = complex(A.scale).real, complex(A.scale).imag
                keep.append(smp)
                ptrs.append(_ptr(smp))
            elif np.isscalar(A):
                ft[k].id_re, ft[k].id_im = complex(A).real, complex(A).imag
                ptrs.append(None)
            else:
                if isinstance(A, np.ndarray) or not hasattr(A, "data_ptr"):
                    A = _colmajor_c128(A)
                else:  # torch tensor: column-major == transpose of a contiguous row-major tensor
                    A = A.t().contiguous().t()
                keep.append(A)
                ptrs.append(_ptr(A))
        self.handle = pmcim_problem_create(self.n, K, ptrs, ft)

    @classmethod
    def from_workload_problem(cls, prob):
        return cls(prob.n, prob.terms)

    def close(self):
        if getattr(self, "handle", None):
            pmcim_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- wrappers returning NumPy arrays --------------------------------
    def moments(self, regions, V, opt=None):
        lib = load()
        V = _colmajor_c128(V)
        n, l, R = self.n, V.shape[1], len(regions)
        C0 = np.zeros((R, l, n), np.complex128)
        C1 = np.zeros((R, l, n), np.complex128)
        ph = np.zeros((R, n), np.complex128)
        pa = np.zeros((R, n), np.float64)
        opt = opt or options()
        _check(lib.pmcim_moments(self.handle, C.byref(opt), R, regions_array(regions), l, _ptr(V), _ptr(C0),
                                 _ptr(C1), _ptr(ph), _ptr(pa)), "pmcim_moments")
        return C0.transpose(0, 2, 1), C1.transpose(0, 2, 1), ph, pa

    def indicator(self, regions, V, opt=None):
        lib = load()
        V = _colmajor_c128(V)
        R, l = len(regions), V.shape[1]
        ind = np.zeros(R)
        pn = np.zeros(R)
        ps = np.zeros(R)
        cand = np.zeros(R, np.uint8)
        opt = opt or options()
        _check(lib.pmcim_indicator(self.handle, C.byref(opt), R, regions_array(regions), l, _ptr(V), _ptr(ind),
                                   _ptr(pn), _ptr(ps), _ptr(cand)), "pmcim_indicator")
        return ind, cand.astype(bool), pn, ps

    def beyn(self, regions, V, cap=None, opt=None, want_vecs=True):
        try:
            return self._beyn(regions, V, cap, opt, want_vecs)
        except PmcimError as e:  # capacity: the library reported the count; retry at that size
            if e.code != -5 or cap is not None:
                raise
            return self._beyn(regions, V, e.count, opt, want_vecs)

    def _beyn(self, regions, V, cap, opt, want_vecs):
        lib = load()
        V = _colmajor_c128(V)
        R, l, n = len(regions), V.shape[1], self.n
        cap = cap if cap is not None else max(64, 4 * l * R)
        lam = np.zeros(cap, np.complex128)
        vecs = np.zeros((cap, n), np.complex128) if want_vecs else None
        rof = np.zeros(cap, np.int32)
        cnt = np.zeros(1, np.int32)
        rst = np.zeros(max(R, 1), np.int32)
        opt = opt or options()
        _check(lib.pmcim_beyn(self.handle, C.byref(opt), R, regions_array(regions), l, _ptr(V), cap, _ptr(lam),
                              _ptr(vecs), _ptr(rof), _ptr(cnt), _ptr(rst)), "pmcim_beyn", cnt)
        k = int(cnt[0])
        return lam[:k], (vecs[:k].T if want_vecs else None), rof[:k], rst[:R]

    def screen_features(self, regions, V, opt=None):
        """(ind3 R x 3 = I_8, I_16, I_N; feats R x 3 float32) of the disks (N a multiple of 16)."""
        lib = load()
        V = _colmajor_c128(V)
        R = len(regions)
        ind3 = np.zeros((max(R, 1), 3))
        feats = np.zeros((max(R, 1), 3), np.float32)
        opt = opt or options()
        _check(lib.pmcim_screen_features(self.handle, C.byref(opt), R, regions_array(regions), V.shape[1], _ptr(V),
                                         _ptr(ind3), _ptr(feats)), "pmcim_screen_features")
        return ind3[:R], feats[:R]

    def verify(self, lam, opt=None):
        lib = load()
        lam = np.ascontiguousarray(np.asarray(lam, np.complex128))
        m = len(lam)
        sig = np.zeros(max(m, 1))
        acc = np.zeros(max(m, 1), np.uint8)
        opt = opt or options()
        _check(lib.pmcim_verify(self.handle, C.byref(opt), m, _ptr(lam), _ptr(sig), _ptr(acc)), "pmcim_verify")
        return sig[:m], acc[:m].astype(bool)

    def certify(self, lam, vecs, opt=None):
        """Upper bounds of sigma_min(T(lambda_i)) from start vectors (n x m, column i for
        lambda_i): the start vector's own residual, then the bordered inverse step's.
        Returns (cert, accept)."""
        lib = load()
        lam = np.ascontiguousarray(np.atleast_1d(np.asarray(lam, np.complex128)))
        m = len(lam)
        vc = np.ascontiguousarray(np.asarray(vecs, np.complex128).reshape(-1, m).T)  # column-major
        cert = np.zeros(max(m, 1))
        acc = np.zeros(max(m, 1), np.uint8)
        opt = opt or options()
        _check(lib.pmcim_certify(self.handle, C.byref(opt), m, _ptr(lam), _ptr(vc), _ptr(cert), _ptr(acc)),
               "pmcim_certify")
        return cert[:m], acc[:m].astype(bool)

    def residual(self, z, V, X, opt=None):
        """R_j = V - T(z_j) X_j on the tensor cores; X is m x n x l (or n x l for one point)."""
        lib = load()
        z = np.ascontiguousarray(np.atleast_1d(np.asarray(z, np.complex128)))
        X = np.asarray(X, np.complex128)
        one = X.ndim == 2
        if one:
            X = X[None]
        m, n, l = X.shape
        Xc = np.ascontiguousarray(X.transpose(0, 2, 1))          # column-major blocks
        Vc = np.ascontiguousarray(np.asarray(V, np.complex128).T)
        R = np.zeros_like(Xc)
        opt = opt or options()
        _check(lib.pmcim_residual(self.handle, C.byref(opt), m, _ptr(z), l, _ptr(Vc), _ptr(Xc), _ptr(R)),
               "pmcim_residual")
        R = R.transpose(0, 2, 1)
        return R[0] if one else R

    def pmcima(self, regions, V, tol_eps=1e-6, cap=None, opt=None, want_vecs=True):
        """pmCIMa with probe column V[:, 0]: returns dict(lam, vecs, sigma_min, stats)."""
        lib = load()
        f = _colmajor_c128(np.asarray(V).reshape(self.n, -1)[:, :1])
        R = len(regions)
        cap = cap if cap is not None else max(64, 8 * R)
        while True:
            lam = np.zeros(cap, np.complex128)
            vecs = np.zeros((cap, self.n), np.complex128) if want_vecs else None
            sig = np.zeros(cap)
            cnt = np.zeros(1, np.int32)
            st = pmcim_stats()
            o = opt or options()
            rc = lib.pmcim_pmcima(self.handle, C.byref(o), R, regions_array(regions), _ptr(f), float(tol_eps), cap,
                                  _ptr(lam), _ptr(vecs), _ptr(sig), _ptr(cnt), C.byref(st))
            if rc == -5 and int(cnt[0]) > cap:
                cap = int(cnt[0])
                continue
            _check(rc, "pmcim_pmcima", cnt)
            k = int(cnt[0])
            return dict(lam=lam[:k], vecs=(vecs[:k].T if want_vecs else None), sigma_min=sig[:k],
                        stats=st.as_dict())

    def solve(self, regions, V, cap=None, opt=None, want_vecs=True):
        """Whole pmCIMb: returns dict(lam, vecs, sigma_min, region_of, ind, status, stats)."""
        try:
            return self._solve(regions, V, cap, opt, want_vecs)
        except PmcimError as e:  # capacity: the library reported the count; retry at that size
            if e.code != -5 or cap is not None:
                raise
            return self._solve(regions, V, e.count, opt, want_vecs)

    def _solve(self, regions, V, cap, opt, want_vecs):
        lib = load()
        V = _colmajor_c128(V)
        R, l, n = len(regions), V.shape[1], self.n
        cap = cap if cap is not None else max(64, 4 * l * R)
        lam = np.zeros(cap, np.complex128)
        vecs = np.zeros((cap, n), np.complex128) if want_vecs else None
        sig = np.zeros(cap)
        rof = np.zeros(cap, np.int32)
        cnt = np.zeros(1, np.int32)
        ind = np.zeros(max(R, 1))
        rst = np.zeros(max(R, 1), np.int32)
        st = pmcim_stats()
        opt = opt or options()
        _check(lib.pmcim_solve(self.handle, C.byref(opt), R, regions_array(regions), l, _ptr(V), cap, _ptr(lam),
                               _ptr(vecs), _ptr(sig), _ptr(rof), _ptr(cnt), _ptr(ind), _ptr(rst), C.byref(st)),
               "pmcim_solve", cnt)
        k = int(cnt[0])
        return dict(lam=lam[:k], vecs=(vecs[:k].T if want_vecs else None), sigma_min=sig[:k], region_of=rof[:k],
                    ind=ind[:R], status=rst[:R], stats=st.as_dict())


def batch_solve(problems, regions_list, V_list, cap=None, opt=None):
    """pmcim_batch_solve over Problem handles with their disks and probe blocks.

    Returns dict(lam, sigma_min, problem_of, region_of, stats).
    """
    try:
        return _batch_solve(problems, regions_list, V_list, cap, opt)
    except PmcimError as e:  # capacity: the library reported the count; retry at that size
        if e.code != -5 or cap is not None:
            raise
        return _batch_solve(problems, regions_list, V_list, e.count, opt)


def _batch_solve(problems, regions_list, V_list, cap, opt):
    lib = load()
    P = len(problems)
    items = (pmcim_batch_item * P)()
    keep = []
    for q, (pr, regs, V) in enumerate(zip(problems, regions_list, V_list)):
        V = _colmajor_c128(V)
        ra = regions_array(regs)
        keep += [V, ra]
        items[q].problem = pr.handle
        items[q].R = len(regs)
        items[q].regions = C.cast(ra, C.c_void_p)
        items[q].l = V.shape[1]
        items[q].V = _ptr(V)
    if cap is None:
        cap = max(64, sum(4 * V.shape[1] * len(r) for r, V in zip(regions_list, V_list)))
    lam = np.zeros(cap, np.complex128)
    sig = np.zeros(cap)
    pof = np.zeros(cap, np.int32)
    rof = np.zeros(cap, np.int32)
    cnt = np.zeros(1, np.int32)
    st = pmcim_stats()
    opt = opt or options()
    _check(lib.pmcim_batch_solve(P, items, C.byref(opt), cap, _ptr(lam), _ptr(sig), _ptr(pof), _ptr(rof),
                                 _ptr(cnt), C.byref(st)), "pmcim_batch_solve", cnt)
    k = int(cnt[0])
    return dict(lam=lam[:k], sigma_min=sig[:k], problem_of=pof[:k], region_of=rof[:k], stats=st.as_dict())
