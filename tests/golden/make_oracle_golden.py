"""Write the stored CPU-oracle results of whole workloads (test infrastructure).

Every expected value in the files this script writes comes from the oracle
(``oracle.pmcimb``, the plain FP64 restatement of pmCIMb steps 1-3) on the
seeded inputs of ``workloads``; nothing else is imported. Disks are
independent (Sec. 3.2: each disk's indicator, Beyn step and filter use only its
own nodes), so the oracle runs one top-level disk at a time (with that disk's
split children) in a process pool started with ``spawn``, one BLAS thread per
process, and the results are merged and sorted as ``pmcimb`` itself sorts them.
When several tol_svd values are asked for, the quadrature moments of a disk are
computed once and reused: ``moments`` is a pure function of the disk and the
inputs, and only the rank decision (step 2.d) depends on tol_svd.

Usage (from the repository root):
  python tests/golden/make_oracle_golden.py delay  [--workers 7]
      -> tests/golden/delay_n1024_oracle.json   (768 disks, tol_svd 1e-6 and 1e-10)
  python tests/golden/make_oracle_golden.py mass_spring_sample [--workers 7]
      -> tests/golden/mass_spring_n2048_sample_oracle.json
         (16 disks whose circle holds an eigenvalue and 16 whose circle holds none,
          chosen by a seeded draw; eigenvalue locations from the 2n companion pencil)
  python tests/golden/make_oracle_golden.py scattering [--workers 7]
      -> tests/golden/scattering_disk_n256_oracle.json
         (the 100 disks of the sound-soft disk's scattering-pole problem, Sec. 4.2)
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_v] = "1"

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

_W = None
_KIND = None


def _workload(kind):
    import workloads as w
    if kind == "delay":
        return w.delay_large()
    if kind == "mass_spring_sample":
        return w.mass_spring()
    if kind == "scattering":
        return w.scattering_disk()
    raise ValueError(kind)


def _init(kind):
    global _W, _KIND
    _KIND = kind
    _W = _workload(kind)


def _one_disk(args):
    """pmcimb on one top-level disk for each tol_svd; moments shared between them."""
    g, tols = args
    import oracle.pmcim_ref as ref
    cache = {}
    plain = ref.moments

    def memo(problem, c, r, N, V):
        key = (complex(c), float(r), int(N), int(V.shape[1]))
        if key not in cache:
            cache[key] = plain(problem, c, r, N, V)
        return cache[key]

    ref.moments = memo
    try:
        out = {}
        reg = _W.regions[g]
        for tol in tols:
            res = ref.pmcimb(_W.problem, [reg], _W.V, tol_ind=_W.tol_ind, tol_svd=tol,
                             tol_verify=_W.tol_verify)
            recs = []
            for rc in res.records:
                s = rc.sigma if rc.sigma is not None else np.zeros(0)
                p = int(rc.p)
                above = float(s[p - 1]) if p >= 1 else None          # smallest sigma counted
                below = float(s[p]) if 0 <= p < len(s) else None     # largest sigma not counted
                recs.append([rc.c.real, rc.c.imag, rc.r, int(rc.depth), float(rc.I), bool(rc.candidate),
                             p, bool(rc.saturated), bool(rc.split), above, below])
            out[repr(tol)] = {
                "records": recs,
                "cand": [[complex(z).real, complex(z).imag, float(s), bool(a)]
                         for z, s, a in zip(res.cand_lam, res.cand_sigma, res.cand_accept)],
            }
        return g, out
    finally:
        ref.moments = plain


def _sample_disks(W, seed=5, per_class=16):
    """Seeded choice of disks with and without an eigenvalue in their circle.

    The eigenvalues of z^2 I + z C + K are those of the 2n companion pencil
    [[0, I], [-K, -C]] - z [[I, 0], [0, I]] (its matrix form, since the leading
    coefficient is I)."""
    import scipy.linalg as sla
    n = W.problem.n
    C = K = None
    for (A, kind, deg, tau) in W.problem.terms:
        if deg == 1 and not np.isscalar(A):
            C = np.asarray(A)
        if deg == 0 and not np.isscalar(A):
            K = np.asarray(A)
    comp = np.zeros((2 * n, 2 * n), dtype=np.complex128)
    comp[:n, n:] = np.eye(n)
    comp[n:, :n] = -K
    comp[n:, n:] = -C
    lam = sla.eigvals(comp)
    cen = np.array([complex(g.c) for g in W.regions])
    rad = np.array([g.r for g in W.regions])
    counts = np.array([int(np.sum(np.abs(lam - cen[i]) < rad[i])) for i in range(len(cen))])
    rng = np.random.default_rng(seed)
    with_eig = np.flatnonzero(counts > 0)
    without = np.flatnonzero(counts == 0)
    pick = sorted(rng.choice(with_eig, per_class, replace=False).tolist()
                  + rng.choice(without, per_class, replace=False).tolist())
    return pick, counts, lam


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["delay", "mass_spring_sample", "scattering"])
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--tol-svd", type=float, nargs="*", default=None)
    ap.add_argument("--out", default=None)
    ap.add_argument("--limit", type=int, default=0, help="first LIMIT disks only (a quick trial)")
    a = ap.parse_args()

    W = _workload(a.workload)
    meta = {"workload": a.workload, "n": W.problem.n, "l": int(W.V.shape[1]), "N": W.regions[0].N,
            "tol_ind": W.tol_ind, "tol_verify": W.tol_verify,
            "written_by": "tests/golden/make_oracle_golden.py " + a.workload,
            "oracle": "oracle.pmcimb (FP64, LAPACK LU per node, SVD/eig, sigma_min by svdvals)"}
    if a.workload == "delay":
        tols = a.tol_svd or [1e-6, 1e-10]
        disks = list(range(len(W.regions)))
        out = a.out or os.path.join(HERE, "delay_n1024_oracle.json")
        meta["disks_note"] = "all disks of Omega = [-3,1] x [-6,6] split 16 x 48, x-major order"
    elif a.workload == "scattering":
        tols = a.tol_svd or [1e-6]
        disks = list(range(len(W.regions)))
        out = a.out or os.path.join(HERE, "scattering_disk_n%d_oracle.json" % W.problem.n)
        meta["disks_note"] = "all disks of Omega = [0.2,3.2] x [-3.2,-0.2] split 10 x 10, x-major order"
    else:
        tols = a.tol_svd or [1e-6]
        disks, counts, lam_comp = _sample_disks(W)
        out = a.out or os.path.join(HERE, "mass_spring_n2048_sample_oracle.json")
        meta["disks_note"] = ("seeded sample (seed 5): 16 disks whose circle holds an eigenvalue of the "
                              "companion pencil, 16 whose circle holds none")
        meta["companion_counts"] = [int(counts[g]) for g in disks]
        inside = [complex(z) for z in lam_comp
                  if any(abs(z - complex(W.regions[g].c)) < W.regions[g].r for g in disks)]
        meta["companion_lam_in_sample"] = [[z.real, z.imag] for z in sorted(inside, key=lambda z: (z.real, z.imag))]
    if a.limit:
        disks = disks[:a.limit]
    meta["disks"] = disks
    meta["tol_svd"] = tols

    t0 = time.time()
    ctx = mp.get_context("spawn")
    results = {}
    with ctx.Pool(a.workers, initializer=_init, initargs=(a.workload,)) as pool:
        for k, (g, res) in enumerate(pool.imap_unordered(_one_disk, [(g, tols) for g in disks])):
            results[g] = res
            if (k + 1) % 16 == 0 or k + 1 == len(disks):
                print("%d/%d disks, %.0f s" % (k + 1, len(disks), time.time() - t0), flush=True)

    runs = {}
    for tol in tols:
        key = repr(tol)
        recs, lam, rej = [], [], []
        for g in disks:
            r = results[g][key]
            recs += [[g] + rc for rc in r["records"]]
            for (re, im, s, acc) in r["cand"]:
                (lam if acc else rej).append([re, im, s, g])
        lam.sort(key=lambda t: (t[0], t[1]))
        rej.sort(key=lambda t: (t[0], t[1]))
        runs[key] = {"tol_svd": tol,
                     "record_fields": ["disk", "c_re", "c_im", "r", "depth", "I", "candidate", "p",
                                       "saturated", "split", "sigma_smallest_counted", "sigma_largest_dropped"],
                     "records": recs,
                     "lam_fields": ["re", "im", "sigma_min", "disk"],
                     "lam": lam, "rejected": rej}
    meta["seconds"] = round(time.time() - t0, 1)
    meta["workers"] = a.workers
    with open(out, "w") as fh:
        json.dump({"meta": meta, "runs": runs}, fh, separators=(",", ":"))
    print("wrote", out, "in %.0f s" % (time.time() - t0))


if __name__ == "__main__":
    main()
