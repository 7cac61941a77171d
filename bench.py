"""Benchmark: T(z)^{-1} V solves per second through the whole pmCIMb hot path.

Workload: the delay-type problem T(z) = -z I + A0 + A1 exp(-z), n = 1024,
l = 16 probes, N = 64 nodes per disk, Omega = [-3,1] x [-6,6] split 16 x 48.
One step runs pmCIMb (indicator, Beyn with splitting, square filter,
verification) on a batch of consecutive disks of that grid; successive steps
take successive batches. value = node solves of all ranks / max time over
ranks. Data are synthetic (seeded generators).

Extra keys: roofline of the dominant kernel (measured live with CUDA events
on its launch stream inside the library), e2e (same metric through the C ABI
with host buffers, host<->device copies inside the timed region), the oracle
CPU baseline on a bounded sample, launches of the library's kernels, clocks.

--impl reference times the CPU oracle itself (the reference arm of this
build) on the same workload, one disk per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "T(z)^-1·V solves/s at n=1024; full pmCIMb time vs plain FP64 at λ err≤1e-10"
UNIT = "solves/s"
FP64_DFMA_PER_SM_CLK = 2          # measured: 1.19-1.20 TFLOP/s at ~2.0 GHz on 152 SMs
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
# DRAM bytes per node of k_factor_solve_fp64, from one ncu capture of a 64-node launch at n = 1024, l = 16
# (dram__bytes_read.sum + dram__bytes_write.sum = 15.16 + 13.45 GB); scaled to a launch by its node count.
FACTOR_FP64_TRAFFIC_PER_NODE = 28.61e9 / 64
# DRAM bytes per node of k_factor_solve_mixed, from one ncu capture of a 384-node launch per form
# (dram__bytes_read.sum + dram__bytes_write.sum); scaled to a launch by its node count. None: no
# capture of the kernel as it stands
MIXED_TRAFFIC_PER_NODE = {"fp32ir": None, "tf32x3": (71.629e9 + 44.950e9) / 384, "bf16x3": None,
                          "tf32x3_fp64res": None}
# sm__pipe_tensor_cycles_active (% of active cycles) of the same capture of the tensor-core form
MIXED_TENSOR_PIPE_PCT = {"tf32x3": 8.66}
# FP32 pipe: 128 FFMA / SM / clock (measured 73.3 TFLOP/s at ~2.0 GHz); at the 2.07 GHz maximum:
FP32_PEAK_TFLOPS = 128 * 2 * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# TF32 tensor peak: the measured dense bf16 burst x the nominal tf32 / bf16 ratio (1.1 / 2.25 PFLOP/s)
TF32_PEAK_TFLOPS = float(_peaks().get("bf16_tflops", 1900.0)) * 1.1 / 2.25
# BF16 tensor peak for a kernel timed inside a long step: the measured sustained figure
BF16_SUSTAINED_TFLOPS = float(_peaks().get("bf16_tflops_sustained", 1700.0))


def fp64_peak_tflops(sm_max_mhz: float) -> float:
    """FP64 pipe peak: 2 DFMA / SM / clock x 2 flops x 152 SMs x max SM clock."""
    return FP64_DFMA_PER_SM_CLK * 2 * SM_COUNT * sm_max_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)

    def window(self, t0=None, t1=None):
        """Median SM clock, its minimum, peak power and throttle reasons of the samples
        taken between monotonic times t0 and t1 (all samples when None)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            if (t0 is not None and ts < t0) or (t1 is not None and ts > t1):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                pw.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_min_mhz": min(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "power_w_max": max(pw) if pw else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def disk_ids(step: int, rank: int, world: int, per_step: int, R: int, offset: int):
    """Disks of one rank in one step: each rank takes its own consecutive block of
    per_step disks, so the ranks' blocks are disjoint (weak scaling, no data-path
    collective)."""
    base = offset + (step * world + rank) * per_step
    return [(base + i) % R for i in range(per_step)]


def reduce_over_ranks(x: float, world: int, op: str) -> float:
    """max or sum of a scalar over ranks (timings and counts only)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(x: float, world: int) -> float:
    return reduce_over_ranks(x, world, "max")


def sum_over_ranks(x: float, world: int) -> float:
    return reduce_over_ranks(x, world, "sum")


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------

def oracle_solves_per_s(W, region_ids):
    import oracle
    t0 = time.perf_counter()
    solves = 0
    res = oracle.pmcimb(W.problem, [W.regions[g] for g in region_ids], W.V, tol_ind=W.tol_ind,
                        tol_svd=W.tol_svd, tol_verify=W.tol_verify)
    for rec in res.records:
        solves += rec.N
    dt = time.perf_counter() - t0
    return solves, dt


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import workloads as w
    W = w.delay_large()
    R = len(W.regions)
    start = args.region_offset
    total_solves, total_t = 0, 0.0
    for k in range(args.warmup + args.steps):
        g = (start + k) % R
        s, dt = oracle_solves_per_s(W, [g])
        if k >= args.warmup:
            total_solves += s
            total_t += dt
    value = total_solves / total_t
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "delay NEP n=1024, l=16, N=64, Omega=[-3,1]x[-6,6] 16x48 disks (one disk per step)",
                   "oracle": "NumPy/SciPy LAPACK, FP64"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "one disk (64 node solves + Beyn + verification) per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_batched(args, world, rank, local):
    """Many independent quadratic problems of uneven size (n ~ U{32..768}) per step.

    One step solves a slice of the 512 seeded problems with pmcim_batch_solve
    (one level = one CUDA graph, one persistent launch per form). Reported for
    the autotuned precision, for FP64 and the precision form forced, and for
    the same problems solved one call each (no batching)."""
    import torch
    from paper_2312_13117_gb300 import pmcim
    import workloads as w
    per = args.problems_per_step
    total = 512

    def seeds(step):
        base = ((step * world + rank) * per) % total
        return [1 + (base + i) % total for i in range(per)]

    def make(step):
        W = w.batched_quadratics(seeds(step))
        if args.disks_per_problem > 0:  # an evenly spread subset of each problem's grid
            for x in W:
                R = len(x.regions)
                keep = sorted({(i * R) // args.disks_per_problem for i in range(min(R, args.disks_per_problem))})
                x.regions = [x.regions[i] for i in keep]
        return [pmcim.Problem(x.problem.n, x.problem.terms) for x in W], W

    steps = list(range(-args.warmup, args.steps))
    prepared = {k: make(k) for k in steps}          # coefficients resident before timing
    stream = torch.cuda.current_stream()
    res = {}
    forms = [("auto", pmcim.PREC_AUTO), ("fp32ir", pmcim.PREC_FP32_IR), ("unbatched_auto", pmcim.PREC_AUTO),
             ("auto_hankel", pmcim.PREC_AUTO)]
    if args.batched_fp64:
        forms.append(("fp64", pmcim.PREC_FP64))
    # the autotuner measures each (n bucket, l, dense terms) on first use: let it do so
    # for every timed problem before timing (one disk each)
    o_auto = pmcim.options(stream=stream.cuda_stream, precision=pmcim.PREC_AUTO)
    for k in steps:
        hs, W = prepared[k]
        pmcim.batch_solve(hs, [x.regions[:1] for x in W], [x.V for x in W], opt=o_auto)
    torch.cuda.synchronize()
    t_start = time.perf_counter()
    for name, prec in forms:
        if time.perf_counter() - t_start > args.time_budget:
            sys.stderr.write("skipping %s: time budget spent\n" % name)
            continue
        o = pmcim.options(stream=stream.cuda_stream, precision=prec,
                          beyn_K=args.beyn_k if name.endswith("hankel") else 1)
        agg = {}
        t_ms = 0.0
        pmcim.pmcim_profile_reset()
        for k in steps:
            hs, W = prepared[k]
            torch.cuda.synchronize()
            pmcim.pmcim_profile_enable(k >= 0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if name.startswith("unbatched"):
                st = {}
                for h, x in zip(hs, W):
                    r = h.solve(x.regions, x.V, opt=o, want_vecs=False)
                    for key, v in r["stats"].items():
                        st[key] = max(st.get(key, 0), v) if key == "node_ctas" else st.get(key, 0) + v
                found = None
            else:
                r = pmcim.batch_solve(hs, [x.regions for x in W], [x.V for x in W], opt=o)
                st = r["stats"]
            e1.record(stream)
            torch.cuda.synchronize()
            if k >= 0:
                t_ms += e0.elapsed_time(e1)
                for key, v in st.items():
                    agg[key] = max(agg.get(key, 0), v) if key == "node_ctas" else agg.get(key, 0) + v
        pmcim.pmcim_profile_enable(False)
        prof = pmcim.pmcim_profile_read()
        t_max = max_over_ranks(t_ms, world)
        sys.stderr.write("%s: %.1f ms/step, %d solves, %d splits\n" % (name, t_max / args.steps, agg["solves"],
                                                                     agg["splits"]))
        res[name] = {"solves_per_s": sum_over_ranks(float(agg["solves"]), world) / (t_max / 1e3),
                     "ms_per_step": t_max / args.steps, "solves": agg["solves"], "splits": agg["splits"],
                     "graphs": agg["graphs"], "tuned_fp64": agg["tuned_fp64"], "tuned_mixed": agg["tuned_mixed"],
                     "tuned_tc": agg.get("tuned_tc", 0), "ir_fallbacks": agg["ir_fallbacks"],
                     "node_ctas": agg.get("node_ctas"),
                     # busy CTA-time of the node kernel over (its launch time x CTAs): the launch tails
                     "node_cta_utilisation": (prof["factor_fp32"]["cta_wall_ns"] /
                                              (prof["factor_fp32"]["ms"] * 1e6 * max(1, agg.get("node_ctas") or 1))
                                              if prof.get("factor_fp32", {}).get("ms") else None),
                     "kernels_ms": {kk: round(v["ms"], 1) for kk, v in prof.items()},
                     "kernel_launches": {kk: v["launches"] for kk, v in prof.items()},
                     "node_phase_share": prof.get("factor_fp32", {}).get("phase_share")}
    if rank == 0:
        ns = [x.problem.n for k in steps if k >= 0 for x in prepared[k][1]]
        print(json.dumps({"metric": "solves/s, batched quadratic NEPs", "value": res["auto"]["solves_per_s"],
                          "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "higher_is_better": True, "scaling": "weak", "dtype": "auto: per problem FP64, FP32 LU + FP64 IR or tensor-core LU + FP64 IR",
                          "data": "synthetic",
                          "config": {"workload": "batched quadratic NEPs, seeds 1..512, %d problems per step%s"
                                                     % (per, ", %d disks of each problem's grid" % args.disks_per_problem
                                                        if args.disks_per_problem > 0 else ""),
                                     "n_range": [min(ns), max(ns)], "l": 8,
                                     "disks": sum(len(x.regions) for k in steps if k >= 0 for x in prepared[k][1])},
                          "forms": res,
                          "speedup_batched_vs_unbatched": (res["unbatched_auto"]["ms_per_step"] / res["auto"]["ms_per_step"]
                                                           if "unbatched_auto" in res else None),
                          "beyn_K_of_hankel_leg": args.beyn_k,
                          "speedup_hankel_vs_auto": (res["auto"]["ms_per_step"] / res["auto_hankel"]["ms_per_step"]
                                                     if "auto_hankel" in res else None)}))
    for k in steps:
        for h in prepared[k][0]:
            h.close()
    return 0


def run_screen(args, world, rank, local):
    """Learned screen on the damped mass-spring problem (n = 2048).

    Untimed set-up: traces of the delay and batched workloads' own generators
    at other seeds and smaller n (features I_8, I_16, r and the full rule's
    decision, about 1e5 disks), computed by the library; the screen trained on
    the GPU; its threshold set so every training positive passes with margin.
    Timed: pmCIMb in the precision form on a block of disks of the 32 x 256
    grid (default 32 x 32), plain, screened, two-pass, and two-pass screened.
    Recall: on the oracle's stored sample of the grid (16 disks with an
    eigenvalue, 16 without), the screened run against the oracle's decisions
    and eigenvalues."""
    import torch
    from paper_2312_13117_gb300 import pmcim
    import workloads as w
    # ---- traces and training (untimed) ----
    t0 = time.perf_counter()
    F, Y = [], []
    n_delay = max(1, args.trace_problems // 100)
    for prob, regs, V in w.config_trace_problems(range(1, 1 + n_delay), range(513, 513 + args.trace_problems)):
        h = pmcim.Problem(prob.n, prob.terms)
        ind3, feats = h.screen_features(regs, V)
        h.close()
        F.append(feats)
        Y.append(ind3[:, 2] > 0.1)
    F = np.concatenate(F)
    Y = np.concatenate(Y).astype(np.uint8)
    t_traces = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    perm = rng.permutation(len(Y))
    F, Y = F[perm], Y[perm]
    W1 = rng.standard_normal((64, 3)) * np.sqrt(2.0 / 3)
    W2 = rng.standard_normal((64, 64)) * np.sqrt(2.0 / 64)
    W3 = rng.standard_normal(64) * np.sqrt(1.0 / 64)
    p0 = np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3, [0.0]]).astype(np.float32)
    t0 = time.perf_counter()
    params, loss = pmcim.screen_train(F, Y, p0, epochs=args.epochs, batch=1024, lr=3e-3, pos_weight=8.0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    prob = pmcim.screen_apply(F, params)
    thr = 0.5 * float(prob[Y == 1].min())
    # ---- the mass-spring slice ----
    W = w.mass_spring(l=args.ms_l)
    c0, r0, side = args.ms_cols[0], args.ms_rows[0], args.ms_side
    cols, rows = range(c0, c0 + side), range(r0, r0 + side)
    regs = [W.regions[i * 256 + j] for i in cols for j in rows]
    h = pmcim.Problem(W.problem.n, W.problem.terms)
    stream = torch.cuda.current_stream()
    out = {}
    legs = (("plain", {}), ("screened", {"screen_params": params, "screen_threshold": thr}),
            ("two_pass", {"indicator_N": args.indicator_n}),
            ("two_pass_screened", {"screen_params": params, "screen_threshold": thr, "indicator_N": args.indicator_n}))
    for name, kw in legs:
        o = pmcim.options(stream=stream.cuda_stream, precision=pmcim.PREC_TF32X3_IR, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = h.solve(regs, W.V, opt=o, want_vecs=False, cap=64 * args.ms_l * len(regs))
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"seconds": e0.elapsed_time(e1) / 1e3, "lam": r["lam"], "ind": r["ind"], "stats": r["stats"],
                     "status": r["status"], "region_of": r["region_of"]}
    plain_cand = out["plain"]["ind"] > 0.1
    passed = (out["screened"]["status"] & pmcim.RS_SCREENED) == 0
    recall = float(np.mean(passed[plain_cand])) if plain_cand.any() else 1.0
    with_eigs = np.zeros(len(regs), bool)
    with_eigs[np.unique(out["plain"]["region_of"])] = True
    recall_eig_disks = float(np.mean(passed[with_eigs])) if with_eigs.any() else 1.0
    a, b = out["plain"]["lam"], out["screened"]["lam"]
    eig_recall = _lam_recall(a, b)
    # ---- recall against the oracle's stored sample of the grid ----
    oracle_recall = None
    gpath = os.path.join(ROOT, "tests", "golden", "mass_spring_n2048_sample_oracle.json")
    if os.path.exists(gpath):
        with open(gpath) as fh:
            gold = json.load(fh)
        disks = gold["meta"]["disks"]
        run = gold["runs"][repr(1e-6)]
        top = {rec[0]: rec for rec in run["records"] if rec[4] == 0}
        o = pmcim.options(stream=stream.cuda_stream, precision=pmcim.PREC_TF32X3_IR, screen_params=params,
                          screen_threshold=thr)
        rs = h.solve([W.regions[g] for g in disks], W.V, opt=o, want_vecs=False, cap=64 * args.ms_l * len(disks))
        skipped = (rs["status"] & pmcim.RS_SCREENED) != 0
        cand = np.array([bool(top[g][6]) for g in disks])
        lam_o = np.array([complex(x[0], x[1]) for x in run["lam"]])
        oracle_recall = {"disks": len(disks), "oracle_candidates": int(cand.sum()),
                         "candidate_recall": float(np.mean(~skipped[cand])) if cand.any() else 1.0,
                         "screened_out": int(skipped.sum()),
                         "oracle_eigenvalues": int(len(lam_o)),
                         "eigenvalue_recall": _lam_recall(lam_o, rs["lam"]),
                         "max_rel_lambda_err": _max_rel_diff(lam_o, rs["lam"])}
    h.close()
    R = len(regs)
    if rank == 0:
        print(json.dumps({
            "metric": "learned screen: subregions/s on the mass-spring NEP (n=2048)",
            "value": R / out["screened"]["seconds"], "unit": "subregions/s", "n_gpus": world,
            "higher_is_better": True, "dtype": "precision form (FP32 LU + FP64-accurate IR); screen BF16/FP32",
            "data": "synthetic",
            "config": {"workload": "mass-spring z^2 I + z C + K, n=2048, l=%d, N=64; disks of grid columns %d-%d x "
                                   "rows %d-%d of the 32 x 256 split of [-1,0] x [0,8]"
                                   % (args.ms_l, c0, c0 + side - 1, r0, r0 + side - 1),
                       "traces": int(len(Y)), "trace_sources": "delay generator (%d seeds, n 64-128) and batched "
                                                               "generator (%d seeds, n 32-128)"
                                                               % (n_delay, args.trace_problems),
                       "trace_positive_fraction": float(Y.mean()),
                       "trace_seconds": t_traces, "train_seconds": t_train, "epochs": args.epochs,
                       "final_loss": float(loss[-1]), "threshold": thr},
            "plain_seconds": out["plain"]["seconds"], "screened_seconds": out["screened"]["seconds"],
            "speedup": out["plain"]["seconds"] / out["screened"]["seconds"],
            "eigenvalue_recall_vs_plain": eig_recall, "recall_disks_with_eigenvalues": recall_eig_disks,
            "candidate_decision_recall_vs_plain": recall, "screened_out": out["screened"]["stats"]["screened_out"],
            "candidates_plain": int(plain_cand.sum()), "eigenvalues_plain": len(a), "eigenvalues_screened": len(b),
            "solves_plain": out["plain"]["stats"]["solves"],
            "solves_screened": out["screened"]["stats"]["solves"] + out["screened"]["stats"]["screen_solves"],
            "two_pass": {name: {"seconds": out[name]["seconds"],
                                "solves": out[name]["stats"]["solves"] + out[name]["stats"]["screen_solves"],
                                "speedup_vs_plain": out["plain"]["seconds"] / out[name]["seconds"],
                                "eigenvalue_recall_vs_plain": _lam_recall(a, out[name]["lam"])}
                         for name in ("two_pass", "two_pass_screened")},
            "gain_of_screen_over_two_pass": out["two_pass"]["seconds"] / out["two_pass_screened"]["seconds"],
            "recall_vs_oracle_sample": oracle_recall,
            "indicator_N": args.indicator_n}))
    return 0


def _lam_recall(ref, got, tol=1e-10):
    """Fraction of the reference eigenvalues that have a value of `got` within tol (relative)."""
    ref, got = np.asarray(ref), np.asarray(got)
    if len(ref) == 0:
        return 1.0
    if len(got) == 0:
        return 0.0
    d = np.abs(ref[:, None] - got[None, :]) / np.maximum(1.0, np.abs(ref[:, None]))
    return float(np.mean(d.min(axis=1) <= tol))


def _max_rel_diff(a, b):
    """Largest relative difference of two eigenvalue lists matched one to one (None when the counts differ)."""
    a, b = np.asarray(a), np.asarray(b)
    if len(a) != len(b):
        return None
    if len(a) == 0:
        return 0.0
    from scipy.optimize import linear_sum_assignment
    ri, ci = linear_sum_assignment(np.abs(a[:, None] - b[None, :]))
    return float(np.max(np.abs(a[ri] - b[ci]) / np.maximum(1.0, np.abs(a[ri]))))


def _oracle_golden():
    """Verified eigenvalues of the CPU oracle on every disk of the n = 1024 delay workload
    (tol_svd = 1e-6), by disk, from the stored results tests/golden/make_oracle_golden.py
    wrote; None when the file is absent."""
    path = os.path.join(ROOT, "tests", "golden", "delay_n1024_oracle.json")
    try:
        with open(path) as fh:
            run = json.load(fh)["runs"][repr(1e-6)]
    except (OSError, KeyError, ValueError):
        return None
    out = {}
    for (re_, im_, _sig, g) in run["lam"]:
        out.setdefault(int(g), []).append(complex(re_, im_))
    return out


def _same_lams(a, b, tol=1e-10):
    """Both eigenvalue lists hold the same values (relative tol), matched one to one."""
    d = _max_rel_diff(a, b)
    return d is not None and d <= tol


def run_paper_quadratic(args, world, rank, local):
    """The paper's quadratic experiment (Sec. 4.1, Table 1) on seeded inputs of its shape:
    n = 100, T_j uniform [0, 1), Omega = [-0.5, 0.5]^2 in 225 squares. Times pmCIMb with the
    Appendix's schedule (indicator on 16 nodes, Beyn on 64, l = 10) in FP64 and in the FP32-LU
    form, and pmCIMa (indicator on 16 nodes, tol_eps = 1e-6) in FP64; each is checked against
    the companion pencil's eigenvalues in Omega. The paper's MATLAB times (12 workers of an
    M1 Ultra) are quoted as context, not as a target."""
    import torch
    import scipy.linalg as sla
    from paper_2312_13117_gb300 import pmcim
    import workloads as w
    if rank != 0:
        return 0
    W = w.paper_quadratic()
    n = W.problem.n
    T0, T1, T2 = [t[0] for t in W.problem.terms]
    Z, I = np.zeros((n, n)), np.eye(n)
    lam_all = sla.eig(np.block([[Z, I], [-T0, -T1]]), np.block([[I, Z], [Z, T2]]), right=False)
    truth = lam_all[(np.abs(lam_all.real) < 0.5) & (np.abs(lam_all.imag) < 0.5)]
    P = pmcim.Problem(n, W.problem.terms)
    regs16 = [w.Region(g.c, g.r, 16) for g in W.regions]
    stream = torch.cuda.current_stream()
    legs = {
        "pmCIMb_fp64": lambda: P.solve(W.regions, W.V, opt=pmcim.options(stream=stream.cuda_stream,
                                                                          indicator_N=16), want_vecs=False),
        "pmCIMb_fp64_tile32": lambda: P.solve(W.regions, W.V, opt=pmcim.options(
            stream=stream.cuda_stream, indicator_N=16, fp64_tile=32), want_vecs=False),
        "pmCIMb_auto": lambda: P.solve(W.regions, W.V, opt=pmcim.options(
            stream=stream.cuda_stream, precision=pmcim.PREC_AUTO, indicator_N=16), want_vecs=False),
        "pmCIMb_fp32ir": lambda: P.solve(W.regions, W.V, opt=pmcim.options(
            stream=stream.cuda_stream, precision=pmcim.PREC_FP32_IR, indicator_N=16), want_vecs=False),
        "pmCIMa_fp64": lambda: P.pmcima(regs16, W.V, tol_eps=1e-6, opt=pmcim.options(stream=stream.cuda_stream),
                                        want_vecs=False),
    }
    out = {}
    for name, fn in legs.items():
        fn()  # untimed: workspace allocation and first launches
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = fn()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        lam = np.asarray(res["lam"])
        out[name] = {"seconds": dt, "eigenvalues": len(lam), "solves": res["stats"]["solves"],
                     "max_rel_err_vs_companion": _max_rel_diff(truth, lam)}
    P.close()
    print(json.dumps({
        "metric": "time to all eigenvalues in Omega, the paper's quadratic experiment (seeded inputs)",
        "unit": "s", "n_gpus": 1, "data": "synthetic",
        "config": {"workload": "T0 + z T1 + z^2 T2, n = 100, T_j uniform [0,1) (seed 0), Omega = [-0.5,0.5]^2 in "
                               "15 x 15 squares, circumscribed disks", "l": 10, "N_beyn": 64, "N_indicator": 16,
                   "tol_eps_pmCIMa": 1e-6},
        "eigenvalues_in_omega_companion": int(len(truth)), "forms": out,
        "paper_context_seconds": {"hardware": "MATLAB R2021a, Apple M1 Ultra, 12 workers (Table 1)",
                                  "pmCIMa": 93.18, "pmCIMb": 7.10, "note": "other inputs (MATLAB rand), context only"}}))
    return 0


def library_lu_leg(W, disk, device="cuda", reps=2):
    """External comparison, not part of the product path: the node solves of one disk,
    T(z_j) X_j = V for its N nodes, through PyTorch's batched LU (torch.linalg.lu_factor and
    lu_solve: cuSOLVER/cuBLAS getrf and getrs on a GPU) in complex128, and in complex64
    (FP32 LU, no refinement: not FP64 accurate, for context). T(z_j) is assembled with torch
    tensor operations before the timed region; the timed region is the factorisation and the
    solve of the whole batch, `reps` times after one untimed run, with CUDA events."""
    import torch
    out = {"disk": disk, "note": "torch.linalg.lu_factor + lu_solve on the batch of the disk's N nodes"}
    try:
        reg = W.regions[disk]
        N, n = reg.N, W.problem.n
        th = 2.0 * np.pi * np.arange(N) / N
        z = torch.tensor(reg.c + reg.r * np.exp(1j * th), dtype=torch.complex128, device=device)
        T = torch.zeros((N, n, n), dtype=torch.complex128, device=device)
        eye = torch.eye(n, dtype=torch.complex128, device=device)
        for (A, kind, deg, tau) in W.problem.terms:
            f = z ** deg if kind == 0 else torch.exp(-tau * z)
            M = eye * complex(A) if np.isscalar(A) else torch.from_numpy(np.ascontiguousarray(A)).to(device)
            T += f[:, None, None] * M[None]
        V = torch.from_numpy(np.ascontiguousarray(W.V)).to(device)
        for name, dt in (("complex128", torch.complex128), ("complex64", torch.complex64)):
            Tb, Vb = T.to(dt), V.to(dt).expand(N, -1, -1)

            def run():
                LU, piv = torch.linalg.lu_factor(Tb)
                return torch.linalg.lu_solve(LU, piv, Vb)
            X = run()
            if device == "cuda":
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    X = run()
                e1.record()
                e1.synchronize()
                sec = e0.elapsed_time(e1) / 1e3 / reps
            else:
                t0 = time.perf_counter()
                for _ in range(reps):
                    X = run()
                sec = (time.perf_counter() - t0) / reps
            res = torch.linalg.matrix_norm(T @ X.to(torch.complex128) - V) / torch.linalg.matrix_norm(V)
            out[name] = {"seconds_per_batch": sec, "solves_per_s": N / sec,
                         "max_rel_residual": float(res.max())}
    except Exception as e:  # a comparison only: report, never fail the benchmark line
        out["error"] = "%s: %s" % (type(e).__name__, e)
    return out


def _hankel_zeros(omega, mmax=12):
    """Zeros of H_m^(1) (0 <= m <= mmax) inside the rectangle: the exact scattering poles of the
    sound-soft unit disk (Sec. 4.2), by Newton's method on SciPy's Hankel functions."""
    from scipy import special
    x0, x1, y0, y1 = omega
    out = []
    for m in range(mmax + 1):
        for a in np.linspace(0.05, x1 + 1.0, 16):
            for b in np.linspace(y0 - 1.0, -0.02, 16):
                z = complex(a, b)
                for _ in range(60):
                    f, d = special.hankel1(m, z), special.h1vp(m, z)
                    if not (np.isfinite(f) and np.isfinite(d)) or d == 0:
                        break
                    dz = f / d
                    z -= dz
                    if abs(dz) < 1e-15 * max(1.0, abs(z)):
                        if (x0 <= z.real <= x1 and y0 <= z.imag <= y1
                                and all(abs(z - q) > 1e-8 for mm, q in out if mm == m)):
                            out.append((m, z))
                        break
    return out


def scattering_leg(pmcim, stream, steps=3, with_pmcima=False, oracle_sample=False):
    """The scattering-pole problem of Sec. 4.2: T(kappa) = (I + K_n(kappa)) / 2 on the unit circle,
    n = 256 Nystrom points, Omega = [0.2, 3.2] x [-3.2, -0.2] in 10 x 10 squares, N = 64, l = 8,
    with PREC_AUTO (the FP32 LU with FP64 refinement for this problem), in plain FP64 and with
    tensor-core trailing updates. Each leg runs once untimed, then `steps`
    times; the median wall time of the synchronous call is reported. The eigenvalues are compared
    with the stored oracle run and with the zeros of the Hankel functions in Omega."""
    import torch
    import workloads as w
    W = w.scattering_disk()
    P = pmcim.Problem(W.problem.n, W.problem.terms)
    gold = None
    gpath = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                         "scattering_disk_n256_oracle.json")
    if os.path.exists(gpath):
        with open(gpath) as fh:
            gold = np.array([complex(a, b) for (a, b, _, _) in json.load(fh)["runs"][repr(1e-6)]["lam"]])
    zeros = np.array([z for m, z in _hankel_zeros(W.omega) for _ in range(2 if m else 1)])
    regs16 = [w.Region(g.c, g.r, 16) for g in W.regions]
    cs = stream.cuda_stream
    legs = {
        "pmCIMb": lambda: P.solve(W.regions, W.V, want_vecs=False,
                                  opt=pmcim.options(stream=cs, precision=pmcim.PREC_AUTO)),
        "pmCIMb_fp64": lambda: P.solve(W.regions, W.V, want_vecs=False,
                                       opt=pmcim.options(stream=cs, fp64_tile=32)),
        "pmCIMb_fp64_tile64": lambda: P.solve(W.regions, W.V, want_vecs=False,
                                              opt=pmcim.options(stream=cs, fp64_tile=64)),
        "pmCIMb_two_pass": lambda: P.solve(W.regions, W.V, want_vecs=False,
                                           opt=pmcim.options(stream=cs, precision=pmcim.PREC_AUTO, indicator_N=16)),
        "pmCIMb_tf32x3": lambda: P.solve(W.regions, W.V, want_vecs=False,
                                         opt=pmcim.options(stream=cs, precision=pmcim.PREC_TF32X3_IR)),
    }
    if with_pmcima:
        legs["pmCIMa"] = lambda: P.pmcima(regs16, W.V, tol_eps=1e-6, want_vecs=False,
                                          opt=pmcim.options(stream=cs, precision=pmcim.PREC_AUTO))
    out = {}
    for name, fn in legs.items():
        fn()
        ts = []
        for _ in range(max(1, steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        dt = float(np.median(ts))
        lam = np.asarray(res["lam"])
        out[name] = {"seconds": dt, "solves": res["stats"]["solves"],
                     "solves_per_s": res["stats"]["solves"] / dt, "eigenvalues": int(len(lam)),
                     "max_rel_err_vs_oracle": _max_rel_diff(gold, lam) if gold is not None and name != "pmCIMa"
                     else None,
                     "max_rel_err_vs_hankel_zeros": (_max_rel_diff(zeros, lam) if name != "pmCIMa" else
                                                     _max_rel_diff(np.unique(np.round(zeros, 9)), lam))}
    # where the time goes (library events on its launch stream), one more run of the first leg
    pmcim.pmcim_profile_reset()
    pmcim.pmcim_profile_enable(True)
    legs["pmCIMb"]()
    pmcim.pmcim_profile_enable(False)
    prof = {k: v for k, v in pmcim.pmcim_profile_read().items() if v["launches"]}
    P.close()
    summary = {"workload": "sound-soft unit disk, T(kappa) = (I + K_n(kappa))/2, Kress Nystrom, n = 256, "
                           "Omega = [0.2,3.2] x [-3.2,-0.2] in 10 x 10 squares, N = 64, l = 8",
               "speedup_auto_vs_fp64": out["pmCIMb_fp64"]["seconds"] / out["pmCIMb"]["seconds"],
               "legs": out, "kernels_ms": {k: v["ms"] for k, v in prof.items()},
               "poles_in_omega": int(len(np.unique(np.round(zeros, 9)))),
               "paper_context_seconds": {"hardware": "MATLAB, 12 workers (Table 1), unknown n; context only",
                                         "pmCIMb": 12.14, "pmCIMa": 66.20}}
    if oracle_sample:
        # the oracle on one disk that holds a pole (64 node solves at n = 256), on the host
        import oracle as o
        g = W.regions[6]
        t0 = time.perf_counter()
        o.pmcimb(W.problem, [g], W.V, W.tol_ind, W.tol_svd, W.tol_verify)
        dt = time.perf_counter() - t0
        summary["cpu_oracle_one_disk"] = {"seconds": dt, "solves_per_s": g.N / dt, "kind": "oracle",
                                          "sample": "disk 6 (64 node solves + Beyn + verification), one process"}
    return summary


def run_scattering(args, world, rank, local):
    import torch
    from paper_2312_13117_gb300 import pmcim
    if rank != 0:
        return 0
    res = scattering_leg(pmcim, torch.cuda.current_stream(), steps=args.steps, with_pmcima=True,
                         oracle_sample=not args.no_cpu_baseline)
    lg = res["legs"]["pmCIMb"]
    print(json.dumps({"metric": "T(z)^{-1} V node solves/s, scattering poles of a sound-soft disk (Sec. 4.2)",
                      "value": lg["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
                      "higher_is_better": True, "dtype": "f32 LU + f64 refinement", "data": "synthetic",
                      "config": {"workload": res["workload"]}, "scattering_poles": res}))
    return 0


def run_full(args, P, W, opt, opt_mixed, opt_tc, world, rank, local):
    """Time to all eigenvalues: one pmCIMb pass over the whole grid per form (opt_tc: the
    precision form with tensor-core trailing updates, opt_mixed: the same on the FMA pipes,
    opt: plain FP64), the tensor-core and FP64 forms also with the two-pass schedule."""
    import torch
    from paper_2312_13117_gb300 import pmcim
    R = len(W.regions)
    mine = [W.regions[g] for g in range(rank, R, world)]
    out = {}
    lams = {}
    o2 = pmcim.options(stream=opt_tc.cuda_stream, precision=opt_tc.precision, indicator_N=args.indicator_n)
    f2 = pmcim.options(stream=opt.cuda_stream, precision=opt.precision, indicator_N=args.indicator_n)
    o3 = pmcim.options(stream=opt_tc.cuda_stream, precision=opt_tc.precision, indicator_N=args.indicator_n,
                       beyn_K=2)
    for name, o in (("precision_form", opt_tc), ("precision_form_fma_pipes", opt_mixed),
                    ("precision_form_two_pass", o2), ("precision_form_two_pass_hankel2", o3), ("fp64", opt),
                    ("fp64_two_pass", f2)):
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        res = P.solve(mine, W.V, cap=64 * W.V.shape[1] * len(mine), opt=o)
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, world)
        lams[name] = res["lam"]
        out[name] = {"seconds": dt, "solves": res["stats"]["solves"], "eigenvalues": len(res["lam"]),
                     "stats": res["stats"]}
    a, b = np.asarray(lams["fp64"]), np.asarray(lams["precision_form"])
    err = None
    if len(a) == len(b) and len(a):
        from scipy.optimize import linear_sum_assignment
        ri, ci = linear_sum_assignment(np.abs(a[:, None] - b[None, :]))
        err = float(np.max(np.abs(a[ri] - b[ci]) / np.maximum(1.0, np.abs(a[ri]))))
    if rank == 0:
        print(json.dumps({"metric": "full pmCIMb time (all %d disks)" % R, "unit": "s", "n_gpus": world,
                          "workload": "delay NEP n=1024, l=16, N=64, Omega=[-3,1]x[-6,6] 16x48",
                          "forms": out, "max_rel_lambda_diff_fp64_vs_precision_form": err,
                          "speedup": out["fp64"]["seconds"] / out["precision_form"]["seconds"],
                          "speedup_fma_pipes_form": out["fp64"]["seconds"] /
                          out["precision_form_fma_pipes"]["seconds"],
                          "max_rel_lambda_diff_fp64_vs_fma_pipes_form": _max_rel_diff(
                              lams["fp64"], lams["precision_form_fma_pipes"]),
                          "indicator_N": args.indicator_n,
                          "speedup_two_pass_precision_vs_fp64": out["fp64"]["seconds"] /
                          out["precision_form_two_pass"]["seconds"],
                          "two_pass_same_eigenvalues": {k: _same_lams(lams["fp64"], lams[k])
                                                        for k in ("precision_form_two_pass", "fp64_two_pass")},
                          "max_rel_lambda_diff_hankel2_vs_fp64": _max_rel_diff(
                              lams["fp64"], lams["precision_form_two_pass_hankel2"]),
                          "speedup_two_pass_hankel2_vs_fp64": out["fp64"]["seconds"] /
                          out["precision_form_two_pass_hankel2"]["seconds"]}))
    P.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--regions-per-step", type=int, default=96,
                    help="disks per step (96 x 64 nodes = 6144; 8 steps make one pass over the 768-disk grid)")
    ap.add_argument("--region-offset", type=int, default=300)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-regions", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the precision-form measurement")
    ap.add_argument("--only-mixed", action="store_true", help="time only the precision forms (profiling runs)")
    ap.add_argument("--mixed-forms", default="fp32ir,tf32x3", help="precision forms --only-mixed times, in order")
    ap.add_argument("--workload", default="delay",
                    choices=["delay", "batched", "screen", "paper_quadratic", "scattering"])
    ap.add_argument("--no-scattering", action="store_true",
                    help="leave the scattering-pole summary out of the default line")
    ap.add_argument("--trace-problems", type=int, default=2400,
                    help="screen traces: batched-generator problems (and one delay problem per 100 of them)")
    ap.add_argument("--ms-cols", type=int, nargs=1, default=[0], help="first grid column of the mass-spring slice")
    ap.add_argument("--ms-rows", type=int, nargs=1, default=[32], help="first grid row of the mass-spring slice")
    ap.add_argument("--ms-side", type=int, default=32, help="disks per side of the mass-spring slice")
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--ms-l", type=int, default=48, help="probe columns on the mass-spring problem")
    ap.add_argument("--problems-per-step", type=int, default=32)
    ap.add_argument("--disks-per-problem", type=int, default=2,
                    help="batched workload: disks of each problem's grid per step (0: all)")
    ap.add_argument("--batched-fp64", action="store_true", help="also time the batched workload in plain FP64")
    ap.add_argument("--time-budget", type=float, default=240.0, help="seconds before remaining legs are skipped")
    ap.add_argument("--beyn-k", type=int, default=4,
                    help="moment pairs of the block Hankel Beyn legs (--workload batched: 4, --full: 2)")
    ap.add_argument("--indicator-n", type=int, default=16,
                    help="coarse indicator rule of the two-pass legs (--full, --workload screen)")
    ap.add_argument("--fp64-residual-leg", action="store_true",
                    help="also time the headline LU with its refinement residuals on the FP64 pipe")
    ap.add_argument("--no-time-to-all", action="store_true",
                    help="skip the passes over every disk (time to all eigenvalues; about 3 minutes)")
    ap.add_argument("--full", action="store_true",
                    help="time pmCIMb over all 768 disks (time to all eigenvalues), FP64 and precision form")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world, rank, local = dist_init(args)
    from paper_2312_13117_gb300 import build, pmcim
    if rank == 0:
        build.build()
    barrier(world)
    pmcim.load()
    if args.workload == "batched":
        return run_batched(args, world, rank, local)
    if args.workload == "screen":
        return run_screen(args, world, rank, local)
    if args.workload == "paper_quadratic":
        return run_paper_quadratic(args, world, rank, local)
    if args.workload == "scattering":
        return run_scattering(args, world, rank, local)
    import workloads as w

    W = w.delay_large()
    n, l = W.problem.n, W.V.shape[1]
    R = len(W.regions)
    B = args.regions_per_step

    def batch(step):
        return [W.regions[g] for g in disk_ids(step, rank, world, B, R, args.region_offset)]

    stream = torch.cuda.current_stream()
    opt = pmcim.options(stream=stream.cuda_stream)
    opt_mixed = pmcim.options(stream=stream.cuda_stream, precision=pmcim.PREC_FP32_IR)
    opt_tc = pmcim.options(stream=stream.cuda_stream, precision=pmcim.PREC_TF32X3_IR)
    opt_bf = pmcim.options(stream=stream.cuda_stream, precision=pmcim.PREC_BF16X3_IR)
    # the same form with its refinement residuals on the FP64 pipe (the tensor-core residual's A/B leg)
    opt_tc64 = pmcim.options(stream=stream.cuda_stream, precision=pmcim.PREC_TF32X3_IR, residual_fp64=True)
    P = pmcim.Problem(n, W.problem.terms)
    cap = 64 * l * B

    if args.full:
        return run_full(args, P, W, opt, opt_mixed, opt_tc, world, rank, local)

    def timed(o, steps, warmup):
        """Warm up, then time `steps` steps on the library's stream; returns (ms, solves, found, stats, prof)."""
        for k in range(warmup):
            P.solve(batch(-1 - k), W.V, cap=cap, opt=o)
        torch.cuda.synchronize()
        pmcim.pmcim_profile_reset()
        pmcim.pmcim_profile_enable(True)
        barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        w0 = time.monotonic()
        solves, found = 0, 0
        agg = {}
        per_step = []
        for k in range(steps):
            res = P.solve(batch(k), W.V, cap=cap, opt=o)
            per_step.append((k, res["lam"], res["region_of"]))
            solves += res["stats"]["solves"]
            found += len(res["lam"])
            for key, v in res["stats"].items():
                agg[key] = agg.get(key, 0) + v
        e1.record(stream)
        torch.cuda.synchronize()
        w1 = time.monotonic()
        barrier(world)
        pmcim.pmcim_profile_enable(False)
        # eigenvalues of the timed steps by grid disk (first visit of a disk only)
        by_disk = {}
        for k, lam, rof in per_step:
            ids = disk_ids(k, rank, world, B, R, args.region_offset)
            step = {}
            for x, q in zip(lam, rof):
                step.setdefault(ids[int(q)], []).append(complex(x))
            for g in ids:
                by_disk.setdefault(g, step.get(g, []))
        return e0.elapsed_time(e1), solves, found, agg, pmcim.pmcim_profile_read(), (w0, w1), by_disk

    # forms: the headline is the faster of the two precision forms (FP32 LU with its
    # trailing updates on the tensor cores or on the FMA pipes, FP64 refinement),
    # both at FP64 accuracy; the other form and plain FP64 are measured on the same
    # disks beside it
    forms = ([("fp64", opt)] if args.no_mixed else
             [("fp32ir", opt_mixed), ("tf32x3", opt_tc), ("bf16x3", opt_bf)])
    if not args.no_mixed and args.fp64_residual_leg:
        forms.append(("tf32x3_fp64res", opt_tc64))
    head_name, head_opt = forms[0]
    clocks = ClockSampler(local)
    clocks.start()
    if args.only_mixed:
        by_name = dict(forms)
        for name, o in [(nm, by_name[nm]) for nm in args.mixed_forms.split(",")]:
            tm_ms, msolves, mfound, aggm, profm, win, _ = timed(o, args.steps, args.warmup)
            if rank == 0:
                print(json.dumps({"form": name, "solves_per_s": msolves / (tm_ms / 1e3), "ms": tm_ms,
                                  "stats": aggm, "kernels": profm}))
        clocks.stop()
        if rank == 0:
            print(json.dumps({"clocks": clocks.window()}))
        P.close()
        return 0
    runs = {name: timed(o, args.steps, args.warmup) for name, o in forms}
    if not args.no_mixed:
        # the headline is the faster precision form on these disks (same work in both; the
        # max over ranks, so that every rank picks the same one)
        t_form = {nm: max_over_ranks(runs[nm][0], world) for nm in ("fp32ir", "tf32x3", "bf16x3")}
        head_name = min(t_form, key=t_form.get)
        head_opt = {"fp32ir": opt_mixed, "tf32x3": opt_tc, "bf16x3": opt_bf}[head_name]
    clk = clocks.window(*runs[head_name][5])  # the headline's timed region
    smax = clk.get("sm_max_mhz") or SM_MAX_MHZ
    peak64 = fp64_peak_tflops(smax)
    k_dense = sum(1 for t in W.problem.terms if not np.isscalar(t[0]))

    # ---- time to all eigenvalues: one pmCIMb pass over every disk of the grid (this
    # rank's share), in the headline form, in its two-pass schedule and in plain FP64
    mine = list(range(rank, R, world))

    def full_pass(o):
        torch.cuda.synchronize()
        pmcim.pmcim_profile_reset()
        pmcim.pmcim_profile_enable(True)
        barrier(world)
        w0 = time.monotonic()
        t0 = time.perf_counter()
        res = P.solve([W.regions[g] for g in mine], W.V, cap=64 * l * len(mine), opt=o)
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, world)
        w1 = time.monotonic()
        pmcim.pmcim_profile_enable(False)
        by_disk = {g: [] for g in mine}
        for x, q in zip(res["lam"], res["region_of"]):
            by_disk[mine[int(q)]].append(complex(x))
        return {"seconds": dt, "res": res, "by_disk": by_disk, "clocks": clocks.window(w0, w1),
                "kernels": pmcim.pmcim_profile_read()}

    tta = {}
    if not args.no_time_to_all:
        o2 = pmcim.options(stream=stream.cuda_stream, precision=head_opt.precision, indicator_N=args.indicator_n)
        legs = [(head_name, head_opt)] if head_name != "fp64" else []
        legs += [(head_name + "_two_pass", o2), ("fp64", opt)]
        for name, o in legs:
            tta[name] = full_pass(o)
    clocks.stop()

    gold = _oracle_golden()

    def lam_diff(a_by_disk, b_by_disk, disks):
        """Largest relative eigenvalue difference over the given disks (one-to-one match
        per disk; None when a disk's counts differ)."""
        worst = 0.0
        for g in disks:
            d = _max_rel_diff(a_by_disk.get(g, []), b_by_disk.get(g, []))
            if d is None:
                return None
            worst = max(worst, d)
        return worst

    def fp64_record(fp):
        res = fp["res"]
        solves = res["stats"]["solves"]
        fac = fp["kernels"]["factor_fp64"]
        flops_per_node = 8.0 * n ** 3 / 3.0 + 8.0 * n * n * l
        achieved = (flops_per_node * solves) / (fac["ms"] / 1e3) / 1e12 if fac["ms"] > 0 else None
        roof = {"bound": "alu", "kernel": "k_factor_solve_fp64 (FP64 pipe)",
                "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                "frac": (achieved / peak64) if achieved else None,
                "traffic": FACTOR_FP64_TRAFFIC_PER_NODE * solves / max(1, fac["launches"]),
                "traffic_note": "ncu DRAM bytes of a 64-node capture, scaled by nodes per launch",
                "peak_source": "2 DFMA/SM/clk x 152 SMs x max SM clock (probe: 1.20 TFLOP/s at 2.0 GHz)",
                "launches": fac["launches"], "avg_launch_ms": fac["ms"] / max(1, fac["launches"])}
        return {"form": "plain FP64 LU (all disks of the grid, one pmCIMb pass)",
                "value": sum_over_ranks(float(solves), world) / fp["seconds"], "unit": UNIT,
                "seconds": fp["seconds"], "eigenvalues_found": len(res["lam"]),
                "roofline": roof, "kernels": fp["kernels"], "clocks": fp["clocks"]}

    def precision_record(name, run):
        tm_ms, msolves, mfound, aggm, profm, win, _ = run
        tm_max = max_over_ranks(tm_ms, world)
        fm = profm["factor_fp32"]
        # FP64 work: per sweep one residual product T(z)X (T(z) assembled in FP64 once per node
        # by the factor group when the problem has two or more dense terms), plus the fallback solves
        w_asm = msolves * 8.0 * k_dense * n * n if (k_dense >= 2 and name == "tf32x3_fp64res") else 0.0
        w_res = aggm["ir_sweeps"] * 8.0 * n * n * l
        w64 = w_res + w_asm + aggm["ir_fallbacks"] * (8.0 * n ** 3 / 3 + 8.0 * n * n * l)
        w32 = msolves * (8.0 * n ** 3 / 3 + 8.0 * n * n * l) + aggm["ir_sweeps"] * 8.0 * n * n * l
        a64 = w64 / (fm["ms"] / 1e3) / 1e12 if fm["ms"] > 0 else None
        a32 = w32 / (fm["ms"] / 1e3) / 1e12 if fm["ms"] > 0 else None
        roof = {"bound": "alu", "kernel": "k_factor_solve_mixed (FP64 pipe: refinement residuals)",
                "achieved": a64, "peak": peak64, "unit": "TFLOP/s",
                "frac": (a64 / peak64) if a64 else None,
                "traffic": (MIXED_TRAFFIC_PER_NODE[name] * msolves / max(1, fm["launches"])
                            if MIXED_TRAFFIC_PER_NODE.get(name) else None),
                "traffic_note": "ncu DRAM bytes of a small capture, scaled by nodes per launch",
                "peak_source": "2 DFMA/SM/clk x 152 SMs x max SM clock",
                "fp32_work_tflops": a32, "fp32_peak_tflops": FP32_PEAK_TFLOPS,
                "launches": fm["launches"], "avg_launch_ms": fm["ms"] / max(1, fm["launches"]),
                "share_of_step": fm["ms"] / tm_ms if tm_ms else None}
        cyc = fm.get("phase_cycles", {})
        upd = sum(8.0 * 32 * (n - k) * (n + l - k) for k in range(32, n, 32))
        if name != "tf32x3_fp64res":
            # refinement residuals on the tensor cores: the kernel's arithmetic is tensor work,
            # 3xTF32 LU trailing updates (tf32x3) and the BF16 digit products of the residuals
            # (34 digit pairs x 2 MMAs of 128 x 32 x 16 per 32 inner indices, row block, dense
            # term and 16-column block), counted in BF16-equivalent flops
            cb, rbn, kcn = -(-l // 16), -(-n // 128), -(-n // 32)
            res_bf16 = aggm["ir_sweeps"] * k_dense * cb * rbn * kcn * 136 * 2.0 * 128 * 32 * 16
            lu_tf32 = 3.0 * upd * msolves if name == "tf32x3" else 0.0
            # BF16 3M: 3 real products x 6 part products per complex multiply-add (upd counts 8 flops)
            lu_bf16 = 4.5 * upd * msolves if name == "bf16x3" else 0.0
            ratio = (2.25 / 1.1)
            t_s = fm["ms"] / 1e3
            ach = (res_bf16 + lu_tf32 * ratio + lu_bf16) / t_s / 1e12 if t_s > 0 else None
            roof = {"bound": "tensor",
                    "kernel": {"tf32x3": "k_factor_solve_mixed (tensor pipe: 3xTF32 LU trailing updates + BF16 "
                                         "digit products of the refinement residuals)",
                               "bf16x3": "k_factor_solve_mixed (tensor pipe: BF16 3M LU trailing updates + BF16 "
                                         "digit products of the refinement residuals)"}.get(
                        name, "k_factor_solve_mixed (tensor pipe: BF16 digit products of the refinement "
                              "residuals; LU on the FMA pipes)"),
                    "achieved": ach, "peak": BF16_SUSTAINED_TFLOPS, "unit": "TFLOP/s (BF16-equivalent)",
                    "frac": (ach / BF16_SUSTAINED_TFLOPS) if ach else None,
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained; TF32 flops x 2.25/1.1",
                    "traffic": (MIXED_TRAFFIC_PER_NODE[name] * msolves / max(1, fm["launches"])
                                if MIXED_TRAFFIC_PER_NODE.get(name) else None),
                    "traffic_note": "ncu DRAM bytes of a 384-node capture, scaled by nodes per launch",
                    "ncu_tensor_pipe_active_pct": MIXED_TENSOR_PIPE_PCT.get(name),
                    "residual_bf16_tflops": res_bf16 / t_s / 1e12 if t_s > 0 else None,
                    "lu_tf32_tflops": lu_tf32 / t_s / 1e12 if t_s > 0 else None,
                    "lu_bf16_tflops": lu_bf16 / t_s / 1e12 if t_s > 0 else None,
                    "residual_fp64_equivalent_tflops": a64,
                    "fp32_work_tflops": a32,
                    "launches": fm["launches"], "avg_launch_ms": fm["ms"] / max(1, fm["launches"]),
                    "share_of_step": fm["ms"] / tm_ms if tm_ms else None}
        if cyc.get("residual_fp64") and name == "tf32x3_fp64res":
            # SM clock cycles of the refine group inside the residual phase, summed over CTAs
            # (one CTA per SM): the FP64 pipe's rate while the residual runs
            roof["residual_dfma_per_sm_clock"] = w_res / 2.0 / cyc["residual_fp64"]
            roof["peak_dfma_per_sm_clock"] = FP64_DFMA_PER_SM_CLK
        rec = {
            "form": {"fp32ir": "FP32 LU + FP64-accurate iterative refinement, residuals on the tensor cores "
                               "(exact BF16 digit products)",
                     "tf32x3": "FP32 LU with 3xTF32 complex trailing updates on the tensor cores (tcgen05, TMEM "
                               "accumulators) + FP64-accurate iterative refinement, residuals on the tensor "
                               "cores (exact BF16 digit products)",
                     "bf16x3": "FP32 LU with BF16 3M complex trailing updates on the tensor cores (each FP32 "
                               "operand as three BF16 parts) + FP64-accurate iterative refinement, residuals on "
                               "the tensor cores (exact BF16 digit products)",
                     "tf32x3_fp64res": "FP32 LU with 3xTF32 tensor-core trailing updates + FP64 iterative "
                                       "refinement, residuals on the FP64 pipe (T(z) assembled in FP64)"}[name],
            "value": sum_over_ranks(float(msolves), world) / (tm_max / 1e3), "unit": UNIT,
            "ms_per_step": tm_max / args.steps, "eigenvalues_found": mfound,
            "ir_sweeps_per_node": aggm["ir_sweeps"] / max(1, msolves), "ir_fallbacks": aggm["ir_fallbacks"],
            "tc_timeouts": aggm.get("tc_timeouts", 0), "certified": aggm.get("certified", 0),
            "unverified": aggm.get("unverified", 0),
            "roofline": roof, "kernels": profm, "clocks": clocks.window(*win),
        }
        if name.startswith("tf32x3"):
            # tensor-pipe work of the trailing updates: 3 split products of the complex
            # rank-32 updates, 8 real flops per complex multiply-add
            lu_cyc = sum(cyc.get(k, 0.0) for k in ("lu_update",))
            tf = 3.0 * upd * msolves / (lu_cyc / (152 * smax * 1e6)) / 1e12 if lu_cyc else None
            rec["tensor"] = {"tf32_tflops_during_update_phase": tf, "tf32_peak_tflops": TF32_PEAK_TFLOPS,
                             "frac_during_update_phase": tf / TF32_PEAK_TFLOPS if tf else None,
                             "peak_source": "measured bf16 burst x nominal tf32/bf16 ratio 1.1/2.25"}
        return rec

    plain = fp64_record(tta["fp64"]) if "fp64" in tta else None
    head = precision_record(head_name, runs[head_name]) if head_name != "fp64" else None
    if head is None:   # --no-mixed: plain FP64 steps only
        tm_ms, msolves, mfound, aggm, profm, win, _ = runs["fp64"]
        tm_max = max_over_ranks(tm_ms, world)
        head = {"form": "plain FP64 LU", "value": sum_over_ranks(float(msolves), world) / (tm_max / 1e3),
                "unit": UNIT, "ms_per_step": tm_max / args.steps, "eigenvalues_found": mfound,
                "roofline": None, "kernels": profm, "clocks": clocks.window(*win)}
    other_name = {"fp32ir": "tf32x3", "tf32x3": "fp32ir", "bf16x3": "tf32x3"}.get(head_name)
    other = precision_record(other_name, runs[other_name]) if other_name in runs else None
    third_name = next((nm for nm in ("fp32ir", "tf32x3", "bf16x3") if nm in runs and nm not in (head_name, other_name)),
                      None)
    third = precision_record(third_name, runs[third_name]) if third_name else None
    fp64res = precision_record("tf32x3_fp64res", runs["tf32x3_fp64res"]) if "tf32x3_fp64res" in runs else None
    if plain is not None:
        for rec in (head, other, third):
            if rec is not None and rec is not plain:
                rec["speedup_vs_fp64_solves_per_s"] = rec["value"] / plain["value"]

    # ---- the accuracy qualifier of the metric, computed in this run: eigenvalues of the
    # timed steps against plain FP64 and against the stored oracle results on the same disks
    head_by_disk = runs[head_name][6]
    step_disks = sorted(head_by_disk)
    lam_err = {"bound": 1e-10,
               "measure": "max |d lambda| / max(1, |lambda|) over one-to-one matched eigenvalues per disk"}
    if "fp64" in tta:
        lam_err["timed_steps_vs_fp64"] = lam_diff(head_by_disk, tta["fp64"]["by_disk"], step_disks)
    if gold is not None:
        lam_err["timed_steps_vs_oracle"] = lam_diff(head_by_disk, gold, step_disks)
    for name, fp in tta.items():
        if "fp64" in tta and name != "fp64":
            lam_err["all_disks_%s_vs_fp64" % name] = lam_diff(fp["by_disk"], tta["fp64"]["by_disk"], mine)
        if gold is not None:
            lam_err["all_disks_%s_vs_oracle" % name] = lam_diff(fp["by_disk"], gold, mine)
    checks = [v for k, v in lam_err.items() if k.startswith(("timed_steps", "all_disks"))]
    lam_err["within_bound"] = bool(checks) and all(v is not None and v <= 1e-10 for v in checks)

    time_to_all = None
    if tta:
        time_to_all = {name: {"seconds": fp["seconds"], "solves": fp["res"]["stats"]["solves"],
                              "eigenvalues": len(fp["res"]["lam"]), "splits": fp["res"]["stats"]["splits"],
                              "ir_fallbacks": fp["res"]["stats"]["ir_fallbacks"],
                              "certified": fp["res"]["stats"]["certified"],
                              "unverified": fp["res"]["stats"]["unverified"],
                              "kernels_ms": {k: v["ms"] for k, v in fp["kernels"].items()},
                              "clocks": fp["clocks"]} for name, fp in tta.items()}
        time_to_all["disks"] = len(mine) * world
        if "fp64" in tta:
            for name in tta:
                if name != "fp64":
                    time_to_all["speedup_%s_vs_fp64" % name] = tta["fp64"]["seconds"] / tta[name]["seconds"]

    # ---- e2e: host buffers through the C ABI, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        Vh = torch.from_numpy(np.ascontiguousarray(W.V.T)).pin_memory()  # column-major n x l, pinned host
        lam_h = torch.zeros(cap, dtype=torch.complex128).pin_memory()
        vec_h = torch.zeros(cap * n, dtype=torch.complex128).pin_memory()
        sig_h = torch.zeros(cap, dtype=torch.float64).pin_memory()
        rof_h = torch.zeros(cap, dtype=torch.int32).pin_memory()
        cnt_h = torch.zeros(1, dtype=torch.int32).pin_memory()
        ind_h = torch.zeros(B, dtype=torch.float64).pin_memory()
        st_h = torch.zeros(B, dtype=torch.int32).pin_memory()
        lib = pmcim.load()
        import ctypes
        stats = pmcim.pmcim_stats()

        def e2e_step(step):
            regs = pmcim.regions_array(batch(step))
            rc = lib.pmcim_solve(P.handle, ctypes.byref(head_opt), B, regs, l, Vh.data_ptr(), cap, lam_h.data_ptr(),
                                 vec_h.data_ptr(), sig_h.data_ptr(), rof_h.data_ptr(), cnt_h.data_ptr(),
                                 ind_h.data_ptr(), st_h.data_ptr(), ctypes.byref(stats))
            assert rc == 0, pmcim.load().pmcim_last_error()
            c = int(cnt_h[0])
            h2d = n * l * 16 + B * 32
            d2h = c * (16 + 8 + 4 + n * 16) + B * (8 + 4) + 4
            return stats.solves, h2d, d2h

        e2e_step(-1)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        es, h2d, d2h = 0, 0, 0
        for k in range(args.steps):
            s, a, b = e2e_step(k)
            es += s
            h2d += a
            d2h += b
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        te = max_over_ranks(te, world)
        es_all = sum_over_ranks(float(es), world)
        e2e = {"value": es_all / te, "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
               "d2h_bytes_per_step": d2h // args.steps, "form": head_name}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        ids = [(args.region_offset + i) % R for i in range(args.cpu_sample_regions)]
        s, dt = oracle_solves_per_s(W, ids)
        cpu = {"value": s / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": "%d disks (%d node solves) through the full oracle pmCIMb, %.1f s" % (len(ids), s, dt)}

    prof = head["kernels"]
    launches = sum(v["launches"] for v in prof.values())
    scat = None
    if rank == 0 and not args.no_scattering:
        scat = scattering_leg(pmcim, stream, steps=2)
    liblu = library_lu_leg(W, args.region_offset) if rank == 0 else None
    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32ir": "f32 LU + f64 refinement",
                      "tf32x3": "f32 LU (3xTF32 tensor-core updates) + f64 refinement"}[head_name],
            "data": "synthetic",
            "config": {"workload": "delay NEP T(z)=-zI+A0+A1 exp(-z), n=1024, l=16, N=64, "
                                   "Omega=[-3,1]x[-6,6] split 16x48; %d disks per step per GPU" % B,
                       "form": head["form"], "regions_per_step": B, "n": n, "l": l, "N": 64,
                       "l2": "working set > L2 (456 factorisation slots of 8.5 MB)",
                       "eigenvalues_found": head["eigenvalues_found"],
                       "lambda_err_max_vs_fp64": lam_err.get("timed_steps_vs_fp64"),
                       "lambda_err_max_vs_oracle": lam_err.get("timed_steps_vs_oracle")},
            "lambda_err": lam_err, "time_to_all_eigenvalues": time_to_all,
            "speedup_vs_plain_fp64": head.get("speedup_vs_fp64_solves_per_s"),
            "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "kernels": prof, "plain_fp64": plain,
            "other_precision_form": other, "third_precision_form": third, "residual_on_fp64_pipe": fp64res,
            "speedup_tensor_core_residual": (runs["tf32x3_fp64res"][0] / runs["tf32x3"][0]
                                             if "tf32x3_fp64res" in runs else None),
            "clocks": clk, "scattering_poles": scat, "library_lu_comparison": liblu,
        }
        for key in ("tensor", "ir_sweeps_per_node", "ir_fallbacks", "tc_timeouts", "certified", "unverified"):
            if key in head:
                line[key] = head[key]
        print(json.dumps(line))
    P.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
