#!/usr/bin/env python3
"""Benchmark of the Embedded-IPC contact stage on one GB300 (or N replicas).

Workload: the bubble-grasp scene (noisy sphere body of 100,820 triangles in a 1,584-node
cage, squeezed by two ellipsoidal membranes of 40,500 triangles in 2,040-node cages,
dhat = 5e-4 m, kappa = 1e4, lagged friction mu = 0.8) along its 60-iterate closing
trajectory.  One step is one Newton iteration's contact stage, all through the C ABI:
  embed x = J q -> LBVH contact set -> (lagged friction state at each time step's first
  iterate) -> barrier/friction energy, gradient, projected Hessian, reduced by the cage
  embedding into g_r and the BSR H_r -> CCD step bound along the iterate's search step.
Metric: active contact pairs evaluated per second over whole steps; CCD candidate pairs
advanced per second is reported beside it.

Timing: W untimed warm-up steps, then K steps bracketed by barrier + synchronize; each step
is timed on the device with CUDA events on the launching stream, and a 256 MiB buffer is
rewritten between steps (outside the events) so every step starts with a cold L2.
`--impl reference` times the CPU oracle instead (host cores, bounded samples).
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "contact pairs/s (barrier+grad+Hess into subspace)"
UNIT = "pairs/s"
WORKLOAD = "bubble_grasp"

# Algorithmic cost per unit of the kernels the roofline may name:
#  eval_barrier: FP64 flops per contact pair; ccd_advance: FP64 flops per candidate;
#  the rest: DRAM bytes per unit (minimum traffic of the kernel's inputs and outputs).
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 300 for the bubble grasp, so that the clock sampler sees "
                         "the timed region, 20 for the other workloads)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="bubble grasp: skip the other workloads reported beside the headline (sphere on pad, "
                         "plate in rack, exact-Hessian HVP, 256-scene batch vs plain)")
    ap.add_argument("--quick", action="store_true", help="small scene (profiling / smoke)")
    ap.add_argument("--json-out", default="")
    ap.add_argument("--cand-cap", type=int, default=0, help="broad-phase candidate capacity (0: library default)")
    ap.add_argument("--rec-cap", type=int, default=0, help="reduction record capacity (0: library default)")
    ap.add_argument("--profile-once", action="store_true", help="eval_by_type: one evaluation per class (for ncu)")
    ap.add_argument("--workload", choices=["bubble_grasp", "batched", "adjoint", "physical", "eval_by_type"],
                    default="bubble_grasp",
                    help="bubble_grasp: one scene; batched: 256 grasp scenes in one CUDA graph per step; "
                         "adjoint: trajectory gradient of the sphere on a rising pad")
    ap.add_argument("--no-plain", action="store_true", help="batched: skip the plain per-scene comparison")
    ap.add_argument("--retune", action="store_true", help="ignore the autotuner cache")
    ap.add_argument("--no-tune", action="store_true", help="library default launch shapes (no autotuning)")
    ap.add_argument("--solver", choices=["auto", "dense", "pcg"], default="auto", help="physical: linear solver")
    ap.add_argument("--launch-mode", choices=["programmatic", "stream"], default="programmatic",
                    help="kernel launch mode: programmatic dependent launch (default) or plain stream order")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 300 if args.workload == "bubble_grasp" and args.impl == "ours" else 20
    return args


def dist_setup(backend):
    import torch
    import torch.distributed as dist
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    return ws, rank, local


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.window = None          # (t0, t1) wall-clock seconds of the timed region

    def mark(self, t0, t1):
        """Keep only the samples taken between t0 and t1 (time.time() seconds)."""
        self.window = (t0, t1)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return parse_clock_samples(out, self.window)


def parse_clock_samples(text, window=None):
    """Median SM clock, maximum SM clock, active slowdown reasons and sample count from the
    CSV lines of ClockSampler.FIELDS; with window = (t0, t1), only the samples whose
    timestamp lies within 50 ms of [t0, t1] (time.time() seconds) count."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in text.strip().splitlines():
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 10:
            continue
        if window is not None:
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            if not (window[0] - 0.05 <= ts <= window[1] + 0.05):
                continue
        try:
            sm.append(float(f[2])); mx.append(float(f[3]))
        except ValueError:
            continue
        for n, v in zip(names, f[6:10]):
            if v.lower().startswith("active"):
                reasons.add(n)
    if not sm:
        return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"], samples=0)
    return dict(sm_mhz=float(np.median(sm)), sm_max_mhz=float(max(mx)), reasons=sorted(reasons), samples=len(sm))


def across_ranks(total_s, total_pairs, total_cand, ws, device):
    """Whole-job totals of the timed steps: the slowest rank's seconds (the job ends with its
    last rank) and the pairs and candidates of all ranks.  One rank: the values as given."""
    if ws <= 1:
        return total_s, total_pairs, total_cand
    import torch
    import torch.distributed as dist
    tt = torch.tensor([total_s, total_pairs, total_cand], dtype=torch.float64, device=device)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = tt.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1]), float(sm[2])


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# Algorithmic work per unit:
#   eval_barrier  FP64 flops per contact pair, counted by ncu on the bubble-grasp workload
#                 ((2 x DFMA + DMUL + DADD) thread instructions / pairs), the lagged
#                 friction of the pairs that carry it included
#   ccd_advance   FP64 flops per advanced CCD candidate (box test, advancement distances)
#   others        DRAM bytes per unit of their minimum input + output traffic
# eval_barrier: 345.20e6 flops over the 115,699 pairs of bubble-grasp iterate 2 (ncu, the
# autotuned shape 64 threads, 170-register variant); see profiles/
FP64_FLOPS_PER_PAIR = 2983.6
FP64_FLOPS_PER_CCD_CAND = 420.0
# DRAM bytes (read + write) per unit from one ncu capture of the same kernel code and shape
# (eval_barrier: 112.4 MB + 239.7 MB for the same 115,699 pairs)
NCU_TRAFFIC_PER_UNIT = {"eval_barrier": 3043.1}


def query_bytes(sc, n_cand):
    """Minimum DRAM bytes of one traversal launch: every query's padded vertex box once
    (32 B per vertex; edge queries reuse their vertices' boxes, plus 8 B of edge ids), every
    node of both hierarchies once (64 B; the trees are L2-resident after that), and 8 B per
    candidate written."""
    return 32.0 * sc.Nv + 8.0 * sc.E + 64.0 * (2 * sc.F + 2 * sc.E) + 8.0 * n_cand


def roofline_figure(name, total_ms, launches, steps, per_step, sc, fp64_probe=None):
    """Roofline of one kernel from its live event timer: total_ms over `launches` launches in
    `steps` steps.  per_step: units per step -- pairs (contact pairs evaluated), ccd
    (candidates the CCD advanced), cand_contact / cand_ccd (broad-phase candidates of the
    contact and CCD traversals).  FP64 kernels are measured against the FP64 peak derived
    from the unit counts and the maximum clock; fp64_probe (the live DFMA-chain
    measurement) is reported beside it."""
    if launches == 0 or total_ms <= 0:
        return dict(bound=None, achieved=None, peak=None, unit=None, frac=None, traffic=None, kernel=name)
    avg_s = total_ms / 1e3 / launches
    per_step_launches = launches / steps
    hbm, src = measured_peaks()
    if name in ("eval_barrier", "ccd_advance", "eval_kernels"):
        units = (per_step["ccd"] if name == "ccd_advance" else per_step["pairs"]) / per_step_launches
        per = FP64_FLOPS_PER_CCD_CAND if name == "ccd_advance" else FP64_FLOPS_PER_PAIR
        tr = NCU_TRAFFIC_PER_UNIT.get(name)
        if name == "eval_kernels":
            # barrier evaluation (with the friction of the pairs that carry it) and the
            # friction items without a contact pair beside it on a second stream, from the
            # fork to the join; the latter's few flops are not counted
            tr = NCU_TRAFFIC_PER_UNIT["eval_barrier"]
        ach = units * per / avg_s / 1e12
        peak = FP64_PEAK_TFLOPS
        out = dict(bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                   traffic=(tr * units if tr else None), kernel=name, launch_ms=avg_s * 1e3,
                   units_per_launch=units, unit_cost=f"{per:.0f} FP64 flop per unit",
                   peak_source="derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (FP64)")
        if fp64_probe:
            out["peak_probe"] = fp64_probe["tflops"]
            out["frac_of_probe"] = ach / fp64_probe["tflops"]
        return out
    # memory-bound kernels: minimum DRAM bytes per launch
    nv, ne, nf = sc.Nv, sc.E, sc.F
    bytes_model = {
        "bvh_build": 0.5 * (nf + ne) * (24 + 8 + 4 + 4 * 4 * 12 + 64 + 8),
        "bvh_query": (query_bytes(sc, per_step.get("cand_contact", 0.0)) + query_bytes(sc, per_step.get("cand_ccd", 0.0)))
                     / max(per_step_launches, 1.0),
        "narrow_phase": 8 * per_step.get("cand_contact", 0.0) + 20 * per_step["pairs"],
        "pair_sort": 5 * per_step["pairs"] * 24 + 20 * per_step["pairs"],
        "hessian_reduce": 0.0,
        "embed": 32 * nv + 48 * nv,
    }
    b = bytes_model.get(name)
    if not b:
        return dict(bound="hbm", achieved=None, peak=hbm, unit="GB/s", frac=None, traffic=None, kernel=name,
                    launch_ms=avg_s * 1e3)
    ach = b / avg_s / 1e9
    tr = NCU_TRAFFIC_PER_UNIT.get(name)
    out = dict(bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm, traffic=tr, kernel=name,
               launch_ms=avg_s * 1e3, bytes_per_launch=b, peak_source=src)
    if name == "bvh_query":
        out["note"] = ("latency-bound (dependent node fetches; see the ncu summary): the fraction is the minimum "
                       "DRAM bytes over the launch time, a model, not measured traffic")
    return out


def build_scene(quick):
    from paper_2409_16385_gb300 import scenes
    return scenes.make_config(2, small=quick)


# --------------------------------------------------------------------------- CPU oracle

def oracle_sample(sc, t, frac, seed=0):
    """The oracle's whole contact stage at iterate t restricted to a random fraction of
    the query primitives (PT queries: vertices; EE queries: edges): brute-force pairs of
    those queries, lagged friction, evaluation, step bound.  Returns (pairs, seconds,
    ccd candidates)."""
    import oracle
    rng = np.random.default_rng(seed + t)
    qv = np.sort(rng.choice(sc.Nv, max(1, int(frac * sc.Nv)), replace=False)).astype(np.int32)
    qe = np.sort(rng.choice(sc.E, max(1, int(frac * sc.E)), replace=False)).astype(np.int32)
    q, qn = sc.iterate(t), sc.iterate(sc.lag_of(t))
    t0 = time.perf_counter()
    x, xn = oracle.embed(sc, q), oracle.embed(sc, qn)
    def sampled_pairs(xx):
        pv = oracle.pairs_of(sc, xx, 0, qv)
        pe = oracle.pairs_of(sc, xx, 1, qe)
        # an EE pair with both edges among the queries is listed once per side: keep one
        ee = np.unique(np.stack([pe["i"], pe["j"]], 1), axis=0).reshape(-1, 2)
        return dict(type=np.concatenate([np.zeros(len(pv["i"]), np.int32), np.ones(len(ee), np.int32)]),
                    i=np.concatenate([pv["i"], ee[:, 0]]).astype(np.int32),
                    j=np.concatenate([pv["j"], ee[:, 1]]).astype(np.int32))

    prs = sampled_pairs(x)
    prn = sampled_pairs(xn)
    lag = oracle.friction_lag(sc, xn, prn)
    oracle.eval_contact(sc, x, prs, lag)
    dx = oracle.embed(sc, sc.dq(t), displacement=True)
    a1 = oracle.accd_of(sc, x, dx, 0, qv)
    a2 = oracle.accd_of(sc, x, dx, 1, qe)
    dt = time.perf_counter() - t0
    return len(prs["type"]), dt, a1["n_candidates"] + a2["n_candidates"]


def _subset(d, idx):
    return {k: np.asarray(v)[idx] for k, v in d.items()}


def swept_overlap(sc, x, dx, cand):
    """Mask of the candidates whose closed FP64 swept boxes over [x, x + dx] overlap (the
    CCD's exact box test), for host arrays x, dx [Nv,3] and cand = (type, i, j)."""
    ct, ci, cj = (np.asarray(a) for a in (cand["type"], cand["i"], cand["j"]))
    st = np.zeros((len(ct), 4), np.int64)
    pt = ct == 0
    st[pt] = np.c_[ci[pt], np.asarray(sc.tris)[cj[pt]]]
    st[~pt] = np.c_[np.asarray(sc.edges)[ci[~pt]], np.asarray(sc.edges)[cj[~pt]]]
    p0, p1 = x[st], x[st] + dx[st]
    lo, hi = np.minimum(p0, p1), np.maximum(p0, p1)
    side_a = np.arange(4)[None, :] < np.where(pt, 1, 2)[:, None]
    loA = np.where(side_a[..., None], lo, np.inf).min(1)
    hiA = np.where(side_a[..., None], hi, -np.inf).max(1)
    loB = np.where(~side_a[..., None], lo, np.inf).min(1)
    hiB = np.where(~side_a[..., None], hi, -np.inf).max(1)
    return ~((loA > hiB) | (loB > hiA)).any(1)


def cpu_stage_baseline(sc, x, xn, dx, pairs, pairs_n, cand, budget_s=8.0, seed=0):
    """The oracle's two timed stages on the lists the GPU used, on all host cores and on
    one core:
      eval: barrier + lagged friction energy, gradient and projected Hessian reduced into
            g_r and H_r (oracle.eval_contact) over the contact pairs `pairs` and the lag
            state of `pairs_n` at xn -- pairs/s;
      ccd:  conservative advancement over the candidates whose swept boxes overlap
            (oracle.accd_list over `cand`) -- queries/s.
    Each stage runs on the whole list when it fits in about budget_s seconds, else on a
    seeded random subset (the same fraction of the friction pairs as of the contact pairs),
    sized by a first run on up to 2,000 entries."""
    import oracle
    oracle.build()
    lag = oracle.friction_lag(sc, xn, pairs_n)
    n_all = oracle.num_threads()
    rng = np.random.default_rng(seed)
    P, L, C = len(pairs["type"]), len(lag["lam"]), len(cand["type"])
    res = {}

    def run_eval(m):
        ip = np.arange(P) if m >= P else np.sort(rng.choice(P, m, replace=False))
        il = np.arange(L) if m >= P else np.sort(rng.choice(L, min(L, int(round(m * L / max(P, 1)))), replace=False))
        sp, sl = _subset(pairs, ip), _subset(lag, il)
        t0 = time.perf_counter()
        oracle.eval_contact(sc, x, sp, sl)
        return len(ip), len(il), time.perf_counter() - t0

    def run_ccd(m, repeat=1):
        ic = np.arange(C) if m >= C else np.sort(rng.choice(C, m, replace=False))
        sub = _subset(cand, ic)
        t0 = time.perf_counter()
        for _ in range(repeat):
            oracle.accd_list(sc, x, dx, sub)
        return len(ic) * repeat, time.perf_counter() - t0

    try:
        for label, threads in (("all", n_all), ("1core", 1)):
            oracle.set_threads(threads)
            if P:
                m0, _, t0 = run_eval(min(P, 2000))
                n, nl, dt = run_eval(min(P, max(m0, int(m0 * budget_s / max(t0, 1e-6)))))
                res[f"eval_{label}"] = dict(value=n / dt, pairs=n, friction_pairs=nl, seconds=dt, threads=threads,
                                            list_pairs=P, list_friction_pairs=L)
            if C:
                # the whole list, repeated until about budget_s / 2 has passed (most
                # candidates settle at their first advancement, so one pass is short)
                m0, t0 = run_ccd(min(C, 2000))
                m = min(C, max(m0, int(m0 * budget_s / 2 / max(t0, 1e-6))))
                n1, t1 = run_ccd(m)
                rep = max(1, int(budget_s / 2 / max(t1, 1e-6))) if m >= C else 1
                n, dt = run_ccd(m, rep) if rep > 1 else (n1, t1)
                res[f"ccd_{label}"] = dict(value=n / dt, queries=n, seconds=dt, threads=threads, list_queries=C,
                                           passes=rep)
    finally:
        oracle.set_threads(n_all)
    return res


def cpu_enumeration(sc, x, n_queries=400, seed=0):
    """The oracle's brute-force O(n^2) contact-pair enumeration, timed apart (it is the
    definition of the pair set, not a fair baseline for the LBVH): n_queries vertex queries
    against every triangle and n_queries edge queries against every edge, and the time a
    whole-scene enumeration would take at that rate."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    qv = np.sort(rng.choice(sc.Nv, min(n_queries, sc.Nv), replace=False)).astype(np.int32)
    qe = np.sort(rng.choice(sc.E, min(n_queries, sc.E), replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    pv = oracle.pairs_of(sc, x, 0, qv)
    t1 = time.perf_counter()
    pe = oracle.pairs_of(sc, x, 1, qe)
    t2 = time.perf_counter()
    full = (t1 - t0) * sc.Nv / len(qv) + (t2 - t1) * sc.E / len(qe)
    return dict(vertex_queries=int(len(qv)), edge_queries=int(len(qe)), pairs_found=int(len(pv["i"]) + len(pe["i"])),
                seconds=t2 - t0, full_enumeration_s_estimate=full, cores=oracle.num_threads(),
                kind="oracle brute force (not a baseline: the definition of the pair set)")


def reference_list(sc, t, frac, seed):
    """The oracle's own contact list at iterate t for a seeded random fraction of the query
    primitives (brute force), its lagged list, and the positions: the input of one
    reference step."""
    import oracle
    rng = np.random.default_rng(seed + t)
    qv = np.sort(rng.choice(sc.Nv, max(1, int(frac * sc.Nv)), replace=False)).astype(np.int32)
    qe = np.sort(rng.choice(sc.E, max(1, int(frac * sc.E)), replace=False)).astype(np.int32)
    x, xn = oracle.embed(sc, sc.iterate(t)), oracle.embed(sc, sc.iterate(sc.lag_of(t)))

    def sampled_pairs(xx):
        pv = oracle.pairs_of(sc, xx, 0, qv)
        pe = oracle.pairs_of(sc, xx, 1, qe)
        ee = np.unique(np.stack([pe["i"], pe["j"]], 1), axis=0).reshape(-1, 2)
        return dict(type=np.concatenate([np.zeros(len(pv["i"]), np.int32), np.ones(len(ee), np.int32)]),
                    i=np.concatenate([pv["i"], ee[:, 0]]).astype(np.int32),
                    j=np.concatenate([pv["j"], ee[:, 1]]).astype(np.int32))

    prs = sampled_pairs(x)
    lag = oracle.friction_lag(sc, xn, sampled_pairs(xn))
    return x, prs, lag


def run_reference(args, ws, rank):
    """`--impl reference`: the CPU oracle as it stands, on the host cores.  A step is the
    oracle's evaluation stage (barrier + lagged friction energy, gradient and projected
    Hessian reduced into the subspace: the metric's own stage) over the contact list of one
    iterate.  The lists come from the oracle's own brute-force enumeration for a seeded
    fraction of the query primitives, found before the timed steps (untimed; their time is
    reported as enumeration_s)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    if ws > 1:
        # the launcher sets OMP_NUM_THREADS=1 for every rank; only this rank works, so the
        # oracle takes every host core it may run on, as in a one-process run
        oracle.set_threads(len(os.sched_getaffinity(0)))
    sc = build_scene(args.quick)
    # the enumeration fraction: about 30 s of brute force per list, calibrated on 1/2000
    t_cal = time.perf_counter()
    reference_list(sc, 0, 5e-4, seed=999)
    t_cal = time.perf_counter() - t_cal
    frac = 1.0 if args.quick else min(1.0 / 12, 5e-4 * 30.0 / max(t_cal, 1e-3))
    its = [sc.lag_of(5), sc.lag_of(5) + 1 if sc.lag_of(5) + 1 < sc.n_iterates else sc.lag_of(5)]
    t_en = time.perf_counter()
    lists = [reference_list(sc, t, frac, seed=7) for t in its]
    t_en = time.perf_counter() - t_en
    for k in range(args.warmup):
        x, prs, lag = lists[k % len(lists)]
        oracle.eval_contact(sc, x, prs, lag)
    pairs = 0; secs = 0.0
    for k in range(args.steps):
        x, prs, lag = lists[k % len(lists)]
        t0 = time.perf_counter()
        oracle.eval_contact(sc, x, prs, lag)
        secs += time.perf_counter() - t0
        pairs += len(prs["type"])
    v = pairs / secs if secs > 0 else 0.0
    cores = oracle.num_threads()
    sample = (f"per step: the oracle's evaluation stage over the contact pairs (and lagged friction pairs) of one "
              f"iterate ({', '.join(str(t) for t in its)}, alternating) found by its own brute force for a "
              f"{frac:.4f} fraction of the vertices and edges as queries; enumeration untimed ({t_en:.1f} s)")
    line = dict(metric=METRIC, value=v, unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * secs / max(1, args.steps), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic (seeded)", impl="reference",
                config=dict(workload=WORKLOAD + ("_small" if args.quick else ""), iterates=sc.n_iterates,
                            l2="n/a (host)", pairs_per_step=pairs / max(1, args.steps)),
                cpu_baseline=dict(value=v, unit=UNIT, cores=cores, kind="oracle", sample=sample),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0),
                enumeration_s=t_en)
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU arm

def pair_split(sc, h):
    """Contact pairs between two bodies and pairs inside one body (self-contact, mostly
    rest-state neighbours when dhat is near the edge length)."""
    body = np.asarray(sc.body)
    t, i, j = (np.asarray(h[k]) for k in ("type", "i", "j"))
    tris, edges = np.asarray(sc.tris), np.asarray(sc.edges)
    va = np.where(t == 0, i, 0)
    vb = np.zeros_like(va)
    pt = t == 0
    vb[pt] = tris[j[pt], 0]
    va[~pt] = edges[i[~pt], 0]
    vb[~pt] = edges[j[~pt], 0]
    inter = body[va] != body[vb]
    return dict(inter_body=int(inter.sum()), intra_body=int((~inter).sum()))


PAIR_CLASSES = ("pt_face", "pt_edge", "pt_vertex", "ee_interior", "ee_edge", "ee_vertex")


def _seg_param(p, e0, e1):
    """Closest-point parameter t in [0, 1] of points p on segments e0 -> e1 and the squared
    distance (vectorised)."""
    e, w = e1 - e0, p - e0
    ee = np.einsum("ij,ij->i", e, e)
    t = np.clip(np.einsum("ij,ij->i", w, e) / np.where(ee > 0, ee, 1.0), 0.0, 1.0)
    r = w - e * t[:, None]
    return t, np.einsum("ij,ij->i", r, r)


def classify_pairs(sc, x, h):
    """Closest-feature class of each contact pair (index into PAIR_CLASSES) and its number
    of distinct cage nodes: the minimum of the distance over the closed primitives is
    attained inside the face / on an edge interior / at a vertex (point-triangle), or at
    interior points of both edges / an endpoint against an edge interior / two endpoints
    (edge-edge).  Host-side numpy, for reporting work per pair type."""
    t, i, j = (np.asarray(h[k]) for k in ("type", "i", "j"))
    tris, edges = np.asarray(sc.tris), np.asarray(sc.edges)
    cls = np.zeros(len(t), np.int32)
    st = np.zeros((len(t), 4), np.int64)
    pt = t == 0
    st[pt] = np.c_[i[pt], tris[j[pt]]]
    st[~pt] = np.c_[edges[i[~pt]], edges[j[~pt]]]
    if pt.any():
        p, a, b, c = (x[st[pt, k]] for k in range(4))
        e1, e2, w = b - a, c - a, p - a
        n = np.cross(e1, e2)
        nn = np.einsum("ij,ij->i", n, n)
        b1 = np.einsum("ij,ij->i", np.cross(w, e2), n) / nn
        b2 = np.einsum("ij,ij->i", np.cross(e1, w), n) / nn
        face = (b1 >= 0) & (b2 >= 0) & (b1 + b2 <= 1)
        segs = [_seg_param(p, a, b), _seg_param(p, b, c), _seg_param(p, c, a)]
        d2 = np.stack([s_[1] for s_ in segs], 1)
        tt = np.stack([s_[0] for s_ in segs], 1)
        kbest = np.argmin(d2, 1)
        tb = tt[np.arange(len(kbest)), kbest]
        inner = (tb > 0) & (tb < 1)
        cls[pt] = np.where(face, 0, np.where(inner, 1, 2))
    if (~pt).any():
        a0, a1, b0, b1_ = (x[st[~pt, k]] for k in range(4))
        ea, eb, w = a1 - a0, b1_ - b0, a0 - b0
        A = np.einsum("ij,ij->i", ea, ea); B = np.einsum("ij,ij->i", ea, eb); C = np.einsum("ij,ij->i", eb, eb)
        D = np.einsum("ij,ij->i", ea, w); E = np.einsum("ij,ij->i", eb, w)
        n = np.cross(ea, eb)
        nn = np.einsum("ij,ij->i", n, n)
        ok = nn > 1e-20 * A * C
        nns = np.where(ok, nn, 1.0)
        s_ = (B * E - C * D) / nns
        t_ = (A * E - B * D) / nns
        interior = ok & (s_ >= 0) & (s_ <= 1) & (t_ >= 0) & (t_ <= 1)
        segs = [_seg_param(a0, b0, b1_), _seg_param(a1, b0, b1_), _seg_param(b0, a0, a1), _seg_param(b1_, a0, a1)]
        d2 = np.stack([q[1] for q in segs], 1)
        tt = np.stack([q[0] for q in segs], 1)
        kbest = np.argmin(d2, 1)
        tb = tt[np.arange(len(kbest)), kbest]
        inner = (tb > 0) & (tb < 1)
        cls[~pt] = np.where(interior, 3, np.where(inner, 4, 5))
    ci = np.asarray(sc.cage_idx)[st]                       # [n, 4 vertices, 4 nodes]
    nodes = np.array([len({int(v) for v in row.ravel() if v >= 0}) for row in ci])
    return cls, nodes


def run_eval_by_type(args, ws, rank, local):
    """The barrier evaluation stage on the bubble grasp's contact pairs split by closest-
    feature class (PAIR_CLASSES): one list per class, evaluated without friction; device
    time per class from the kernel's event timer.  With --profile-once each class is
    evaluated exactly once, in PAIR_CLASSES order, so that an ncu launch list of
    k_eval_barrier gives each class's FP64 instruction counts (launch k = class k)."""
    import torch
    from paper_2409_16385_gb300 import ContactScene, PairList
    dev = torch.device("cuda", local)
    sc = build_scene(args.quick)
    cs = ContactScene(sc, pair_capacity=1 << 21, bsr_capacity=1 << 21)
    t0 = 5 % sc.n_iterates
    q = torch.tensor(sc.iterate(t0), dtype=torch.float64, device=dev)
    h = cs.build_candidates(q).host()
    cls, nodes = classify_pairs(sc, cs.embed(q).cpu().numpy(), h)
    out = {}
    reps = 1 if args.profile_once else 10
    for c, name in enumerate(PAIR_CLASSES):
        sel = np.nonzero(cls == c)[0]
        if len(sel) == 0:
            continue
        m = len(sel)
        pl = PairList(torch.tensor(h["type"][sel], dtype=torch.int32, device=dev),
                      torch.tensor(h["i"][sel], dtype=torch.int32, device=dev),
                      torch.tensor(h["j"][sel], dtype=torch.int32, device=dev),
                      torch.zeros(m, dtype=torch.float64, device=dev),
                      torch.tensor([m], dtype=torch.int64, device=dev))
        if not args.profile_once:
            cs.eval_contact(q, pl, None)
        cs.timing_enable(["eval_barrier"])
        for _ in range(reps):
            cs.eval_contact(q, pl, None)
        torch.cuda.synchronize()
        ms, n_l = cs.timing_read().get("eval_barrier", (0.0, 0))
        cs.timing_enable([])
        out[name] = dict(pairs=m, mean_cage_nodes=float(nodes[sel].mean()), kernel_ms=ms / max(n_l, 1),
                         pairs_per_s=m / (ms / max(n_l, 1) / 1e3) if ms > 0 else None)
    st = cs.status()
    cs.close()
    if st["flags"] & ~64:
        raise RuntimeError(f"eval by type: device status {st}")
    line = dict(workload=sc.name, iterate=t0, classes=out, reps=reps,
                note="k_eval_barrier time per class (no friction items); FP64 instruction counts per class "
                     "come from an ncu launch list of the --profile-once run")
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_ours(args, ws, rank, local):
    import torch
    import torch.distributed as dist
    from paper_2409_16385_gb300 import ContactScene, binding

    dev = torch.device("cuda", local)
    sc = build_scene(args.quick)
    n_it = sc.n_iterates
    cs = ContactScene(sc, pair_capacity=1 << 21, bsr_capacity=1 << 21, cand_capacity=args.cand_cap,
                      rec_capacity=args.rec_cap)
    lib = binding.load()
    # the device's FP64 rate, measured first, on an idle GPU
    fp64 = binding.fp64_peak()
    Q = torch.tensor(np.stack([sc.iterate(t) for t in range(n_it)]), dtype=torch.float64, device=dev)
    DQ = torch.tensor(np.stack([sc.dq(t) for t in range(n_it)]), dtype=torch.float64, device=dev)
    lag_of = [sc.lag_of(t) for t in range(n_it)]
    pairs = cs.new_pairs()
    lag = cs.new_lag()
    H = cs.new_bsr()
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.zeros((sc.Ns, 3), dtype=torch.float64, device=dev)
    x = torch.empty((sc.Nv, 3), dtype=torch.float64, device=dev)
    dx = torch.empty((sc.Nv, 3), dtype=torch.float64, device=dev)
    alpha = torch.zeros(1, dtype=torch.float64, device=dev)
    ncand = torch.zeros(1, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(t, q, dq):
        if lag_of[t] == t:
            cs.build_candidates(q, out=pairs)
            cs.friction_lag(q, pairs, out=lag)
        else:
            cs.build_candidates(q, out=pairs)
        cs.eval_contact(q, pairs, lag, E=E, g_r=g, H=H)
        cs.embed(q, out=x)
        cs.embed(dq, out=dx, displacement=True)
        cs.accd_toi(x, dx, alpha=alpha, n_candidates=ncand)

    # the lag state of the first timed iterates comes from its time step's first iterate
    t0 = args.warmup % n_it
    first = lag_of[t0]
    cs.build_candidates(Q[first], out=pairs)
    cs.friction_lag(Q[first], pairs, out=lag)

    # launch shapes from the autotuner (cached per device and workload)
    tuned = {}
    if not args.no_tune:
        from paper_2409_16385_gb300 import autotune
        tuned = autotune.tune(cs, lambda: step(t0, Q[t0], DQ[t0]), WORKLOAD + ("_small" if args.quick else ""),
                              force=args.retune)
        cs.build_candidates(Q[first], out=pairs)
        cs.friction_lag(Q[first], pairs, out=lag)

    # warm-up with every kernel timer on: the three largest kernels are then timed inside
    # the timed steps, and the largest of them there is the roofline's kernel
    cs.timing_enable(None)
    start_t = (t0 - args.warmup) % n_it
    for k in range(args.warmup):
        t = (start_t + k) % n_it
        if k == 0 and lag_of[t] != t:
            cs.build_candidates(Q[lag_of[t]], out=pairs)
            cs.friction_lag(Q[lag_of[t]], pairs, out=lag)
        step(t, Q[t], DQ[t])
    torch.cuda.synchronize()
    warm = cs.timing_read()
    # the barrier and friction kernels run inside eval_kernels' span (the friction kernel on
    # a second stream, its own span stretched by the barrier kernel beside it).  Timed inside
    # the timed steps: the largest of the other timers and eval_barrier (for its own
    # roofline); no more, since every timer's events sit between two launches of the stream
    # and cut their programmatic overlap
    ranked = sorted((k for k in warm if k not in ("eval_barrier", "eval_friction")), key=lambda k: -warm[k][0])
    timed = ranked[:1] + ["eval_barrier"]
    cs.timing_enable(timed)
    st = cs.status()
    if st["flags"] & ~64:
        raise RuntimeError(f"device status after warm-up: {st}")

    K = args.steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    counts = torch.zeros((K, 2), dtype=torch.int64, device=dev)
    clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    launches0 = lib.eipc_launch_count()
    clocks.start()
    time.sleep(0.3)                  # the sampler is running before the timed region starts
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    tw0 = time.time()
    wall0 = time.perf_counter()
    for k in range(K):
        t = (t0 + k) % n_it
        flush.zero_()
        evs[k][0].record(stream)
        step(t, Q[t], DQ[t])
        evs[k][1].record(stream)
        counts[k, 0].copy_(pairs.count[0])
        counts[k, 1].copy_(ncand[0])
    torch.cuda.synchronize()
    tw1 = time.time()
    wall = time.perf_counter() - wall0
    if ws > 1:
        dist.barrier()
    clocks.mark(tw0, tw1)
    clk = clocks.stop()
    launches = lib.eipc_launch_count() - launches0
    step_ms = np.array([a.elapsed_time(b) for a, b in evs])
    cnt = counts.cpu().numpy()
    kt = cs.timing_read()
    st = cs.status()
    if st["flags"] & ~64:
        raise RuntimeError(f"device status after the timed steps: {st}")
    total_s = step_ms.sum() / 1e3
    total_pairs = float(cnt[:, 0].sum())
    total_cand = float(cnt[:, 1].sum())
    total_s_all, total_pairs_all, total_cand_all = across_ranks(total_s, total_pairs, total_cand, ws, dev)
    value = total_pairs_all / total_s_all
    dominant = max(timed, key=lambda k: kt.get(k, (0.0, 0))[0])
    kernel_ms_timed = {k: dict(ms_per_step=kt.get(k, (0.0, 0))[0] / K, launches_per_step=kt.get(k, (0.0, 0))[1] / K)
                       for k in timed}

    # ---- stage-only throughputs (same iterates, pairs precomputed); the broad-phase
    # candidate counts of both traversals per iterate, for the traversal's bytes
    stage = {}
    cs.timing_enable([])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev_ms = 0.0; n_p = 0
    cand_contact = []
    fric_items = []
    for k in range(K):
        t = (t0 + k) % n_it
        cs.build_candidates(Q[t], out=pairs)
        cand_contact.append(cs.work_counts()["candidates"])
        n_p += int(pairs.count.item())
        flush.zero_()
        ev0.record(stream)
        cs.eval_contact(Q[t], pairs, lag, E=E, g_r=g, H=H)
        ev1.record(stream)
        torch.cuda.synchronize()
        ev_ms += ev0.elapsed_time(ev1)
        wk = cs.work_counts()
        fric_items.append(wk["items"] - wk["pairs"])
    stage["eval_pairs_per_s"] = n_p / (ev_ms / 1e3)
    work = cs.work_counts()          # the last iterate's contact build and evaluation
    work.update(pair_split(sc, pairs.host()))
    ac_ms = 0.0; n_c = 0
    cand_ccd = []
    for k in range(K):
        t = (t0 + k) % n_it
        cs.embed(Q[t], out=x)
        cs.embed(DQ[t], out=dx, displacement=True)
        flush.zero_()
        ev0.record(stream)
        cs.accd_toi(x, dx, alpha=alpha, n_candidates=ncand)
        ev1.record(stream)
        torch.cuda.synchronize()
        ac_ms += ev0.elapsed_time(ev1)
        n_c += int(ncand.item())
        cand_ccd.append(cs.work_counts()["candidates"])
    stage["ccd_queries_per_s"] = n_c / (ac_ms / 1e3)
    stage["ccd_queries_per_s_in_step"] = total_cand / total_s
    if ws == 1:
        stage["graph_replay"] = graph_steps(sc, Q, DQ, lag_of, t0, K, flush, dev,
                                            {k: v["shape"] for k, v in tuned.items()})
    wc = cs.work_counts()
    work["ccd_candidates"], work["ccd_advanced"] = wc["candidates"], wc["ccd_advanced"]

    # ---- rooflines: every kernel timed inside the timed steps; the headline is the one
    # with the largest time there
    per_step = dict(pairs=total_pairs / K, ccd=total_cand / K, cand_contact=float(np.mean(cand_contact)),
                    cand_ccd=float(np.mean(cand_ccd)), friction_items=float(np.mean(fric_items)))
    roofs = {k: roofline_figure(k, *kt.get(k, (0.0, 0)), K, per_step, sc, fp64) for k in timed}
    roof = dict(roofs[dominant])
    roof["chosen_by"] = "largest device time inside the timed steps (per-kernel CUDA events on the launching stream)"

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(cs, sc, Q, DQ, lag_of, t0, K, flush, dev)

    # ---- CPU baselines (rank 0, one GPU only): the oracle's stages on the GPU's own lists
    cpu, cpu_more = None, {}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        tl = lag_of[t0]
        pn = cs.build_candidates(Q[tl], out=cs.new_pairs()).host()
        pr = cs.build_candidates(Q[t0], out=cs.new_pairs()).host()
        cs.accd_toi(cs.embed(Q[t0]), cs.embed(DQ[t0], displacement=True))
        cand = dict(zip(("type", "i", "j"), (a.cpu().numpy() for a in cs.candidates())))
        xo, xno = oracle.embed(sc, sc.iterate(t0)), oracle.embed(sc, sc.iterate(tl))
        dxo = oracle.embed(sc, sc.dq(t0), displacement=True)
        cand = _subset(cand, np.nonzero(swept_overlap(sc, xo, dxo, cand))[0])
        pl = lambda h: dict(type=h["type"], i=h["i"], j=h["j"])
        stg = cpu_stage_baseline(sc, xo, xno, dxo, pl(pr), pl(pn), cand, budget_s=1.0 if args.quick else 8.0)
        cores = oracle.num_threads()

        def entry(key, unit, what):
            r = stg.get(key)
            if r is None:
                return None
            n = r.get("pairs", r.get("queries"))
            of = r.get("list_pairs", r.get("list_queries"))
            reps = f" ({r['passes']} passes over it)" if r.get("passes", 1) > 1 else ""
            return dict(value=r["value"], unit=unit, cores=r["threads"], kind="oracle",
                        sample=f"iterate {t0}, {what}: {n // r.get('passes', 1)} of the GPU's {of}{reps} "
                               f"in {r['seconds']:.2f} s")

        cpu = entry("eval_all", UNIT, "evaluation stage (barrier + lagged friction, gradient, projected Hessian, "
                                      "reduction) over the GPU's contact and lagged pair lists")
        cpu_more = dict(
            cpu_baseline_1core=entry("eval_1core", UNIT, "the same evaluation stage on one core"),
            cpu_baseline_ccd=entry("ccd_all", "queries/s", "CCD advancement over the GPU's candidates whose swept "
                                                           "boxes overlap"),
            cpu_baseline_ccd_1core=entry("ccd_1core", "queries/s", "the same CCD stage on one core"),
            cpu_enumeration=cpu_enumeration(sc, xo))
        if cpu is not None:
            cpu["host_cores"] = cores

    # ---- the other workloads, reported beside the headline (one GPU only)
    extras = {}
    if ws == 1 and not args.no_extras:
        extras["adjoint_hvp"] = dict(workload=WORKLOAD, **hvp_stage(cs, sc, Q, lag_of, t0, min(K, 30), flush, dev))
        cs.close()
        extras["sphere_on_pad"] = bench_sphere_on_pad(dev)
        extras["plate_in_rack"] = bench_plate_in_rack(args, dev, fp64)
        extras["batched_vs_plain"] = batched_summary(args, ws, rank, local)

    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=K, warmup=args.warmup,
                ms_per_step=float(step_ms.mean()), higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic (seeded)",
                config=dict(workload=WORKLOAD + ("_small" if args.quick else ""), iterates=n_it,
                            triangles=sc.F, vertices=sc.Nv, edges=sc.E, cage_nodes=sc.Ns,
                            dhat=sc.params["dhat"], mu=sc.params["mu"], parallelism=f"replicas x{ws}",
                            l2="flushed between steps (256 MiB rewrite)", launch_mode=args.launch_mode,
                            pairs_per_step=total_pairs / K, ccd_candidates_per_step=total_cand / K,
                            broad_phase_candidates_per_step=dict(contact=per_step["cand_contact"],
                                                                 ccd=per_step["cand_ccd"]),
                            work_last_iterate=work),
                clocks=clk, gpu_launches=int(launches), wall_s=wall, roofline=roof, rooflines=roofs,
                fp64_probe=fp64, kernel_ms_timed=kernel_ms_timed,
                ccd_queries_per_s=total_cand_all / total_s_all, stages=stage,
                e2e=e2e, cpu_baseline=cpu, **cpu_more, kernel_ms_warmup={k: v[0] for k, v in warm.items()},
                autotune={k: dict(shape=v["shape"], ms=v["ms"], default_ms=v["default_ms"], cached=v["cached"])
                          for k, v in tuned.items()},
                **extras)
    if rank == 0:
        print(json.dumps(line), flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                json.dump(line, f, indent=1)
    if not extras:
        cs.close()


def bench_sphere_on_pad(dev, warmup=10, calls=50):
    """Latency of the sphere-on-pad scene (a few hundred pairs): median over `calls` calls,
    after `warmup`, of the whole contact stage and of its parts, each call timed with CUDA
    events and the L2 flushed before it."""
    import torch
    from paper_2409_16385_gb300 import ContactScene, scenes
    sc = scenes.make_config(1)
    cs = ContactScene(sc, pair_capacity=1 << 16, bsr_capacity=1 << 18)
    q = torch.tensor(sc.iterate(0), dtype=torch.float64, device=dev)
    dq = torch.tensor(sc.dq(0), dtype=torch.float64, device=dev)
    pairs, H = cs.new_pairs(), cs.new_bsr()
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.zeros((sc.Ns, 3), dtype=torch.float64, device=dev)
    x = torch.empty((sc.Nv, 3), dtype=torch.float64, device=dev)
    dx = torch.empty_like(x)
    alpha = torch.zeros(1, dtype=torch.float64, device=dev)
    lag = cs.friction_lag(q, cs.build_candidates(q, out=pairs))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    parts = {
        "build_candidates": lambda: cs.build_candidates(q, out=pairs),
        "eval_contact": lambda: cs.eval_contact(q, pairs, lag, E=E, g_r=g, H=H),
        "accd_toi": lambda: (cs.embed(q, out=x), cs.embed(dq, out=dx, displacement=True), cs.accd_toi(x, dx, alpha=alpha)),
    }
    parts["whole_stage"] = lambda: (parts["build_candidates"](), parts["eval_contact"](), parts["accd_toi"]())
    stream = torch.cuda.current_stream()
    out = {}
    for name, fn in parts.items():
        for _ in range(warmup):
            fn()
        ms = []
        for _ in range(calls):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        out[name] = float(np.median(ms))
    n = int(pairs.count.item())
    st = cs.status()
    cs.close()
    if st["flags"] & ~64:
        raise RuntimeError(f"sphere on pad: device status {st}")
    return dict(workload=sc.name, triangles=sc.F, vertices=sc.Nv, cage_nodes=sc.Ns, pairs=n,
                median_ms=out, calls=calls, warmup=warmup, pairs_per_s=n / (out["whole_stage"] / 1e3),
                timing="CUDA events per call, L2 flushed before each call")


def bench_plate_in_rack(args, dev, fp64=None):
    """The plate-in-rack scene (Sec. IV-B stand-in; many near-parallel edge-edge pairs) over
    its 100 lowering iterates, one step = one Newton iteration's contact stage as in the
    headline: pairs/s over whole steps, the evaluation kernel's FP64 roofline."""
    import torch
    from paper_2409_16385_gb300 import ContactScene, scenes
    sc = scenes.make_config(3, small=args.quick)
    n_it = sc.n_iterates
    cs = ContactScene(sc, pair_capacity=1 << 21, bsr_capacity=1 << 21)
    Q = torch.tensor(np.stack([sc.iterate(t) for t in range(n_it)]), dtype=torch.float64, device=dev)
    DQ = torch.tensor(np.stack([sc.dq(t) for t in range(n_it)]), dtype=torch.float64, device=dev)
    lag_of = [sc.lag_of(t) for t in range(n_it)]
    pairs, lag, H = cs.new_pairs(), cs.new_lag(), cs.new_bsr()
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.zeros((sc.Ns, 3), dtype=torch.float64, device=dev)
    x = torch.empty((sc.Nv, 3), dtype=torch.float64, device=dev)
    dx = torch.empty_like(x)
    alpha = torch.zeros(1, dtype=torch.float64, device=dev)
    nc = torch.zeros(1, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(t):
        cs.build_candidates(Q[t], out=pairs)
        if lag_of[t] == t:
            cs.friction_lag(Q[t], pairs, out=lag)
        cs.eval_contact(Q[t], pairs, lag, E=E, g_r=g, H=H)
        cs.embed(Q[t], out=x)
        cs.embed(DQ[t], out=dx, displacement=True)
        cs.accd_toi(x, dx, alpha=alpha, n_candidates=nc)

    cs.friction_lag(Q[lag_of[0]], cs.build_candidates(Q[lag_of[0]], out=pairs), out=lag)
    for t in range(min(5, n_it)):
        step(t)
    torch.cuda.synchronize()
    cs.timing_enable(["eval_barrier"])
    ms, np_, nq = [], 0, 0
    for t in range(n_it):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(t)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        np_ += int(pairs.count.item())
        nq += int(nc.item())
    kt = cs.timing_read()
    work = cs.work_counts()
    work.update(pair_split(sc, pairs.host()))
    st = cs.status()
    cs.close()
    if st["flags"] & ~64:
        raise RuntimeError(f"plate in rack: device status {st}")
    total_s = float(np.sum(ms)) / 1e3
    per_step = dict(pairs=np_ / n_it, ccd=nq / n_it)
    roof = roofline_figure("eval_barrier", *kt.get("eval_barrier", (0.0, 0)), n_it, per_step, sc, fp64)
    return dict(workload=sc.name, triangles=sc.F, vertices=sc.Nv, cage_nodes=sc.Ns, iterates=n_it,
                value=np_ / total_s, unit=UNIT, ms_per_step=float(np.mean(ms)), pairs_per_step=np_ / n_it,
                ccd_queries_per_s=nq / total_s, roofline_eval_barrier=roof, work_last_iterate=work,
                timing="every iterate once, CUDA events per step, L2 flushed before each")


def run_e2e(cs, sc, Q, DQ, lag_of, t0, K, flush, dev):
    """Same steps through the public API with pinned host buffers: every step copies q and
    dq in, runs the stage and reads E, g_r, alpha and the BSR Hessian back."""
    import torch
    n_it = sc.n_iterates
    qh = [Q[t].cpu().pin_memory() for t in range(n_it)]
    dqh = [DQ[t].cpu().pin_memory() for t in range(n_it)]
    q = torch.empty_like(Q[0]); dq = torch.empty_like(DQ[0])
    pairs, lag, H = cs.new_pairs(), cs.new_lag(), cs.new_bsr()
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.zeros((sc.Ns, 3), dtype=torch.float64, device=dev)
    x = torch.empty((sc.Nv, 3), dtype=torch.float64, device=dev)
    dx = torch.empty_like(x)
    alpha = torch.zeros(1, dtype=torch.float64, device=dev)
    Eh = torch.zeros(1, dtype=torch.float64).pin_memory()
    gh = torch.zeros((sc.Ns, 3), dtype=torch.float64).pin_memory()
    ah = torch.zeros(1, dtype=torch.float64).pin_memory()
    nh = torch.zeros(1, dtype=torch.int64).pin_memory()
    rph = torch.zeros(sc.Ns + 1, dtype=torch.int32).pin_memory()
    colh = torch.zeros(H.col.shape[0], dtype=torch.int32).pin_memory()
    valh = torch.zeros(H.val.shape, dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream()
    first = lag_of[t0]
    q.copy_(qh[first], non_blocking=True)
    cs.build_candidates(q, out=pairs)
    cs.friction_lag(q, pairs, out=lag)
    torch.cuda.synchronize()
    tot_ms, tot_pairs, bi, bo = 0.0, 0, 0, 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(K):
        t = (t0 + k) % n_it
        flush.zero_()
        ev0.record(stream)
        q.copy_(qh[t], non_blocking=True)
        dq.copy_(dqh[t], non_blocking=True)
        cs.build_candidates(q, out=pairs)
        if lag_of[t] == t:
            cs.friction_lag(q, pairs, out=lag)
        cs.eval_contact(q, pairs, lag, E=E, g_r=g, H=H)
        cs.embed(q, out=x)
        cs.embed(dq, out=dx, displacement=True)
        cs.accd_toi(x, dx, alpha=alpha)
        Eh.copy_(E, non_blocking=True)
        gh.copy_(g, non_blocking=True)
        ah.copy_(alpha, non_blocking=True)
        nh.copy_(H.nnzb, non_blocking=True)
        rph.copy_(H.row_ptr, non_blocking=True)
        stream.synchronize()
        nb = int(nh[0])
        colh[:nb].copy_(H.col[:nb], non_blocking=True)
        valh[:nb].copy_(H.val[:nb], non_blocking=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        tot_ms += ev0.elapsed_time(ev1)
        tot_pairs += int(pairs.count.item())
        bi += 2 * Q[0].numel() * 8
        bo += 8 + gh.numel() * 8 + 8 + 8 + rph.numel() * 4 + nb * (4 + 72)
    return dict(value=tot_pairs / (tot_ms / 1e3), unit=UNIT, h2d_bytes_per_step=bi // K, d2h_bytes_per_step=bo // K,
                ms_per_step=tot_ms / K)


# --------------------------------------------------------------------------- batched

BATCH_WORKLOAD = "batched_grasp_256"


def _grow(caps, need):
    """Capacities after an overflow: at least 1.3x what the device reported as needed."""
    names = ("pair", "cand", "rec", "bsr")
    out = dict(caps)
    for n, v in zip(names, need):
        if v > 0:
            out[n] = max(out[n], int(1.3 * v) + 1024)
    return out


class _Stage:
    """One contact stage of a (batched) scene through the C ABI, on preallocated buffers so
    that it can be captured in a CUDA graph: static inputs q, dq; outputs E, g_r, H_r,
    per-group energy, alpha and per-group alpha."""

    def __init__(self, sc, caps, groups, dev, group_outputs=True):
        import torch
        from paper_2409_16385_gb300 import ContactScene
        self.sc, self.caps, self.groups = sc, caps, group_outputs
        self.cs = ContactScene(sc, pair_capacity=caps["pair"], bsr_capacity=caps["bsr"], cand_capacity=caps["cand"],
                               rec_capacity=caps["rec"])
        ng = 1
        if groups is not None:
            self.cs.set_groups(groups[0], groups[1])
            ng = groups[1]
        f64 = dict(dtype=torch.float64, device=dev)
        self.q = torch.zeros((sc.Ns, 3), **f64)
        self.dq = torch.zeros((sc.Ns, 3), **f64)
        self.pairs, self.lag, self.H = self.cs.new_pairs(), self.cs.new_lag(), self.cs.new_bsr()
        self.E = torch.zeros(1, **f64)
        self.g = torch.zeros((sc.Ns, 3), **f64)
        self.Eg = torch.zeros(ng, **f64)
        self.ag = torch.zeros(ng, **f64)
        self.x = torch.zeros((sc.Nv, 3), **f64)
        self.dx = torch.zeros((sc.Nv, 3), **f64)
        self.alpha = torch.zeros(1, **f64)
        self.ncand = torch.zeros(1, dtype=torch.int64, device=dev)

    def __call__(self, lag_step):
        cs = self.cs
        cs.build_candidates(self.q, out=self.pairs)
        if lag_step:
            cs.friction_lag(self.q, self.pairs, out=self.lag)
        cs.eval_contact(self.q, self.pairs, self.lag, E=self.E, g_r=self.g, H=self.H)
        if self.groups:
            cs.group_energy(out=self.Eg)
        cs.embed(self.q, out=self.x)
        cs.embed(self.dq, out=self.dx, displacement=True)
        cs.accd_toi(self.x, self.dx, alpha=self.alpha, n_candidates=self.ncand)
        if self.groups:
            cs.group_alpha(out=self.ag)


def capture_step_graphs(st, q_warm, dq_warm, R):
    """One CUDA graph of the whole contact stage per (lag step, hierarchy rebuild) case:
    the rebuild-or-refit choice is made on the host when a call is enqueued, so each case is
    captured with the rebuild interval forced to it.  Returns ({case: graph}, {case: kernels})."""
    import torch
    from paper_2409_16385_gb300 import binding
    lib = binding.load()
    graphs, kernels = {}, {}
    side = torch.cuda.Stream()
    for lag_step in (False, True):
        for rebuild in (True, False):
            st.cs.set_rebuild_interval(1 if rebuild else 1 << 30)
            st.q.copy_(q_warm); st.dq.copy_(dq_warm)
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                st(lag_step)                      # warm-up on the side stream
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            n0 = lib.eipc_launch_count()
            with torch.cuda.graph(g):
                st(lag_step)
            kernels[(lag_step, rebuild)] = lib.eipc_launch_count() - n0
            graphs[(lag_step, rebuild)] = g
    st.cs.set_rebuild_interval(R)
    torch.cuda.synchronize()
    return graphs, kernels


def graph_steps(sc, Q, DQ, lag_of, t0, K, flush, dev, shapes):
    """The headline's steps replayed from CUDA graphs (the library's calls are capturable:
    no host read-back), with the same launch shapes, iterates, L2 flush and CUDA-event
    timing: how much of the eager step is host launch overhead."""
    import torch
    n_it = sc.n_iterates
    R = 8
    st = _Stage(sc, dict(pair=1 << 21, bsr=1 << 21, cand=0, rec=0), None, dev, group_outputs=False)
    for k, shape in shapes.items():
        st.cs.set_launch(k, *shape)
    graphs, kernels = capture_step_graphs(st, Q[t0], DQ[t0], R)
    st.q.copy_(Q[lag_of[t0]])
    st(True)
    stream = torch.cuda.current_stream()
    ms, n_p = [], torch.zeros(K, dtype=torch.int64, device=dev)
    for k in range(K):
        t = (t0 + k) % n_it
        st.q.copy_(Q[t]); st.dq.copy_(DQ[t])
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graphs[(lag_of[t] == t, k % R == 0)].replay()
        e1.record(stream)
        n_p[k].copy_(st.pairs.count[0])
        ms.append((e0, e1))
    torch.cuda.synchronize()
    step_ms = np.array([a.elapsed_time(b) for a, b in ms])
    stt = st.cs.status()
    st.cs.close()
    if stt["flags"] & ~64:
        raise RuntimeError(f"graph steps: device status {stt}")
    pairs = float(n_p.sum().item())
    return dict(ms_per_step=float(step_ms.mean()), pairs_per_s=pairs / (step_ms.sum() / 1e3),
                kernels_per_step={f"lag={a},rebuild={c}": int(n) for (a, c), n in kernels.items()},
                timing="CUDA events around each replay, L2 flushed before each, the headline's iterates")


def _sized_stage(sc, caps, groups, dev, Q, DQ, lag_of, ts):
    """A _Stage whose capacities hold every iterate in `ts` (grown and rebuilt on overflow)."""
    import torch
    for _ in range(4):
        st = _Stage(sc, caps, groups, dev)
        need = [0, 0, 0, 0]
        bad = 0
        for t in ts:
            st.q.copy_(Q[lag_of[t]])
            st(True)
            st.q.copy_(Q[t]); st.dq.copy_(DQ[t])
            st(False)
            torch.cuda.synchronize()
            s = st.cs.status()
            bad |= s["flags"] & ~64
            need = [max(a, b) for a, b in zip(need, s["needed"])]
        if not bad:
            return st
        if bad & ~(2 | 4 | 8 | 16 | 128):
            raise RuntimeError(f"device status {s}")
        st.cs.close()
        del st
        caps = _grow(caps, need)
        if need[0] == 0 and bad & 128:
            caps["pair"] *= 2
    raise RuntimeError("capacities did not converge")


def batched_oracle_sample(b, t, budget_s=20.0, seed=0, max_tris=8000):
    """The oracle's whole contact stage at iterate t on whole scenes of the batch, drawn
    in a seeded random order among those of at most max_tris triangles (the brute-force
    enumeration is quadratic in the scene size, so a large scene alone would exceed the
    budget), until about budget_s seconds of host time are spent."""
    import oracle
    oracle.build()
    order = np.random.default_rng(seed).permutation(b.n_scenes)
    pairs, secs, used = 0, 0.0, []
    for s in order:
        if secs >= budget_s:
            break
        if b.parts[int(s)][0].F > max_tris:
            continue
        one = b.part_scene(int(s))
        p, dt, _ = oracle_sample(one, t, 1.0)
        pairs += p; secs += dt; used.append(int(s))
    tris = sum(b.parts[s][0].F for s in used)
    return dict(value=pairs / secs if secs > 0 else 0.0, unit=UNIT, cores=oracle.num_threads(), kind="oracle",
                sample=f"iterate {t}: whole contact stage (brute-force contact set, lagged friction, evaluation, CCD) "
                       f"of {len(used)} of the {b.n_scenes} scenes ({tris} triangles), drawn in seeded random order "
                       f"among those of at most {max_tris} triangles; "
                       f"{pairs} pairs in {secs:.1f} s")


def batched_summary(args, ws, rank, local):
    """The 256-scene batch beside the headline: 20 graph-replayed steps and the plain
    per-scene path on the same iterates (no CPU leg, no end-to-end pass)."""
    import copy
    a = copy.copy(args)
    a.steps, a.warmup = 20, max(3, min(args.warmup, 5))
    a.no_cpu_baseline, a.no_e2e, a.no_plain = True, True, False
    a.cand_cap, a.rec_cap = 0, 0
    line = run_batched(a, ws, rank, local, emit=False)
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "plain_per_scene", "speedup_vs_plain", "roofline",
            "clocks", "gpu_launches", "kernels_per_graph", "autotune", "ccd_queries_per_s", "scene_generation_s")
    out = {k: line[k] for k in keep if k in line}
    out["config"] = line["config"]
    return out


def run_batched(args, ws, rank, local, emit=True):
    """256 independent grasp scenes (surface sizes log-uniform in [2k, 50k] triangles, own
    closing phase each) in one scene with one group per scene.  One step is one CUDA graph
    replay of the whole contact stage of all scenes; the plain per-scene path (one
    ContactScene per scene, called scene after scene, eager) runs the same iterates beside
    it.  Metric: contact pairs evaluated per second over whole steps."""
    import torch
    import torch.distributed as dist
    from paper_2409_16385_gb300 import autotune, binding, scenes

    dev = torch.device("cuda", local)
    lib = binding.load()
    t_gen = time.perf_counter()
    b = scenes.make_config(4, small=args.quick)
    gen_s = time.perf_counter() - t_gen
    G, n_it = b.n_scenes, b.n_iterates
    lag_of = [b.lag_of(t) for t in range(n_it)]
    Q = torch.tensor(np.stack([b.iterate(t) for t in range(n_it)]), dtype=torch.float64, device=dev)
    DQ = torch.tensor(np.stack([b.dq(t) for t in range(n_it)]), dtype=torch.float64, device=dev)
    K, W = args.steps, args.warmup
    t0 = W % n_it
    size_ts = sorted({t0, (t0 + 3) % n_it, (t0 + 29) % n_it, (t0 + 47) % n_it})
    # starting capacities; the sizing pass grows whichever overflows
    caps = dict(pair=1 << 20, bsr=1 << 20, cand=args.cand_cap or (1 << 24), rec=args.rec_cap or (1 << 24))
    st = _sized_stage(b, caps, (b.body, G), dev, Q, DQ, lag_of, size_ts)

    # ---- autotuned launch shapes (cached per device and workload)
    def tune_stage():
        st(False)
    st.q.copy_(Q[t0]); st.dq.copy_(DQ[t0])
    tuned = {}
    if not args.no_tune:
        tuned = autotune.tune(st.cs, tune_stage, f"{BATCH_WORKLOAD if not args.quick else 'batched_grasp_16'}",
                              force=args.retune)

    # ---- one graph per (lag step, hierarchy rebuild) combination
    R = 8
    graphs, kernels_per_graph = capture_step_graphs(st, Q[t0], DQ[t0], R)

    def replay(k, t):
        st.q.copy_(Q[t]); st.dq.copy_(DQ[t])
        key = (lag_of[t] == t, k % R == 0)
        graphs[key].replay()
        return kernels_per_graph[key]

    # lag state of the first timed iterates, then warm-up replays
    start_t = (t0 - W) % n_it
    st.q.copy_(Q[lag_of[start_t]])
    st(True)
    for k in range(W):
        replay(k, (start_t + k) % n_it)
    torch.cuda.synchronize()
    s0 = st.cs.status()
    if s0["flags"] & ~64:
        raise RuntimeError(f"device status after warm-up: {s0}")

    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    counts = torch.zeros((K, 2), dtype=torch.int64, device=dev)
    clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    clocks.start()
    time.sleep(0.3)                  # the sampler is running before the timed region starts
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    tw0 = time.time()
    wall0 = time.perf_counter()
    launches = 0
    for k in range(K):
        t = (t0 + k) % n_it
        flush.zero_()
        evs[k][0].record(stream)
        launches += replay(W + k, t)
        evs[k][1].record(stream)
        counts[k, 0].copy_(st.pairs.count[0])
        counts[k, 1].copy_(st.ncand[0])
    torch.cuda.synchronize()
    tw1 = time.time()
    wall = time.perf_counter() - wall0
    if ws > 1:
        dist.barrier()
    clocks.mark(tw0, tw1)
    clk = clocks.stop()
    s1 = st.cs.status()
    if s1["flags"] & ~64:
        raise RuntimeError(f"device status after the timed steps: {s1}")
    step_ms = np.array([a.elapsed_time(c) for a, c in evs])
    cnt = counts.cpu().numpy()
    total_s, total_pairs, total_cand = step_ms.sum() / 1e3, float(cnt[:, 0].sum()), float(cnt[:, 1].sum())
    total_s_all, total_pairs_all, total_cand_all = across_ranks(total_s, total_pairs, total_cand, ws, dev)
    value = total_pairs_all / total_s_all
    Eg_last = st.Eg.cpu().numpy()
    ag_last = st.ag.cpu().numpy()

    # ---- dominant kernel and its roofline: the same steps eagerly, kernel timers on
    st.cs.set_rebuild_interval(R)
    st.cs.timing_enable(None)
    st.q.copy_(Q[lag_of[t0]]); st(True)
    for k in range(K):
        t = (t0 + k) % n_it
        st.q.copy_(Q[t]); st.dq.copy_(DQ[t])
        flush.zero_()
        st(lag_of[t] == t)
    torch.cuda.synchronize()
    kt = st.cs.timing_read()
    st.cs.timing_enable([])
    dominant = max(kt.items(), key=lambda kv: kv[1][0])[0]
    dom_ms, dom_n = kt[dominant]
    roof = roofline_figure(dominant, dom_ms, dom_n, K, dict(pairs=total_pairs / K, ccd=total_cand / K), b)
    roof["timed"] = "eager replay of the timed steps with per-kernel CUDA-event timers"

    # ---- end to end: pinned host q, dq in; E per scene, alpha per scene, g_r out
    e2e = None
    if not args.no_e2e:
        qh = [Q[t].cpu().pin_memory() for t in range(n_it)]
        dqh = [DQ[t].cpu().pin_memory() for t in range(n_it)]
        Egh = torch.zeros(G, dtype=torch.float64).pin_memory()
        agh = torch.zeros(G, dtype=torch.float64).pin_memory()
        gh = torch.zeros((b.Ns, 3), dtype=torch.float64).pin_memory()
        st.q.copy_(Q[lag_of[t0]]); st(True)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot_ms, tot_pairs = 0.0, 0
        for k in range(K):
            t = (t0 + k) % n_it
            flush.zero_()
            ev0.record(stream)
            st.q.copy_(qh[t], non_blocking=True)
            st.dq.copy_(dqh[t], non_blocking=True)
            graphs[(lag_of[t] == t, k % R == 0)].replay()
            Egh.copy_(st.Eg, non_blocking=True)
            agh.copy_(st.ag, non_blocking=True)
            gh.copy_(st.g, non_blocking=True)
            ev1.record(stream)
            torch.cuda.synchronize()
            tot_ms += ev0.elapsed_time(ev1)
            tot_pairs += int(st.pairs.count.item())
        e2e = dict(value=tot_pairs / (tot_ms / 1e3), unit=UNIT, h2d_bytes_per_step=2 * b.Ns * 3 * 8,
                   d2h_bytes_per_step=2 * G * 8 + b.Ns * 3 * 8, ms_per_step=tot_ms / K,
                   api="q, dq from pinned host memory; per-scene E and alpha and g_r back to pinned host memory")

    # ---- the plain per-scene path on the same iterates
    plain = None
    if not args.no_plain:
        parts = [b.part_scene(s) for s in range(G)]
        stages = []
        for s, one in enumerate(parts):
            n0, ns = b.node_ranges[s]
            pc = dict(pair=max(1 << 14, 4 * one.Nv), bsr=max(1 << 14, 64 * one.Ns), cand=0,
                      rec=max(1 << 18, 96 * one.Nv))
            Qs, DQs = Q[:, n0:n0 + ns], DQ[:, n0:n0 + ns]
            stages.append((_sized_stage(one, pc, None, dev, Qs, DQs, lag_of, size_ts), Qs, DQs))
        for stg, Qs, _ in stages:
            stg.cs.set_rebuild_interval(R)
            stg.q.copy_(Qs[lag_of[start_t]]); stg(True)
        for k in range(W):
            t = (start_t + k) % n_it
            for stg, Qs, DQs in stages:
                stg.q.copy_(Qs[t]); stg.dq.copy_(DQs[t]); stg(lag_of[t] == t)
        torch.cuda.synchronize()
        pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        pcount = torch.zeros((K, G), dtype=torch.int64, device=dev)
        l0 = lib.eipc_launch_count()
        for k in range(K):
            t = (t0 + k) % n_it
            flush.zero_()
            pev[k][0].record(stream)
            for s, (stg, Qs, DQs) in enumerate(stages):
                stg.q.copy_(Qs[t]); stg.dq.copy_(DQs[t])
                stg(lag_of[t] == t)
                pcount[k, s].copy_(stg.pairs.count[0])
            pev[k][1].record(stream)
        torch.cuda.synchronize()
        pl = lib.eipc_launch_count() - l0
        pms = np.array([a.elapsed_time(c) for a, c in pev])
        ppairs = float(pcount.sum().item())
        for stg, _, _ in stages:
            if stg.cs.status()["flags"] & ~64:
                raise RuntimeError("plain path overflowed")
        # the last iterate's per-scene energy and step bound, against the batch's
        same_E = all(stg.Eg.item() == Eg_last[s] for s, (stg, _, _) in enumerate(stages))
        same_a = all(stg.alpha.item() == ag_last[s] for s, (stg, _, _) in enumerate(stages))
        plain = dict(value=ppairs / (pms.sum() / 1e3), unit=UNIT, ms_per_step=float(pms.mean()),
                     launches_per_step=pl / K, pairs_per_step=ppairs / K,
                     last_step_bitwise_equal=dict(energy_per_scene=bool(same_E), alpha_per_scene=bool(same_a)))
        for stg, _, _ in stages:
            stg.cs.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = batched_oracle_sample(b, t0, budget_s=20.0)

    sizes = [sc.F for sc, _ in b.parts]
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=K, warmup=W,
                ms_per_step=float(step_ms.mean()), higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic (seeded)",
                config=dict(workload=BATCH_WORKLOAD if not args.quick else "batched_grasp_16", scenes=G,
                            triangles=b.F, vertices=b.Nv, edges=b.E, cage_nodes=b.Ns,
                            triangles_per_scene=[int(min(sizes)), int(np.median(sizes)), int(max(sizes))],
                            dhat=b.params["dhat"], mu=b.params["mu"], parallelism=f"replicas x{ws}",
                            l2="flushed between steps (256 MiB rewrite)", pairs_per_step=total_pairs / K,
                            ccd_candidates_per_step=total_cand / K, rebuild_interval=R,
                            graph="one CUDA graph replay per step (4 graphs: lag step x hierarchy rebuild)"),
                clocks=clk, gpu_launches=int(launches), wall_s=wall, roofline=roof,
                ccd_queries_per_s=total_cand_all / total_s_all, e2e=e2e, cpu_baseline=cpu,
                plain_per_scene=plain, speedup_vs_plain=(value / plain["value"]) if plain else None,
                autotune={k: dict(shape=v["shape"], ms=v["ms"], default_ms=v["default_ms"], cached=v["cached"],
                                  candidates=v.get("candidates"))
                          for k, v in tuned.items()},
                kernels_per_graph={f"lag={a},rebuild={c}": int(n) for (a, c), n in kernels_per_graph.items()},
                capacities=st.caps, scene_generation_s=gen_s,
                kernel_ms_eager={k: v[0] for k, v in kt.items()})
    st.cs.close()
    if not emit:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                json.dump(line, f, indent=1)


# --------------------------------------------------------------------------- adjoint

def hvp_stage(cs, sc, Q, lag_of, t0, K, flush, dev):
    """Stage-only device time of the exact-Hessian HVP beside the projected evaluation on
    the same pairs (bubble-grasp iterates): contact pairs per second of each."""
    import torch
    stream = torch.cuda.current_stream()
    pairs, lag = cs.new_pairs(), cs.new_lag()
    first = lag_of[t0]
    cs.build_candidates(Q[first], out=pairs)
    cs.friction_lag(Q[first], pairs, out=lag)
    v = torch.randn((sc.Ns, 3), dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(0))
    out = torch.empty_like(v)
    out_kin = torch.empty(3, dtype=torch.float64, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.zeros((sc.Ns, 3), dtype=torch.float64, device=dev)
    H = cs.new_bsr()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    t_h = t_e = 0.0
    n_p = 0
    for k in range(K):
        t = (t0 + k) % sc.n_iterates
        cs.build_candidates(Q[t], out=pairs)
        n_p += int(pairs.count.item())
        flush.zero_()
        ev[0].record(stream)
        cs.contact_hvp(Q[t], pairs, v, lag=lag, out=out, out_kin=out_kin)
        ev[1].record(stream)
        flush.zero_()
        ev[2].record(stream)
        cs.eval_contact(Q[t], pairs, lag, E=E, g_r=g, H=H)
        ev[3].record(stream)
        torch.cuda.synchronize()
        t_h += ev[0].elapsed_time(ev[1])
        t_e += ev[2].elapsed_time(ev[3])
    return dict(hvp_pairs_per_s=n_p / (t_h / 1e3), eval_pairs_per_s=n_p / (t_e / 1e3), hvp_ms=t_h / K,
                eval_ms=t_e / K, pairs_per_call=n_p / K)


def run_adjoint(args, ws, rank, local):
    """The trajectory gradient of the sphere on a rising pad (20 backward-Euler steps of the
    reduced Newton driver, checkpoints every 5): dL/dtheta and dL/dkappa for L = ||g_c(q_20)||^2
    by the HVP kernel and implicit steps, timed forward and backward; plus the HVP kernel's
    stage throughput on the bubble-grasp pairs beside the projected evaluation."""
    import torch
    from paper_2409_16385_gb300 import ContactScene, scenes
    from paper_2409_16385_gb300.adjoint import trajectory_loss
    from paper_2409_16385_gb300.sim import Simulator

    dev = torch.device("cuda", local)
    sc = scenes.make_config(5, small=args.quick)
    sim = Simulator(sc, device=str(dev))
    K, W = max(1, args.steps // 10), max(1, args.warmup // 3)
    stream = torch.cuda.current_stream()
    th0, ka0 = sc.theta, sc.params["kappa"]
    fwd, bwd, newton = [], [], []
    for k in range(W + K):
        th = torch.tensor(th0, dtype=torch.float64, device=dev, requires_grad=True)
        ka = torch.tensor(ka0, dtype=torch.float64, device=dev, requires_grad=True)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        e0.record(stream)
        L = trajectory_loss(sim, th, ka, sc.n_steps, sc.checkpoint_every)
        e1.record(stream)
        L.backward()
        e2.record(stream)
        torch.cuda.synchronize()
        if k >= W:
            fwd.append(e0.elapsed_time(e1)); bwd.append(e1.elapsed_time(e2))
    _, _, infos = sim.trajectory(th0, ka0)
    newton = [i.iterations for i in infos]
    # central differences of the same trajectory (h = 1e-7 on theta, 1e-3 relative on kappa)
    def loss(t, k_):
        with torch.no_grad():
            return float(trajectory_loss(sim, torch.tensor(t, dtype=torch.float64, device=dev),
                                         torch.tensor(k_, dtype=torch.float64, device=dev), sc.n_steps, 0))
    fd_t = (loss(th0 + 1e-7, ka0) - loss(th0 - 1e-7, ka0)) / 2e-7
    fd_k = (loss(th0, ka0 * (1 + 1e-3)) - loss(th0, ka0 * (1 - 1e-3))) / (2e-3 * ka0)
    d_t, d_k = float(th.grad), float(ka.grad)
    # HVP kernel throughput on the bubble-grasp workload
    sb = scenes.make_config(2, small=args.quick)
    cs = ContactScene(sb, pair_capacity=1 << 21, bsr_capacity=1 << 21)
    Q = torch.tensor(np.stack([sb.iterate(t) for t in range(sb.n_iterates)]), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stage = hvp_stage(cs, sb, Q, [sb.lag_of(t) for t in range(sb.n_iterates)], 5, max(5, args.steps), flush, dev)
    steps_s = sc.n_steps / ((np.mean(fwd) + np.mean(bwd)) / 1e3)
    line = dict(metric="trajectory gradient: time steps differentiated per second", value=steps_s,
                unit="steps/s", n_gpus=ws, steps=K, warmup=W, ms_per_step=float(np.mean(fwd) + np.mean(bwd)) / sc.n_steps,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic (seeded)",
                config=dict(workload=sc.name, steps_per_trajectory=sc.n_steps, checkpoint_every=sc.checkpoint_every,
                            cage_nodes=sc.Ns, vertices=sc.Nv, triangles=sc.F, theta=th0, kappa=ka0,
                            solver="dense adjoint solves, exact Hessian; HVP kernel for the loss and theta terms"),
                trajectory_ms=dict(forward=float(np.mean(fwd)), backward=float(np.mean(bwd))),
                newton_iterations=newton,
                gradient=dict(dL_dtheta=d_t, dL_dkappa=d_k, fd_dL_dtheta=fd_t, fd_dL_dkappa=fd_k,
                              rel_err_theta=abs(fd_t - d_t) / abs(d_t), rel_err_kappa=abs(fd_k - d_k) / abs(d_k)),
                hvp_stage=dict(workload=sb.name, **stage))
    if rank == 0:
        print(json.dumps(line), flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                json.dump(line, f, indent=1)


# --------------------------------------------------------------------------- physical

def run_physical(args, ws, rank, local):
    """The bubble grasp simulated by the reduced Newton driver (membranes' outer cage layers
    position-controlled, body and membranes elastic under gravity, friction lagged every
    step): time per backward-Euler step, Newton and Krylov iterations, and the contact-stage
    share.  --solver auto picks the dense solve up to 12k free DoFs (this scene has 7.6k)."""
    import torch
    from paper_2409_16385_gb300 import scenes
    from paper_2409_16385_gb300.sim import Simulator

    dev = torch.device("cuda", local)
    sc = scenes.bubble_grasp_physical(small=args.quick)
    sim = Simulator(sc, device=str(dev), solver=args.solver, pair_capacity=1 << 21, bsr_capacity=1 << 21,
                    rec_capacity=1 << 24)
    sim.pcg_rtol = 1e-8
    K = max(2, args.steps // 5)
    kappa = sc.params["kappa"]
    lag = sim.initial_lag(kappa)
    qs = [sim.q0.clone(), sim.q0.clone()]
    stream = torch.cuda.current_stream()
    sim.cs.timing_enable(None)
    ms, infos, pairs = [], [], []
    zero = torch.zeros(3, dtype=torch.float64, device=dev)
    for n in range(1, K + 1):
        if n > 1:
            lag = sim.cs.friction_lag(qs[-1], sim.cs.build_candidates(qs[-1], out=sim.cs.new_pairs()))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        q, info = sim.step(qs[-1], qs[-2], zero, kappa, lag, rtol=1e-8, q_fixed=sim.prescribed(n), strict=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1)); infos.append(info)
        pairs.append(int(sim.cs.build_candidates(q).count.item()))
        qs.append(q)
    kt = sim.cs.timing_read()
    contact_ms = sum(v[0] for v in kt.values())
    line = dict(metric="physical simulation: backward-Euler steps per second", value=1e3 / float(np.mean(ms)),
                unit="steps/s", n_gpus=ws, steps=K, warmup=0, ms_per_step=float(np.mean(ms)), higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic (seeded)",
                config=dict(workload=sc.name, cage_nodes=sc.Ns, free_dofs=int(sim.free.sum()) * 3, vertices=sc.Nv,
                            triangles=sc.F, closing_per_step=1e-4, newton_rtol=1e-8, solver=sim.solver,
                            pcg_rtol=sim.pcg_rtol),
                newton_iterations=[i.iterations for i in infos], pcg_iterations=[i.krylov_iterations for i in infos],
                residuals=[i.residual for i in infos], stop_reasons=[i.reason for i in infos], contact_pairs=pairs,
                contact_stage_ms_total=contact_ms, step_ms=ms,
                kernel_ms_total={k: round(v[0], 3) for k, v in kt.items()})
    if rank == 0:
        print(json.dumps(line), flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                json.dump(line, f, indent=1)


def main():
    args = parse()
    backend = "gloo" if args.impl == "reference" else "nccl"
    ws, rank, local = dist_setup(backend)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return finish(ws)
    from paper_2409_16385_gb300 import binding
    binding.set_programmatic_launch(args.launch_mode == "programmatic")
    if args.workload == "batched":
        run_batched(args, ws, rank, local)
    elif args.workload == "adjoint":
        run_adjoint(args, ws, rank, local)
    elif args.workload == "physical":
        run_physical(args, ws, rank, local)
    elif args.workload == "eval_by_type":
        run_eval_by_type(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)
    finish(ws)


def finish(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
