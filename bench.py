#!/usr/bin/env python3
"""Benchmark: IMM seconds-to-seeds on one GB300 (plus sampling GTEPS and the
roofline of the dominant kernel), through the C ABI.

Default workload (one step = one whole IMM run, every hot-path step):
  IC, R-MAT 1,048,576 vertices / 16,777,216 edges, p ~ U[0, 0.1] fp32,
  k = 50, eps = 0.13, ell = 1, rng seed 2.
The graph is resident in HBM before the timed region (value); the e2e number
repeats the step through the same public calls from pinned host buffers, with
the graph upload and the seed read-back inside the timed region.

After that line's measurements, a one-GPU default run also measures the other
workloads and attaches them under "workloads" in the same JSON line:
  lt_4m       LT, R-MAT 4,194,304 / 67,108,864, w = 1/indeg, k=100, eps=0.5
  ic_wc_4k    IC, R-MAT 4,096 / 32,768, p = 1/indeg, k=10, eps=0.5
  ic_u1_256k  IC, R-MAT 262,144 / 4,194,304, p ~ U[0, 1], k=50, eps=0.5
              (the paper's IC weight law), with RRR-set coverage of V
  opim_*      the OPIM-style early stop (imm_run_opim) on lt_4m and ic_u1_256k
  batch64     64 IMM instances through imm_run_batch (queries/s)
  served      10,000 Poisson queries at 200/s through imm_server (queries/s,
              p50/p99 latency)
Each result is checked against the oracle (its full run, or the stored
oracle results under tests/golden/) or against the same query run alone.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
  python bench.py --profile-case --workload W --theta T [--select K]

--impl reference times the oracle (plain single-threaded C on the host) on a
bounded sample of the same workload and scales it to the whole run's exact
schedule.  --profile-case runs one sampling call (and optionally one
selection) of a workload, the small case the ncu captures under profiles/ use.
Multi-GPU: replicas only (each rank runs the same workload on its own GPU);
the timed region is bracketed by a barrier and the max over ranks is taken.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IMM seconds-to-seeds"

# IC sampling is bound by integer issue, not by DRAM: its roofline counts coin
# evaluations, one per (RRR set, in-edge quad) pair the BFS examines, each a
# Philox4x32-10 draw (10 rounds of 2 wide 32x32 multiplies + 2 three-input
# xors = 40 instructions) and 4 threshold compares, against the issue rate of
# the GPU (SMs x 4 schedulers x 32 lanes x max SM clock).
ALU_OPS_PER_QUAD_EVAL = 44
# DRAM bytes per quad evaluation of the dominant IC kernel on the 1M-vertex
# workload, from one ncu capture (profiles/ic_group_kernel__ic_u01_1m_first20000sets.md)
IC_DRAM_BYTES_PER_QUAD_EVAL = 32.628760e9 / 12215037853
# DRAM bytes per member of the LT walk sampler on the 4M-vertex LT workload,
# from one ncu capture of a 46,669-set call with 2,105,421 members
# (profiles/lt_samplers_and_select_coop__lt_4m_46669sets_k100.md)
LT_DRAM_BYTES_PER_MEMBER = (329.627904e6 + 7.699712e6) / 2105421
WORKLOADS = ("ic_u01_1m", "lt_4m", "ic_wc_4k", "ic_u1_256k", "batch64", "served")
GOLDEN = os.path.join(ROOT, "tests", "golden")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("gpu", "reference"), default="gpu")
    ap.add_argument("--workload", choices=WORKLOADS, default="ic_u01_1m")
    ap.add_argument("--cpu-sample-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--served-queries", type=int, default=10000)
    ap.add_argument("--served-rate", type=float, default=200.0)
    ap.add_argument("--served-solo", type=int, default=200, help="queries timed one at a time for comparison")
    ap.add_argument("--no-extras", action="store_true", help="measure the --workload line only")
    ap.add_argument("--extra-steps", type=int, default=5)
    ap.add_argument("--profile-case", action="store_true")
    ap.add_argument("--theta", type=int, default=2000)
    ap.add_argument("--select", type=int, default=0)
    ap.add_argument("--repeat", type=int, default=1)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group("gloo", rank=self.rank, world_size=self.world)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for nm, val in zip(names, p[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# stored oracle results (tests/golden/, written by tests/golden/make_golden.py
# from the oracle alone)
# ---------------------------------------------------------------------------
def golden(name: str):
    p = os.path.join(GOLDEN, name + ".json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        return json.load(f)


def same_as_golden(seeds, st, rec) -> bool:
    r = st.rounds
    return ([int(x) for x in seeds] == rec["seeds"] and r == rec["rounds"]
            and [int(st.theta_i[i]) for i in range(r)] == rec["theta_i"]
            and [int(st.covered_i[i]) for i in range(r)] == rec["covered_i"]
            and float(st.lb).hex() == rec["lb_hex"] and st.theta == rec["theta"]
            and st.num_sets == rec["num_sets"] and st.covered == rec["covered"] and st.members == rec["members"])


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands on a bounded sample of the workload
# ---------------------------------------------------------------------------
def run_schedule(w, st=None):
    """Sets per selection of the workload's whole IMM run (one selection per
    sampling round, then the final one) and its total members.  From the
    GPU's own run statistics when given (they equal the oracle's; the tests
    check this), else from the oracle's stored complete run."""
    rec = golden(w.name)
    if st is not None:
        sets = [int(st.sets_i[i]) for i in range(st.rounds)] + [int(st.num_sets)]
        out = {"sets_per_selection": sets, "num_sets": int(st.num_sets), "members": int(st.members),
               "source": "this run's statistics (equal to the oracle's run)"}
        if rec is not None:
            out["full_run_s"] = rec["oracle_seconds"]
        return out
    if rec is None:
        return None
    return {"sets_per_selection": rec["sets_i"] + [rec["num_sets"]], "num_sets": rec["num_sets"],
            "members": rec["members"], "full_run_s": rec["oracle_seconds"],
            "source": f"the oracle's complete run stored in tests/golden/{w.name}.json"}


def cpu_baseline(w, budget_s: float, sched: dict, k: int, part: int = 0, parts: int = 1):
    """The oracle as it stands, single-threaded on one host core.  When its
    whole IMM run fits the budget it is timed directly.  Otherwise set ids
    drawn at random from the whole run's stream (part `part` of `parts`
    disjoint draws) are sampled one by one for about budget_s seconds, one
    k-selection runs over them, and the two rates are scaled to the run's
    exact schedule: sampling s/set x sets drawn + selection s/member x members
    in the stream at each selection."""
    import numpy as np

    import oracle
    g = w.graph
    o = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model)
    full_sets = sched["num_sets"]
    fr = sched.get("full_run_s")  # the oracle's complete run, timed when its stored results were written
    if (fr is not None and fr < budget_s) or (fr is None and full_sets <= 20000 and g.m <= (1 << 20)):
        t1 = time.perf_counter()
        seeds, _ = o.run(k, w.epsilon, w.ell, w.seed)
        t_run = time.perf_counter() - t1
        if t_run < 4 * budget_s:
            o.close()
            return {"seconds": t_run, "sample": "the oracle's whole IMM run on this workload (not scaled)",
                    "cores": 1, "sets_per_s": full_sets / t_run, "scaled": False}
    rng = np.random.default_rng(12345)
    ids = rng.permutation(full_sets)[part::parts]
    t0 = time.perf_counter()
    off, mem = [0], []
    done = 0
    while done < len(ids) and time.perf_counter() - t0 < budget_s:
        s = o.sample_one(w.seed, int(ids[done]))
        mem.append(s)
        off.append(off[-1] + len(s))
        done += 1
    t_sample = time.perf_counter() - t0
    members = off[-1]
    offa = np.array(off, dtype=np.uint64)
    mema = np.concatenate(mem).astype(np.uint32) if mem else np.zeros(0, dtype=np.uint32)
    t1 = time.perf_counter()
    oracle.select_sets(g.n, offa, mema, min(k, g.n))
    t_select = time.perf_counter() - t1
    o.close()
    per_set = t_sample / done
    per_member_select = t_select / max(members, 1)
    avg_len = sched["members"] / full_sets
    select_members = sum(s * avg_len for s in sched["sets_per_selection"])
    est = per_set * full_sets + per_member_select * select_members
    return {
        "seconds": est, "cores": 1, "sets_per_s": done / t_sample, "scaled": True,
        "sample": (f"scaled estimate: the oracle sampled {done} set ids drawn at random from the run's "
                   f"{full_sets}-set stream ({members} members) in {t_sample:.1f} s and ran one k={k} selection "
                   f"over them in {t_select:.2f} s; scaled to the run's exact schedule "
                   f"({len(sched['sets_per_selection'])} selections over {sched['sets_per_selection']} sets, "
                   f"schedule from {sched['source']})"),
    }


def run_reference(args, dist: Dist):
    import graphgen
    if dist.rank != 0:
        return
    w = graphgen.plain_workload(args.workload if args.workload in graphgen.PLAIN else "ic_u01_1m")
    sched = run_schedule(w)
    same = sched is not None
    if sched is None:
        # no stored run: the stream size comes from the oracle's own theta math
        # and a short pilot (an estimate of where the LB test fires)
        import math

        import oracle
        g = w.graph
        o = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model)
        prm = oracle.theta_params(g.n, w.k, w.epsilon, w.ell)
        pilot = 200
        o.sample(pilot, w.seed)
        _, cov = o.select(w.k)
        nF = g.n * cov / pilot
        eps_p = 2 ** 0.5 * w.epsilon
        sets, lb = [], 1.0
        for i in range(1, prm["rounds"] + 1):
            x = g.n / 2.0 ** i
            sets.append(math.ceil(prm["lambda_prime"] / x))
            if nF >= (1 + eps_p) * x:
                lb = nF / (1 + eps_p)
                break
        full = max(math.ceil(prm["lambda_star"] / lb), sets[-1] if sets else 0)
        sched = {"sets_per_selection": sets + [full], "num_sets": full, "members": o.num_members * full // pilot,
                 "source": "a 200-set pilot (estimate)"}
        o.close()
    steps = args.warmup + args.steps
    per_step = max(3.0, 150.0 / max(steps, 1))
    times, rates, res = [], [], None
    for it in range(steps):
        res = cpu_baseline(w, per_step, sched, w.k, part=it, parts=steps)
        if it >= args.warmup:
            times.append(res["seconds"])
            rates.append(res["sets_per_s"])
    val = statistics.mean(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": val * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": w.desc, "l2": "n/a (host)"},
        "cpu_baseline": {"value": val, "unit": "s", "cores": res["cores"], "kind": "oracle",
                         "sample": res["sample"]},
        "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_sets_per_s": statistics.mean(rates) if rates else None,
        "schedule": {"sets_per_selection": sched["sets_per_selection"], "num_sets": sched["num_sets"],
                     "same_as_gpu_run": same, "source": sched["source"]},
        "scaled_estimate": bool(res.get("scaled")),
    }
    if sched.get("full_run_s"):
        line["oracle_full_run_s_build_host"] = sched["full_run_s"]
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def quad_evals(imm, ctx, g) -> float:
    """(set, in-edge quad) coin evaluations of the current stream:
    sum over vertices of occurrences x in-edge quads."""
    import numpy as np
    cnt = imm.imm_get_counts(ctx, g.n).astype(np.float64)
    row = g.row.astype(np.int64)
    deg = np.diff(row)
    quads = np.where(deg > 0, ((row[1:] - 1) >> 2) - (row[:-1] >> 2) + 1, 0).astype(np.float64)
    return float((cnt * quads).sum())


def coverage_of_v(imm, ctx, g, num_sets: int) -> dict:
    """RRR-set sizes as a fraction of |V| (the paper's Table I reports the
    average and maximum over a run's sets)."""
    import numpy as np
    sizes = []
    first = 0
    while first < num_sets:
        cnt = min(1 << 20, num_sets - first)
        off, _ = imm.imm_get_sets(ctx, first, cnt, members=False)
        sizes.append(np.diff(off.astype(np.int64)))
        first += cnt
    sz = np.concatenate(sizes) if sizes else np.zeros(1)
    return {"avg_pct_of_V": float(100.0 * sz.mean() / g.n), "max_pct_of_V": float(100.0 * sz.max() / g.n),
            "paper_table1_ic_eps05": "avg 1.6-68.0%, max 5.4-88.0% (SNAP graphs)"}


def run_plain(args, dist: Dist, name: str, steps: int, warmup: int, e2e_on: bool, cpu_on: bool,
              cpu_budget: float):
    """One plain-IMM workload: `steps` timed whole runs with the graph
    resident, the sampler roofline, optionally e2e and the CPU oracle."""
    import numpy as np
    import torch

    import graphgen
    from paper_2411_09473_gb300 import imm

    dev = dist.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    w = graphgen.plain_workload(name)
    g = w.graph
    ctx = imm.imm_create(device=dev, stream=stream)
    imm.imm_load_graph(ctx, g.n, g.m, g.row, g.src, g.weight, g.model)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=f"cuda:{dev}")  # 256 MB > L2

    def step():
        return imm.imm_run(ctx, g.model, w.k, w.epsilon, w.ell, w.seed)

    for _ in range(warmup):
        seeds, st = step()
        flush.fill_(1.0)
    torch.cuda.synchronize()

    clocks = ClockSampler(dev)
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    evs = []
    stats = []
    for _ in range(steps):
        flush.fill_(2.0)  # L2 flush between timed iterations, outside the events
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        seeds, st = step()
        b.record(stream)
        evs.append((a, b))
        stats.append(st)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in evs]
    ms_step = dist.max(statistics.mean(ms))

    # roofline of the dominant kernel: the samplers, timed by CUDA events on
    # the launching stream inside the library, over the timed steps
    ms_sample = sum(s.ms_sample for s in stats)
    edges = sum(s.sample_edges for s in stats)
    members = sum(s.sample_members for s in stats)
    launches = sum(s.sample_launches for s in stats)
    st = stats[-1]
    if g.model == graphgen.IC:
        # every step samples the same stream: count its quad evaluations once
        evals = quad_evals(imm, ctx, g) * len(stats)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = clk.get("sm_max_mhz") or 2070.0
        peak = sms * 4 * 32 * mhz * 1e6 / 1e12
        achieved = ALU_OPS_PER_QUAD_EVAL * evals / (ms_sample / 1e3) / 1e12 if ms_sample > 0 else 0.0
        roof = {"kernel": "RRR sampling (IC): ic_group_kernel / ic_large_kernel + ic_small_kernel",
                "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "peak_kind": f"derived: {sms} SMs x 4 schedulers x 32 lanes x {mhz:.0f} MHz",
                "traffic": (IC_DRAM_BYTES_PER_QUAD_EVAL * evals / max(launches, 1)
                            if name == "ic_u01_1m" else None),
                "traffic_source": "ncu dram__bytes_read+write per quad evaluation of the dominant kernel, "
                                  "scaled to the average timed launch",
                "algorithmic_ops": f"{ALU_OPS_PER_QUAD_EVAL} integer instructions per (set, in-edge quad) "
                                   "coin evaluation",
                "quad_evals_per_launch": evals / max(launches, 1), "launches": launches}
    else:
        algo_bytes = 8.0 * edges + 16.0 * members
        achieved = algo_bytes / (ms_sample / 1e3) / 1e9 if ms_sample > 0 else 0.0
        peak, peak_kind = measured_peaks()
        roof = {"kernel": "RRR sampling (LT): lt_small_kernel + lt_mid_kernel + lt_long_kernel", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": peak_kind,
                "traffic": (LT_DRAM_BYTES_PER_MEMBER * members / max(launches, 1) if name == "lt_4m" else None),
                "traffic_source": "ncu dram__bytes_read+write per member of lt_small_kernel, scaled to the "
                                  "average timed launch",
                "algorithmic_bytes": "8 B per walk step + 16 B per member",
                "algorithmic_bytes_per_launch": algo_bytes / max(launches, 1), "launches": launches}
    gteps = (st.sample_edges / (st.ms_sample / 1e3)) / 1e9 if st.ms_sample > 0 else 0.0
    cover = coverage_of_v(imm, ctx, g, st.num_sets) if name == "ic_u1_256k" else None

    # parity of this very run: the oracle's stored complete run, else its
    # complete run now when that is cheap
    parity = None
    rec = golden(name)
    if rec is not None:
        parity = {"equal": same_as_golden(seeds, st, rec), "against": f"tests/golden/{name}.json (oracle run)"}
    elif g.m <= (1 << 20):
        import oracle
        want, ost = oracle.Oracle(g.n, g.row, g.src, g.weight, g.model).run(w.k, w.epsilon, w.ell, w.seed)
        parity = {"equal": bool(np.array_equal(want, seeds) and ost.theta == st.theta
                                and ost.covered == st.covered), "against": "the oracle's run, now"}

    e2e = None
    if e2e_on:
        # public API from pinned host buffers: upload + run + seeds read back
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        hrow, hsrc, hw = pin(g.row), pin(g.src), pin(g.weight)
        h2d = hrow.nbytes + hsrc.nbytes + hw.nbytes
        d2h = 4 * w.k + 8 * 2
        ctx2 = imm.imm_create(device=dev, stream=stream)
        tt = []
        for it in range(warmup + steps):
            flush.fill_(3.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            imm.imm_load_graph(ctx2, g.n, g.m, hrow, hsrc, hw, g.model)
            s2, _ = imm.imm_run(ctx2, g.model, w.k, w.epsilon, w.ell, w.seed)
            torch.cuda.synchronize()
            if it >= warmup:
                tt.append(time.perf_counter() - t0)
            assert np.array_equal(s2, seeds)
        imm.imm_destroy(ctx2)
        e2e = {"value": dist.max(statistics.mean(tt)), "unit": "s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    cpu = None
    if dist.rank == 0 and dist.world == 1 and cpu_on:
        r = cpu_baseline(w, cpu_budget, run_schedule(w, st), w.k)
        cpu = {"value": r["seconds"], "unit": "s", "cores": r["cores"], "kind": "oracle", "sample": r["sample"],
               "sets_per_s": r["sets_per_s"]}
    imm.imm_destroy(ctx)
    del flush
    line = {
        "metric": METRIC,
        "value": ms_step / 1e3,
        "unit": "s",
        "n_gpus": dist.world,
        "steps": steps,
        "warmup": warmup,
        "ms_per_step": ms_step,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": w.desc, "graph": "R-MAT a=.57 b=.19 c=.19, transposed CSR",
                   "l2": "256 MB buffer written between timed steps (outside the events)",
                   "parallelism": f"replicas x{dist.world}"},
        "sampling_gteps" if g.model == graphgen.IC else "walk_steps_per_s_g": gteps,
        "sets_per_s": st.num_sets / (st.ms_sample / 1e3) if st.ms_sample > 0 else None,
        "imm": {"theta": st.theta, "num_sets": st.num_sets, "members": st.members, "rounds": st.rounds,
                "lb": st.lb, "covered": st.covered, "ms_sample": st.ms_sample, "ms_index": st.ms_index,
                "ms_select": st.ms_select, "seeds_head": [int(x) for x in seeds[:10]]},
        "parity": parity,
        "roofline": roof,
        "gpu_launches": int(sum(s.kernel_launches for s in stats)),
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if cover:
        line["rrr_coverage"] = cover
    return line


def run_opim(args, dist: Dist, name: str, steps: int, warmup: int):
    """OPIM-style early stop (imm_run_opim) on a plain workload: one step =
    one whole run (two RR collections doubling until the bound ratio holds),
    compared with the oracle's stored run."""
    import torch

    import graphgen
    from paper_2411_09473_gb300 import imm

    dev = dist.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    w = graphgen.plain_workload(name)
    g = w.graph
    ctx = imm.imm_create(device=dev, stream=stream)
    imm.imm_load_graph(ctx, g.n, g.m, g.row, g.src, g.weight, g.model)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=f"cuda:{dev}")
    for _ in range(warmup):
        seeds, st = imm.imm_run_opim(ctx, g.model, w.k, w.epsilon, w.ell, w.seed)
    clocks = ClockSampler(dev)
    torch.cuda.synchronize()
    clocks.start()
    evs, launches = [], 0
    for _ in range(steps):
        flush.fill_(2.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        seeds, st = imm.imm_run_opim(ctx, g.model, w.k, w.epsilon, w.ell, w.seed)
        b.record(stream)
        evs.append((a, b))
        launches += int(st.kernel_launches)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    imm.imm_destroy(ctx)
    r = st.rounds
    parity = None
    gold = golden("opim")
    rec = next((x for x in gold["runs"] if x["workload"] == name), None) if gold else None
    if rec is not None:
        eq = ([int(x) for x in seeds] == rec["seeds"] and r == rec["rounds"]
              and [int(st.cov1_i[i]) for i in range(r)] == rec["cov1_i"]
              and [int(st.cov2_i[i]) for i in range(r)] == rec["cov2_i"]
              and [float(st.upper_i[i]).hex() for i in range(r)] == rec["upper_hex"]
              and [float(st.lower_i[i]).hex() for i in range(r)] == rec["lower_hex"])
        parity = {"equal": bool(eq), "against": "tests/golden/opim.json (oracle run)"}
    return {
        "metric": "IMM seconds-to-seeds (OPIM-style early stop)", "value": ms / 1e3, "unit": "s",
        "n_gpus": dist.world, "steps": steps, "warmup": warmup, "ms_per_step": ms, "higher_is_better": False,
        "dtype": "u32", "data": "synthetic", "config": {"workload": w.desc},
        "rounds": r, "i_max": int(st.i_max), "sets_per_collection": int(st.sets_i[r - 1]),
        "alpha": st.alpha, "target": 1.0 - 1.0 / 2.718281828459045 - w.epsilon,
        "parity": parity, "gpu_launches": launches, "clocks": clk,
    }


def run_batch(args, dist: Dist, steps: int, warmup: int):
    """64 independent IMM instances (R-MAT, n log-uniform over 2^10..2^18,
    average degree 8..32, IC/LT alternating, k 5..100, eps 0.1..0.5), one
    step = the whole batch through imm_run_batch; the one-at-a-time path
    (imm_run per instance, in order) is timed beside it, and every instance
    is compared with its solo run and with the oracle's stored run."""
    import numpy as np
    import torch

    import graphgen
    from paper_2411_09473_gb300 import imm

    dev = dist.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    b = graphgen.batch_workload(count=64)
    ctxs = []
    for g in b.graphs:
        c = imm.imm_create(device=dev, stream=stream)
        imm.imm_load_graph(c, g.n, g.m, g.row, g.src, g.weight, g.model)
        ctxs.append(c)
    queries = [(ctxs[q.graph_id], q.k, q.epsilon, q.ell, q.seed) for q in b.queries]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=f"cuda:{dev}")
    # the library's autotuner picks the batch's tuning (outside the timed region)
    ta = time.perf_counter()
    best, table = imm.imm_autotune_batch(queries, reps=1)
    tune_s = time.perf_counter() - ta
    for _ in range(warmup):
        seeds, stats, status = imm.imm_run_batch(queries)
        assert status == [0] * len(queries), status
    clocks = ClockSampler(dev)
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times = []
    launches = 0
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        seeds, stats, status = imm.imm_run_batch(queries)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        launches += int(sum(st.kernel_launches for st in stats))
    dist.barrier()
    clk = clocks.stop()
    step_s = dist.max(statistics.mean(times))
    # one at a time, same instances, same results
    solo = []
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, q in enumerate(b.queries):
            g = b.graphs[q.graph_id]
            s2, _ = imm.imm_run(ctxs[q.graph_id], g.model, q.k, q.epsilon, q.ell, q.seed)
            if rep == 0:
                assert np.array_equal(s2, seeds[i]), i
        torch.cuda.synchronize()
        solo.append(time.perf_counter() - t0)
    solo_s = min(solo)
    gold = golden("batch64")
    parity = None
    if gold is not None:
        eq = sum(same_as_golden(seeds[i], stats[i], gold["instances"][i]) for i in range(len(queries)))
        parity = {"equal": eq == len(queries), "instances_equal": int(eq),
                  "against": "tests/golden/batch64.json (oracle runs)"}
    for c in ctxs:
        imm.imm_destroy(c)
    nq = len(queries)
    return {
        "metric": "batched IMM queries/s", "value": dist.sum(nq / step_s) if dist.world > 1 else nq / step_s,
        "unit": "queries/s", "n_gpus": dist.world, "steps": steps, "warmup": warmup,
        "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": "64 IMM instances: R-MAT n=2^U(10,18), avg degree U(8,32), IC/LT alternating, "
                               "k=U{5..100}, eps=U(0.1,0.5), batch seed 4", "l2": "256 MB write between steps",
                   "parallelism": f"replicas x{dist.world}"},
        "one_at_a_time": {"value": nq / solo_s, "unit": "queries/s", "s_per_batch": solo_s,
                          "results_identical": True},
        "batched_over_solo": solo_s / step_s,
        "parity": parity,
        "autotune": {"best": best, "seconds": tune_s,
                     "candidates_ms": [[c["cluster_min_n"], c["select_cand"], c["batch_sets"], round(ms, 2)]
                                       for c, ms in table],
                     "columns": ["cluster_min_n", "select_cand", "batch_sets", "mean_ms"]},
        "theta_total": int(sum(st.num_sets for st in stats)),
        "members_total": int(sum(st.members for st in stats)),
        "gpu_launches": launches, "clocks": clk,
    }


def run_served(args, dist: Dist):
    """Served IMM: 8 resident R-MAT graphs (n log-spaced 2^16..2^20, average
    degree 16, IC/LT alternating, w = 1/indeg), a Poisson stream of queries
    (rate --served-rate, k = U{10..200}, eps = U(0.1, 0.5), graph uniform),
    replayed in real time against imm_server; latency = completion - arrival.
    The first queries' results are compared with the oracle's stored runs."""
    import numpy as np
    import torch

    import graphgen
    from paper_2411_09473_gb300 import imm

    dev = dist.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    graphs = graphgen.served_graphs()
    ctxs = []
    for g in graphs:
        c = imm.imm_create(device=dev, stream=stream)
        imm.imm_load_graph(c, g.n, g.m, g.row, g.src, g.weight, g.model)
        ctxs.append(c)
    qs = graphgen.served_queries(count=args.served_queries, rate_per_s=args.served_rate, num_graphs=len(graphs))
    gold = golden("served") if args.served_rate == 200.0 else None
    n_gold = len(gold["results"]) if gold else 0
    srv = imm.imm_server_create(ctxs, memory_budget_bytes=96 << 30, max_active=128)
    # warm-up: a few queries through the server
    for q in qs[:max(args.warmup, 1) * 4]:
        imm.imm_server_submit(srv, q.graph_id, q.k, q.epsilon, q.ell, 10 ** 9 + q.seed)
    got = 0
    t_w = time.perf_counter()
    while got < max(args.warmup, 1) * 4:
        for (qid, status, _, _) in imm.imm_server_poll(srv):
            if status == 0:
                imm.imm_server_take(srv, qid, 256)
            got += 1
        if time.perf_counter() - t_w > 120:
            raise RuntimeError(f"served warm-up did not complete: {imm.imm_server_info(srv)}")
        time.sleep(0.001)
    clocks = ClockSampler(dev)
    clocks.start()
    ids, lat, failed = {}, {}, 0
    keep = {}
    gold_ok = 0
    t0 = time.perf_counter()
    i, n = 0, len(qs)
    limit_s = max(60.0, 4.0 * qs[-1].arrival_s)  # the run reports what completed by then
    last_note = 0.0
    while len(lat) + failed < n:
        now = time.perf_counter() - t0
        if now > limit_s:
            break
        if now - last_note > 10.0:
            last_note = now
            print(f"served: t={now:.0f}s submitted={i} done={len(lat)} failed={failed} "
                  f"{imm.imm_server_info(srv)}", file=sys.stderr, flush=True)
        while i < n and qs[i].arrival_s <= now:
            q = qs[i]
            ids[imm.imm_server_submit(srv, q.graph_id, q.k, q.epsilon, q.ell, q.seed)] = i
            i += 1
        for (qid, status, latency_ms, queue_ms) in imm.imm_server_poll(srv):
            j = ids[qid]
            if status != 0:
                failed += 1
                continue
            # latency from the scheduled arrival (submission can lag it slightly)
            lat[j] = (time.perf_counter() - t0 - qs[j].arrival_s) * 1e3
            seeds, st = imm.imm_server_take(srv, qid, qs[j].k)
            if j < 20:
                keep[j] = seeds
            if j < n_gold:
                gold_ok += same_as_golden(seeds, st, gold["results"][j])
        time.sleep(0.0005)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    info = imm.imm_server_info(srv)
    imm.imm_server_destroy(srv)
    # one at a time on the same contexts: capacity of the plain path
    m = min(args.served_solo, n)
    torch.cuda.synchronize()
    ts = time.perf_counter()
    for j in range(m):
        q = qs[j]
        s2, _ = imm.imm_run(ctxs[q.graph_id], graphs[q.graph_id].model, q.k, q.epsilon, q.ell, q.seed)
        if j in keep:
            assert np.array_equal(s2, keep[j]), j
    torch.cuda.synchronize()
    solo_s = time.perf_counter() - ts
    for c in ctxs:
        imm.imm_destroy(c)
    lats = np.array([lat[j] for j in sorted(lat)])
    checked = len([j for j in lat if j < n_gold])
    return {
        "metric": "served IMM queries/s", "value": len(lat) / wall, "unit": "queries/s", "n_gpus": dist.world,
        "steps": 1, "warmup": args.warmup, "ms_per_step": wall * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"{n} queries, Poisson {args.served_rate:g}/s, 8 resident R-MAT graphs "
                               "2^16..2^20 (avg deg 16, IC/LT alternating, w=1/indeg), k=U{10..200}, "
                               "eps=U(0.1,0.5), stream seed 5", "parallelism": f"replicas x{dist.world}"},
        "latency_ms": ({"p50": float(np.percentile(lats, 50)), "p99": float(np.percentile(lats, 99)),
                        "max": float(lats.max()), "mean": float(lats.mean())} if len(lats) else None),
        "offered_rate": args.served_rate, "completed": int(len(lat)), "failed": int(failed),
        "submitted": int(i), "time_limited": bool(len(lat) + failed < n),
        "one_at_a_time": {"value": m / solo_s, "unit": "queries/s", "queries": m,
                          "results_identical_checked": len([j for j in keep if j < m])},
        "parity": ({"equal": gold_ok == checked, "queries_checked": checked, "queries_equal": int(gold_ok),
                    "against": "tests/golden/served.json (oracle runs)"} if n_gold else None),
        "server": info, "gpu_launches": None, "clocks": clk,
    }


def run_gpu(args, dist: Dist):
    if args.workload == "batch64":
        line = run_batch(args, dist, args.steps, args.warmup)
    elif args.workload == "served":
        line = run_served(args, dist)
    else:
        line = run_plain(args, dist, args.workload, args.steps, args.warmup, not args.no_e2e,
                         not args.no_cpu_baseline, args.cpu_sample_seconds)
    if args.workload == "ic_u01_1m" and dist.world == 1 and not args.no_extras:
        # the other workloads, measured after the headline's own numbers
        extra = {}
        es, ew = max(1, min(args.extra_steps, args.steps)), 3
        for name in ("lt_4m", "ic_wc_4k", "ic_u1_256k"):
            extra[name] = run_plain(args, dist, name, es, ew, False, not args.no_cpu_baseline, 10.0)
        for name in ("lt_4m", "ic_u1_256k"):
            extra["opim_" + name] = run_opim(args, dist, name, es, ew)
        extra["batch64"] = run_batch(args, dist, es, ew)
        extra["served"] = run_served(args, dist)
        line["workloads"] = extra
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def run_profile_case(args):
    """One sampling call (and optionally one selection) of a named workload
    through the C ABI: the small case the kernel captures under profiles/
    run, smaller than a whole IMM run."""
    import numpy as np
    import torch

    import graphgen
    from paper_2411_09473_gb300 import imm

    w = graphgen.plain_workload(args.workload)
    g = w.graph
    ctx = imm.imm_create(device=0)
    imm.imm_load_graph(ctx, g.n, g.m, g.row, g.src, g.weight, g.model)
    out = []
    for _ in range(args.repeat):
        imm.imm_reset_sets(ctx)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        imm.imm_sample(ctx, g.model, args.theta, w.seed)
        rec = {"theta": args.theta}
        if args.select:
            seeds, cov = imm.imm_select(ctx, args.select)
            rec["covered"] = cov
            rec["seeds_head"] = [int(x) for x in seeds[:5]]
        torch.cuda.synchronize()
        rec["s"] = time.perf_counter() - t0
        rec["sets"], rec["members"] = imm.imm_stream_size(ctx)
        cnt = imm.imm_get_counts(ctx, g.n).astype(np.uint64)
        indeg = np.diff(g.row.astype(np.int64)).astype(np.uint64)
        rec["edges"] = int((cnt * indeg).sum())
        rec["quad_evals"] = int(quad_evals(imm, ctx, g))
        out.append(rec)
    print(json.dumps(out))
    imm.imm_destroy(ctx)


def main():
    args = parse()
    if args.profile_case:
        run_profile_case(args)
        return
    dist = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        else:
            run_gpu(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
