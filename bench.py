#!/usr/bin/env python3
"""Benchmark of the forest hot path on the 111,000-row AIWC-shaped workload.

One step = fit a 500-tree forest (presort/rank, Philox bootstrap, breadth-first growth, pack)
on 111,000 rows x 32 features, predict 1,000,000 queries, and select the fastest of 15
devices for 64 kernels. Inputs are resident in device memory when the timed region starts;
L2 is flushed between steps. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (oracle/, plain C, trees spread over the host cores) on
a bounded sample of the same workload and metric.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# one hardware queue per stream for the selection server's streams (read when CUDA initialises)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from paper_1811_00156_gb300 import synth  # noqa: E402

ROWS_TREES_UNIT = "rows·trees/s"
METRIC = "fit rows·trees/s (bit-exact forest) + predict queries/s"
T_TREES, MTRY, MIN_NODE = 500, 10, 5
N_QUERIES = 1_000_000
SEL_KERNELS, SEL_DEVICES = 64, 15
WORKLOAD = ("aiwc-111000: fit 500 trees (mtry 10, min_node 5, bootstrap) on 111,000 rows x 32 "
            "features + predict 1,000,000 queries + select device for 64 kernels x 15 devices")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the OOB and LOKO reports")
    ap.add_argument("--write-counters", metavar="CSV", default=None,
                    help="merge into profiles/counters.json the per-launch counters of an ncu --csv capture "
                         "(dram__bytes_read.sum, dram__bytes_write.sum, smsp__inst_executed.sum, "
                         "l1tex__data_pipe_lsu_wavefronts_mem_shared.sum) and exit")
    ap.add_argument("--counters-command", default="", help="the ncu command that made the CSV (recorded)")
    ap.add_argument("--counters-scale", nargs="*", default=None, metavar="CLASS=FACTOR",
                    help="keep only these classes, their instruction and wavefront counts multiplied by FACTOR "
                         "(a smaller case scaled to the full launch)")
    ap.add_argument("--trees", type=int, default=T_TREES,
                    help="forest size per GPU; smaller values are for profiler captures only")
    ap.add_argument("--queries", type=int, default=N_QUERIES,
                    help="query count; smaller values are for profiler captures only")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


# ------------------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.path = os.path.join(tempfile.gettempdir(), f"aiwcrf_clocks_{os.getpid()}.csv")
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------ oracle timing
def oracle_fit_sample(wl, n_trees: int, threads: int, first: int = 0):
    """Oracle as it stands, one tree per task, tasks spread over `threads` host threads."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda t: oracle.fit(wl.X, wl.y, T_TREES, MTRY, MIN_NODE, seed=synth.FOREST_SEED,
                                         t0=t, t1=t + 1), range(first, first + n_trees)))
    return time.perf_counter() - t0


def cpu_baseline(wl):
    cores = os.cpu_count() or 1
    n_trees = max(8, 8 * cores)
    secs = oracle_fit_sample(wl, n_trees, cores)
    return {"value": wl.n_rows * n_trees / secs, "unit": ROWS_TREES_UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_trees} of the 500 trees on all 111,000 rows ({secs:.1f} s wall, "
                      f"one tree per thread task)"}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    wl = synth.scaled_forest_workload()
    cores = os.cpu_count() or 1
    per_step = max(2, cores)
    for w in range(args.warmup):
        oracle_fit_sample(wl, min(per_step, 2), cores, first=w)
    times = []
    for k in range(args.steps):
        times.append(oracle_fit_sample(wl, per_step, cores, first=(k * per_step) % T_TREES))
    tot = sum(times)
    value = wl.n_rows * per_step * args.steps / tot
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": ROWS_TREES_UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "rows": wl.n_rows, "features": 32,
                                           "trees": T_TREES, "sample_trees_per_step": per_step},
           "cpu_baseline": {"value": value, "unit": ROWS_TREES_UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{per_step} trees per step on all 111,000 rows, one tree per thread task"},
           "e2e": {"value": value, "unit": ROWS_TREES_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ------------------------------------------------------------------------------ ours
# the sources of each kernel class: its ncu counters are reported only while these are unchanged
CLASS_SOURCES = {"tree": ("fit.cu", "internal.cuh"), "level_big": ("fit.cu", "internal.cuh"),
                 "level_small": ("fit.cu", "internal.cuh"), "walk": ("predict.cu", "internal.cuh"),
                 "predict": ("predict.cu", "sort.cu", "internal.cuh")}


def source_sha(cls: str | None = None):
    h = hashlib.sha256()
    for f in CLASS_SOURCES.get(cls, ("fit.cu", "predict.cu", "sort.cu", "internal.cuh")):
        h.update(open(os.path.join(ROOT, "paper_1811_00156_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_counter(kernel: str, metric: str, sha: str, path: str | None = None):
    """A per-launch counter of a kernel class from the committed ncu summary
    (profiles/counters.json: dram_bytes, inst, smem_wavefronts), if it was taken on the current
    kernel source; else None."""
    p = path or os.path.join(ROOT, "profiles", "counters.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(kernel)
    if not e or e.get("source_sha") != sha:
        return None
    return e.get(metric)


def ncu_traffic(kernel: str, sha: str, path: str | None = None):
    """Per-launch DRAM traffic (read + write bytes) of a kernel class, or None."""
    return ncu_counter(kernel, "dram_bytes", sha, path)


class L2Flush:
    """Between steps: write a 256 MB buffer (> the 129 MB L2), then read another 256 MB one, so
    that L2 holds no data of the step and none of its lines is dirty (the write-back of the
    written lines happens here, not inside the next step's kernels and their DRAM counters)."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.r = torch.zeros(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def __call__(self, k):
        self.w.fill_(float(k))
        self.r.sum()


def run_ours(args):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_1811_00156_gb300 import aiwcrf as A
    A.load()

    dev = torch.device("cuda", local_rank)
    wl = synth.scaled_forest_workload()
    N, F = wl.n_rows, wl.n_features
    n_trees, n_queries = args.trees, args.queries
    Xq_h = synth.queries(n_queries)
    kfeat_h = np.ascontiguousarray(synth.queries(SEL_KERNELS, seed=99)[:30])
    X = torch.from_numpy(wl.X).to(dev)
    y = torch.from_numpy(wl.y).to(dev)
    Xq = torch.from_numpy(Xq_h).to(dev)
    kfeat = torch.from_numpy(kfeat_h).to(dev)
    psum = torch.empty(n_queries, dtype=torch.int64, device=dev)
    pred = torch.empty(n_queries, dtype=torch.int64, device=dev)
    best = torch.empty(SEL_KERNELS, dtype=torch.int32, device=dev)
    selp = torch.empty(SEL_KERNELS * SEL_DEVICES, dtype=torch.int64, device=dev)
    flush = L2Flush(dev)
    devices = list(range(SEL_DEVICES))
    T_total = n_trees * world
    params = A.params(n_trees, MTRY, MIN_NODE, seed=synth.FOREST_SEED, first_tree=rank * n_trees)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev: ev[0].record(stream)
        forest = A.aiwcrf_fit(params, X, y)
        if ev: ev[1].record(stream)
        if world == 1:
            A.aiwcrf_predict(forest, Xq, pred)
        else:
            A.aiwcrf_predict_sum(forest, Xq, psum)
            dist.all_reduce(psum)
            A.aiwcrf_round_mean(psum, T_total, pred)
        if ev: ev[2].record(stream)
        A.aiwcrf_select_device(forest, kfeat, 2, devices, best, selp)
        if ev: ev[3].record(stream)
        return forest

    FIT_CLASSES = ("tree", "level_small", "level_big")
    dom_fit, dom = "tree", "predict"
    for w in range(args.warmup):
        last = w == args.warmup - 1
        if last:               # the last warm-up step finds the dominant kernels of the fit and the step
            A.aiwcrf_profile_classes([*FIT_CLASSES, "predict"])
            A.aiwcrf_profile_enable(True)
            A.aiwcrf_profile_read()
        step()
        if last:
            torch.cuda.synchronize()
            p0 = A.aiwcrf_profile_read()
            A.aiwcrf_profile_enable(False)
            dom_fit = max(FIT_CLASSES, key=lambda c: p0[c][1])
            dom = max((*FIT_CLASSES, "predict"), key=lambda c: p0[c][1])
    torch.cuda.synchronize()

    clocks = Clocks(local_rank)
    clocks.start()
    # inside the timed steps, events bracket the dominant kernels' launches only: every pair
    # costs the stream about 2 us, and bracketing every class would add ~5 % to the fit
    A.aiwcrf_profile_classes(sorted({dom, dom_fit, "walk"}))
    A.aiwcrf_profile_enable(True)
    A.aiwcrf_profile_read()
    launches0 = A.aiwcrf_launch_count()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    stats = None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush(k)                                   # write 256 MB (> L2) between steps
        f = step(evs[k])
        stats = f.stats()
        del f
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = A.aiwcrf_launch_count() - launches0
    prof_dom = A.aiwcrf_profile_read()
    A.aiwcrf_profile_enable(False)
    clk = clocks.stop()
    # the kernel classes' shares: K more (untimed) steps with every class bracketed
    A.aiwcrf_profile_classes(["tree", "level_small", "level_big", "predict", "select"])
    A.aiwcrf_profile_enable(True)
    A.aiwcrf_profile_read()
    for k in range(args.steps):
        flush(k)
        del_f = step()
        del del_f
    torch.cuda.synchronize()
    prof = A.aiwcrf_profile_read()
    A.aiwcrf_profile_enable(False)
    A.aiwcrf_profile_classes(None)

    fit_ms = sum(e[0].elapsed_time(e[1]) for e in evs)
    pred_ms = sum(e[1].elapsed_time(e[2]) for e in evs)
    sel_ms = sum(e[2].elapsed_time(e[3]) for e in evs)
    step_ms = sum(e[0].elapsed_time(e[3]) for e in evs)
    t = torch.tensor([fit_ms, pred_ms, sel_ms, step_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    fit_ms, pred_ms, sel_ms, step_ms = t.tolist()
    K = args.steps
    value = N * n_trees * world * K / (fit_ms / 1e3)

    # roofline of the dominant kernel class, from the events recorded around each launch
    peak, peak_kind = measured_peaks()
    sm_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    big_rows = stats["entries_evaluated"] - stats["entries_evaluated_small"]
    big_part = stats["entries_partitioned"] - stats["entries_partitioned_small"]
    per_eval = 16 + stats["rank_bytes"] * MTRY     # 16-byte entry + the tried features' ranks
    per_part = 16 + stats["rank_bytes"] + 16       # entry and chosen rank read, entry written
    alg = {
        "level_big": K * (big_rows * per_eval + big_part * per_part),
        "level_small": K * (stats["entries_evaluated_small"] * per_eval + stats["entries_partitioned_small"] * per_part),
        "tree": K * (stats["entries_evaluated"] * per_eval + stats["entries_partitioned"] * per_part),
        "predict": K * n_queries * (F * 4 + 8),
    }
    kernels = {}
    for name, (n_launch, ms) in prof.items():
        if n_launch == 0:
            continue
        entry = {"launches": n_launch, "total_ms": ms, "share_of_profiled": None}
        if name in alg and ms > 0:
            entry["alg_bytes"] = alg[name]
            entry["achieved_gbs"] = alg[name] / (ms / 1e3) / 1e9
        kernels[name] = entry
    tot_ms = sum(v["total_ms"] for v in kernels.values()) or 1.0
    for v in kernels.values():
        v["share_of_profiled"] = v["total_ms"] / tot_ms
    timing = "CUDA events around each launch of this kernel inside the timed steps"

    def hbm_roofline(name):
        n_l, ms = prof_dom[name]
        achieved = alg[name] / (ms / 1e3) / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"hbm_gbs of {peak_kind} peaks",
                "traffic": ncu_traffic(name, source_sha(name)), "alg_bytes_per_launch": alg[name] / n_l,
                "ms_per_launch": ms / n_l, "timing": timing}

    def issue_roofline(name):
        """A kernel whose working set is in shared memory and registers: bound by instruction
        issue. achieved = warp instructions per launch (ncu smsp__inst_executed.sum, same
        source) / event-timed duration; peak = 152 SMs x 4 schedulers x 1 warp instruction per
        cycle at the median SM clock sampled in the timed region."""
        n_l, ms = prof_dom[name]
        inst = ncu_counter(name, "inst", source_sha(name))
        pk = 152 * 4 * sm_mhz * 1e6 / 1e12                  # T warp-instructions/s
        r = {"kernel": name, "bound": "alu", "unit": "T warp-inst/s", "peak": pk,
             "peak_source": f"152 SMs x 4 issue slots x {sm_mhz:.0f} MHz (median sampled SM clock)",
             "ms_per_launch": ms / n_l, "timing": timing, "traffic": ncu_traffic(name, source_sha(name)),
             "alg_bytes_per_launch": alg[name] / n_l, "inst_per_launch": inst,
             "achieved": None, "frac": None}
        if inst:
            r["achieved"] = inst / (ms / n_l / 1e3) / 1e12
            r["frac"] = r["achieved"] / pk
        # context: the entry bytes it evaluates, as a rate against HBM (not its bound)
        r["entry_bytes_gbs"] = alg[name] / n_l / (ms / n_l / 1e3) / 1e9
        return r

    roofline = hbm_roofline(dom) if dom in ("predict", "level_big", "level_small") else issue_roofline(dom)
    if dom == "predict" and prof_dom.get("walk", (0, 0.0))[0]:
        # The predict call's dominant kernel is the walk, whose working set (tree slots and
        # query codes) is in shared memory: it is bound by instruction issue and shared-memory
        # wavefronts together. Reported against the issue peak, with the wavefront fraction and
        # the whole call's HBM floor (136 B per query) beside it.
        n_w, ms_w = prof_dom["walk"]
        wf = ncu_counter("walk", "smem_wavefronts", source_sha("walk"))
        wi = ncu_counter("walk", "inst", source_sha("walk"))
        smem_peak = 152 * sm_mhz * 1e6 / 1e9                  # G wavefronts/s
        issue_peak = 152 * 4 * sm_mhz * 1e6 / 1e12            # T warp-instructions/s
        floor = roofline
        if wi and wf:
            t_w = ms_w / n_w / 1e3
            roofline = {"kernel": "walk (predict4_kernel)", "bound": "alu", "unit": "T warp-inst/s",
                        "achieved": wi / t_w / 1e12, "peak": issue_peak, "frac": wi / t_w / 1e12 / issue_peak,
                        "peak_source": f"152 SMs x 4 issue slots x {sm_mhz:.0f} MHz (median sampled SM clock)",
                        "traffic": ncu_traffic("walk", source_sha("walk")), "inst_per_launch": wi,
                        "ms_per_launch": ms_w / n_w, "timing": timing,
                        "smem": {"wavefronts_per_launch": wf, "achieved_gwf_s": wf / t_w / 1e9,
                                 "peak_gwf_s": smem_peak, "frac": wf / t_w / 1e9 / smem_peak,
                                 "peak_source": f"152 SMs x 1 wavefront x {sm_mhz:.0f} MHz"},
                        "hbm_floor": floor}
            roofline["smem_frac"] = roofline["smem"]["frac"]
        else:
            # counters not taken on these sources: the call's HBM floor alone
            roofline["walk"] = {"ms_per_launch": ms_w / n_w, "smem_peak_gwf_s": smem_peak,
                                "issue_peak_tinst_s": issue_peak}
    roofline_fit = (issue_roofline(dom_fit) if dom_fit == "tree" else hbm_roofline(dom_fit))

    out = {"metric": METRIC, "value": value, "unit": ROWS_TREES_UNIT, "n_gpus": world, "steps": K,
           "warmup": args.warmup, "ms_per_step": step_ms / K, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "config": {"workload": WORKLOAD if (n_trees, n_queries) == (T_TREES, N_QUERIES) else
                      f"profiling case: {n_trees} trees, {n_queries} queries", "rows": N, "features": F,
                      "trees_per_gpu": n_trees, "queries": n_queries, "select": f"{SEL_KERNELS}x{SEL_DEVICES}",
                      "seeds": {"data": synth.DATA_SEED, "forest": synth.FOREST_SEED, "queries": synth.QUERY_SEED},
                      "l2": "flushed between steps (256 MB write, then 256 MB read: no dirty lines left); fit working set and queries exceed L2",
                      "parallelism": f"tree-sharded x{world}" if world > 1 else "1 GPU"},
           "predict": {"value": n_queries * K / (pred_ms / 1e3), "unit": "queries/s", "ms": pred_ms / K,
                       "trees": T_total},
           "select": {"ms": sel_ms / K, "kernels": SEL_KERNELS, "devices": SEL_DEVICES},
           "fit_ms": fit_ms / K, "fit_stats": stats, "roofline": roofline, "roofline_fit": roofline_fit,
           "kernels": {"timing": "CUDA events around every launch of these classes, in K further untimed steps",
                       **kernels},
           "gpu_launches": launches, "clocks": clk, "parity": "bit-exact vs oracle (tests/test_gpu_parity.py)"}

    if not args.no_e2e:
        out["e2e"] = e2e(A, wl, Xq_h, kfeat_h, params, devices, world, dev, max(1, min(K, 5)))
    if rank == 0 and not args.no_extras:
        out["fit_graph"] = fit_graph_report(A, params, X, y, stats)
        f = A.aiwcrf_fit(params, X, y)
        out["oob"] = oob_report(A, wl, X, f)
        del f
        out["loko"] = loko_report(A, dev)
        out["tune"] = tune_report(A, dev)
        out["per_row"] = per_row_report(A, dev)
        f = A.aiwcrf_fit(params, X, y)
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        out["surrogate"], sg = surrogate_report(A, f, Xq, bf16_peak_tflops=peaks.get("bf16_tflops"))
        del f
        # the earlier reports' forests, plans and networks are freed now, not by the garbage
        # collector in the middle of the load test
        gc.collect()
        torch.cuda.synchronize()
        out["serving"] = serving_report(A, wl, surrogate=sg)
        del sg
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def e2e(A, wl, Xq_h, kfeat_h, params, devices, world, dev, steps):
    """The same step through the C ABI with pinned HOST buffers: the library copies inputs in
    and results out inside the timed region."""
    import torch
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()        # noqa: E731
    X, y, Xq, kf = pin(wl.X), pin(wl.y), pin(Xq_h), pin(kfeat_h)
    pred = torch.empty(Xq.shape[1], dtype=torch.int64).pin_memory().numpy()
    best = torch.empty(kf.shape[1], dtype=torch.int32).pin_memory().numpy()
    selp = torch.empty(kf.shape[1] * len(devices), dtype=torch.int64).pin_memory().numpy()
    f = A.aiwcrf_fit(params, X, y)                    # one untimed step: the staging pool is warm
    A.aiwcrf_predict(f, Xq, pred)
    A.aiwcrf_select_device(f, kf, 2, devices, best, selp)
    del f
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        f = A.aiwcrf_fit(params, X, y)
        A.aiwcrf_predict(f, Xq, pred)
        A.aiwcrf_select_device(f, kf, 2, devices, best, selp)
        del f
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    h2d = X.nbytes + y.nbytes + Xq.nbytes + kf.nbytes + 4 * len(devices)
    d2h = pred.nbytes + best.nbytes + selp.nbytes
    return {"value": wl.n_rows * params.num_trees * world * steps / secs, "unit": ROWS_TREES_UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * secs / steps,
            "steps": steps, "note": "host clock around fit + predict + select with pinned host arrays (X, y staged by "
                                     "the library; the query features read in place by the coding kernel)"}


def fit_graph_report(A, params, X, y, stats, steps: int = 5):
    """The benchmark fit as a fit plan: one captured CUDA graph (presort, groups, bootstrap and a
    device-side loop over the tree levels) replayed, launch schedule from the autotuner; checked
    byte for byte against aiwcrf_fit."""
    import torch
    t0 = time.perf_counter()
    plan = A.FitPlan(params, X, y)
    build_s = time.perf_counter() - t0
    chosen, tried = plan.tune(reps=2)
    ref = A.aiwcrf_fit(params, X, y).serialize()
    ms, same = [], True
    flush = L2Flush(X.device)
    for k in range(steps + 1):
        flush(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        f = plan.run()[0]
        e1.record()
        torch.cuda.synchronize()
        if k > 0:
            ms.append(e0.elapsed_time(e1))
        same = same and f.serialize() == ref
        del f
    plan.close()
    fit_ms = statistics.median(ms)
    return {"fit_ms": fit_ms, "rows_trees_per_s": int(X.shape[1]) * params.num_trees / (fit_ms / 1e3),
            "forest_identical_to_aiwcrf_fit": same, "schedule": chosen, "schedules_tried": tried,
            "build_s": build_s}


def per_row_report(A, dev, n_trees: int = T_TREES, steps: int = 1):
    """The 111,000-row, 500-tree fit on the per-row reading of the features (every row its own
    AIWC vector: about 111,000 distinct values in 24 of the 32 columns, four-byte ranks, no two
    rows grouped), where the scan passes stream every active in-bag row: the automatic choice
    takes the presorted-list search. roofline on the scan passes' algorithmic bytes: 33 B per
    active in-bag row and level (4 B row id + 1 B multiplicity + 8 B target + 10 tried ranks x
    2 B) plus 10 B per partitioned row (row id and multiplicity read and written), over the
    level kernels' event-timed time (the two level kernels run concurrently, so their summed
    times overstate the span) and over the whole fit."""
    import torch
    wl = synth.per_row_forest_workload()
    X, y = torch.from_numpy(wl.X).to(dev), torch.from_numpy(wl.y).to(dev)
    params = A.params(n_trees, MTRY, MIN_NODE, seed=synth.FOREST_SEED)
    f = A.aiwcrf_fit(params, X, y)                                     # warm-up
    st = f.stats()
    del f
    A.aiwcrf_profile_classes(["level_small", "level_big", "list_partition", "finalize", "tree"])
    A.aiwcrf_profile_enable(True)
    A.aiwcrf_profile_read()
    ms = 0.0
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        f = A.aiwcrf_fit(params, X, y)
        e1.record()
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        st = f.stats()
        del f
    prof = A.aiwcrf_profile_read()
    A.aiwcrf_profile_enable(False)
    A.aiwcrf_profile_classes(None)
    peak, peak_kind = measured_peaks()
    scan_ms = sum(prof.get(c, (0, 0.0))[1] for c in ("level_small", "level_big", "list_partition", "tree")) / steps
    alg = 33 * st["entries_evaluated"] + 10 * st["entries_partitioned"]
    achieved = alg / (scan_ms / 1e3) / 1e9 if scan_ms else None
    achieved_fit = alg / (ms / steps / 1e3) / 1e9
    return {"workload": f"aiwc-111000 per-row features: fit {n_trees} trees (mtry 10, min_node 5) on 111,000 "
                        "rows x 32 features, every row its own feature vector",
            "trees": n_trees,
            "fit_ms": ms / steps, "rows_trees_per_s": wl.n_rows * n_trees * steps / (ms / 1e3),
            "stats": st,
            "roofline_fit": {"kernels": "level_big (presorted-list scans, argmax, entry and list partition) + "
                                        "level_small (warp bitonic search and partition)",
                             "bound": "hbm", "alg_bytes_per_fit": alg,
                             "alg_bytes": "33 B per active in-bag row-level (entries_evaluated) + 10 B per "
                                          "partitioned row-level (entries_partitioned)",
                             "ms_per_fit": scan_ms, "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak if achieved else None,
                             "achieved_over_whole_fit": achieved_fit, "frac_over_whole_fit": achieved_fit / peak,
                             "peak_source": f"hbm_gbs of {peak_kind} peaks",
                             "timing": "CUDA events around every level kernel launch of the fit"},
            "kernels_ms": {c: prof[c][1] / steps for c in ("level_small", "level_big", "list_partition", "finalize", "tree")
                           if c in prof and prof[c][0]}}


def tune_report(A, dev, steps: int = 40):
    """Simulated-annealing tuning of num.trees, mtry and min.node.size against the out-of-bag
    error (Sec. III-C) on the 2,220-row workload: 40 candidates from (128, 10, 5), num.trees in
    [16, 512], mtry in [1, 32], min.node.size in [1, 20]; every candidate a GPU fit and its
    exact out-of-bag error."""
    import torch
    wl = synth.plain_forest_workload()
    X, y = torch.from_numpy(wl.X).to(dev), torch.from_numpy(wl.y).to(dev)
    tp = A.tune_params(steps=steps, trees=(16, 512), mtry=(1, 32), node=(1, 20), t0=0.1, cooling=0.93, seed=1811)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    best, mse, trace = A.aiwcrf_tune_sa(tp, A.params(128, MTRY, MIN_NODE, seed=synth.FOREST_SEED), X, y)
    secs = time.perf_counter() - t0
    distinct = len({(t["num_trees"], t["mtry"], t["min_node_size"]) for t in trace})
    return {"workload": "aiwc-2220", "candidates": steps, "distinct_fits": distinct, "s": secs,
            "start": {"num_trees": 128, "mtry": MTRY, "min_node_size": MIN_NODE, "oob_mse": trace[0]["oob_mse"]},
            "best": {"num_trees": best.num_trees, "mtry": best.mtry, "min_node_size": best.min_node_size,
                     "oob_mse": mse},
            "accepted": sum(t["accepted"] for t in trace[1:])}


def loko_report(A, dev, steps: int = 2):
    """Leave-one-kernel-out cross-validation (Alg. 1 / Table III, here without the simulated-
    annealing re-tuning): 37 forests x 256 trees grown together by one batched fit; per-fold
    mean absolute percentage error of the predicted runtime (10^log10 t) on the held-out rows
    (Sec. V reports the same relative error)."""
    import torch
    wl, folds = synth.loko_folds()
    X, y = torch.from_numpy(wl.X).to(dev), torch.from_numpy(wl.y).to(dev)
    offs = np.cumsum([0] + [len(tr) for tr, _ in folds]).astype(np.int64)
    rows = torch.from_numpy(np.concatenate([tr for tr, _ in folds]).astype(np.int32)).to(dev)
    params = A.params(256, MTRY, MIN_NODE, seed=synth.FOREST_SEED)
    forests = A.aiwcrf_fit_subsets(params, X, y, offs, rows)          # warm-up
    ms = []
    for _ in range(steps):
        del forests
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        forests = A.aiwcrf_fit_subsets(params, X, y, offs, rows)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    mape = []
    for g, (tr, te) in enumerate(folds):
        Xt = torch.from_numpy(np.ascontiguousarray(wl.X[:, te])).to(dev)
        out = torch.empty(len(te), dtype=torch.int64, device=dev)
        A.aiwcrf_predict(forests[g], Xt, out)
        pred = out.cpu().numpy() / 2.0 ** 32
        truth = wl.y[te] / 2.0 ** 32
        mape.append(float(np.mean(np.abs(10.0 ** pred - 10.0 ** truth) / 10.0 ** truth)))
    rows_trees = int(sum(len(tr) for tr, _ in folds)) * 256
    # the same 37 fits as one captured graph (device-side level loop), schedule from the autotuner
    t0 = time.perf_counter()
    plan = A.FitPlan(params, X, y, offs, rows)
    build_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    chosen, tried = plan.tune(reps=2)
    tune_s = time.perf_counter() - t0
    pms = []
    same = True
    ref = [f.serialize() for f in forests]
    for k in range(steps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pf = plan.run()
        e1.record()
        torch.cuda.synchronize()
        if k > 0:
            pms.append(e0.elapsed_time(e1))
        same = same and [f.serialize() for f in pf] == ref
        del pf
    plan.close()
    # strict leave-one-kernel-out (Alg. 1): each fold trains on the other 36 kernels' rows and is
    # scored on every row of the held-out kernel
    kern = wl.meta["kernel"]
    strict = [(np.flatnonzero(kern != k), np.flatnonzero(kern == k)) for k in range(synth.N_KERNELS)]
    soffs = np.cumsum([0] + [len(tr) for tr, _ in strict]).astype(np.int64)
    srows = torch.from_numpy(np.concatenate([tr for tr, _ in strict]).astype(np.int32)).to(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sforests = A.aiwcrf_fit_subsets(params, X, y, soffs, srows)
    e1.record()
    torch.cuda.synchronize()
    strict_ms = e0.elapsed_time(e1)
    smape = []
    for g, (tr, te) in enumerate(strict):
        Xt = torch.from_numpy(np.ascontiguousarray(wl.X[:, te])).to(dev)
        out = torch.empty(len(te), dtype=torch.int64, device=dev)
        A.aiwcrf_predict(sforests[g], Xt, out)
        pred = out.cpu().numpy() / 2.0 ** 32
        truth = wl.y[te] / 2.0 ** 32
        smape.append(float(np.mean(np.abs(10.0 ** pred - 10.0 ** truth) / 10.0 ** truth)))
    del sforests
    return {"folds": len(folds), "trees_per_fold": 256, "train_rows": [int(min(len(t) for t, _ in folds)),
                                                                      int(max(len(t) for t, _ in folds))],
            "fit_ms": min(ms), "rows_trees_per_s": rows_trees / (min(ms) / 1e3),
            "graph": {"fit_ms": min(pms), "rows_trees_per_s": rows_trees / (min(pms) / 1e3),
                      "speedup_vs_batched_fit": min(ms) / min(pms), "forests_identical": same,
                      "schedule": chosen, "schedules_tried": tried, "build_s": build_s, "tune_s": tune_s},
            "mape_mean": float(np.mean(mape)), "mape_median": float(np.median(mape)),
            "mape_max": float(np.max(mape)), "batched": "one aiwcrf_fit_subsets call for all folds; "
            "graph: one aiwcrf_fit_plan_run (captured CUDA graph, autotuned schedule)",
            "strict": {"reading": "train on the other 36 kernels (2,160 rows), score every row of the held-out "
                                  "kernel (60 rows)", "fit_ms": strict_ms,
                       "mape_mean": float(np.mean(smape)), "mape_median": float(np.median(smape)),
                       "mape_max": float(np.max(smape))}}


def surrogate_report(A, forest, Xq, n_train=4_000_000, n_near=1_000_000, epochs=20, bf16_peak_tflops=None):
    """The learned surrogate distilled from the benchmark forest: 4,000,000 samples labelled by
    the forest -- 3,000,000 of the query distribution and 1,000,000 neighbours of the training
    kernels (synth.neighbour_queries, the scheduler's own use: kernels like those it was trained
    on) -- Adam (lr 1e-3, batch 4096, 20 epochs); then both models predict the benchmark's
    1,000,000 queries and 200,000 fresh neighbour queries. Error against the forest on both
    populations for the BF16 tensor-core network and, on a 20,000-query sample, for the same
    weights evaluated in FP64 by the oracle. Returns (report, surrogate)."""
    import torch
    from oracle import mlp as M
    dev = Xq.device
    Xs = torch.from_numpy(np.concatenate([synth.queries(n_train - n_near, seed=4242),
                                          synth.neighbour_queries(n_near, seed=4343)], axis=1)).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sg = A.aiwcrf_surrogate_fit(A.surrogate_params(epochs=epochs, batch=4096), forest, Xs)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del Xs
    Q = Xq.shape[1]
    ref = torch.empty(Q, dtype=torch.int64, device=dev)
    out = torch.empty(Q, dtype=torch.float32, device=dev)
    for _ in range(3):
        A.aiwcrf_predict(forest, Xq, ref)
        sg.predict(Xq, out)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(); A.aiwcrf_predict(forest, Xq, ref); e[1].record()
    e[2].record(); sg.predict(Xq, out); e[3].record()
    torch.cuda.synchronize()
    f_ms, s_ms = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
    f = ref.cpu().numpy() / 2.0 ** 32
    s = out.cpu().numpy().astype(np.float64)
    err = np.abs(s - f)
    P, mu, sd, lg = sg.export()
    idx = np.arange(0, Q, max(1, Q // 20000))
    Xh = Xq[:, idx].cpu().numpy()
    r64, _ = M.forward(P.astype(np.float64), M.encode(Xh, mu, sd, lg, 15, 4), rounding=False)
    flops = 2.0 * Q * (64 * 256 + 256 * 256 + 256)
    Xn = torch.from_numpy(synth.neighbour_queries(200_000, seed=4444)).to(dev)
    refn = torch.empty(Xn.shape[1], dtype=torch.int64, device=dev)
    outn = torch.empty(Xn.shape[1], dtype=torch.float32, device=dev)
    A.aiwcrf_predict(forest, Xn, refn)
    sg.predict(Xn, outn)
    errn = np.abs(outn.cpu().numpy().astype(np.float64) - refn.cpu().numpy() / 2.0 ** 32)
    del Xn, refn, outn
    rep = {"train_samples": n_train, "train_samples_neighbours": n_near, "epochs": epochs, "train_s": train_s,
           "stats": sg.stats(),
           "queries_per_s": Q / (s_ms / 1e3), "forest_queries_per_s": Q / (f_ms / 1e3),
           "speedup_vs_forest": f_ms / s_ms, "mae_vs_forest_log10": float(err.mean()),
           "p99_abs_err_log10": float(np.percentile(err, 99)),
           "mae_vs_forest_fp64_oracle_log10": float(np.abs(r64 - f[idx]).mean()),
           "mae_of_mean_predictor_log10": float(np.abs(f - f.mean()).mean()),
           "neighbours": {"queries": int(errn.size), "mae_vs_forest_log10": float(errn.mean()),
                          "p99_abs_err_log10": float(np.percentile(errn, 99))},
           "tensor_tflops": flops / (s_ms / 1e3) / 1e12}
    if bf16_peak_tflops:
        rep["tensor_frac_of_measured_bf16"] = rep["tensor_tflops"] / bf16_peak_tflops
    rep["gated_selection"] = gated_selection_report(A, forest, sg)
    return rep, sg


GATE_SETTINGS = ([("var", z, True) for z in (0.1, 0.25, 0.5, 1.0, 2.0)] +
                 [("tau", t, ood) for ood in (True, False) for t in (0.01, 0.02, 0.05, 0.1, 0.2)] +
                 [("alone", None, False)])


def gated_selection_report(A, forest, sg, K=65536, var_trees=32, settings=GATE_SETTINGS):
    """The gated selection on two kernel populations: fresh draws of the feature distributions
    (far from the 37 training kernels) and neighbours of the training kernels."""
    far = np.ascontiguousarray(synth.queries(K, seed=555)[:synth.N_AIWC])
    near = synth.kernel_neighbours(K, 2, jitter=0.05, seed=556)
    return {"random_kernels": gated_selection_case(A, forest, sg, far, var_trees, settings),
            "training_neighbours": gated_selection_case(A, forest, sg, near, var_trees, settings)}


def gated_selection_case(A, forest, sg, kf_h, var_trees, settings):
    """Device selection for K kernels x 15 devices: the forest alone, and the surrogate whose
    choice falls back to the forest (ood: on out-of-range features) when its margin between the
    two best devices is within z standard deviations of their ensemble spread over the forest's
    first 32 trees ("var"), or below tau log10 seconds ("tau"), or never ("alone"). Agreement
    and regret are judged by the forest's own predictions."""
    import torch
    dev = torch.device("cuda")
    K = kf_h.shape[1]
    kf = torch.from_numpy(kf_h).to(dev)
    devices = list(range(SEL_DEVICES))
    fb_best = torch.empty(K, dtype=torch.int32, device=dev)
    fb_pred = torch.empty(K * SEL_DEVICES, dtype=torch.int64, device=dev)
    best = torch.empty(K, dtype=torch.int32, device=dev)
    flags = torch.empty(K, dtype=torch.uint8, device=dev)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts), out

    t_forest, _ = timed(lambda: A.aiwcrf_select_device(forest, kf, 2, devices, fb_best, fb_pred))
    fp = fb_pred.view(K, SEL_DEVICES).cpu().numpy().astype(np.float64) / 2.0 ** 32
    fbest = fb_best.cpu().numpy()
    rep = {"kernels": K, "devices": SEL_DEVICES, "var_trees": var_trees,
           "forest": {"ms": 1e3 * t_forest, "queries_per_s": K * SEL_DEVICES / t_forest}, "gated": []}
    for kind, x, ood in settings:
        g = {"var": lambda: A.gate_params(var_trees, x, ood=ood), "tau": lambda: A.gate_params(1, 0.0, ood=ood, tau=x),
             "alone": lambda: A.gate_params(1, 0.0, ood=False)}[kind]()
        t, st = timed(lambda: A.aiwcrf_select_device_gated(forest, sg, g, kf, 2, devices, best, None, flags))
        b = best.cpu().numpy()
        regret = fp[np.arange(K), b] - fp[np.arange(K), fbest]
        rep["gated"].append({"gate": kind, "z" if kind == "var" else "tau": x, "ood": ood, "ms": 1e3 * t,
                             "queries_per_s": K * SEL_DEVICES / t,
                             "speedup_vs_forest": t_forest / t, "fallback_frac": st["fallback"] / K,
                             "fallback_ood": st["fallback_ood"], "fallback_var": st["fallback_var"],
                             "agreement_with_forest": float((b == fbest).mean()),
                             "mean_regret_log10": float(regret.mean()), "p99_regret_log10": float(np.percentile(regret, 99))})
    return rep


def serving_report(A, wl, rates=(5000.0, 20000.0, 50000.0), n_requests=20000, refit_every=10000, surrogate=None,
                   gated_rates=(20000.0, 50000.0), gate_z=0.5, gate_var_trees=32):
    """The device-selection server under open-loop Poisson load: a 500-tree forest of the
    111,000-row workload resident, requests of 1-64 kernels (uniform) x 15 devices x one size
    class (uniform), a refit every 10,000 requests on 2,220 appended rows. Latency runs from the
    scheduled arrival to the completed batch being seen on the host. A sample of the answers is
    checked against aiwcrf_select_device on the creation forest. With a surrogate, the same load
    again with every request gated (the surrogate resident in the server, the forest answering
    where the gate falls back; no refits): throughput, latency, fallback share and agreement of
    the gated devices with the forest's own choice."""
    rng = np.random.default_rng(2024)
    pool = np.ascontiguousarray(synth.queries(4096, seed=77)[:synth.N_AIWC])
    devices = np.arange(SEL_DEVICES, dtype=np.int32)
    fp = A.params(T_TREES, MTRY, MIN_NODE, seed=synth.FOREST_SEED)
    sp = A.server_params(n_streams=4, max_request_kernels=64, batch_kernels=1024, arena_bytes=64 << 20,
                         refit_every=refit_every, refit_rows=synth.N_KERNELS * SEL_DEVICES * synth.N_SIZES)
    out = {"trees": T_TREES, "train_rows": wl.n_rows, "devices": SEL_DEVICES, "kernels_per_request": "1-64",
           "refit_every": refit_every, "refit_rows": sp.refit_rows, "streams": sp.n_streams,
           "batch_kernels": sp.batch_kernels, "arena_bytes": sp.arena_bytes, "runs": []}
    with A.Server(sp, fp, wl.X, wl.y, devices) as srv:
        # a lone request at a time: the latency floor
        lat = []
        for i in range(200):
            t0 = time.perf_counter()
            srv.wait(srv.submit(np.ascontiguousarray(pool[:, i:i + 64]), i % synth.N_SIZES))
            lat.append((time.perf_counter() - t0) * 1e6)
        out["lone_64_kernel_request_us"] = {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))}
        # the selection kernel alone, from events around its launches: lone 64-kernel requests,
        # then 1,024-kernel batches (16 requests queued while the dispatcher is paused)
        A.aiwcrf_profile_enable(True)
        A.aiwcrf_profile_read()
        for i in range(100):
            srv.wait(srv.submit(np.ascontiguousarray(pool[:, i:i + 64]), 1))
        n64, ms64 = A.aiwcrf_profile_read()["serve"]
        for r in range(20):
            srv.pause(True)
            ts = [srv.submit(np.ascontiguousarray(pool[:, 64 * j:64 * j + 64]), r % 4) for j in range(16)]
            srv.pause(False)
            for t in ts:
                srv.wait(t)
        n1k, ms1k = A.aiwcrf_profile_read()["serve"]
        A.aiwcrf_profile_enable(False)
        out["kernel"] = {
            "batch_64_us": 1e3 * ms64 / max(n64, 1), "batch_64_launches": n64,
            "batch_1024_us": 1e3 * ms1k / max(n1k, 1), "batch_1024_launches": n1k,
            "batch_1024_queries_per_s": 1024 * SEL_DEVICES * n1k / (ms1k / 1e3) if ms1k else None}
        # answers checked against the forest fitted at creation
        ref = {}
        f0 = A.aiwcrf_fit(fp, wl.X, wl.y)
        for s_ in range(synth.N_SIZES):
            b = np.zeros(pool.shape[1], np.int32)
            A.aiwcrf_select_device(f0, pool, s_, devices, b)
            ref[s_] = b
        del f0
        blk = 0
        for rate in rates:
            n_refit = n_requests // refit_every + 1
            for _ in range(n_refit):
                e = synth.plain_forest_workload(seed=synth.DATA_SEED + 100 + blk)
                blk += 1
                srv.append(e.X, e.y)
            k = rng.integers(1, 65, n_requests).astype(np.int32)
            first = (rng.integers(0, pool.shape[1] - 64, n_requests)).astype(np.int64)
            size = rng.integers(0, synth.N_SIZES, n_requests).astype(np.int32)
            c0 = srv.stats()
            rep, best, gen, lat = srv.run_load(pool, first, k, size, rate_per_s=rate, seed=int(rate),
                                               timeout_ms=600000)
            c1 = srv.stats()
            rep["refit_ms"] = (c1["refit_us_total"] - c0["refit_us_total"]) / 1e3
            # where the tail comes from: host enqueue time and GPU (copies + kernel) time per batch
            bt, rt = srv.trace()
            nb = int(rep["batches"])
            bt = bt[-nb:] if nb else bt[:0]
            if nb:
                gpu = (bt["t_done_ns"] - bt["t_enqueued_ns"]) / 1e3
                enq = (bt["t_enqueued_ns"] - bt["t_formed_ns"]) / 1e3
                form = np.sort(bt["t_formed_ns"])
                rep["batch_gpu_us"] = {"p50": float(np.median(gpu)), "p99": float(np.percentile(gpu, 99)),
                                       "max": float(gpu.max())}
                rep["batch_enqueue_us"] = {"p50": float(np.median(enq)), "max": float(enq.max())}
                rep["max_gap_between_batches_ms"] = float(np.diff(form).max() / 1e6) if nb > 1 else 0.0
                slow = bt[(gpu > 5000) | (enq > 5000)]
                # where a slow batch's time went: the dispatcher's CPU time and context switches
                # while enqueuing, and the longest gap between its completion polls
                rep["slow_batches"] = [{"t_ms": float((b["t_formed_ns"] - form[0]) / 1e6),
                                        "gpu_ms": float((b["t_done_ns"] - b["t_enqueued_ns"]) / 1e6),
                                        "enqueue_ms": float((b["t_enqueued_ns"] - b["t_formed_ns"]) / 1e6),
                                        "enqueue_cpu_ms": float(b["enqueue_cpu_ns"] / 1e6),
                                        "enqueue_voluntary_switches": int(b["enqueue_voluntary_switches"]),
                                        "enqueue_involuntary_switches": int(b["enqueue_involuntary_switches"]),
                                        "poll_gap_max_ms": float(b["poll_gap_max_ns"] / 1e6)} for b in slow[:8]]
                rep["refit_windows_ms"] = [[float((r["t_start_ns"] - form[0]) / 1e6),
                                            float((r["t_swapped_ns"] - form[0]) / 1e6)]
                                           for r in rt if r["t_start_ns"] >= form[0]]
            rep["requests_over_1ms"] = int((lat > 1_000_000).sum())
            rep["requests_over_10ms"] = int((lat > 10_000_000).sum())
            checked = mism = 0
            off = 0
            for i in range(n_requests):
                if gen[i] == 0:
                    checked += 1
                    mism += int((best[off:off + k[i]] != ref[int(size[i])][first[i]:first[i] + k[i]]).any())
                off += k[i]
            rep["generation_0_requests_checked"] = checked
            rep["generation_0_mismatches"] = mism
            out["runs"].append(rep)
        out["counters"] = srv.stats()
    if surrogate is not None:
        out["gated"] = {"z": gate_z, "var_trees": gate_var_trees, "runs": []}
        sp0 = A.server_params(n_streams=4, max_request_kernels=64, batch_kernels=1024, arena_bytes=64 << 20)
        with A.Server(sp0, fp, wl.X, wl.y, devices) as srv:
            srv.set_surrogate(surrogate, A.gate_params(gate_var_trees, gate_z, ood=True))
            for rate in gated_rates:
                k = rng.integers(1, 65, n_requests).astype(np.int32)
                first = (rng.integers(0, pool.shape[1] - 64, n_requests)).astype(np.int64)
                size = rng.integers(0, synth.N_SIZES, n_requests).astype(np.int32)
                c0 = srv.stats()
                rep, best, gen, lat = srv.run_load(pool, first, k, size, rate_per_s=rate, seed=int(rate) + 1,
                                                   timeout_ms=600000, gated=np.ones(n_requests, np.uint8))
                c1 = srv.stats()
                gk = c1["gated_kernels"] - c0["gated_kernels"]
                rep["fallback_frac"] = (c1["gated_fallback"] - c0["gated_fallback"]) / max(gk, 1)
                agree = tot = 0
                off = 0
                for i in range(n_requests):
                    want = ref[int(size[i])][first[i]:first[i] + k[i]]
                    agree += int((best[off:off + k[i]] == want).sum())
                    tot += int(k[i])
                    off += k[i]
                rep["agreement_with_forest"] = agree / tot
                rep["requests_over_1ms"] = int((lat > 1_000_000).sum())
                out["gated"]["runs"].append(rep)
            out["gated"]["counters"] = srv.stats()
    return out


def oob_report(A, wl, X, forest):
    import torch
    y = torch.from_numpy(wl.y).to(X.device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    mse, rows = A.aiwcrf_oob_error(forest, X, y)
    e1.record()
    torch.cuda.synchronize()
    return {"mse_log10_s2": mse, "rows_out_of_bag": rows / wl.n_rows, "ms": e0.elapsed_time(e1)}


COUNTER_METRICS = {"dram__bytes_read.sum": "dram_bytes", "dram__bytes_write.sum": "dram_bytes",
                   "smsp__inst_executed.sum": "inst", "l1tex__data_pipe_lsu_wavefronts_mem_shared.sum": "smem_wavefronts"}


def write_counters(csv_path: str, command: str, out_path: str | None = None, scale: dict | None = None) -> dict:
    """Per-launch ncu counters of each kernel class from an ncu --csv capture (metrics of
    COUNTER_METRICS), keyed by the kernel source hash so that the bench reports them only while
    the kernels are unchanged. Classes: tree, level_big, level_small (one kernel each); walk
    (the compact or 8-byte predict walk); predict (every launch from the query coding to the
    walk, summed per call)."""
    import csv
    rows = list(csv.reader(open(csv_path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hi]
    ki, ii, mi, ui, vi = (hdr.index(c) for c in ("Kernel Name", "ID", "Metric Name", "Metric Unit", "Metric Value"))
    unit = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9, "": 1,
            "inst": 1, "warp": 1}
    launches = {}                                   # launch ID -> [kernel name, {counter: value}]
    for r in rows[hi + 1:]:
        if len(r) != len(hdr) or r[mi] not in COUNTER_METRICS:
            continue
        name = r[ki].split("(")[0].split("<")[0].split("::")[-1].replace("void ", "").strip()
        e = launches.setdefault(int(r[ii]), [name, {}])
        c = COUNTER_METRICS[r[mi]]
        e[1][c] = e[1].get(c, 0.0) + float(r[vi].replace(",", "")) * unit.get(r[ui], 1)
    per = {}                                        # class -> list of per-launch (or per-call) counters
    in_predict, acc = False, {}
    for lid in sorted(launches):
        name, cnt = launches[lid]
        if name == "code_queries_kernel":
            in_predict, acc = True, {}
        if in_predict:
            for k, v in cnt.items():
                acc[k] = acc.get(k, 0.0) + v
        if name in ("predict4_kernel", "predict_kernel"):
            per.setdefault("walk", []).append(cnt)
            if in_predict:
                per.setdefault("predict", []).append(acc)
                in_predict = False
        elif name in ("level_small_kernel", "level_big_kernel", "tree_grow_kernel"):
            cls = {"tree_grow_kernel": "tree"}.get(name, name.replace("_kernel", ""))
            per.setdefault(cls, []).append(cnt)
    out = {}
    for cls, v in per.items():
        if scale is not None and cls not in scale:
            continue
        keys = sorted({k for c in v for k in c})
        out[cls] = {k: sum(c.get(k, 0.0) for c in v) / len(v) for k in keys}
        out[cls].update({"launches": len(v), "source_sha": source_sha(cls), "command": command})
        if scale is not None:
            # a smaller case scaled to a full launch by the units it processes: instructions and
            # shared wavefronts grow in proportion; DRAM bytes (cache reuse) do not and are dropped
            out[cls] = {k: (x * scale[cls] if k in ("inst", "smem_wavefronts") else x)
                        for k, x in out[cls].items() if k != "dram_bytes"}
            out[cls]["scaled_by"] = scale[cls]
    path = out_path or os.path.join(ROOT, "profiles", "counters.json")
    old = json.load(open(path)) if os.path.exists(path) else {}
    for cls, e in out.items():
        prev = old.get(cls, {})
        if prev.get("source_sha") != e["source_sha"]:
            prev = {}                                   # counters of changed kernels are dropped
        cmds = prev.get("commands", [prev["command"]] if "command" in prev else [])
        merged = {**prev, **e}
        merged.pop("command", None)
        merged["commands"] = cmds + [command] if command not in cmds else cmds
        old[cls] = merged
    with open(path, "w") as fh:
        json.dump(old, fh, indent=1, sort_keys=True)
    return out


def main():
    args = parse()
    if args.write_counters:
        scale = None
        if args.counters_scale is not None:
            scale = {kv.split("=")[0]: float(kv.split("=")[1]) for kv in args.counters_scale}
        print(json.dumps(write_counters(args.write_counters, args.counters_command, scale=scale)))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
