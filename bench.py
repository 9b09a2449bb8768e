"""Benchmark of the fused-BPT hot path on GB300.

One step = RR sampling of 1,048,576 samples on the R-MAT scale-22 weighted-
cascade graph (fbpt_sample) plus greedy max-coverage k = 100
(fbpt_select_seeds), inputs resident in HBM.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank samples its own range of sample ids on a
replica of the graph (no data-path collective; weak scaling); the step time is
the maximum over ranks.  --impl reference times the CPU oracle on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "rmat_s22_wc"
# DRAM bytes (read + write) per 4-edge group of a k_expand launch (start
# vertices, expand and sweep), from an ncu capture of the current kernel on the
# s22 workload in degree order (five launches, levels 600-604: 774,158,592 B over
# 21,148,211 groups); the bench scales it by its own groups per launch.  None
# when the kernel has changed since the capture.
EXPAND_DRAM_BYTES_PER_GROUP = ((151935488 + 151389696 + 152336640 + 151331328 + 151704320) +
                               (5079808 + 2358016 + 2384128 + 2474752 + 3164416)) / 21148211
EXPAND_TRAFFIC_NOTE = ("ncu dram__bytes_read + dram__bytes_write per group of the current kernel "
                       "(s22, degree order, levels 600-604) x this run's groups per launch")
METRIC = "RR samples/s (bit-exact RR sets + greedy seeds, R-MAT s22 WC, 1,048,576 samples, k=100)"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def build_workload(name=WORKLOAD):
    w = synth.WORKLOADS[name]()
    return w, w.graphs[0]


def rank_samples(rank: int, S: int):
    """Sample ids of one rank under weak scaling: every rank samples S ids of
    its own range on a replica of the graph (no data-path collective)."""
    return rank * S, S


def max_over_ranks(dist, value: float, device: str) -> float:
    """The step time of the whole job: the slowest rank's."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(g, seed, sample_count):
    """The oracle as it stands (per-sample BFS + greedy), all host cores."""
    import oracle
    t = time.perf_counter()
    rr = oracle.rr_sets(g, seed, 0, sample_count)
    oracle.greedy(g.n, rr, 100)
    dt = time.perf_counter() - t
    return {"value": sample_count / dt, "unit": "RR samples/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"first {sample_count} sample ids of the workload (per-sample BFS + greedy k=100 over them), "
                      f"{dt:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, g = build_workload()
    cnt = 8192
    vals = []
    for _ in range(args.warmup + args.steps if args.steps else 1):
        vals.append(cpu_baseline(g, w.seeds[0], cnt))
    v = statistics.median([x["value"] for x in vals[args.warmup:]] or [vals[-1]["value"]])
    cb = dict(vals[-1])
    cb["value"] = v
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "RR samples/s",
                      "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                      "higher_is_better": True, "dtype": "u64", "data": "synthetic",
                      "config": {"workload": WORKLOAD, "graph": g.name, "n": g.n, "m": g.m, "samples": cnt, "k": 100},
                      "cpu_baseline": cb,
                      "e2e": {"value": v, "unit": "RR samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def bench_batched(fbpt, torch, stream, steps, schedule):
    """The 32-graph workload (R-MAT scales 12-20, edge factors 8-32, uniform p
    in [0.01, 0.1], 4,096-262,144 samples per graph), from the plain fused form
    to the learned batched form one change at a time (each arm warmed up once,
    then `steps` timed calls; all arms give the same bits):
      plain            graph after graph, one host launch per level, 8-word
                       batches run to completion, push levels
      lane_refill      the same with lane refill
      tuned            each graph at its autotuned row width and CTA count, its
                       levels in one CUDA-graph launch, push levels
      batched_push     the tuned shapes, every graph in ONE CUDA-graph launch
      batched_heuristic / batched_learned   the same shapes under the degree-
                       ratio heuristic / the policy network's schedule
      learned_batched  the autotuner's pick of shape and schedule (it judges
                       the learned schedule against the heuristic and push)."""
    w = synth.batched_32()
    total = sum(w.S)
    firsts = [0] * len(w.graphs)
    dgs = [fbpt.Graph.from_synth(g, stream) for g in w.graphs]
    t0 = time.perf_counter()
    tuned = [fbpt.autotune(dg, seed, S, schedule=schedule) for dg, seed, S in zip(dgs, w.seeds, w.S)]
    tune_s = time.perf_counter() - t0
    arms = {}

    def run_arm(name, call):
        ms, st = timed_calls(torch, stream, call, steps)
        arms[name] = {"value": total / (ms / 1e3), "unit": "RR samples/s", "ms_per_step": ms,
                      "colour_edge_visits_per_s": st.colour_edge_visits / (ms / 1e3), "levels": int(st.levels),
                      "rr_entries": int(st.rr_total)}

    def batched(**kw):
        def call():
            outs, st = fbpt.sample_batched(dgs, w.seeds, firsts, w.S, stream=stream, **kw)
            del outs
            return st
        return call

    def one_by_one(kws):
        def call():
            agg = fbpt.Stats()
            for dg, seed, S, kw in zip(dgs, w.seeds, w.S, kws):
                rr = fbpt.sample(dg, seed, 0, S, stream=stream, **kw)
                for k in ("levels", "colour_edge_visits", "rr_total"):
                    setattr(agg, k, getattr(agg, k) + getattr(rr.stats, k))
                del rr
            return agg
        return call

    run_arm("plain", batched(launch="host", words=8, slots=1, refill="batch", schedule="push"))
    run_arm("lane_refill", batched(launch="host", words=8, slots=1, refill="lane", schedule="push"))
    shapes = [dict(words=t["words"], slots=t["slots"], blocks=t["blocks"], refill="lane") for t in tuned]
    run_arm("tuned", one_by_one([dict(s, schedule="push", launch="graph") for s in shapes]))
    for sched in ("push", "heuristic", "learned"):
        for dg, sh in zip(dgs, shapes):
            fbpt.set_tuning(dg, sh["words"], sh["slots"], "lane", sh["blocks"], sched)
        run_arm("batched_" + sched, batched(schedule=sched))
    for dg, t in zip(dgs, tuned):
        fbpt.set_tuning(dg, t["words"], t["slots"], "lane", t["blocks"], t["schedule"])
    run_arm("learned_batched", batched(schedule=schedule))
    for dg in dgs:
        dg.close()
    base = arms["plain"]["value"]
    out = {"graphs": len(w.graphs), "samples": total, "steps": steps, "tune_s": tune_s,
           "tuned_schedules": {k: sum(1 for t in tuned if t["schedule"] == k) for k in ("push", "heuristic", "learned")},
           **arms}
    out["speedup"] = arms["learned_batched"]["value"] / base
    out["steps_over_plain"] = {k: v["value"] / base for k, v in arms.items()}
    out["learned_over_heuristic"] = arms["batched_learned"]["value"] / arms["batched_heuristic"]["value"]
    return out


def timed_calls(torch, stream, call, steps):
    """call() once untimed, then `steps` calls between CUDA events on stream;
    returns (ms per call, the last call's result)."""
    res = call()
    del res
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        res = call()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, res


def bench_fused_unfused(fbpt, torch, stream, steps):
    """R-MAT s20 weighted cascade, 65,536 samples: the plain fused form of
    Listing 1 in batches of W = 1, 2, 4, 8 words (64 W colours per batch, a new
    batch when all have finished, push levels, one graph launch) against the
    same samples unfused (one traversal unit per colour, every colour reading
    every edge itself; the same kernels and bits).  RR samples/s and
    colour-edge visits/s per arm; edge accesses are what Theorem 1 bounds."""
    w = synth.rmat_s20_wc()
    g, S, seed = w.graphs[0], w.S[0], w.seeds[0]
    dg = fbpt.Graph.from_synth(g, stream)
    out = {"workload": "rmat_s20_wc", "samples": S, "steps": steps}
    for W in (1, 2, 4, 8):
        row = {}
        for arm, unf in (("fused", False), ("unfused", True)):
            kw = dict(words=W, slots=1, refill="batch", schedule="push", launch="graph", unfused=unf)

            def call():
                rr = fbpt.sample(dg, seed, 0, S, **kw)
                return rr.stats
            ms, st = timed_calls(torch, stream, call, steps)
            row[arm] = {"value": S / (ms / 1e3), "unit": "RR samples/s", "ms_per_step": ms,
                        "colour_edge_visits_per_s": st.colour_edge_visits / (ms / 1e3),
                        "edge_accesses": int(st.edge_accesses), "philox_calls": int(st.philox_calls),
                        "levels": int(st.levels), "ms_expand": st.ms_expand}
        row["fused_over_unfused"] = row["fused"]["value"] / row["unfused"]["value"]
        out[f"W{W}"] = row
    dg.close()
    return out


def bench_s24(fbpt, torch, stream, samples, chunk, words=8):
    """R-MAT scale 24 with trivalency p per edge (16,777,216 vertices, ~263M
    in-edges), sample ids 0 .. samples-1 in calls of `chunk` samples (each
    call's RR sets are built in full, then released: the whole output would
    not fit in memory), at 8-word rows with lane refill, under the policy
    network's schedule and under the degree-ratio heuristic.  Greedy k = 200
    runs on the first chunk's sets."""
    w = synth.rmat_s24_tri()
    g, seed = w.graphs[0], w.seeds[0]
    t0 = time.perf_counter()
    dg = fbpt.Graph.from_synth(g, stream)
    upload_s = time.perf_counter() - t0
    out = {"workload": "rmat_s24_tri", "n": g.n, "m": g.m, "samples": samples, "chunk": chunk, "words": words,
           "upload_s": upload_s}
    for sched in ("learned", "heuristic"):
        kw = dict(words=words, slots=1, refill="lane", schedule=sched, launch="graph")
        warm = fbpt.sample(dg, seed, 0, min(chunk, 1024), stream=stream, **kw)
        del warm
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        agg = {"levels": 0, "pull_levels": 0, "colour_edge_visits": 0, "rr_total": 0, "philox_calls": 0}
        e0.record(stream)
        for c0 in range(0, samples, chunk):
            rr = fbpt.sample(dg, seed, c0, min(chunk, samples - c0), stream=stream, **kw)
            if c0 == 0 and sched == "learned":
                seeds, _ = fbpt.select_seeds(rr, w.k)
            st = rr.stats
            for k in agg:
                agg[k] += int(getattr(st, k))
            del rr
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[sched] = {"value": samples / (ms / 1e3), "unit": "RR samples/s", "ms": ms,
                      "colour_edge_visits_per_s": agg["colour_edge_visits"] / (ms / 1e3), **agg}
    out["learned_over_heuristic"] = out["learned"]["value"] / out["heuristic"]["value"]
    dg.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--words", type=int, default=0, help="0 = the autotuned shape")
    ap.add_argument("--slots", type=int, default=0)
    ap.add_argument("--schedule", default="learned")
    ap.add_argument("--launch", default="graph")
    ap.add_argument("--samples", type=int, default=1 << 20)
    ap.add_argument("--batched-steps", type=int, default=1,
                    help="timed steps of the 32-graph batched comparison (0 = skip)")
    ap.add_argument("--workload", default=WORKLOAD, choices=["rmat_s20_wc", "rmat_s22_wc"],
                    help="single-graph workload (profiling runs; the reported line is rmat_s22_wc)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-fused comparison on this workload")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffers) measurement")
    ap.add_argument("--order", default="degree", choices=["identity", "rcm", "degree", "random", "cluster"],
                    help="vertex order of the sampled graph (host preprocessing, outside the timed steps)")
    ap.add_argument("--sorted-starts", action=argparse.BooleanOptionalAction, default=True,
                    help="samples take lanes by (relabelled) start vertex")
    ap.add_argument("--fused-steps", type=int, default=2,
                    help="timed calls per arm of the fused-vs-unfused W sweep on R-MAT s20 (0 = skip)")
    ap.add_argument("--s24-samples", type=int, default=65536,
                    help="samples of the R-MAT s24 trivalency measurement (0 = skip; 4194304 = the full workload)")
    ap.add_argument("--s24-chunk", type=int, default=8192, help="samples per sampling call on R-MAT s24")
    ap.add_argument("--only", default=None, choices=["batched", "fused", "s24"],
                    help="run one comparison alone and print its object")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2311_10201_gb300 as fbpt
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    fbpt.build()
    if args.only:
        stream = torch.cuda.current_stream()
        if args.only == "batched":
            res = bench_batched(fbpt, torch, stream, max(args.batched_steps, 1), args.schedule)
        elif args.only == "fused":
            res = bench_fused_unfused(fbpt, torch, stream, max(args.fused_steps, 1))
        else:
            res = bench_s24(fbpt, torch, stream, args.s24_samples, args.s24_chunk)
        print(json.dumps({"only": args.only, args.only: res}))
        return
    w, g = build_workload(args.workload)
    S = args.samples
    k = w.k or 100
    seed = w.seeds[0]
    first, S = rank_samples(rank, S)
    stream = torch.cuda.current_stream()
    dg = fbpt.Graph.from_synth(g, stream)
    perm = None
    order_s = 0.0
    if args.order != "identity" or args.sorted_starts:
        t0 = time.perf_counter()
        perm = fbpt.order_compute(g.n, g.row_ptr, g.col, args.order)
        order_s = time.perf_counter() - t0
        dg.set_order(perm, args.sorted_starts)
    # launch shape: measured by the autotuner before the timed region (like a
    # library's algorithm search), unless given on the command line
    if args.words:
        kw = dict(words=args.words, slots=args.slots, schedule=args.schedule, launch=args.launch)
        tuned = None
    else:
        tuned = fbpt.autotune(dg, seed, S, schedule=args.schedule)
        kw = dict(words=tuned["words"], slots=tuned["slots"], blocks=tuned["blocks"], refill="lane",
                  schedule=tuned["schedule"], launch=args.launch)

    def step():
        rr = fbpt.sample(dg, seed, first, S, **kw)
        seeds, gains = fbpt.select_seeds(rr, k)
        return rr, seeds

    for _ in range(args.warmup):
        rr, seeds = step()
        del rr
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stats = []
    ev0.record(stream)
    for _ in range(args.steps):
        rr, seeds = step()
        stats.append(rr.stats)
        del rr
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    if dist:
        ms = max_over_ranks(dist, ms, "cuda")
        dist.barrier()
    ms_step = ms / args.steps
    value = S * world * args.steps / (ms / 1e3)

    st = stats[-1]

    # ---- the plain fused form on the same workload: Listing 1 with 512
    # colours per batch, a new batch only when every colour has finished,
    # push levels only, one host-driven launch per level ----
    plain_kw = dict(words=8, slots=1, refill="batch", schedule="push", launch="host")
    plain = None
    if rank == 0 and world == 1 and not args.no_plain:
        def plain_step():
            rr = fbpt.sample(dg, seed, first, S, **plain_kw)
            fbpt.select_seeds(rr, k)
            return rr
        warm = plain_step()
        del warm
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        psteps = max(1, min(args.steps, 3))
        e0.record(stream)
        for _ in range(psteps):
            prr = plain_step()
            del prr
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / psteps
        plain = {"value": S / (pms / 1e3), "unit": "RR samples/s", "ms_per_step": pms, "steps": psteps,
                 "shape": plain_kw, "speedup": (S / (ms_step / 1e3)) / (S / (pms / 1e3))}

    # ---- the consumer of the path: IMM seed selection (k = 100, epsilon = 0.1,
    # ell = 1) on the same graph and shape, sampling and greedy included ----
    imm = None
    if rank == 0 and world == 1 and not args.no_plain:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, ires, ist = fbpt.imm(dg, k, 0.1, 1.0, seed, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        imm = {"k": k, "epsilon": 0.1, "ell": 1.0, "seconds": dt, "samples": ires["samples"],
               "theta": ires["theta"], "rounds": ires["rounds"], "lower_bound": ires["lower_bound"],
               "coverage": ires["coverage"], "samples_per_s": ires["samples"] / dt}

    # ---- the same step in the other vertex order (Section 5: vertices
    # relabelled by decreasing degree, samples taking lanes by start vertex,
    # against the caller's order): the order is host preprocessing like the
    # graph upload, outside the timed steps, and the RR sets are the same bits ----
    ordered = None
    if rank == 0 and world == 1 and not args.no_plain:
        try:
            t0 = time.perf_counter()
            if perm is None:
                operm, o_name, o_sorted = fbpt.order_compute(g.n, g.row_ptr, g.col, "degree"), "degree", True
            else:
                operm, o_name, o_sorted = None, "identity", False
            host_s = time.perf_counter() - t0
            dg.set_order(operm, o_sorted)
            warm, _ = step()
            ref_total = warm.total
            del warm
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            osteps = max(1, min(args.steps, 3))
            e0.record(stream)
            for _ in range(osteps):
                orr, _ = step()
                ost = orr.stats
                del orr
            e1.record(stream)
            torch.cuda.synchronize()
            oms = e0.elapsed_time(e1) / osteps
            ordered = {"order": o_name, "sorted_starts": o_sorted, "value": S / (oms / 1e3), "unit": "RR samples/s",
                       "ms_per_step": oms, "steps": osteps, "host_order_s": host_s, "levels": int(ost.levels),
                       "groups_expanded": int(ost.groups_expanded), "rr_total": int(ref_total),
                       "same_rr_total": int(ref_total) == int(st.rr_total),
                       "headline_over_this": (S / (ms_step / 1e3)) / (S / (oms / 1e3))}
        except Exception as ex:  # reported, never fatal to the line
            ordered = {"error": str(ex)[:200]}
        finally:
            try:
                dg.set_order(perm, args.sorted_starts if perm is not None else False)
            except Exception:
                pass

    # ---- the linear-threshold model on the same graph (WC weights sum to at
    # most 1 per row): RR walks instead of cascades, same shape, seeds included ----
    lt = None
    if rank == 0 and world == 1 and not args.no_plain:
        try:
            lkw = dict(words=8, slots=8, refill="lane", schedule="push", launch=args.launch, model="lt")

            def lt_step():
                lrr = fbpt.sample(dg, seed, first, S, **lkw)
                fbpt.select_seeds(lrr, k)
                return lrr
            warm = lt_step()
            del warm
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            lsteps = max(1, min(args.steps, 2))
            e0.record(stream)
            for _ in range(lsteps):
                lrr = lt_step()
                lst = lrr.stats
                ltotal = lrr.total
                del lrr
            e1.record(stream)
            torch.cuda.synchronize()
            lms = e0.elapsed_time(e1) / lsteps
            lt = {"model": "lt", "value": S / (lms / 1e3), "unit": "RR samples/s", "ms_per_step": lms,
                  "steps": lsteps, "levels": int(lst.levels), "rr_total": int(ltotal)}
        except Exception as ex:  # reported, never fatal to the line
            lt = {"error": str(ex)[:200]}

    batched = None
    if rank == 0 and world == 1 and args.batched_steps > 0:
        batched = bench_batched(fbpt, torch, stream, args.batched_steps, args.schedule)
    fused = None
    if rank == 0 and world == 1 and args.fused_steps > 0:
        fused = bench_fused_unfused(fbpt, torch, stream, args.fused_steps)
    s24 = None
    if rank == 0 and world == 1 and args.s24_samples > 0:
        try:
            s24 = bench_s24(fbpt, torch, stream, args.s24_samples, args.s24_chunk)
        except Exception as ex:  # reported, never fatal to the line
            s24 = {"error": str(ex)[:200]}

    # ---- roofline of the dominant kernel (the level's first kernel), per launch ----
    # HBM is the roofline: nothing on the path is a dense contraction.  The
    # kernel places the new start vertices, expands the frontier and sweeps the
    # finished lanes.  Algorithmic bytes of one launch: expand, 8 B of col + thr
    # per in-edge read (edge accesses), 40 B per frontier unit (its record and
    # chunk-map entry), 8 B per colour word of a unit (stage word); init, 40 B per
    # started sample (start id, next and occupancy words read and written, a
    # pending entry); sweep, 32 B per RR entry (segment entry read, staging
    # entry written, visited word and vertex count read and written; 36 B with
    # a vertex order, whose inverse is read).  The launch duration is measured
    # with CUDA events around every expand launch of one host-launched call of
    # the same shape right after the timed steps (inside the timed graph launch
    # all levels run within one launch); the device %globaltimer brackets of the
    # expand phase in the timed steps are reported beside it.  Secondary view:
    # the liveness draws against the measured rate of a Philox-only kernel.
    launches = max(int(st.levels), 1)
    sweep_b = 36 if perm is not None else 32
    alg_bytes = (8 * st.edge_accesses + 40 * st.units_expanded + 8 * st.mask_words + 40 * S
                 + sweep_b * st.rr_total) / launches
    pk, pk_kind = peaks()
    ev_rr = fbpt.sample(dg, seed, first, S, **dict(kw, launch="host"))
    ev = ev_rr.stats
    del ev_rr
    ev_launches = max(int(ev.levels), 1)
    launch_s = ev.ms_expand_events * 1e-3 / ev_launches
    achieved = alg_bytes / launch_s / 1e9 if launch_s > 0 else 0.0
    exp_s = st.ms_expand * 1e-3
    philox_peak = fbpt.philox_rate(seed, 16384)
    calls_s = st.philox_calls / exp_s if exp_s else 0.0
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
            "traffic": (EXPAND_DRAM_BYTES_PER_GROUP * st.groups_expanded / launches
                        if EXPAND_DRAM_BYTES_PER_GROUP else None),
            "traffic_note": EXPAND_TRAFFIC_NOTE,
            "kernel": "k_expand", "peak_kind": pk_kind + " (copy bandwidth, MEASURED_PEAKS.json)",
            "algorithmic_bytes_per_launch": alg_bytes, "launches_per_step": launches,
            "launch_us_events": launch_s * 1e6, "event_pass_levels": int(ev.levels),
            "expand_ms_per_step_globaltimer": st.ms_expand,
            "launch_us_globaltimer": st.ms_expand * 1e3 / launches,
            "limiter": "latency: issue-active and DRAM throughput both low in the ncu capture (profiles/)",
            "alu_view": {"philox_calls_per_s": calls_s, "peak_calls_per_s": philox_peak,
                         "frac": calls_s / philox_peak if philox_peak else None,
                         "peak_kind": "measured: fbpt_philox_rate (Philox-only kernel, CUDA events)",
                         "sms": sms}}

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        h_rp, h_col, h_thr = pin(g.row_ptr.view(np.int64)), pin(g.col.view(np.int32)), pin(g.thr.view(np.int32))
        e2e_steps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d = d2h = 0
        for _ in range(e2e_steps):
            hg = fbpt.Graph(g.n, h_rp.numpy().view(np.uint64), h_col.numpy().view(np.uint32),
                            h_thr.numpy().view(np.uint32), stream)
            if perm is not None:
                hg.set_order(perm, args.sorted_starts)
            rr = fbpt.sample(hg, seed, first, S, **kw)
            seeds, gains = fbpt.select_seeds(rr, k)
            off = torch.empty(S + 1, dtype=torch.int64, pin_memory=True)
            verts = torch.empty(max(rr.total, 1), dtype=torch.int32, pin_memory=True)
            fbpt.lib().fbpt_rrsets_copy_to_host(fbpt.ctypes.byref(rr.c), off.data_ptr(), verts.data_ptr(), None, None)
            h2d = g.row_ptr.nbytes + g.col.nbytes + g.thr.nbytes + (perm.nbytes if perm is not None else 0)
            d2h = off.numel() * 8 + rr.total * 4 + k * 12
            del rr
            hg.close()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        if dist:
            e2e_s = max_over_ranks(dist, e2e_s, "cuda")
        e2e = {"value": S * world / e2e_s, "unit": "RR samples/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}


    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(g, seed, 40960)  # about 10 s of the oracle on 16 cores

    # kernels per step: 3 or 4 per level (expand with start vertices and sweep,
    # commit, scheduler; + the filtered/pull expand when the schedule may pick
    # it), the final sweep, the row-length scan (3), the three row-ordering
    # kernels, greedy 2 per pick + 3
    per_level = 3 + (1 if kw.get("schedule", "push") != "push" else 0)
    launches_step = per_level * int(st.levels) + 1 + 3 + 3 + 2 * k + 3
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "RR samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.workload, "graph": g.name, "n": g.n, "m": g.m, "samples_per_gpu": S, "k": k,
                       "shape": kw, "autotuned": tuned, "order": args.order, "sorted_starts": args.sorted_starts,
                       "host_order_s": order_s,
                       "l2": "inputs larger than L2 (in-CSR + thresholds %.0f MB)" % ((g.m * 8 + g.n * 8) / 1e6)},
            "plain_fused": plain, "ordered": ordered, "lt": lt, "batched_32": batched, "imm": imm,
            "fused_vs_unfused_s20": fused, "s24_tri": s24,
            "colour_edge_visits_per_s": st.colour_edge_visits * world / (ms_step / 1e3),
            "stats": st.as_dict(),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches_step * args.steps,
        }))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
