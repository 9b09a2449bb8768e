"""Collect per-level traces under fixed schedules and fit the schedule network.

Level actions (outputs 0..4).  For each workload and each fixed schedule --
push, filtered push and pull with the pending queue, push and filtered push
with the scan of the occupancy masks (pull only where the row width allows
it) -- one sampling run records its level trace; every level gives a training
row: the six features the scheduler computed on the device for that level
(the trace rows carry them), the action it ran with, and the log2 of its
expand + commit device time.  A level's frontier does not depend on how it is
expanded, so the runs list the same levels.

Row width (outputs 5..7).  For each workload, runs at rows of 4, 16 and 64
words (lane refill, push) are timed; every level of a reference run (8 words x
1 slot, as fbpt_policy_width probes) gives three rows: its features, the
output of that width and the log2 of the ns per sample measured at it.

fbpt_policy_train fits the network on the GPU; the parameters are written as
text (one float per line).

    python -m paper_2311_10201_gb300.train_policy --out policy.txt
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import paper_2311_10201_gb300 as fbpt  # noqa: E402
import synth  # noqa: E402

# fixed schedules and the network output (action) each one trains
RUNS = (("push", "queue", 0), ("filtered", "queue", 1), ("pull", "queue", 2), ("push", "scan", 3),
        ("filtered", "scan", 4))
WIDTHS = (4, 16, 64)   # words; outputs 5, 6, 7
WIDTH_OUT = 5


def action_of(trace):
    d = trace["direction"].astype(np.uint32)
    scan = (trace["compaction"] == 1) & (d != 2)
    return d + 3 * scan.astype(np.uint32)


def rows_of(trace):
    """Training rows of one trace: the device-computed features of each level
    with a frontier, the action it ran with, log2 of its expand + commit ns."""
    keep = trace["units"] > 0
    keep[0] = False  # row 0's level had no schedule step before it
    t = trace[keep]
    X = t["features"].astype(np.float64)
    A = action_of(t)
    Y = np.log2(1.0 + t["expand_ns"].astype(np.float64) + t["commit_ns"].astype(np.float64))
    return X, A, Y


def collect(dg, seed, S, shapes, first=0):
    Xs, As, Ys = [], [], []
    for words, slots, refill in shapes:
        for sched, comp, _ in RUNS:
            if sched == "pull" and words * slots > 8:
                continue
            kw = dict(words=words, slots=slots, refill=refill, schedule=sched, compaction=comp, launch="graph")
            fbpt.sample(dg, seed, first, S, **kw)  # warm-up (workspace, out-CSR)
            rr = fbpt.sample(dg, seed, first, S, trace_cap=1 << 20, **kw)
            X, A, Y = rows_of(rr.trace)
            Xs.append(X); As.append(A); Ys.append(Y)
    return np.concatenate(Xs), np.concatenate(As), np.concatenate(Ys)


def width_rows(dg, seed, S):
    """Rows for outputs 5..7: the reference run's level features, each with
    the measured log2 ns per sample of the run at every width."""
    import torch
    ys = []
    for w in WIDTHS:
        kw = dict(words=min(w, 8), slots=max(w // 8, 1), refill="lane", schedule="push", launch="graph")
        fbpt.sample(dg, seed, 0, S, **kw)
        torch.cuda.synchronize()
        rr = fbpt.sample(dg, seed, 0, S, **kw)
        ms = rr.stats.ms_total
        del rr
        ys.append(np.log2(1e6 * ms / S))
    tr = fbpt.sample(dg, seed, 0, min(S, 8192), words=8, slots=1, refill="lane", schedule="push", launch="graph",
                     trace_cap=1 << 16).trace
    keep = tr["units"] > 0
    keep[0] = False
    X = tr[keep]["features"].astype(np.float64)
    Xs = np.concatenate([X] * len(WIDTHS))
    As = np.concatenate([np.full(len(X), WIDTH_OUT + k, np.uint32) for k in range(len(WIDTHS))])
    Ys = np.concatenate([np.full(len(X), ys[k]) for k in range(len(WIDTHS))])
    return Xs, As, Ys, ys


def training_graphs(quick=False):
    """(graph, seed, samples, shapes) of the training workloads: the ER 1k and
    R-MAT s20 WC workloads, denser uniform-p R-MATs (so that pull and scan
    levels are represented) and R-MATs of other scales and densities."""
    out = []
    w = synth.er_1k()
    out.append((w.graphs[0], w.seeds[0], 4096, [(1, 1, "batch"), (2, 4, "lane")]))
    out.append((synth.rmat_wc(16 if quick else 20), synth.SAMPLE_SEED, 16384 if quick else 65536,
                [(8, 8, "lane"), (8, 1, "batch"), (1, 1, "batch")]))
    for scale, p, seed, S in ((14 if quick else 16, 0.1, 91, 2048), (14, 0.05, 92, 8192), (13, 0.2, 93, 1024),
                              (15, 0.03, 94, 16384)):
        rp, col = synth.rmat_graph(scale, 16, seed)
        g = synth.Graph(len(rp) - 1, rp, col, synth.thr_uniform(col.size, p), f"rmat{scale}-p{p}")
        out.append((g, synth.SAMPLE_SEED, S, [(8, 1, "batch"), (4, 2, "lane")]))
    for scale in ((14,) if quick else (14, 18)):
        out.append((synth.rmat_wc(scale, seed=900 + scale), synth.SAMPLE_SEED, 32768, [(8, 4, "lane")]))
    return out


def training_set(quick=False):
    Xs, As, Ys = [], [], []
    for g, seed, S, shapes in training_graphs(quick):
        dg = fbpt.Graph.from_synth(g)
        X, A, Y = collect(dg, seed, S, shapes)
        Xw, Aw, Yw, ys = width_rows(dg, seed, max(S, 16384))
        print(f"{g.name}: {len(Y)} level rows, width log2 ns/sample {[round(y, 2) for y in ys]}", flush=True)
        Xs += [X, Xw]; As += [A, Aw]; Ys += [Y, Yw]
        dg.close()
    return np.concatenate(Xs), np.concatenate(As), np.concatenate(Ys)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "policy_default.txt"))
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--save-rows", default=None)
    args = ap.parse_args()
    fbpt.build()
    X, A, Y = training_set(args.quick)
    if args.save_rows:
        np.savez(args.save_rows, X=X, A=A, Y=Y)
    pol, loss = fbpt.policy_train(X, A, Y, steps=args.steps, lr=3e-3, seed=1)
    np.savetxt(args.out, pol.params(), fmt="%.9g")
    print(f"{len(Y)} rows, loss {loss:.4f}, actions {np.bincount(A, minlength=8).tolist()} -> {args.out}")


if __name__ == "__main__":
    main()
