"""Collect per-level traces under fixed schedules and fit the schedule network.

For each workload and each direction (push, filtered push, pull where the row
width allows it) one sampling run records its level trace; every level gives a
training row: the six scheduler features, the direction it ran with, and the
log2 of its expand + commit device time.  fbpt_policy_train fits the network on
the GPU; the parameters are written as text (one float per line).

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

DIRECTIONS = {"push": 0, "filtered": 1, "pull": 2}


def features(trace, m):
    u = trace["units"].astype(np.float64)
    g = trace["groups"].astype(np.float64)
    c = trace["colours"].astype(np.float64)
    lanes = trace["frontier_lanes"].astype(np.float64)
    return np.stack([np.log2(1 + u), np.log2(1 + g), np.log2(1 + c), np.log2(1 + lanes),
                     np.log2(1 + 4 * g) - np.log2(1 + float(m)), np.log2(1 + c / np.maximum(u, 1))], axis=1)


def rows_of(trace, m):
    keep = trace["units"] > 0
    t = trace[keep]
    X = features(t, m)
    A = t["direction"].astype(np.uint32)
    Y = np.log2(1.0 + t["expand_ns"].astype(np.float64) + t["commit_ns"].astype(np.float64))
    return X, A, Y


def collect(graph, seed, S, shapes, schedules, first=0):
    dg = fbpt.Graph.from_synth(graph)
    Xs, As, Ys = [], [], []
    for words, slots, refill in shapes:
        for sched in schedules:
            if sched == "pull" and words * slots > 8:
                continue
            kw = dict(words=words, slots=slots, refill=refill, schedule=sched, launch="graph")
            fbpt.sample(dg, seed, first, S, **kw)  # warm-up (workspace, out-CSR)
            rr = fbpt.sample(dg, seed, first, S, trace_cap=1 << 20, **kw)
            X, A, Y = rows_of(rr.trace, graph.m)
            Xs.append(X); As.append(A); Ys.append(Y)
    dg.close()
    return np.concatenate(Xs), np.concatenate(As), np.concatenate(Ys)


def training_set(quick=False):
    """Traces of the ER 1k and R-MAT s20 WC workloads (plus a denser uniform-p
    R-MAT so that pull levels are represented)."""
    scheds = ("push", "filtered", "pull")
    parts = []
    w = synth.er_1k()
    parts.append(collect(w.graphs[0], w.seeds[0], 4096, [(1, 1, "batch"), (2, 4, "lane")], scheds))
    g20 = synth.rmat_wc(16 if quick else 20)
    parts.append(collect(g20, synth.SAMPLE_SEED, 16384 if quick else 65536,
                         [(8, 8, "lane"), (8, 1, "batch"), (1, 1, "batch")], scheds))
    rp, col = synth.rmat_graph(14 if quick else 16, 16, 91)
    dense = synth.Graph(len(rp) - 1, rp, col, synth.thr_uniform(col.size, 0.1), "rmat-dense")
    parts.append(collect(dense, synth.SAMPLE_SEED, 2048, [(8, 1, "batch"), (4, 2, "lane")], scheds))
    X = np.concatenate([p[0] for p in parts])
    A = np.concatenate([p[1] for p in parts])
    Y = np.concatenate([p[2] for p in parts])
    return X, A, Y


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
    print(f"{len(Y)} rows, loss {loss:.4f}, actions {np.bincount(A, minlength=3).tolist()} -> {args.out}")


if __name__ == "__main__":
    main()
