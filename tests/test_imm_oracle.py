"""Pins of the IMM oracle (oracle/imm.py) against facts outside it: a graph
whose sampling rounds and theta follow by hand, the (1 - 1/e - eps)
approximation guarantee against the exact optimum of tiny graphs (influence by
enumeration of every live-edge world), and the monotone dependence of theta on
epsilon and k.  CPU only."""
import itertools
import math

import numpy as np
import pytest

import synth
from oracle import imm as oimm


def graph(n, edges, p):
    """In-CSR from directed edges (u -> v), uniform p."""
    order = sorted(range(len(edges)), key=lambda i: (edges[i][1], edges[i][0]))
    row_ptr = np.zeros(n + 1, np.uint64)
    col = np.zeros(len(edges), np.uint32)
    for k, i in enumerate(order):
        u, v = edges[i]
        row_ptr[v + 1] += 1
        col[k] = u
    row_ptr = np.cumsum(row_ptr).astype(np.uint64)
    g = synth.Graph(n, row_ptr, col, synth.thr_uniform(len(edges), p), "imm-test")
    return g, [edges[i] for i in order]


def exact_influence(n, edges, p, S):
    """sigma(S): expected number of vertices reached forward from S over every
    live-edge world (each edge live with probability p)."""
    total = 0.0
    for alive in itertools.product([0, 1], repeat=len(edges)):
        w = 1.0
        adj = [[] for _ in range(n)]
        for (u, v), a in zip(edges, alive):
            w *= p if a else 1 - p
            if a:
                adj[u].append(v)
        seen = set(S)
        stack = list(S)
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if y not in seen:
                    seen.add(y)
                    stack.append(y)
        total += w * len(seen)
    return total


def test_star_rounds_and_theta_by_hand():
    """p = 1 on a star whose centre 0 points at every other vertex: every RR
    set holds its start and 0, so greedy's first pick is 0 and covers every
    set.  The first round (x = n/2) already passes n * 1 >= (1 + eps') n/2,
    so LB = n / (1 + eps') and theta = ceil(lambda* / LB)."""
    n, eps, ell = 64, 0.5, 1.0
    g, _ = graph(n, [(0, v) for v in range(1, n)], 1.0)
    seeds, gains, info = oimm.imm(g, 1, eps, ell, 17)
    epsp, lam_p, lam_s = oimm.imm_params(n, 1, eps, ell)
    assert info["rounds"] == 1
    assert info["lower_bound"] == n / (1.0 + epsp)
    assert info["theta"] == math.ceil(lam_s / (n / (1.0 + epsp)))
    # the final selection runs over theta fresh sets, after the round's lambda' / (n / 2)
    assert info["samples"] == info["theta"]
    assert info["first_final_id"] == math.ceil(lam_p / (n / 2.0))
    assert seeds.tolist() == [0] and gains.tolist() == [info["samples"]]
    assert info["coverage"] == 1.0


def test_isolated_vertices_need_every_round():
    """No edges: every RR set is its start alone, so one seed covers about a
    1/n share and n F (~1.4 here) stays below (1 + eps') x (>= 3.4) in every
    round i = 1 .. ceil(log2 32) - 1 = 4: LB stays 1 and theta = ceil(lambda*)."""
    n, eps, ell = 32, 0.5, 1.0
    g = synth.Graph(n, np.zeros(n + 1, np.uint64), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    seeds, gains, info = oimm.imm(g, 1, eps, ell, 5)
    epsp, lam_p, lam_s = oimm.imm_params(n, 1, eps, ell)
    assert info["rounds"] == math.ceil(math.log2(n)) - 1
    assert info["lower_bound"] == 1.0
    assert info["theta"] == math.ceil(lam_s) == info["samples"]


@pytest.mark.parametrize("gseed", [1, 2, 3, 4])
def test_guarantee_against_the_exact_optimum(gseed):
    """sigma(IMM seeds) >= (1 - 1/e - eps) OPT on random graphs of 7 vertices
    and 11 edges (p = 0.4), OPT over every pair of vertices, both by exact
    enumeration of the 2^11 worlds."""
    rng = np.random.default_rng(gseed)
    n, k, eps = 7, 2, 0.25
    pairs = [(u, v) for u in range(n) for v in range(n) if u != v]
    idx = rng.choice(len(pairs), 11, replace=False)
    g, edges = graph(n, [pairs[i] for i in idx], 0.4)
    seeds, gains, info = oimm.imm(g, k, eps, 1.0, 100 + gseed)
    p = int(g.thr[0]) / 2**32
    opt = max(exact_influence(n, edges, p, S) for S in itertools.combinations(range(n), k))
    got = exact_influence(n, edges, p, [int(s) for s in seeds])
    assert got >= (1 - 1 / math.e - eps) * opt
    # the estimate n * F_R(S) is close to sigma(S) at IMM's sample size
    assert abs(n * info["coverage"] - got) <= 0.1 * got


def test_theta_grows_as_epsilon_shrinks_and_k_grows():
    g = synth.rmat_wc(10)
    a = oimm.imm(g, 5, 0.5, 1.0, 3)[2]
    b = oimm.imm(g, 5, 0.3, 1.0, 3)[2]
    c = oimm.imm(g, 20, 0.3, 1.0, 3)[2]
    assert b["lambda_star"] > a["lambda_star"] and b["samples"] >= a["samples"]
    assert c["lambda_star"] > b["lambda_star"] and c["lambda_prime"] > b["lambda_prime"]
