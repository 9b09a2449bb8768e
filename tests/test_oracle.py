"""Pins of the CPU oracle against facts fixed outside it: published Philox
vectors, closed forms, exact enumeration of live-edge worlds, library graph
search, the greedy approximation bound and Theorem 1.  CPU only."""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import breadth_first_order

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_graph(edges, n, probs):
    """In-CSR from a list of directed edges (u -> v) with per-edge p."""
    order = sorted(range(len(edges)), key=lambda i: (edges[i][1], edges[i][0]))
    row_ptr = np.zeros(n + 1, np.uint64)
    col = np.zeros(len(edges), np.uint32)
    thr = np.zeros(len(edges), np.uint32)
    for k, i in enumerate(order):
        u, v = edges[i]
        row_ptr[v + 1] += 1
        col[k] = u
        thr[k] = synth.threshold(probs[i])
    row_ptr = np.cumsum(row_ptr).astype(np.uint64)
    return synth.Graph(n, row_ptr, col, thr, "small"), [edges[i] for i in order], [probs[i] for i in order]


# ---- Philox4x32-10 -------------------------------------------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox(v[0:4], v[4:6]) == v[6:10]


def test_philox_bits_balanced():
    ones = np.zeros(32)
    N = 20000
    for i in range(N):
        w = oracle.philox([i, 7, 0, 0], [0x12345678, 0x9abcdef0])[i & 3]
        ones += (w >> np.arange(32)) & 1
    frac = ones / N
    assert np.all(np.abs(frac - 0.5) < 5 * math.sqrt(0.25 / N))


# ---- The liveness rule -----------------------------------------------------------

def test_threshold_encoding():
    assert synth.threshold(0.1) == 429496729
    assert synth.threshold(0.01) == 42949672
    assert synth.threshold(0.001) == 4294967
    assert synth.threshold(1.0) == 0xFFFFFFFF
    assert synth.threshold(0.0) == 0
    assert synth.threshold(0.5) == 1 << 31


@pytest.mark.parametrize("p", [0.1, 0.5, 0.9])
def test_live_marginal_and_independence(p):
    thr = synth.threshold(p)
    seed = 99
    N = 40000
    rng = np.random.default_rng(1)
    s = rng.integers(0, 1 << 40, N)
    e = (rng.integers(0, 1 << 30, N) // 4) * 4
    a = np.array([oracle.live(seed, int(si), int(ei), thr) for si, ei in zip(s, e)])
    b = np.array([oracle.live(seed, int(si), int(ei) + 1, thr) for si, ei in zip(s, e)])   # same Philox call
    c = np.array([oracle.live(seed, int(si) + 1, int(ei), thr) for si, ei in zip(s, e)])   # next sample
    pe = thr / 2**32
    tol = 5 * math.sqrt(pe * (1 - pe) / N)
    assert abs(a.mean() - pe) < tol
    assert abs((a & b).mean() - pe * pe) < 5 * math.sqrt(pe * pe * (1 - pe * pe) / N)
    assert abs((a & c).mean() - pe * pe) < 5 * math.sqrt(pe * pe * (1 - pe * pe) / N)


def test_live_special_thresholds():
    for s in range(50):
        for e in range(20):
            assert oracle.live(5, s, e, 0xFFFFFFFF)
            assert not oracle.live(5, s, e, 0)


def test_start_uniform_and_in_range():
    n = 13
    counts = np.zeros(n)
    N = 26000
    for s in range(N):
        v = oracle.start(42, s, n)
        assert 0 <= v < n
        counts[v] += 1
    chi2 = ((counts - N / n) ** 2 / (N / n)).sum()
    assert chi2 < 45  # 12 dof; p ~ 1e-5


# ---- RR sets: special cases of Definition 2 -----------------------------------------

def test_p1_equals_reverse_reachability():
    import synth as S
    rp, col = S.er_graph(300, 600, 7)
    g = S.Graph(300, rp, col, S.thr_uniform(col.size, 1.0))
    A = sp.csr_matrix((np.ones(col.size), col.astype(np.int64), rp.astype(np.int64)), shape=(300, 300))
    rr = oracle.rr_sets(g, 3, 0, 60)
    for j in range(60):
        st = int(rr.starts[j])
        ref = np.sort(breadth_first_order(A, st, directed=True, return_predecessors=False))
        assert np.array_equal(rr.row(j), ref)


def test_p0_gives_singletons():
    rp, col = synth.er_graph(200, 800, 8)
    g = synth.Graph(200, rp, col, np.zeros(col.size, np.uint32))
    rr = oracle.rr_sets(g, 11, 5, 100)
    assert np.array_equal(np.diff(rr.offsets), np.ones(100))
    assert np.array_equal(rr.verts, rr.starts)


def test_subset_ids_match_contiguous(er_workload):
    g = er_workload.graphs[0]
    full = oracle.rr_sets(g, 77, 1000, 64)
    ids = np.array([1063, 1000, 1031, 1007], np.uint64)
    sub = oracle.rr_sets(g, 77, ids=ids)
    for k, i in enumerate(ids):
        assert np.array_equal(sub.row(k), full.row(int(i) - 1000))


# ---- Exact enumeration of live-edge worlds ------------------------------------------------

TINY_EDGES = [(1, 0), (2, 0), (2, 1), (3, 2), (4, 2), (0, 3), (4, 1), (5, 4), (3, 5), (1, 5)]
TINY_P = [0.5, 0.3, 0.7, 0.6, 0.2, 0.4, 0.9, 0.5, 0.35, 0.8]


def reach(n, edges, alive, src, forward):
    adj = [[] for _ in range(n)]
    for (u, v), a in zip(edges, alive):
        if a:
            if forward:
                adj[u].append(v)
            else:
                adj[v].append(u)
    seen = {src}
    stack = [src]
    while stack:
        x = stack.pop()
        for y in adj[x]:
            if y not in seen:
                seen.add(y)
                stack.append(y)
    return seen


def test_hashed_world_bfs_matches_materialized_world():
    g, edges, _ = small_graph(TINY_EDGES, 6, TINY_P)
    seed = 1234
    rr = oracle.rr_sets(g, seed, 0, 300)
    for j in range(300):
        alive = [oracle.live(seed, j, e, int(g.thr[e])) for e in range(len(edges))]
        ref = sorted(reach(6, edges, alive, int(rr.starts[j]), forward=False))
        assert list(rr.row(j)) == ref


def exact_inclusion(g, edges):
    """P[u in RR | start = v] over all 2^m worlds, p_e = thr_e / 2^32."""
    n, m = g.n, len(edges)
    pe = [(1.0 if int(t) == 0xFFFFFFFF else int(t) / 2**32) for t in g.thr]
    P = np.zeros((n, n))
    for alive in itertools.product([0, 1], repeat=m):
        w = 1.0
        for a, p in zip(alive, pe):
            w *= p if a else 1 - p
        for v in range(n):
            for u in reach(n, edges, alive, v, forward=False):
                P[v, u] += w
    return P


def test_inclusion_frequencies_match_enumeration():
    g, edges, _ = small_graph(TINY_EDGES, 6, TINY_P)
    P = exact_inclusion(g, edges)
    N = 120000
    rr = oracle.rr_sets(g, 555, 0, N)
    sizes = np.diff(rr.offsets).astype(np.int64)
    rows = np.repeat(rr.starts.astype(np.int64), sizes)
    hits = np.zeros((6, 6))
    np.add.at(hits, (rows, rr.verts), 1)
    per_start = np.bincount(rr.starts, minlength=6)
    freq = hits / per_start[:, None]
    sd = np.sqrt(P * (1 - P) / per_start[:, None]) + 1e-12
    assert np.all(np.abs(freq - P) < 5 * sd + 1e-9)


def test_borgs_identity_fixes_direction():
    """sigma({u}) = n * Pr[u in RR(v)], v uniform: the expected forward
    influence of u equals n times its inclusion rate in RR sets (Section 2,
    RIS).  On this asymmetric graph the same identity with the edges reversed
    is off by far more than the tolerance, so a traversal over out-edges
    instead of in-edges fails it."""
    g, edges, _ = small_graph(TINY_EDGES, 6, TINY_P)
    pe = [int(t) / 2**32 for t in g.thr]
    sigma = np.zeros(6)
    sigma_rev = np.zeros(6)
    for alive in itertools.product([0, 1], repeat=len(edges)):
        w = np.prod([p if a else 1 - p for a, p in zip(alive, pe)])
        for u in range(6):
            sigma[u] += w * len(reach(6, edges, alive, u, forward=True))
            sigma_rev[u] += w * len(reach(6, edges, alive, u, forward=False))
    N = 120000
    rr = oracle.rr_sets(g, 909, 0, N)
    rate = np.bincount(rr.verts, minlength=6) / N
    tol = 5 * np.sqrt(rate * (1 - rate) / N) * 6 + 1e-9
    assert np.all(np.abs(6 * rate - sigma) < tol)
    assert np.max(np.abs(sigma_rev - sigma) - 10 * tol) > 0


# ---- Listing 1 (fused) equals the per-sample definition; Theorem 1 -----------------------

@pytest.mark.parametrize("W,count,first", [(1, 64, 0), (1, 150, 3), (2, 200, 17), (4, 300, 1 << 33)])
def test_fused_equals_unfused(W, count, first):
    rp, col = synth.rmat_graph(11, 8, 5)
    g = synth.Graph(1 << 11, rp, col, synth.thr_uniform(col.size, 0.08))
    plain = oracle.rr_sets(g, 2024, first, count)
    fused, acc = oracle.rr_sets_fused(g, 2024, first, count, W)
    assert np.array_equal(plain.offsets, fused.offsets)
    assert np.array_equal(plain.verts, fused.verts)
    # Theorem 1: fused edge accesses <= the edges the separate traversals scan
    indeg = g.indeg()
    assert acc <= int(indeg[plain.verts].sum())


def test_fused_equals_unfused_wc():
    g = synth.rmat_wc(12)
    plain = oracle.rr_sets(g, 31, 0, 256)
    fused, acc = oracle.rr_sets_fused(g, 31, 0, 256, 4)
    assert np.array_equal(plain.verts, fused.verts) and np.array_equal(plain.offsets, fused.offsets)
    assert acc <= int(g.indeg()[plain.verts].sum())


def test_rows_sorted_and_contain_start(er_workload):
    g = er_workload.graphs[0]
    rr = oracle.rr_sets(g, er_workload.seeds[0], 0, 64)
    for j in range(64):
        r = rr.row(j)
        assert np.all(np.diff(r.astype(np.int64)) > 0)
        assert int(rr.starts[j]) in set(r.tolist())


# ---- Greedy max-k-cover ---------------------------------------------------------------

def coverage(rows, chosen):
    c = set(chosen)
    return sum(1 for r in rows if c & set(r))


def test_greedy_bound_against_brute_force():
    rng = np.random.default_rng(3)
    for trial in range(5):
        n = 10
        rows = [sorted(set(rng.integers(0, n, rng.integers(1, 4)).tolist())) for _ in range(25)]
        off = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.uint64)
        rr = oracle.RRSets(off, np.array([x for r in rows for x in r], np.uint32))
        k = 3
        seeds, gains = oracle.greedy(n, rr, k)
        opt = max(coverage(rows, c) for c in itertools.combinations(range(n), k))
        got = coverage(rows, seeds.tolist())
        assert got >= (1 - 1 / math.e) * opt
        assert int(gains.sum()) == got


def test_greedy_picks_are_marginal_argmax():
    rng = np.random.default_rng(4)
    n = 30
    rows = [sorted(set(rng.integers(0, n, rng.integers(1, 6)).tolist())) for _ in range(80)]
    off = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.uint64)
    rr = oracle.RRSets(off, np.array([x for r in rows for x in r], np.uint32))
    seeds, gains = oracle.greedy(n, rr, 12)
    covered = [False] * len(rows)
    chosen = []
    for u, gval in zip(seeds.tolist(), gains.tolist()):
        marg = [sum(1 for i, r in enumerate(rows) if not covered[i] and v in r) if v not in chosen else -1
                for v in range(n)]
        best = max(marg)
        assert marg[u] == best == gval
        assert u == marg.index(best)  # smallest id on ties
        chosen.append(u)
        for i, r in enumerate(rows):
            if u in r:
                covered[i] = True


def test_greedy_exhaustion_and_limits():
    rows = [[2], [2, 5], [5]]
    off = np.array([0, 1, 3, 4], np.uint64)
    rr = oracle.RRSets(off, np.array([2, 2, 5, 5], np.uint32))
    seeds, gains = oracle.greedy(7, rr, 7)
    assert seeds.tolist()[:2] in ([2, 5], [5, 2])
    assert seeds.tolist() == [2, 5, 0, 1, 3, 4, 6]
    assert gains.tolist() == [2, 1, 0, 0, 0, 0, 0]
    with pytest.raises(ValueError):
        oracle.greedy(7, rr, 8)
