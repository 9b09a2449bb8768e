"""Pins of the linear-threshold (LT) oracle (oracle_rr_lt, oracle_lt_choice)
against facts outside it: the choice frequencies against the weights, a chain
whose walks follow by hand, zero weights, exact enumeration of every live-edge
world of a small graph (each vertex keeps one in-edge or none), and the RIS
identity under LT (which fixes the direction of the walk).  CPU only."""
import itertools

import numpy as np

import oracle
import synth


def lt_graph(n, edges, weights):
    """In-CSR from directed edges (u -> v) with LT weights (sum per head <= 1)."""
    order = sorted(range(len(edges)), key=lambda i: (edges[i][1], edges[i][0]))
    row_ptr = np.zeros(n + 1, np.uint64)
    col = np.zeros(len(edges), np.uint32)
    thr = np.zeros(len(edges), np.uint32)
    for k, i in enumerate(order):
        u, v = edges[i]
        row_ptr[v + 1] += 1
        col[k] = u
        thr[k] = synth.threshold(weights[i])
    row_ptr = np.cumsum(row_ptr).astype(np.uint64)
    return synth.Graph(n, row_ptr, col, thr, "lt"), [edges[i] for i in order]


def w_of(t):
    return 1.0 if int(t) == 0xFFFFFFFF else int(t) / 2**32


def test_choice_frequencies_match_the_weights():
    g, _ = lt_graph(4, [(0, 3), (1, 3), (2, 3)], [0.5, 0.2, 0.1])
    N = 60000
    picks = np.array([oracle.lt_choice(g, 77, s, 3) for s in range(N)])
    for e, t in enumerate(g.thr):
        p = w_of(t)
        f = np.mean(picks == e)
        assert abs(f - p) < 5 * np.sqrt(p * (1 - p) / N)
    p_none = 1 - sum(w_of(t) for t in g.thr)
    assert abs(np.mean(picks == -1) - p_none) < 5 * np.sqrt(p_none * (1 - p_none) / N)


def test_chain_walks_back_to_the_root():
    n = 10
    g, _ = lt_graph(n, [(i, i + 1) for i in range(n - 1)], [1.0] * (n - 1))
    rr = oracle.rr_sets(g, 3, 0, 200, model="lt")
    for j in range(200):
        v = int(rr.starts[j])
        assert rr.row(j).tolist() == list(range(v + 1))


def test_zero_weights_give_singletons():
    rp, col = synth.er_graph(300, 1200, 4)
    g = synth.Graph(300, rp, col, np.zeros(col.size, np.uint32))
    rr = oracle.rr_sets(g, 9, 0, 500, model="lt")
    assert np.array_equal(np.diff(rr.offsets), np.ones(500))
    assert np.array_equal(rr.verts, rr.starts)


SMALL_EDGES = [(0, 1), (2, 1), (1, 3), (4, 3), (3, 5), (0, 5), (5, 2), (4, 0)]
SMALL_W = [0.35, 0.4, 0.5, 0.3, 0.45, 0.25, 0.6, 0.7]


def lt_worlds(n, g):
    """Every live-edge world: each vertex keeps one of its in-edges or none,
    with its weight.  Yields (probability, kept source per vertex or -1)."""
    rows = []
    for v in range(n):
        a, b = int(g.row_ptr[v]), int(g.row_ptr[v + 1])
        opts = [(-1, 1 - sum(w_of(g.thr[e]) for e in range(a, b)))]
        opts += [(int(g.col[e]), w_of(g.thr[e])) for e in range(a, b)]
        rows.append(opts)
    for combo in itertools.product(*rows):
        p = 1.0
        for _, w in combo:
            p *= w
        yield p, [u for u, _ in combo]


def test_inclusion_and_ris_identity_by_enumeration():
    """Exact P[u in RR(v)] (v uniform) over every world, against the oracle's
    inclusion frequencies; and the RIS identity sigma({u}) = n P[u in RR]
    with sigma from forward reach in each world (the walk must go backward
    along kept in-edges: the reversed walk breaks the identity)."""
    n = 6
    g, _ = lt_graph(n, SMALL_EDGES, SMALL_W)
    incl = np.zeros(n)
    sigma = np.zeros(n)
    for p, keep in lt_worlds(n, g):
        for v in range(n):  # backward walk from v
            seen, x = set(), v
            while x >= 0 and x not in seen:
                seen.add(x)
                x = keep[x]
            for u in seen:
                incl[u] += p / n
        for u in range(n):  # forward reach from u: v is reached if its kept edge comes from a reached vertex
            reached = {u}
            grew = True
            while grew:
                grew = False
                for v in range(n):
                    if v not in reached and keep[v] in reached:
                        reached.add(v)
                        grew = True
            sigma[u] += p * len(reached)
    N = 200000
    rr = oracle.rr_sets(g, 2024, 0, N, model="lt")
    freq = np.bincount(rr.verts, minlength=n) / N
    tol = 5 * np.sqrt(incl * (1 - incl) / N) + 1e-9
    assert np.all(np.abs(freq - incl) < tol)
    assert np.allclose(n * incl, sigma, atol=1e-12)
