"""Host-side vertex orders (fbpt_order_compute; Section 5's reordering) against
facts outside them: every method yields a permutation; reverse Cuthill-McKee
recovers a banded labelling of a shuffled path (bandwidth 1) and of a shuffled
grid (no wider than the grid's side), keeps each connected component
contiguous, and is no wider than scipy's RCM on random graphs; the degree order
is non-increasing in degree with ties by id; the random order is a seeded,
uniform-looking shuffle; the clustering (Louvain) order lays planted
communities out contiguously, larger ones first.  No GPU."""
import numpy as np
import pytest

import synth
import paper_2311_10201_gb300 as fbpt


@pytest.fixture(scope="module", autouse=True)
def built():
    fbpt.build()


def in_csr(n, edges):
    """In-edge CSR of directed edges (u -> v), rows in order of v then u."""
    edges = sorted(edges, key=lambda e: (e[1], e[0]))
    rp = np.zeros(n + 1, np.uint64)
    for _, v in edges:
        rp[v + 1] += 1
    return np.cumsum(rp).astype(np.uint64), np.array([u for u, _ in edges], np.uint32)


def bandwidth(perm, edges):
    return max((abs(int(perm[u]) - int(perm[v])) for u, v in edges if u != v), default=0)


def shuffled(n, edges, seed):
    lab = np.random.default_rng(seed).permutation(n)
    return [(int(lab[u]), int(lab[v])) for u, v in edges]


@pytest.mark.parametrize("method", ["identity", "rcm", "degree", "random", "cluster"])
def test_every_method_gives_a_permutation(method):
    g = synth.rmat_wc(10)
    p = fbpt.order_compute(g.n, g.row_ptr, g.col, method, 3)
    assert np.array_equal(np.sort(p), np.arange(g.n))
    assert np.array_equal(p, fbpt.order_compute(g.n, g.row_ptr, g.col, method, 3))  # deterministic


def test_rcm_recovers_a_shuffled_path():
    n = 200
    edges = shuffled(n, [(i, i + 1) for i in range(n - 1)], 1)
    rp, col = in_csr(n, edges)
    p = fbpt.order_compute(n, rp, col, "rcm")
    assert bandwidth(p, edges) == 1


def test_rcm_bands_a_shuffled_grid():
    w, h = 12, 30
    grid = [(y * w + x, y * w + x + 1) for y in range(h) for x in range(w - 1)]
    grid += [(y * w + x, (y + 1) * w + x) for y in range(h - 1) for x in range(w)]
    n = w * h
    edges = shuffled(n, grid, 2)
    rp, col = in_csr(n, edges)
    p = fbpt.order_compute(n, rp, col, "rcm")
    random_bw = bandwidth(np.random.default_rng(5).permutation(n), edges)
    assert bandwidth(p, edges) <= w + 1 < random_bw


def test_rcm_keeps_components_contiguous():
    # three paths, a triangle and isolated vertices, labels shuffled
    parts = [(0, 1), (1, 2), (2, 3), (10, 11), (11, 12), (20, 21), (21, 22), (22, 20), (30, 31)]
    n = 40
    edges = shuffled(n, parts, 3)
    rp, col = in_csr(n, edges)
    p = fbpt.order_compute(n, rp, col, "rcm")
    lab = np.random.default_rng(3).permutation(n)  # the shuffle applied above
    for a, b in [(0, 3), (10, 12), (20, 22), (30, 31)]:
        labels = sorted(int(p[lab[x]]) for x in range(a, b + 1))
        assert labels == list(range(labels[0], labels[0] + len(labels)))


def test_rcm_no_wider_than_scipy():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(7)
    for trial in range(4):
        n = 300
        base = [(i, i + 1) for i in range(n - 1)] + [(i, i + 3) for i in range(0, n - 3, 2)]
        extra = [(int(a), int(b)) for a, b in rng.integers(0, n, size=(40, 2)) if abs(int(a) - int(b)) < 8]
        edges = shuffled(n, base + extra, 10 + trial)
        rp, col = in_csr(n, edges)
        ours = bandwidth(fbpt.order_compute(n, rp, col, "rcm"), edges)
        u = np.array([e[0] for e in edges])
        v = np.array([e[1] for e in edges])
        A = sp.coo_matrix((np.ones(len(edges)), (u, v)), shape=(n, n)).tocsr()
        A = A + A.T
        order = csgraph.reverse_cuthill_mckee(A, symmetric_mode=True)
        theirs = bandwidth(np.argsort(order), edges)
        assert ours <= int(1.5 * theirs) + 2


def test_degree_order_is_non_increasing_with_ties_by_id():
    g = synth.rmat_wc(11)
    rp = g.row_ptr.astype(np.int64)
    dst = np.repeat(np.arange(g.n), np.diff(rp))
    src = g.col.astype(np.int64)
    keep = src != dst
    deg = np.bincount(dst[keep], minlength=g.n) + np.bincount(src[keep], minlength=g.n)
    p = fbpt.order_compute(g.n, g.row_ptr, g.col, "degree")
    inv = np.argsort(p)
    assert np.all(np.diff(deg[inv]) <= 0)
    same = np.diff(deg[inv]) == 0
    assert np.all(np.diff(inv)[same] > 0)


def test_random_order_is_seeded_and_spread():
    g = synth.rmat_wc(10)
    a = fbpt.order_compute(g.n, g.row_ptr, g.col, "random", 1)
    b = fbpt.order_compute(g.n, g.row_ptr, g.col, "random", 2)
    assert not np.array_equal(a, b)
    # about 1 fixed point expected for a uniform permutation; far from sorted
    assert np.sum(a == np.arange(g.n)) < 10
    assert abs(np.corrcoef(a, np.arange(g.n))[0, 1]) < 0.15


def test_bad_arguments_rejected():
    g = synth.rmat_wc(8)
    with pytest.raises(fbpt.FbptError) as ei:
        fbpt.order_compute(g.n, g.row_ptr, g.col, 7)
    assert ei.value.code == fbpt.EINVAL
    bad = g.col.copy()
    bad[0] = g.n
    with pytest.raises(fbpt.FbptError) as ei:
        fbpt.order_compute(g.n, g.row_ptr, bad, "rcm")
    assert ei.value.code == fbpt.EINVAL


def test_cluster_order_lays_out_planted_communities():
    # cliques of different sizes joined in a ring by single edges, labels shuffled:
    # Louvain keeps each clique a community, laid out contiguously, bigger first
    sizes = [14, 9, 12, 7, 11, 8, 10, 13]
    edges, start = [], 0
    starts = []
    for sz in sizes:
        starts.append(start)
        edges += [(start + a, start + b) for a in range(sz) for b in range(a + 1, sz)]
        start += sz
    n = start
    for i in range(len(sizes)):
        edges.append((starts[i], starts[(i + 1) % len(sizes)]))
    edges = shuffled(n, edges, 4)
    rp, col = in_csr(n, edges)
    p = fbpt.order_compute(n, rp, col, "cluster")
    lab = np.random.default_rng(4).permutation(n)
    first = []
    for st, sz in zip(starts, sizes):
        labels = sorted(int(p[lab[st + x]]) for x in range(sz))
        assert labels == list(range(labels[0], labels[0] + sz))
        first.append(labels[0])
    by_pos = [sz for _, sz in sorted(zip(first, sizes))]
    assert by_pos == sorted(sizes, reverse=True)


def test_cluster_order_without_edges_is_the_identity():
    n = 50
    p = fbpt.order_compute(n, np.zeros(n + 1, np.uint64), np.zeros(0, np.uint32), "cluster")
    assert np.array_equal(p, np.arange(n))
