"""The five workloads at their full sizes, in the launch configuration the
benchmark times (autotuned shape, learned schedule, CUDA-graph launch), against
the CPU oracle.

Where the oracle finishes in seconds (the ER 1k and R-MAT s20 workloads) every
RR set is compared.  Elsewhere sampled rows are compared bit-exactly with the
oracle's BFS of the same sample ids, and properties that hold at any size are
checked on the whole output (CSR shape, strictly ascending rows, start vertex in
its own row, per-vertex counts); the greedy seeds are compared with the
oracle's greedy run over the GPU's RR sets (so that, given the sampled-row
parity, the seed step is checked bit-exactly at full size)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fbpt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2311_10201_gb300 as f
    f.build()
    return f


def check_csr(off, verts, starts, vcount, n, S):
    """CSR invariants of an RR-set output of S rows over n vertices."""
    assert off.size == S + 1 and off[0] == 0 and off[-1] == verts.size
    lens = np.diff(off.astype(np.int64))
    assert lens.min() >= 1                       # start(s) is always in its own row
    assert int(verts.max(initial=0)) < n
    d = np.diff(verts.astype(np.int64))
    inside = np.ones(d.size, bool)
    inside[off[1:-1].astype(np.int64) - 1] = False  # pairs that straddle two rows
    assert np.all(d[inside] > 0)                 # rows strictly ascending
    row = np.repeat(np.arange(S, dtype=np.int64), lens)
    key = row * n + verts
    want = np.arange(S, dtype=np.int64) * n + starts
    at = np.searchsorted(key, want)
    assert np.all(key[np.minimum(at, key.size - 1)] == want)  # start in its row
    assert np.array_equal(vcount, np.bincount(verts, minlength=n).astype(np.uint32))


def check_sampled_rows(g, seed, first, off, verts, starts, rows):
    ref = oracle.rr_sets(g, seed, ids=np.asarray(rows, np.uint64) + np.uint64(first))
    for i, j in enumerate(rows):
        got = verts[off[j]:off[j + 1]]
        assert np.array_equal(got, ref.row(i)), f"row {j}"
        assert starts[j] == ref.starts[i]


def tuned_kw(fbpt, dg, seed, S, **cap):
    t = fbpt.autotune(dg, seed, S, schedule="learned", **cap)
    return dict(words=t["words"], slots=t["slots"], blocks=t["blocks"], refill="lane", schedule=t["schedule"],
                launch="graph")


# ---- ER 1k: 64 samples, W = 1, k = 4 (every row and the seeds) ---------------------

def test_er_1k_full(fbpt):
    w = synth.er_1k()
    g = w.graphs[0]
    dg = fbpt.Graph.from_synth(g)
    rr = fbpt.sample(dg, w.seeds[0], 0, w.S[0], words=1, slots=1, refill="batch", schedule="push")
    ref = oracle.rr_sets(g, w.seeds[0], 0, w.S[0])
    off, verts, starts, vcount = rr.to_host()
    assert np.array_equal(off, ref.offsets) and np.array_equal(verts, ref.verts)
    assert np.array_equal(starts, ref.starts)
    seeds, gains = fbpt.select_seeds(rr, w.k)
    rs, rg = oracle.greedy(g.n, ref, w.k)
    assert np.array_equal(seeds, rs) and np.array_equal(gains, rg)
    dg.close()


# ---- R-MAT s20 WC: 65,536 samples, W = 1, 2, 4, 8, fused and unfused (every row) ----

@pytest.fixture(scope="module")
def s20():
    w = synth.rmat_s20_wc()
    g = w.graphs[0]
    return w, g, oracle.rr_sets(g, w.seeds[0], 0, w.S[0])


@pytest.mark.parametrize("words", [1, 2, 4, 8])
def test_rmat_s20_full_fused(fbpt, s20, words):
    w, g, ref = s20
    dg = fbpt.Graph.from_synth(g)
    rr = fbpt.sample(dg, w.seeds[0], 0, w.S[0], words=words, slots=1, refill="batch", schedule="push",
                     launch="graph")
    off, verts, starts, vcount = rr.to_host()
    assert np.array_equal(off, ref.offsets) and np.array_equal(verts, ref.verts)
    assert np.array_equal(starts, ref.starts)
    assert np.array_equal(vcount, np.bincount(ref.verts, minlength=g.n).astype(np.uint32))
    dg.close()


def test_rmat_s20_full_unfused_and_tuned(fbpt, s20):
    """The unfused form (one colour per traversal) and the tuned learned form
    give the same bits; the fused form reads fewer edges (Theorem 1)."""
    w, g, ref = s20
    dg = fbpt.Graph.from_synth(g)
    un = fbpt.sample(dg, w.seeds[0], 0, w.S[0], words=1, slots=1, unfused=True, refill="batch", launch="graph")
    fu = fbpt.sample(dg, w.seeds[0], 0, w.S[0], words=1, slots=1, refill="batch", launch="graph")
    tu = fbpt.sample(dg, w.seeds[0], 0, w.S[0], **tuned_kw(fbpt, dg, w.seeds[0], w.S[0]))
    for rr in (un, tu):
        off, verts, _, _ = rr.to_host()
        assert np.array_equal(off, ref.offsets) and np.array_equal(verts, ref.verts)
    assert fu.stats.edge_accesses <= un.stats.edge_accesses
    dg.close()


# ---- R-MAT s22 WC: 1,048,576 samples, k = 100 (the benchmark's step) -----------------

def test_rmat_s22_full_size(fbpt):
    w = synth.rmat_s22_wc()
    g, S, seed = w.graphs[0], w.S[0], w.seeds[0]
    dg = fbpt.Graph.from_synth(g)
    rr = fbpt.sample(dg, seed, 0, S, **tuned_kw(fbpt, dg, seed, S))
    off, verts, starts, vcount = rr.to_host()
    check_csr(off, verts, starts, vcount, g.n, S)
    rng = np.random.default_rng(22)
    rows = np.unique(np.concatenate([rng.choice(S, 3000, replace=False), [0, S - 1],
                                     np.argsort(np.diff(off))[-20:]]))  # the longest rows too
    check_sampled_rows(g, seed, 0, off, verts, starts, rows)
    seeds, gains = fbpt.select_seeds(rr, w.k)
    rs, rg = oracle.greedy(g.n, oracle.RRSets(off, verts), w.k)
    assert np.array_equal(seeds, rs) and np.array_equal(gains, rg)
    dg.close()


# ---- R-MAT s24 trivalency: the full graph, rows of at most 8 words, k = 200 -----------
#
# Its RR sets are bimodal: about 90% of samples stay at their start vertex and
# about 10% reach a giant in-component of ~1.83M vertices (mean ~1.9e5 entries
# per sample), so 4,194,304 samples would hold ~7.9e11 entries (3.2 TB as
# uint32), beyond one GPU.  The full graph is sampled for the first 8,192
# sample ids (~1.5e9 entries); rows are checked in chunks to bound host memory.

S24 = 8192


def test_rmat_s24_full_graph(fbpt):
    w = synth.rmat_s24_tri()
    g, seed = w.graphs[0], w.seeds[0]
    dg = fbpt.Graph.from_synth(g)
    rr = fbpt.sample(dg, seed, 0, S24, **tuned_kw(fbpt, dg, seed, S24, words=8, slots=1))
    off, starts, vcount = rr.index_to_host()
    lens = np.diff(off.astype(np.int64))
    assert off[0] == 0 and off[-1] == rr.total and lens.min() >= 1
    assert (lens > 100000).mean() > 0.02 and np.median(lens) < 10  # the bimodal shape
    count = np.zeros(g.n, np.uint64)
    for a in range(0, S24, 256):
        o, v = rr.rows(a, min(256, S24 - a))
        sub = o - o[0]
        check_csr(sub, v, starts[a:a + len(sub) - 1], np.bincount(v, minlength=g.n).astype(np.uint32), g.n,
                  len(sub) - 1)
        count += np.bincount(v, minlength=g.n).astype(np.uint64)
    assert np.array_equal(count.astype(np.uint32), vcount)
    rng = np.random.default_rng(24)
    rows = np.unique(np.concatenate([rng.choice(S24, 48, replace=False), [0, S24 - 1],
                                     np.argsort(lens)[-2:]]))
    ref = oracle.rr_sets(g, seed, ids=rows.astype(np.uint64))
    for i, j in enumerate(rows):
        o, v = rr.rows(int(j), 1)
        assert np.array_equal(v, ref.row(i)), f"row {j}"
        assert starts[j] == ref.starts[i]
    seeds, gains = fbpt.select_seeds(rr, w.k)
    full = rr.to_host()
    rs, rg = oracle.greedy(g.n, oracle.RRSets(full[0], full[1]), w.k)
    assert np.array_equal(seeds, rs) and np.array_equal(gains, rg)
    dg.close()


# ---- 32 graphs in one batched launch (20.8G RR entries) -------------------------------

def test_batched_32_full_size(fbpt):
    """Learned schedule, per-graph tuned shapes, one CUDA-graph launch; then
    the plain form graph after graph.  Sampled rows of every graph against the
    oracle; row offsets and per-vertex counts of the two forms identical."""
    w = synth.batched_32()
    dgs = [fbpt.Graph.from_synth(g) for g in w.graphs]
    for dg, seed, S in zip(dgs, w.seeds, w.S):
        fbpt.autotune(dg, seed, S, schedule="learned")
    firsts = [0] * len(dgs)
    outs, st = fbpt.sample_batched(dgs, w.seeds, firsts, w.S, schedule="learned")
    rng = np.random.default_rng(32)
    index = []
    for g, rr, seed, S in zip(w.graphs, outs, w.seeds, w.S):
        off, starts, vcount = rr.index_to_host()
        assert off[0] == 0 and off[-1] == rr.total and np.all(np.diff(off.astype(np.int64)) >= 1)
        assert int(vcount.sum(dtype=np.uint64)) == rr.total
        index.append((off, vcount))
        rows = np.unique(np.concatenate([rng.choice(S, 3, replace=False), [S - 1]]))
        ref = oracle.rr_sets(g, seed, ids=rows.astype(np.uint64))
        for i, j in enumerate(rows):
            o, v = rr.rows(int(j), 1)
            assert np.array_equal(v, ref.row(i)), f"{g.name} row {j}"
    assert st.rr_total == sum(rr.total for rr in outs)
    del outs
    plain, _ = fbpt.sample_batched(dgs, w.seeds, firsts, w.S, launch="host", words=8, slots=1, refill="batch",
                                   schedule="push")
    for rr, (off, vcount) in zip(plain, index):
        off2, _, vcount2 = rr.index_to_host()
        assert np.array_equal(off2, off) and np.array_equal(vcount2, vcount)
    del plain
    for dg in dgs:
        dg.close()
