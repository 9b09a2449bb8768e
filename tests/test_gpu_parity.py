"""GPU path vs the CPU oracle, through the C ABI.  Integer work: every
comparison is bit-exact (RR rows, starts, per-vertex counts, seeds, gains)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SEED = synth.SAMPLE_SEED


@pytest.fixture(scope="module")
def fbpt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2311_10201_gb300 as f
    f.build()
    return f


def assert_same(rr, ref, g=None):
    off, verts, starts, vcount = rr.to_host()
    assert np.array_equal(off, ref.offsets)
    assert np.array_equal(verts, ref.verts)
    if ref.starts is not None:
        assert np.array_equal(starts, ref.starts)
    if g is not None:
        assert np.array_equal(vcount, np.bincount(ref.verts, minlength=g.n).astype(np.uint32))
    return off, verts, starts, vcount


# ---- the bit-level contract ------------------------------------------------------

def test_device_philox_matches_oracle(fbpt):
    rng = np.random.default_rng(0)
    s = rng.integers(0, 2**63, 4000, dtype=np.uint64)
    e = rng.integers(0, 2**39, 4000, dtype=np.uint64)
    s[:8] = [0, 1, 2, 3, 2**32 - 1, 2**32, 2**63 - 1, 12345]
    e[:8] = [0, 1, 2, 3, 4, 5, 2**32 + 3, 2**39 - 1]
    got = fbpt.edge_draws(SEED, s, e)
    want = np.array([oracle.edge_draw(SEED, int(a), int(b)) for a, b in zip(s, e)], np.uint32)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n", [1, 2, 1000, 2**24, 2**26])
def test_device_starts_match_oracle(fbpt, n):
    s = np.arange(0, 3000, dtype=np.uint64) * 7919 + 5
    got = fbpt.start_vertices(SEED, s, n)
    want = np.array([oracle.start(SEED, int(x), n) for x in s], np.uint32)
    assert np.array_equal(got, want)


# ---- the ER 1k workload (1,024 vertices, 8,192 edges, p = 0.1, 64 samples, k = 4) -----------

@pytest.mark.parametrize("launch", ["host", "graph", "persistent"])
@pytest.mark.parametrize("words,slots", [(1, 1), (1, 0), (2, 0), (8, 1)])
def test_er1k_bit_exact(fbpt, er_workload, launch, words, slots):
    w = er_workload
    g = w.graphs[0]
    dg = fbpt.Graph.from_synth(g)
    rr = fbpt.sample(dg, w.seeds[0], 0, w.S[0], words=words, slots=slots, launch=launch)
    ref = oracle.rr_sets(g, w.seeds[0], 0, w.S[0])
    assert_same(rr, ref, g)
    seeds, gains = fbpt.select_seeds(rr, w.k)
    rs, rg = oracle.greedy(g.n, ref, w.k)
    assert np.array_equal(seeds, rs) and np.array_equal(gains, rg)


def test_er1k_unfused_same_bits_more_edges(fbpt, er_workload):
    w = er_workload
    g = w.graphs[0]
    dg = fbpt.Graph.from_synth(g)
    fused = fbpt.sample(dg, w.seeds[0], 0, 640, words=1)
    unf = fbpt.sample(dg, w.seeds[0], 0, 640, words=1, unfused=True)
    ref = oracle.rr_sets(g, w.seeds[0], 0, 640)
    assert_same(fused, ref, g)
    assert_same(unf, ref, g)
    # Theorem 1: the fused traversal reads no more edges than the separate ones
    assert fused.stats.edge_accesses <= unf.stats.edge_accesses
    # colour-edge visits = sum over rows of in-degrees, from the oracle's rows
    cev = int(g.indeg()[ref.verts].sum())
    assert fused.stats.colour_edge_visits == cev == unf.stats.colour_edge_visits


# ---- ragged batches, odd sample ids, several W and slot counts -------------------------------

@pytest.fixture(scope="module")
def rmat12():
    rp, col = synth.rmat_graph(12, 16, 77)
    return synth.Graph(1 << 12, rp, col, synth.thr_uniform(col.size, 0.06), "rmat12-p0.06")


@pytest.fixture(scope="module")
def rmat13_wc():
    return synth.rmat_wc(13)


@pytest.mark.parametrize("refill", ["lane", "batch"])
@pytest.mark.parametrize("words,slots,first,S", [
    (1, 3, 0, 1000), (2, 0, 3, 1337), (4, 2, 2**33 + 1, 700), (8, 8, 17, 4100), (8, 1, 0, 1)])
def test_rmat_uniform_bit_exact(fbpt, rmat12, words, slots, first, S, refill):
    g = rmat12
    dg = fbpt.Graph.from_synth(g)
    rr = fbpt.sample(dg, SEED, first, S, words=words, slots=slots, refill=refill)
    assert_same(rr, oracle.rr_sets(g, SEED, first, S), g)


@pytest.mark.parametrize("launch", ["host", "graph", "persistent"])
def test_plain_batches_equal_lane_refill(fbpt, rmat12, launch):
    """The plain fused algorithm (one group of 64 colours at a time, run to
    completion) and lane refill give the same bits."""
    g = rmat12
    dg = fbpt.Graph.from_synth(g)
    ref = oracle.rr_sets(g, SEED, 5, 900)
    plain = fbpt.sample(dg, SEED, 5, 900, words=1, slots=1, refill="batch", launch=launch)
    lanes = fbpt.sample(dg, SEED, 5, 900, words=1, slots=1, refill="lane", launch=launch)
    assert_same(plain, ref, g)
    assert_same(lanes, ref, g)
    assert lanes.stats.levels <= plain.stats.levels


@pytest.mark.parametrize("launch", ["host", "graph", "persistent"])
def test_rmat_wc_bit_exact(fbpt, rmat13_wc, launch):
    g = rmat13_wc
    dg = fbpt.Graph.from_synth(g)
    ref = oracle.rr_sets(g, SEED, 100, 5000)
    for words in (1, 2, 4, 8):
        rr = fbpt.sample(dg, SEED, 100, 5000, words=words, launch=launch)
        assert_same(rr, ref, g)
    seeds, gains = fbpt.select_seeds(rr, 40)
    rs, rg = oracle.greedy(g.n, ref, 40)
    assert np.array_equal(seeds, rs) and np.array_equal(gains, rg)


# ---- degenerate inputs -----------------------------------------------------------------------

def test_p_one_and_p_zero(fbpt):
    rp, col = synth.er_graph(500, 1500, 9)
    for p in (1.0, 0.0):
        g = synth.Graph(500, rp, col, synth.thr_uniform(col.size, p))
        dg = fbpt.Graph.from_synth(g)
        rr = fbpt.sample(dg, 5, 0, 300, words=2)
        ref = oracle.rr_sets(g, 5, 0, 300)
        assert_same(rr, ref, g)
        if p == 0.0:
            assert np.array_equal(np.diff(ref.offsets), np.ones(300))


def test_single_vertex_and_edgeless(fbpt):
    g = synth.Graph(1, np.zeros(2, np.uint64), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    rr = fbpt.sample(fbpt.Graph.from_synth(g), 1, 0, 70)
    off, verts, starts, vcount = rr.to_host()
    assert np.array_equal(off, np.arange(71)) and not verts.any() and vcount[0] == 70
    seeds, gains = fbpt.select_seeds(rr, 1)
    assert seeds.tolist() == [0] and gains.tolist() == [70]
    g = synth.Graph(50, np.zeros(51, np.uint64), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    rr = fbpt.sample(fbpt.Graph.from_synth(g), 2, 0, 130, words=1, slots=2)
    assert_same(rr, oracle.rr_sets(g, 2, 0, 130), g)


def test_invalid_graphs_rejected(fbpt):
    bad = [
        (3, np.array([0, 2, 1, 3], np.uint64), np.array([0, 1, 2], np.uint32)),   # decreasing row_ptr
        (3, np.array([1, 2, 3, 3], np.uint64), np.array([0, 1, 2], np.uint32)),   # row_ptr[0] != 0
        (3, np.array([0, 1, 2, 2], np.uint64), np.array([0, 1, 2], np.uint32)),   # row_ptr[n] != m
        (3, np.array([0, 1, 2, 3], np.uint64), np.array([0, 5, 2], np.uint32)),   # col >= n
    ]
    for n, rp, col in bad:
        with pytest.raises(fbpt.FbptError) as ei:
            fbpt.Graph(n, rp, col, np.zeros(col.size, np.uint32))
        assert ei.value.code == fbpt.EINVAL


def test_bad_options_rejected(fbpt, er_workload):
    dg = fbpt.Graph.from_synth(er_workload.graphs[0])
    for kw in ({"words": 3}, {"words": 8, "slots": 9}):
        with pytest.raises(fbpt.FbptError) as ei:
            fbpt.sample(dg, 1, 0, 10, **kw)
        assert ei.value.code == fbpt.EINVAL
    rr = fbpt.sample(dg, 1, 0, 10)
    with pytest.raises(fbpt.FbptError):
        fbpt.select_seeds(rr, 2000)


# ---- level schedules: push, filtered push, pull, heuristic, learned ----------------------------

@pytest.fixture(scope="module")
def rmat12_dense():
    rp, col = synth.rmat_graph(12, 16, 78)
    return synth.Graph(1 << 12, rp, col, synth.thr_uniform(col.size, 0.3), "rmat12-p0.3")


def random_policy(fbpt, seed):
    rng = np.random.default_rng(seed)
    n = fbpt.lib().fbpt_policy_param_count()
    p = rng.normal(0, 0.5, n).astype(np.float32)
    p[:6] = rng.normal(10, 2, 6)
    p[6:12] = rng.uniform(1, 4, 6)
    return fbpt.Policy(p)


@pytest.mark.parametrize("launch", ["host", "graph", "persistent"])
@pytest.mark.parametrize("schedule", ["pull", "filtered", "heuristic", "learned"])
@pytest.mark.parametrize("which", ["rmat12", "rmat12_dense"])
def test_schedules_give_the_same_bits(fbpt, request, which, schedule, launch):
    g = request.getfixturevalue(which)
    dg = fbpt.Graph.from_synth(g)
    policy = random_policy(fbpt, 5) if schedule == "learned" else None
    ref = oracle.rr_sets(g, SEED, 11, 1500)
    for words, slots, refill in ((4, 2, "lane"), (1, 1, "batch")):
        rr = fbpt.sample(dg, SEED, 11, 1500, words=words, slots=slots, refill=refill, schedule=schedule,
                         launch=launch, policy=policy)
        assert_same(rr, ref, g)
        if schedule == "pull":
            assert rr.stats.pull_levels > 0 and rr.stats.push_levels == 0


def test_heuristic_pulls_on_dense_frontiers(fbpt, rmat12_dense):
    dg = fbpt.Graph.from_synth(rmat12_dense)
    rr = fbpt.sample(dg, SEED, 0, 512, words=8, slots=1, refill="batch", schedule="heuristic", trace_cap=4096)
    assert rr.stats.pull_levels > 0
    assert set(np.unique(rr.trace["direction"])) <= {0, 1, 2}
    assert_same(rr, oracle.rr_sets(rmat12_dense, SEED, 0, 512), rmat12_dense)


def test_pull_limits(fbpt, rmat12):
    dg = fbpt.Graph.from_synth(rmat12)
    for kw in ({"words": 8, "slots": 8}, {"words": 1, "slots": 1, "unfused": True}):
        with pytest.raises(fbpt.FbptError) as ei:
            fbpt.sample(dg, 1, 0, 700, schedule="pull", **kw)
        assert ei.value.code == fbpt.EUNSUPPORTED


def test_long_rr_sets_grow_the_spill_log(fbpt):
    """Supercritical uniform p: RR sets of ~n vertices overflow the lanes'
    segments into the spill log, which grows (and the run repeats) until they
    fit; the output stays exact."""
    rp, col = synth.rmat_graph(14, 16, 93)
    g = synth.Graph(1 << 14, rp, col, synth.thr_uniform(col.size, 0.3), "rmat14-p0.3")
    dg = fbpt.Graph.from_synth(g)
    rr = fbpt.sample(dg, SEED, 0, 2048, words=8, slots=4)
    ref = oracle.rr_sets(g, SEED, 0, 2048)
    assert np.diff(ref.offsets).max() > 1024
    assert rr.stats.overflow_reruns >= 1
    assert_same(rr, ref, g)


# ---- frontier compaction: pending queue vs scan of the occupancy masks -----------------------

@pytest.mark.parametrize("launch", ["host", "graph", "persistent"])
@pytest.mark.parametrize("schedule", ["push", "filtered"])
@pytest.mark.parametrize("which", ["rmat12", "rmat12_dense", "rmat13_wc"])
def test_scan_compaction_gives_the_same_bits(fbpt, request, which, schedule, launch):
    """Levels whose reached vertices are found by scanning every vertex's
    word-occupancy mask (no pending list, no returned atomics in the expand)
    give the same RR sets as the queue."""
    g = request.getfixturevalue(which)
    dg = fbpt.Graph.from_synth(g)
    ref = oracle.rr_sets(g, SEED, 3, 1200)
    for words, slots, refill in ((4, 2, "lane"), (1, 1, "batch"), (8, 8, "lane")):
        rr = fbpt.sample(dg, SEED, 3, 1200, words=words, slots=slots, refill=refill, schedule=schedule,
                         launch=launch, compaction="scan", trace_cap=1 << 14 if launch == "host" else 0)
        assert_same(rr, ref, g)
        if rr.trace is not None:
            tr = rr.trace[1:]
            assert np.all(tr["compaction"][tr["units"] > 0] == 1)


def test_heuristic_switches_compaction_on_dense_levels(fbpt, rmat12_dense):
    """The heuristic scans when a level reached more than n / 16 vertices:
    on a supercritical graph both modes occur in one run, with the same bits."""
    dg = fbpt.Graph.from_synth(rmat12_dense)
    rr = fbpt.sample(dg, SEED, 0, 2048, words=4, slots=2, schedule="heuristic", launch="graph", trace_cap=8192)
    modes = set(np.unique(rr.trace["compaction"]).tolist())
    assert modes == {0, 1}
    assert_same(rr, oracle.rr_sets(rmat12_dense, SEED, 0, 2048), rmat12_dense)


@pytest.mark.parametrize("launch", ["graph", "persistent"])
def test_unfused_wide_units_bit_exact(fbpt, rmat13_wc, launch):
    """Unfused runs on a weighted-cascade graph whose hubs have at least 32
    4-edge groups: each (vertex, colour) unit of a hub gets chunks of its own."""
    g = rmat13_wc
    assert int(np.max(np.diff(g.row_ptr.astype(np.int64)))) >= 4 * 32
    dg = fbpt.Graph.from_synth(g)
    ref = oracle.rr_sets(g, SEED, 0, 1500)
    for compaction in ("queue", "scan"):
        rr = fbpt.sample(dg, SEED, 0, 1500, words=2, slots=1, refill="batch", unfused=True, launch=launch,
                         compaction=compaction)
        assert_same(rr, ref, g)
