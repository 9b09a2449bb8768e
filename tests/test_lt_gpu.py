"""RR sets under the linear-threshold model (FBPT_MODEL_LT) against the LT
oracle (oracle_rr_lt): bit-exact rows, starts and per-vertex counts for every
shape, launch form and refill mode, and the seeds over them."""
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


def assert_same(rr, ref, n):
    off, verts, starts, vcount = rr.to_host()
    assert np.array_equal(off, ref.offsets)
    assert np.array_equal(verts, ref.verts)
    assert np.array_equal(starts, ref.starts)
    assert np.array_equal(vcount, np.bincount(ref.verts, minlength=n).astype(np.uint32))


@pytest.fixture(scope="module")
def wc13():
    return synth.rmat_wc(13)


@pytest.mark.parametrize("launch", ["host", "graph", "persistent"])
@pytest.mark.parametrize("words,slots,refill,first,S", [
    (1, 1, "batch", 0, 700), (2, 0, "lane", 3, 5000), (8, 8, "lane", 2**33 + 5, 9000), (8, 1, "batch", 1, 64)])
def test_lt_rmat_wc_bit_exact(fbpt, wc13, launch, words, slots, refill, first, S):
    g = wc13
    dg = fbpt.Graph.from_synth(g)
    rr = fbpt.sample(dg, SEED, first, S, words=words, slots=slots, refill=refill, launch=launch, model="lt")
    assert_same(rr, oracle.rr_sets(g, SEED, first, S, model="lt"), g.n)
    dg.close()


def test_lt_er_chain_and_seeds(fbpt):
    rp, col = synth.er_graph(2000, 12000, 31)
    g = synth.Graph(2000, rp, col, synth.thr_wc(rp), "er-2k-wc")
    dg = fbpt.Graph.from_synth(g)
    rr = fbpt.sample(dg, 7, 0, 3000, words=4, model="lt", launch="graph", schedule="learned")
    ref = oracle.rr_sets(g, 7, 0, 3000, model="lt")
    assert_same(rr, ref, g.n)
    seeds, gains = fbpt.select_seeds(rr, 25)
    rs, rg = oracle.greedy(g.n, ref, 25)
    assert np.array_equal(seeds, rs) and np.array_equal(gains, rg)
    dg.close()
    n = 50  # a chain with weight 1: every walk runs back to vertex 0
    rp = np.concatenate([[0], np.arange(n, dtype=np.uint64)]).astype(np.uint64)
    chain = synth.Graph(n, rp, np.arange(n - 1, dtype=np.uint32), np.full(n - 1, 0xFFFFFFFF, np.uint32))
    dc = fbpt.Graph.from_synth(chain)
    rr = fbpt.sample(dc, 1, 0, 300, words=2, model="lt")
    off, verts, starts, _ = rr.to_host()
    for j in range(300):
        assert verts[off[j]:off[j + 1]].tolist() == list(range(int(starts[j]) + 1))
    dc.close()


def test_lt_rejects_bad_weights_and_directions(fbpt, wc13):
    rp, col = synth.rmat_graph(10, 16, 5)
    heavy = synth.Graph(1 << 10, rp, col, synth.thr_uniform(col.size, 0.5), "heavy")
    dh = fbpt.Graph.from_synth(heavy)
    with pytest.raises(fbpt.FbptError) as ei:
        fbpt.sample(dh, 1, 0, 100, model="lt")
    assert ei.value.code == fbpt.EINVAL
    dh.close()
    dg = fbpt.Graph.from_synth(wc13)
    for kw in ({"schedule": "pull", "words": 1, "slots": 1}, {"schedule": "filtered"}, {"unfused": True}):
        with pytest.raises(fbpt.FbptError) as ei:
            fbpt.sample(dg, 1, 0, 100, model="lt", **kw)
        assert ei.value.code == fbpt.EUNSUPPORTED
    dg.close()


def test_lt_batched_and_full_size_s20(fbpt):
    w = synth.rmat_s20_wc()
    g20 = w.graphs[0]
    g13 = synth.rmat_wc(13)
    d20, d13 = fbpt.Graph.from_synth(g20), fbpt.Graph.from_synth(g13)
    outs, _ = fbpt.sample_batched([d20, d13], [w.seeds[0], 3], [0, 10], [w.S[0], 4000], model="lt",
                                  words=8, slots=8)
    assert_same(outs[0], oracle.rr_sets(g20, w.seeds[0], 0, w.S[0], model="lt"), g20.n)
    assert_same(outs[1], oracle.rr_sets(g13, 3, 10, 4000, model="lt"), g13.n)
    d20.close()
    d13.close()
