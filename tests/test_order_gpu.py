"""Vertex orders on the GPU (fbpt_graph_set_order; Section 5's reordering and
sorted start list): a relabelled graph samples exactly the oracle's RR sets,
starts and counts of the caller's graph, under every order method, with and
without sorted starts, in every launch form and refill mode, for IC and LT,
in batched runs, and inside IMM; restoring the identity restores the graph;
bad permutations and pull levels are rejected."""
import numpy as np
import pytest

import oracle
import synth
from oracle import imm as oimm

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


@pytest.fixture(scope="module")
def wc13():
    return synth.rmat_wc(13)


def assert_same(rr, ref, n):
    off, verts, starts, vcount = rr.to_host()
    assert np.array_equal(off, ref.offsets)
    assert np.array_equal(verts, ref.verts)
    assert np.array_equal(starts, ref.starts)
    assert np.array_equal(vcount, np.bincount(ref.verts, minlength=n).astype(np.uint32))


def ordered(fbpt, g, method, sorted_starts, seed=9):
    dg = fbpt.Graph.from_synth(g)
    dg.set_order(fbpt.order_compute(g.n, g.row_ptr, g.col, method, seed), sorted_starts)
    return dg


@pytest.mark.parametrize("method", ["rcm", "degree", "random", "cluster"])
@pytest.mark.parametrize("sorted_starts", [False, True])
@pytest.mark.parametrize("launch", ["graph", "host", "persistent"])
def test_ordered_graph_bit_exact(fbpt, wc13, method, sorted_starts, launch):
    g = wc13
    dg = ordered(fbpt, g, method, sorted_starts)
    rr = fbpt.sample(dg, SEED, 5, 9000, words=8, slots=8, refill="lane", launch=launch)
    assert_same(rr, oracle.rr_sets(g, SEED, 5, 9000), g.n)
    dg.close()


def test_sorted_starts_alone_and_batch_refill(fbpt, wc13):
    g = wc13
    dg = fbpt.Graph.from_synth(g)
    dg.set_order(None, True)
    assert dg.get_order()[1]
    ref = oracle.rr_sets(g, SEED, 0, 5000)
    assert_same(fbpt.sample(dg, SEED, 0, 5000, words=2, slots=1, refill="batch", launch="graph"), ref, g.n)
    assert_same(fbpt.sample(dg, SEED, 0, 5000, words=8, slots=8, launch="graph"), ref, g.n)
    dg.close()


def test_ordered_schedules_and_pull_rejected(fbpt, wc13):
    g = wc13
    dg = ordered(fbpt, g, "rcm", True)
    ref = oracle.rr_sets(g, SEED, 0, 4000)
    for sched in ("heuristic", "learned", "filtered"):
        assert_same(fbpt.sample(dg, SEED, 0, 4000, words=1, slots=1, schedule=sched, launch="graph"), ref, g.n)
    with pytest.raises(fbpt.FbptError) as ei:
        fbpt.sample(dg, SEED, 0, 100, words=1, slots=1, schedule="pull")
    assert ei.value.code == fbpt.EUNSUPPORTED
    dg.close()


def test_ordered_lt(fbpt, wc13):
    g = wc13
    dg = ordered(fbpt, g, "degree", True)
    rr = fbpt.sample(dg, 3, 0, 6000, words=8, slots=8, model="lt", launch="graph")
    assert_same(rr, oracle.rr_sets(g, 3, 0, 6000, model="lt"), g.n)
    dg.close()


def test_ordered_batched_with_plain_graph(fbpt, wc13):
    g2 = synth.rmat_wc(12)
    d1 = ordered(fbpt, wc13, "rcm", True)
    d2 = fbpt.Graph.from_synth(g2)
    outs, _ = fbpt.sample_batched([d1, d2, d1], [SEED, 7, 11], [0, 0, 100], [3000, 2000, 2500], schedule="learned")
    assert_same(outs[0], oracle.rr_sets(wc13, SEED, 0, 3000), wc13.n)
    assert_same(outs[1], oracle.rr_sets(g2, 7, 0, 2000), g2.n)
    assert_same(outs[2], oracle.rr_sets(wc13, 11, 100, 2500), wc13.n)
    d1.close()
    d2.close()


def test_seeds_and_imm_on_an_ordered_graph(fbpt):
    g = synth.rmat_wc(12)
    dg = ordered(fbpt, g, "rcm", True)
    rr = fbpt.sample(dg, SEED, 0, 6000, words=8, slots=8, launch="graph")
    seeds, gains = fbpt.select_seeds(rr, 20)
    rs, rg = oracle.greedy(g.n, oracle.rr_sets(g, SEED, 0, 6000), 20)
    assert np.array_equal(seeds, rs) and np.array_equal(gains, rg)
    seeds, gains, res, _ = fbpt.imm(dg, 10, 0.5, 1.0, 4, words=8, slots=8, launch="graph")
    rs, rg, info = oimm.imm(g, 10, 0.5, 1.0, 4)
    assert np.array_equal(seeds, rs) and np.array_equal(gains, rg)
    assert res["theta"] == info["theta"] and res["samples"] == info["samples"]
    dg.close()


def test_identity_restores_and_bad_perm_rejected(fbpt, wc13):
    g = wc13
    dg = ordered(fbpt, g, "random", False)
    perm = fbpt.order_compute(g.n, g.row_ptr, g.col, "random", 9)
    got, ss = dg.get_order()
    assert np.array_equal(got, perm) and not ss
    dg.set_order(None, False)
    got, ss = dg.get_order()
    assert np.array_equal(got, np.arange(g.n)) and not ss
    ref = oracle.rr_sets(g, SEED, 0, 3000)
    assert_same(fbpt.sample(dg, SEED, 0, 3000, words=1, slots=1, schedule="pull", launch="graph"), ref, g.n)
    bad = perm.copy()
    bad[0] = bad[1]
    with pytest.raises(fbpt.FbptError) as ei:
        dg.set_order(bad)
    assert ei.value.code == fbpt.EINVAL
    dg.close()


def test_ordered_full_size_s20(fbpt):
    w = synth.rmat_s20_wc()
    g = w.graphs[0]
    dg = ordered(fbpt, g, "rcm", True)
    rr = fbpt.sample(dg, w.seeds[0], 0, w.S[0], launch="graph")
    assert_same(rr, oracle.rr_sets(g, w.seeds[0], 0, w.S[0]), g.n)
    dg.close()
