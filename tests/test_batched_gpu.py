"""Batched sampling (many graphs, one CUDA-graph launch) and the autotuner,
against the CPU oracle.  Every comparison is bit-exact: neither the batch,
nor the shape the autotuner picks, may change a bit of any graph's RR sets."""
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


def assert_same(rr, ref, n):
    off, verts, starts, vcount = rr.to_host()
    assert np.array_equal(off, ref.offsets)
    assert np.array_equal(verts, ref.verts)
    assert np.array_equal(starts, ref.starts)
    assert np.array_equal(vcount, np.bincount(ref.verts, minlength=n).astype(np.uint32))


def small_batch(count=12, max_scale=13, cap=700):
    """The 32-graph batch recipe at small scales (12-13) and at most `cap`
    samples per graph, so that the oracle runs in seconds."""
    w = synth.batched_32(max_scale=max_scale, count=count)
    return w.graphs, [min(S, cap) for S in w.S], w.seeds


def test_batched_matches_oracle(fbpt):
    graphs, Ss, seeds = small_batch()
    dgs = [fbpt.Graph.from_synth(g) for g in graphs]
    # a third of the graphs tuned (their own shapes), the rest on the default shape
    for dg, S, seed in list(zip(dgs, Ss, seeds))[::3]:
        t = fbpt.autotune(dg, seed, S)
        assert t["words"] in (1, 2, 4, 8) and t["words"] * t["slots"] <= 64 and t["blocks"] >= 1
    firsts = [7 * i for i in range(len(graphs))]
    outs, st = fbpt.sample_batched(dgs, seeds, firsts, Ss)
    plain, _ = fbpt.sample_batched(dgs, seeds, firsts, Ss, launch="host", refill="batch")
    for g, rr, pr, S, seed, first in zip(graphs, outs, plain, Ss, seeds, firsts):
        ref = oracle.rr_sets(g, seed, first, S)
        assert_same(rr, ref, g.n)
        assert_same(pr, ref, g.n)
    assert st.rr_total == sum(rr.total for rr in outs)
    for dg in dgs:
        dg.close()


def test_batched_tasks_sharing_a_graph(fbpt):
    """Three sample ranges of one graph (chained on its workspace) and one
    other graph, in one launch."""
    graphs, Ss, seeds = small_batch(count=2)
    a, b = (fbpt.Graph.from_synth(g) for g in graphs)
    tasks = [(a, graphs[0], 11, 0, 300), (b, graphs[1], 12, 5, 500), (a, graphs[0], 11, 300, 257),
             (a, graphs[0], 99, 0, 64)]
    outs, _ = fbpt.sample_batched([t[0] for t in tasks], [t[2] for t in tasks], [t[3] for t in tasks],
                                  [t[4] for t in tasks], words=2, slots=2)
    for (dg, g, seed, first, S), rr in zip(tasks, outs):
        assert_same(rr, oracle.rr_sets(g, seed, first, S), g.n)
    a.close()
    b.close()


def test_batched_reruns_tasks_that_outgrow_their_buffers(fbpt):
    """Supercritical uniform p on a fresh graph: the first task's RR sets
    overflow the spill log inside the batched launch; it runs again alone, and
    so does the later task on the same (now dirty) workspace."""
    rp, col = synth.rmat_graph(14, 16, 93)
    g = synth.Graph(1 << 14, rp, col, synth.thr_uniform(col.size, 0.3), "rmat14-p0.3")
    er = synth.er_1k().graphs[0]
    dg, de = fbpt.Graph.from_synth(g), fbpt.Graph.from_synth(er)
    outs, st = fbpt.sample_batched([dg, de, dg], [1, 2, 3], [0, 0, 100], [2048, 512, 1024], words=8, slots=4)
    assert st.overflow_reruns >= 1
    assert_same(outs[0], oracle.rr_sets(g, 1, 0, 2048), g.n)
    assert_same(outs[1], oracle.rr_sets(er, 2, 0, 512), er.n)
    assert_same(outs[2], oracle.rr_sets(g, 3, 100, 1024), g.n)
    dg.close()
    de.close()


def test_autotune_probe_statistics(fbpt):
    """The tuner's RR mean is the exact mean size of the probe samples
    (ids 0 .. P - 1, with P = S here since S <= 4096), and the stored shape
    is what it returned."""
    g = synth.rmat_wc(12)
    dg = fbpt.Graph.from_synth(g)
    t = fbpt.autotune(dg, 5, 3000)
    assert t == fbpt.tuning(dg)
    assert t["probe_samples"] == 3000
    ref = oracle.rr_sets(g, 5, 0, 3000)
    assert t["rr_per_sample"] == pytest.approx(ref.offsets[-1] / 3000, rel=1e-12)
    assert t["candidates"] >= 4
    rr = fbpt.sample(dg, 5, 0, 3000, words=t["words"], slots=t["slots"], blocks=t["blocks"])
    assert_same(rr, ref, g.n)
    with pytest.raises(fbpt.FbptError):
        fresh = fbpt.Graph.from_synth(g)
        try:
            fbpt.tuning(fresh)
        finally:
            fresh.close()
    dg.close()


def test_copy_rows_matches_full_copy(fbpt):
    g = synth.rmat_wc(12)
    dg = fbpt.Graph.from_synth(g)
    rr = fbpt.sample(dg, 8, 0, 1000)
    off, verts, _, _ = rr.to_host()
    for first, count in [(0, 1), (0, 1000), (37, 100), (999, 1), (500, 0)]:
        o, v = rr.rows(first, count)
        assert np.array_equal(o, off[first:first + count + 1])
        assert np.array_equal(v, verts[off[first]:off[first + count]])
    with pytest.raises(fbpt.FbptError):
        rr.rows(990, 11)
    dg.close()
