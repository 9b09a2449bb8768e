"""fbpt_imm (the IMM sampling loop over the GPU sampler and greedy) against the
IMM oracle (oracle/imm.py over oracle_rr and oracle_greedy).  The control
values are computed by the same formulas in double on both sides and every
RR set and pick is bit-exact, so rounds, sample sizes, bounds and seeds must
be equal."""
import numpy as np
import pytest

import synth
from oracle import imm as oimm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fbpt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2311_10201_gb300 as f
    f.build()
    return f


def check(fbpt, g, k, eps, ell, seed, **kw):
    dg = fbpt.Graph.from_synth(g)
    seeds, gains, res, st = fbpt.imm(dg, k, eps, ell, seed, **kw)
    rs, rg, info = oimm.imm(g, k, eps, ell, seed)
    assert np.array_equal(seeds, rs) and np.array_equal(gains, rg)
    for key in ("theta", "samples", "first_final_id", "rounds", "lower_bound", "coverage", "lambda_prime",
                "lambda_star"):
        assert res[key] == info[key], key
    dg.close()
    return res, st


def test_imm_star_and_isolated(fbpt):
    n = 64
    rp = np.arange(n + 1, dtype=np.uint64) - 1
    rp[0] = 0
    star = synth.Graph(n, rp, np.zeros(n - 1, np.uint32), synth.thr_uniform(n - 1, 1.0))
    res, _ = check(fbpt, star, 1, 0.5, 1.0, 17)
    assert res["rounds"] == 1 and res["coverage"] == 1.0
    iso = synth.Graph(32, np.zeros(33, np.uint64), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    res, _ = check(fbpt, iso, 1, 0.5, 1.0, 5)
    assert res["lower_bound"] == 1.0


@pytest.mark.parametrize("k,eps", [(4, 0.3), (10, 0.5)])
def test_imm_er_and_rmat(fbpt, k, eps):
    check(fbpt, synth.er_1k().graphs[0], k, eps, 1.0, 11)
    rp, col = synth.rmat_graph(12, 16, 77)
    g = synth.Graph(1 << 12, rp, col, synth.thr_uniform(col.size, 0.06), "rmat12-p0.06")
    check(fbpt, g, k, eps, 1.0, 12, words=8, slots=2)


def test_imm_full_size_rmat_s22(fbpt):
    """The scale-22 WC graph, k = 100, epsilon = 0.5, in the benchmark's shape."""
    w = synth.rmat_s22_wc()
    res, st = check(fbpt, w.graphs[0], 100, 0.5, 1.0, w.seeds[0], words=8, slots=8, launch="graph")
    assert res["samples"] >= res["theta"] > 1000


def test_imm_limits(fbpt):
    g = synth.er_1k().graphs[0]
    dg = fbpt.Graph.from_synth(g)
    with pytest.raises(fbpt.FbptError) as ei:
        fbpt.imm(dg, 4, 0.3, 1.0, 1, max_samples=100)
    assert ei.value.code == fbpt.EINVAL
    for bad in ({"k": 0}, {"k": 2000}, {"epsilon": 0.0}, {"ell": -1.0}):
        a = dict(k=4, epsilon=0.3, ell=1.0)
        a.update(bad)
        with pytest.raises(fbpt.FbptError):
            fbpt.imm(dg, a["k"], a["epsilon"], a["ell"], 1)
    dg.close()
