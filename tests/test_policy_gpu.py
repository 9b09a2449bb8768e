"""The schedule network's CUDA training kernels against the FP64 oracle
(oracle/mlp.py): loss and gradient to FP32 tolerance, and Adam recovering a
teacher network.  The schedule it drives never changes the output bits
(tests/test_gpu_parity.py::test_schedules_give_the_same_bits)."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fbpt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2311_10201_gb300 as f
    f.build()
    return f


def problem(seed, rows=600):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.4, mlp.N_PARAMS)
    P = mlp.unpack(p)
    P["mu"][:] = rng.normal(0, 1, mlp.N_IN)
    P["sd"][:] = rng.uniform(0.5, 2, mlp.N_IN)
    X = rng.normal(0, 2, (rows, mlp.N_IN))
    a = rng.integers(0, 3, rows)
    y = rng.normal(0, 1, rows)
    return p, X, a, y


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gpu_gradient_matches_fp64_oracle(fbpt, seed):
    p, X, a, y = problem(seed)
    p32 = p.astype(np.float32)
    # the oracle sees exactly the FP32-rounded parameters and inputs
    L_ref, g_ref = mlp.loss_grad(p32.astype(np.float64), X.astype(np.float32).astype(np.float64), a,
                                 y.astype(np.float32).astype(np.float64))
    L, g = fbpt.policy_loss_grad(p32, X, a, y)
    assert abs(L - L_ref) <= 1e-5 * max(1.0, abs(L_ref))
    tol = 2e-5 * np.max(np.abs(g_ref)) + 1e-7
    assert np.max(np.abs(g - g_ref)) <= tol


def test_gpu_training_recovers_a_teacher(fbpt):
    teacher, X, a, _ = problem(7, rows=800)
    y = mlp.forward(teacher, X)[0][np.arange(len(a)), a]
    init = problem(8)[0]
    init[:2 * mlp.N_IN] = teacher[:2 * mlp.N_IN]
    L0 = mlp.loss(init, X, a, y)
    pol, L = fbpt.policy_train(X, a, y, steps=3000, lr=3e-3, init=init)
    params = pol.params().astype(np.float64)
    assert L < L0 / 100
    assert abs(mlp.loss(params, X, a, y) - L) <= 1e-3 * max(L, 1e-3) + 1e-5
    assert np.all(params[:2 * mlp.N_IN] == init[:2 * mlp.N_IN].astype(np.float32))


# ---- what the trained network gains over the degree-ratio heuristic --------------------

DIRS = ("push", "filtered", "pull")


def level_costs(fbpt, dg, seed, S, **kw):
    """Per-level expand + commit device time (ns) under each forced direction.
    A level's frontier does not depend on the direction it is expanded in, so
    the three traces list the same levels row by row."""
    cols = []
    ref = None
    for d in DIRS:
        fbpt.sample(dg, seed, 0, S, schedule=d, launch="graph", **kw)
        tr = fbpt.sample(dg, seed, 0, S, schedule=d, launch="graph", trace_cap=1 << 18, **kw).trace
        if ref is None:
            ref = tr
        assert np.array_equal(tr["units"], ref["units"]) and np.array_equal(tr["colours"], ref["colours"])
        cols.append(tr["expand_ns"].astype(np.float64) + tr["commit_ns"].astype(np.float64))
    return np.stack(cols, 1)


def chosen(fbpt, dg, seed, S, schedule, **kw):
    """Directions a schedule picks, level by level, and its measured level time."""
    fbpt.sample(dg, seed, 0, S, schedule=schedule, launch="graph", **kw)
    tr = fbpt.sample(dg, seed, 0, S, schedule=schedule, launch="graph", trace_cap=1 << 18, **kw).trace
    return tr["direction"].astype(np.int64), float(np.sum(tr["expand_ns"]) + np.sum(tr["commit_ns"]))


def held_out_workloads():
    """Graphs and seeds the shipped network was not trained on: a smaller
    Erdos-Renyi graph, a denser uniform-p R-MAT and a weighted-cascade R-MAT of
    another scale and graph seed."""
    import synth
    rp, col = synth.er_graph(2048, 16384, 4242)
    er = synth.Graph(2048, rp, col, synth.thr_uniform(col.size, 0.1), "er-2k")
    rp, col = synth.rmat_graph(15, 16, 4243)
    dense = synth.Graph(len(rp) - 1, rp, col, synth.thr_uniform(col.size, 0.1), "rmat15-p0.1")
    wc = synth.rmat_wc(17, seed=4244)
    return [(er, 3, 4096, dict(words=1, slots=1, refill="batch")),
            (dense, 5, 2048, dict(words=4, slots=2, refill="lane")),
            (wc, 7, 16384, dict(words=8, slots=1, refill="batch"))]


def test_trained_network_gains_over_the_heuristic(fbpt):
    """The shipped network (the "learned" schedule) against the degree-ratio
    heuristic on held-out workloads, scored two ways: the per-level cost of the
    directions each one picked, read from the forced-direction traces (a
    paired comparison, little timing noise), and each schedule's own measured
    level time.  Output bits never depend on the schedule."""
    rows = []
    for g, seed, S, kw in held_out_workloads():
        dg = fbpt.Graph.from_synth(g)
        T = level_costs(fbpt, dg, seed, S, **kw)
        idx = np.arange(T.shape[0])
        dh, meas_h = chosen(fbpt, dg, seed, S, "heuristic", **kw)
        dl, meas_l = chosen(fbpt, dg, seed, S, "learned", **kw)
        a = fbpt.sample(dg, seed, 0, S, schedule="learned", launch="graph", **kw)
        b = fbpt.sample(dg, seed, 0, S, schedule="push", launch="graph", **kw)
        assert all(np.array_equal(x, y) for x, y in zip(a.to_host(), b.to_host()))
        dg.close()
        row = dict(graph=g.name, levels=T.shape[0], push=T[:, 0].sum(), heuristic=T[idx, dh].sum(),
                   learned=T[idx, dl].sum(), best=T.min(1).sum(), meas_h=meas_h, meas_l=meas_l)
        rows.append(row)
        print({k: (round(v / 1e6, 3) if isinstance(v, float) else v) for k, v in row.items()})
        # never much worse than the best single direction, level by level
        assert row["learned"] <= 1.10 * min(T.sum(0)[:2].min(), row["heuristic"])
    tot = {k: sum(r[k] for r in rows) for k in ("heuristic", "learned", "meas_h", "meas_l")}
    print("gain over heuristic: paired %.2fx, measured %.2fx" % (tot["heuristic"] / tot["learned"],
                                                               tot["meas_h"] / tot["meas_l"]))
    assert tot["learned"] < 0.9 * tot["heuristic"]
    assert tot["meas_l"] < tot["meas_h"]


def test_policy_file_round_trip(fbpt, tmp_path):
    """The shipped policy loads through fbpt_policy_load, saves through
    fbpt_policy_save and reads back to the same float32 parameters."""
    ref = np.loadtxt(fbpt.DEFAULT_POLICY_FILE, dtype=np.float64).astype(np.float32)
    p = fbpt.Policy.load(fbpt.DEFAULT_POLICY_FILE)
    assert np.array_equal(p.params(), ref)
    out = tmp_path / "policy.txt"
    p.save(out)
    assert np.array_equal(np.loadtxt(out, dtype=np.float64).astype(np.float32), ref)
    q = fbpt.Policy.load(out)
    assert np.array_equal(q.params(), ref)
    p.close()
    q.close()
