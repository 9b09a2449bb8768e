"""The N > 1 path of the benchmark on CPU: two gloo ranks (127.0.0.1), each
sampling its own range of sample ids on a replica of the graph, as bench.py
does under torchrun.  The union of the ranks' RR sets equals one run over the
whole range (sample ids key every draw, so any split is bit-identical), and
the job's step time is the slowest rank's."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, S, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import oracle
    import synth
    import torch
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = synth.rmat_wc(11)
    first, count = bench.rank_samples(rank, S)
    rr = oracle.rr_sets(g, 99, first, count)
    sizes = torch.from_numpy(np.diff(rr.offsets).astype(np.int64))
    verts = torch.from_numpy(rr.verts.astype(np.int64))
    all_sizes = [torch.zeros(count, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(all_sizes, sizes)
    n_verts = torch.tensor([verts.numel()], dtype=torch.int64)
    all_n = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(all_n, n_verts)
    width = int(max(k.item() for k in all_n))  # gloo gathers equal sizes: pad, then trim
    padded = torch.full((width,), -1, dtype=torch.int64)
    padded[:verts.numel()] = verts
    all_verts = [torch.zeros(width, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(all_verts, padded)
    all_verts = [v[:int(k.item())] for v, k in zip(all_verts, all_n)]
    slowest = bench.max_over_ranks(dist, 1.5 + rank, "cpu")
    if rank == 0:
        out.put((torch.cat(all_sizes).numpy(), torch.cat(all_verts).numpy(), slowest))
    dist.destroy_process_group()


def test_two_gloo_ranks_split_the_sample_ids():
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    S, world = 700, 2
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, S, out)) for r in range(world)]
    for p in procs:
        p.start()
    sizes, verts, slowest = out.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = oracle.rr_sets(synth.rmat_wc(11), 99, 0, world * S)
    assert np.array_equal(sizes, np.diff(ref.offsets).astype(np.int64))
    assert np.array_equal(verts, ref.verts.astype(np.int64))
    assert slowest == 2.5
