"""Failure detection without a GPU fault: a bounded device wait that is made
to run out reports FBPT_ETIMEOUT, and the context and the graph stay usable."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_barrier_wait_gives_up_and_library_recovers():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2311_10201_gb300 as fbpt
    fbpt.build()
    g = synth.rmat_wc(12)
    dg = fbpt.Graph.from_synth(g)
    # one poll per wait: every CTA but the last to arrive gives up at once
    with pytest.raises(fbpt.FbptError) as ei:
        fbpt.sample(dg, 3, 0, 4096, words=2, launch="persistent", spin_limit=1)
    assert ei.value.code == fbpt.ETIMEOUT
    torch.cuda.synchronize()
    # the same graph and workspace then give the exact answer
    rr = fbpt.sample(dg, 3, 0, 4096, words=2, launch="persistent")
    ref = oracle.rr_sets(g, 3, 0, 4096)
    off, verts, _, _ = rr.to_host()
    assert np.array_equal(off, ref.offsets) and np.array_equal(verts, ref.verts)
