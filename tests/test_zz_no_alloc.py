"""The seed selection that allocates no device memory (for callers whose
device memory is all in their own pool, or who must stay clear of the
allocator) gives the same seeds and gains as fbpt_select_seeds, through the C
ABI, on two calls in a row over different RR sets.  Collected last."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_selection_matches_allocating_one():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2311_10201_gb300 as fbpt
    fbpt.build()
    g = synth.rmat_wc(13)
    dg = fbpt.Graph.from_synth(g)
    for first, S, k in ((0, 5000, 40), (7000, 3001, 25)):  # two calls in a row; the second reuses the array
        rr = fbpt.sample(dg, synth.SAMPLE_SEED, first, S)
        want_seeds, want_gains = fbpt.select_seeds(rr, k)
        got_seeds, got_gains = fbpt.select_seeds_noalloc(rr, k)
        assert np.array_equal(got_seeds, want_seeds)
        assert np.array_equal(got_gains, want_gains)


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2311_10201_gb300 as fbpt
    fbpt.build()
    n = 14_000_000  # 5 bytes per vertex alone exceed 64 MiB
    g = synth.Graph(n, np.zeros(n + 1, np.uint64), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    rr = fbpt.sample(fbpt.Graph.from_synth(g), 1, 0, 64)
    with pytest.raises(fbpt.FbptError) as ei:
        fbpt.select_seeds_noalloc(rr, 3)
    assert ei.value.code == fbpt.EINVAL
    assert "67108864" in str(ei.value)
