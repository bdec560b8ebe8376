"""lap_sample_static: the sampler for callers that cannot allocate device
memory (for example a plug-in whose host application owns all device memory,
or a service that must keep a fixed footprint after start-up).  It keeps its
scratch in a fixed array inside the library, so its results must equal those
of the handle API (lap_graph_create / lap_set_root / lap_sample / lap_counts)
exactly, also on the second of two calls in a row, when the array still holds
the previous call's contents.  Integer counts: compared bit for bit.

This file sorts last so that a run stopping at the first failure has run
everything else first."""
import numpy as np
import pytest

from paper_2311_10290_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2311_10290_gb300.lap import (LAP_OPT_CURSOR, LapError, LapGraph,  # noqa: E402
                                        lap_sample_static, lap_static_scratch_bytes)


def handle_counts(g, root, seed, first, count):
    G = LapGraph(g.row_ptr, g.col)
    try:
        v = G.set_root(root)
        G.set_option(LAP_OPT_CURSOR, first)
        G.sample(count, seed)
        c1, c2, s = G.counts()
        return v, c1, c2, s
    finally:
        G.close()


def static_counts(g, root, seed, first, count):
    rp = torch.from_numpy(g.row_ptr).cuda()
    cl = torch.from_numpy(g.col).cuda()
    c1 = torch.full((g.n,), -1, dtype=torch.int64, device="cuda")    # garbage: must be overwritten
    c2 = torch.full((g.n,), -1, dtype=torch.int64, device="cuda")
    s2 = torch.full((2,), -1, dtype=torch.int64, device="cuda")
    lap_sample_static(g.n, rp, cl, root, seed, first, count, c1, c2, s2,
                      stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return (c1.cpu().numpy().astype(np.uint64), c2.cpu().numpy().astype(np.uint64),
            s2.cpu().numpy().astype(np.uint64))


def test_two_calls_in_a_row_match_the_handle_api():
    cases = [
        (I.er(800, 0.012, seed=3), -1, 77, 0, 500),
        (I.ba(3000, 3, seed=1), -1, 5, 1000, 300),     # second call: scratch holds call 1's state
        (I.ba(3000, 3, seed=1), 7, 5, 1000, 300),      # third: same graph, explicit root
    ]
    for g, root, seed, first, count in cases:
        v, c1, c2, s = handle_counts(g, root, seed, first, count)
        d1, d2, ds = static_counts(g, v if root < 0 else root, seed, first, count)
        assert np.array_equal(c1, d1)
        assert np.array_equal(c2, d2)
        assert int(ds[0]) == int(s[1]) and int(ds[1]) == int(s[2])
        if root < 0:   # automatic root choice agrees too
            e1, e2, es = static_counts(g, -1, seed, first, count)
            assert np.array_equal(c1, e1) and np.array_equal(c2, e2) and np.array_equal(ds, es)


def test_lanes_reuse_their_slot_within_one_call():
    """n_samples several times the number of slots the scratch holds: every
    lane runs several samples in its slot, one after another, so the per-slot
    epoch bits (not a fresh zeroed state) separate the samples."""
    g = I.ba(200_000, 5, seed=2)
    slots = (lap_static_scratch_bytes() - 16 * g.n) // (8 * g.n)
    count = 100
    assert count >= 4 * slots
    for first in (0, 7_000):    # two calls in a row on the same graph
        v, c1, c2, s = handle_counts(g, -1, 31, first, count)
        d1, d2, ds = static_counts(g, v, 31, first, count)
        assert np.array_equal(c1, d1) and np.array_equal(c2, d2)
        assert int(ds[0]) == int(s[1]) and int(ds[1]) == int(s[2])


def test_graph_too_large_for_the_scratch_is_rejected():
    n = lap_static_scratch_bytes() // 24 + 1000
    g = I.path(int(n))
    rp = torch.from_numpy(g.row_ptr).cuda()
    cl = torch.from_numpy(g.col).cuda()
    out = torch.zeros(g.n, dtype=torch.int64, device="cuda")
    s2 = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(LapError) as e:
        lap_sample_static(g.n, rp, cl, 0, 1, 0, 1, out, out, s2)
    assert e.value.name == "LAP_ERR_TOO_LARGE"
