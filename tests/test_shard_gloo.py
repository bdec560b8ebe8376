"""Multi-process path on CPU (gloo, world size 2): sample-id sharding and the
one exchange step (all-reduce of the integer counts).  Each rank runs the
oracle on its own id range; the merged counts must equal one run over all
ids, and so must the finalized ECC and Kemeny estimates."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_2311_10290_gb300 import inputs as I  # noqa: E402
from paper_2311_10290_gb300.shard import allreduce_counts, id_range  # noqa: E402

SEED, TOTAL, FIRST = 99, 301, 17


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = I.ba(300, 3, seed=2)
        v = oracle.root_max_degree(g.row_ptr)
        start, count = id_range(rank, world, TOTAL, FIRST)
        c = oracle.sample(g.row_ptr, g.col, v, SEED, start, count, keep_per_sample=False)
        sums = np.array([count, c.sum_y1, c.sum_y2], dtype=np.uint64)
        c1, c2, s3 = allreduce_counts(c.cnt1, c.cnt2, sums)
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), c1=c1, c2=c2, s3=s3)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run(world, tmp_path):
    mp.spawn(_worker, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)
    return [np.load(tmp_path / ("rank%d.npz" % r)) for r in range(world)]


@pytest.mark.parametrize("world", [2])
def test_sharded_counts_merge_exactly(world, tmp_path):
    res = _run(world, tmp_path)
    g = I.ba(300, 3, seed=2)
    v = oracle.root_max_degree(g.row_ptr)
    full = oracle.sample(g.row_ptr, g.col, v, SEED, FIRST, TOTAL, keep_per_sample=False)
    for r in res:                                   # every rank holds the totals
        assert np.array_equal(r["c1"], full.cnt1)
        assert np.array_equal(r["c2"], full.cnt2)
        assert [int(x) for x in r["s3"]] == [TOTAL, full.sum_y1, full.sum_y2]
    ld, ec, kc = oracle.finalize(g.row_ptr, v, TOTAL, res[0]["c1"], res[0]["c2"], int(res[0]["s3"][1]),
                                 int(res[0]["s3"][2]))
    ld_f, ec_f, kc_f = oracle.finalize(g.row_ptr, v, TOTAL, full.cnt1, full.cnt2, full.sum_y1, full.sum_y2)
    assert np.array_equal(ec, ec_f) and kc == kc_f


def test_id_ranges_partition_the_ids():
    for world in (1, 2, 3, 8):
        for total in (0, 1, 7, 64, 1001):
            parts = [id_range(r, world, total, 5) for r in range(world)]
            ids = [i for s, c in parts for i in range(s, s + c)]
            assert ids == list(range(5, 5 + total))
            sizes = [c for _, c in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        id_range(2, 2, 10)
