"""CPU checks of the batch work queue (lap_batch_schedule: host logic only,
no device use) and of the uneven-batch input recipe."""
import numpy as np
import pytest

from paper_2311_10290_gb300 import inputs as I


@pytest.fixture(scope="module")
def lap():
    from paper_2311_10290_gb300 import build
    build.build()
    from paper_2311_10290_gb300 import lap as L
    return L


@pytest.mark.parametrize("claim", [1, 3, 16, 100])
@pytest.mark.parametrize("order", [0, 1, 2])
def test_schedule_covers_every_sample_once(lap, order, claim):
    n = [500, 20, 3000, 20, 7, 999]
    samples = 37
    ug, uf = lap.lap_batch_schedule(n, order, samples, claim)
    seen = set()
    for g, f in zip(ug.tolist(), uf.tolist()):
        assert 0 <= g < len(n) and f % claim == 0 and f < samples
        for i in range(f, min(f + claim, samples)):
            assert (g, i) not in seen
            seen.add((g, i))
    assert len(seen) == len(n) * samples
    assert len(ug) == len(n) * -(-samples // claim)


def test_schedule_orders(lap):
    n = [500, 20, 3000, 20, 7, 999]
    first = lambda ug: list(dict.fromkeys(ug.tolist()))     # graphs in order of first appearance
    assert first(lap.lap_batch_schedule(n, 0, 4, 1)[0]) == [2, 5, 0, 1, 3, 4]   # largest first, ties by index
    assert first(lap.lap_batch_schedule(n, 1, 4, 1)[0]) == [4, 1, 3, 0, 5, 2]   # smallest first
    assert first(lap.lap_batch_schedule(n, 2, 4, 1)[0]) == [0, 1, 2, 3, 4, 5]   # caller's order
    # Units of one graph are contiguous and ascending.
    ug, uf = lap.lap_batch_schedule(n, 0, 10, 3)
    for g in range(len(n)):
        idx = np.nonzero(ug == g)[0]
        assert np.all(np.diff(idx) == 1) and np.all(np.diff(uf[idx].astype(np.int64)) == 3)


def test_schedule_rejects_bad_arguments(lap):
    with pytest.raises(lap.LapError):
        lap.lap_batch_schedule([10, 10], 3, 4, 1)
    with pytest.raises(lap.LapError):
        lap.lap_batch_schedule([10, 10], 0, 4, 0)


def test_uneven_batch_recipe():
    spec = I.batch_spec()
    assert len(spec) == 512
    fam = [s[0] for s in spec]
    assert fam[:6] == ["er", "ba", "rmat", "er", "ba", "rmat"]
    n = np.array([s[1] for s in spec], dtype=np.float64)
    deg = np.array([s[2] for s in spec])
    assert n.min() >= 1000 and n.max() <= 1_000_000
    assert 4.0 <= deg.min() and deg.max() <= 32.0
    # log-uniform sizes: the mean of ln n is near the midpoint of [ln 1e3, ln 1e6]
    assert abs(np.log(n).mean() - 0.5 * (np.log(1e3) + np.log(1e6))) < 0.3
    assert spec == I.batch_spec()                              # deterministic
    g = I.batch_graphs(spec[:3] + [("ba", 1200, 6.0, 9)], threads=2)
    for x in g:
        rp = x.row_ptr.astype(np.int64)
        assert rp[0] == 0 and np.all(np.diff(rp) > 0)          # connected generators: every degree >= 1
