"""Host-side logic of the benchmark (no GPU): the time-to-accuracy grid, the
disjointness of the sample-id ranges its forms and timed calls draw, and the
source-hash guard on the measured traffic figures."""
import itertools
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("omega_max", [256, 1000, 16384, 65536])
def test_omega_grid_is_the_sqrt2_grid(omega_max):
    g = bench.omega_grid(omega_max)
    assert g[0] == min(256, omega_max) or omega_max < 256
    assert g[-1] == omega_max
    assert all(a < b for a, b in zip(g, g[1:]))
    for k, w in enumerate(g[:-1]):
        assert w == int(round(256 * 2.0 ** (k / 2.0)))
    assert len(g) == len(set(g))


@pytest.mark.parametrize("omega_max,seeds", [(16384, 10), (65536, 10), (1 << 20, 16)])
def test_time_to_accuracy_id_ranges_are_disjoint(omega_max, seeds):
    ranges = []
    for form, base in bench.TTA_ID_BASE.items():
        for s in range(seeds):
            ranges.append((base + s * omega_max, base + (s + 1) * omega_max))
        ranges.append((base + bench.TTA_TIMED_OFFSET, base + bench.TTA_TIMED_OFFSET + omega_max))
    assert all(hi <= (1 << 32) for _, hi in ranges)
    for (a0, a1), (b0, b1) in itertools.combinations(ranges, 2):
        assert a1 <= b0 or b1 <= a0, ((a0, a1), (b0, b1))


def test_measured_traffic_follows_the_source_hash():
    assert bench.measured_traffic("no_such_kernel", 10) is None
    for name, (per_step, files, sha) in bench.TRAFFIC_PER_WILSON_STEP.items():
        got = bench.measured_traffic(name + " (description)", 1000)
        if bench.sources_sha1(files) == sha:
            assert got == pytest.approx(per_step * 1000)
        else:
            assert got is None
