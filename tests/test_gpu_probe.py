"""The random-access probe (lap_probe_random_rw, a measurement aid) touches
exactly the bytes its SplitMix64 addresses name, all inside the buffer: on a
zeroed buffer the nonzero bytes after a launch are the addresses recomputed
here on the CPU."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2311_10290_gb300.probe import ProbeError, lap_probe_random_rw  # noqa: E402


def splitmix64(z):
    z = z.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def test_probe_touches_exactly_its_addresses():
    nbytes, blocks, rounds, salt = (1 << 20) + 17, 3, 5, 12345
    buf = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    lap_probe_random_rw(buf, blocks, rounds, salt=salt, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = np.nonzero(buf.cpu().numpy())[0]
    t = np.arange(blocks * 256, dtype=np.uint64)[:, None, None]
    r = np.arange(rounds, dtype=np.uint64)[None, :, None]
    j = np.arange(4, dtype=np.uint64)[None, None, :]
    with np.errstate(over="ignore"):
        key = np.uint64(salt) + t * np.uint64(0x9E3779B97F4A7C15) + r * np.uint64(4) + j
    want = np.unique(splitmix64(key) % np.uint64(nbytes)).astype(np.int64)
    assert np.array_equal(got, want)


def test_probe_rejects_empty_launch():
    buf = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(ProbeError):
        lap_probe_random_rw(buf, 0, 1)
