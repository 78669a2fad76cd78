"""The memory-system probes (include/mem_probe.h) compute what their interface
defines: every gather chain's sum equals a host replay of the same gathers
(same hash, same float32 additions in the same order), and the L2 / L1 reads
visit every word the stated number of times."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fmix32(h):
    h = h ^ (h >> np.uint32(16))
    h = h * np.uint32(0x85EBCA6B)
    h = h ^ (h >> np.uint32(13))
    h = h * np.uint32(0xC2B2AE35)
    return h ^ (h >> np.uint32(16))


@pytest.mark.parametrize("n_cells,steps,blocks", [(1, 3, 1), (4096, 17, 3)])
def test_probe_chains_match_a_host_replay(n_cells, steps, blocks):
    from paper_2305_07253_gb300 import mem_probe
    rng = np.random.default_rng(5)
    cells = rng.normal(size=(n_cells, 8)).astype(np.float32)
    out = mem_probe.random_gather(torch.from_numpy(cells).cuda(), steps, blocks).cpu().numpy()
    mask = np.uint32(n_cells - 1)
    with np.errstate(over="ignore"):
        idx = _fmix32(np.arange(1, blocks * 128 + 1, dtype=np.uint32)) & mask
        acc = np.zeros(blocks * 128, dtype=np.float32)
        bits = cells.view(np.uint32)
        for s in range(steps):
            v = cells[idx]
            acc = acc + (v[:, 0] + v[:, 7])
            idx = _fmix32(idx ^ bits[idx, 3] ^ np.uint32(s)) & mask
    assert np.array_equal(out.view(np.uint32), acc.view(np.uint32))


def test_l2_and_l1_reads_visit_every_word():
    """With x lanes holding small integers the float sums are exact: the total
    over all threads is reps x the sum of the x lanes of the buffer (L2), or of
    every block's window (L1)."""
    from paper_2305_07253_gb300 import mem_probe
    words = 4096 * 3 + 5
    x = np.zeros((words, 4), dtype=np.float32)
    x[:, 0] = np.arange(words) % 7
    buf = torch.from_numpy(x).cuda()
    out = mem_probe.l2_read(buf, 3, 5).cpu().numpy().astype(np.float64)
    assert out.sum() == 3 * x[:, 0].astype(np.float64).sum()
    window, blocks = 8192, 4
    w = window // 16
    out = mem_probe.l1_read(buf, window, 2, blocks).cpu().numpy().astype(np.float64)
    assert out.sum() == 2 * x[: w * blocks, 0].astype(np.float64).sum()
    with pytest.raises(ValueError):
        mem_probe.l1_read(buf, window, 2, 100)  # buffer shorter than blocks x window
