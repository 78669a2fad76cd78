"""The memory-system probe follows the chains its interface defines: every
chain's sum equals a host replay of the same gathers (same hash, same float32
additions in the same order)."""
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
    import paper_2305_07253_gb300 as rq
    rng = np.random.default_rng(5)
    cells = rng.normal(size=(n_cells, 8)).astype(np.float32)
    out = rq.rt_gather_probe(torch.from_numpy(cells).cuda(), steps, blocks).cpu().numpy()
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
