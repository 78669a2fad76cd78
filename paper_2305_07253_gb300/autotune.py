"""Launch autotuner: times a workload under each candidate tuning and keeps the fastest.

The candidates cover the knobs of rt_set_tuning: kernel (wavefront stages with
per-lane refill, or one thread per query), threads per block, resident blocks
per SM, the refill threshold, the grid layout (cell-corner copy or plain
grid), the tree width, and the query order (bits of the origin lattice, or
none).  Results never depend on the tuning, only the time does.
"""
from __future__ import annotations

import itertools
import statistics

import torch

from . import (KERNEL_SIMPLE, KERNEL_WAVEFRONT, LAYOUT_CELLS, LAYOUT_PLAIN, rt_get_tuning, rt_set_tuning)


def default_space() -> list[dict]:
    space = []
    for width, block, refill, refill_f, per_sm in itertools.product((8, 2), (64, 128, 256), (8, 16, 32), (8, 16, 24),
                                                                   (0, 4)):
        space.append(dict(kernel=KERNEL_WAVEFRONT, block=block, refill_min=refill, refill_min_field=refill_f,
                          blocks_per_sm=per_sm, grid_layout=LAYOUT_CELLS, bvh_width=width))
    space.append(dict(kernel=KERNEL_WAVEFRONT, block=128, refill_min=16, refill_min_field=16, blocks_per_sm=0,
                      grid_layout=LAYOUT_PLAIN, bvh_width=8))
    for width, block, layout in itertools.product((8, 2), (64, 128, 256), (LAYOUT_CELLS, LAYOUT_PLAIN)):
        space.append(dict(kernel=KERNEL_SIMPLE, block=block, refill_min=16, refill_min_field=16, blocks_per_sm=0,
                          grid_layout=layout, bvh_width=width))
    # the query order on the default launch shape of each kernel (the entries
    # above keep the default order, 4 bits)
    for kernel, bits in itertools.product((KERNEL_WAVEFRONT, KERNEL_SIMPLE), (0, 2, 3, 5)):
        space.append(dict(kernel=kernel, block=128, refill_min=32, refill_min_field=16, blocks_per_sm=0,
                          grid_layout=LAYOUT_CELLS, bvh_width=2, order_bits=bits))
    for cand in space:
        cand.setdefault("order_bits", 4)
    return space


def time_fn(fn, reps: int = 5, warmup: int = 2) -> float:
    """Median device time of fn() in ms (CUDA events on the current stream)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def autotune(fn, space: list[dict] | None = None, reps: int = 5, warmup: int = 2, apply: bool = True):
    """Return (best tuning dict, [(tuning dict, ms), ...]); sets the best one if `apply`."""
    prev = rt_get_tuning()
    results = []
    try:
        for cand in space or default_space():
            rt_set_tuning(**cand)
            results.append((dict(cand), time_fn(fn, reps, warmup)))
    finally:
        rt_set_tuning(prev)
    best = min(results, key=lambda r: r[1])[0]
    if apply:
        rt_set_tuning(**best)
    return best, results
