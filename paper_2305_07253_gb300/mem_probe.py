"""Binding of the memory-system probes (include/mem_probe.h, _build/libmem_probe.so).

Measurement only: the benchmark reports these rates beside the roofline of
the query kernels (the random-gather ceiling of the field stage's access, and
the L2 / L1 read bandwidths that bound the triangle stages, whose node and
triangle reads are mostly served from those caches).  Argument marshalling
only; every buffer is checked here before the call.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmem_probe.so")
EXPORTS = ("mp_random_gather", "mp_l2_read", "mp_l1_read", "mp_last_error")
READ_BLOCK = 256

_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2305_07253_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            L.mp_random_gather.argtypes = [P, i64, i32, i32, P, P]
            L.mp_l2_read.argtypes = [P, i64, i32, i32, P, P]
            L.mp_l1_read.argtypes = [P, i32, i32, i32, P, P]
            for f in (L.mp_random_gather, L.mp_l2_read, L.mp_l1_read):
                f.restype = ctypes.c_int
            L.mp_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise RuntimeError(f"mem_probe: {lib().mp_last_error().decode()}")


def _out(out, n: int, device) -> torch.Tensor:
    if out is None:
        return torch.empty(n, dtype=torch.float32, device=device)
    if (not isinstance(out, torch.Tensor) or out.dtype != torch.float32 or not out.is_cuda
            or out.device != device or not out.is_contiguous() or out.numel() < n):
        raise ValueError(f"out must be a contiguous float32 CUDA tensor on {device} with at least {n} elements")
    return out


def _buffer(buf: torch.Tensor, what: str):
    if not isinstance(buf, torch.Tensor) or not buf.is_cuda or not buf.is_contiguous():
        raise ValueError(f"{what} must be a contiguous CUDA tensor")
    return buf.numel() * buf.element_size()


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def random_gather(cells: torch.Tensor, steps: int, blocks: int, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """Chains of dependent random 32-byte gathers over `cells` (a power-of-two
    number of 32-byte cells); returns each chain's sum (blocks * 128 float32)."""
    nbytes = _buffer(cells, "cells")
    if nbytes % 32:
        raise ValueError("cells must hold a whole number of 32-byte cells")
    out = _out(out, blocks * 128, cells.device)
    _check(lib().mp_random_gather(ctypes.c_void_p(cells.data_ptr()), nbytes // 32, int(steps), int(blocks),
                                  ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def l2_read(buf: torch.Tensor, reps: int, blocks: int, out: torch.Tensor | None = None, stream=None):
    """Read all of `buf` reps times through L2 (16-byte loads); per-thread sums."""
    nbytes = _buffer(buf, "buf")
    out = _out(out, blocks * READ_BLOCK, buf.device)
    _check(lib().mp_l2_read(ctypes.c_void_p(buf.data_ptr()), nbytes, int(reps), int(blocks),
                            ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def l1_read(buf: torch.Tensor, window: int, reps: int, blocks: int, out: torch.Tensor | None = None, stream=None):
    """Block b reads bytes [b * window, (b + 1) * window) of `buf` reps times
    through L1 (16-byte loads); per-thread sums."""
    nbytes = _buffer(buf, "buf")
    if nbytes < int(window) * int(blocks):
        raise ValueError(f"buf holds {nbytes} bytes, fewer than blocks x window = {int(window) * int(blocks)}")
    out = _out(out, blocks * READ_BLOCK, buf.device)
    _check(lib().mp_l1_read(ctypes.c_void_p(buf.data_ptr()), int(window), int(reps), int(blocks),
                            ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out
