"""The C interface: the library builds for sm_103a, loads without a GPU and
exports every entry point the public header declares; host-side argument
checks reject bad input before any device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rt_api.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def rtlib():
    from paper_2305_07253_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ("rt_scene_build", "rt_sdf_bake", "rt_trace_combined", "rt_trace_bvh", "rt_trace_sdf",
              "rt_trace_combined_backward"):
        assert n in names


def test_library_exports_every_declared_symbol(rtlib):
    missing = [n for n in _declared() if not hasattr(rtlib, n)]
    assert not missing, missing


def test_binding_export_list_matches_header():
    import paper_2305_07253_gb300 as rq
    assert sorted(rq.EXPORTS) == _declared()


def test_stage_names_match_the_header_enum():
    """rt_trace_combined_timed reports each part's RT_STAGE_* kind; the binding
    names them from the header's enum (RT_STAGE_BVH_NEAR -> "bvh_near")."""
    import paper_2305_07253_gb300 as rq
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    enum = {int(v): k.lower() for k, v in re.findall(r"\bRT_STAGE_([A-Z_]+)\s*=\s*(\d+)", src)}
    assert len(enum) >= 9 and enum[8] == "bvh_near_rest"
    assert rq.STAGE_NAMES == enum


def test_struct_sizes_match_header():
    import paper_2305_07253_gb300 as rq
    assert ctypes.sizeof(rq.rt_split_params) == 32
    assert ctypes.sizeof(rq.rt_scene_info) == 8 * 3 + 4 * 2 + 8 + 4 * 2 + 4 * 6 + 8
    assert ctypes.sizeof(rq.rt_tuning) == 32
    assert ctypes.sizeof(rq.rt_batch) == 8 * 3 + 32


def test_ctypes_structs_match_the_c_header(tmp_path):
    """Sizes and field offsets of the binding's structs equal what a C compiler
    makes of include/rt_api.h."""
    import shutil
    import subprocess

    import paper_2305_07253_gb300 as rq
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"rt_split_params": rq.rt_split_params, "rt_tuning": rq.rt_tuning, "rt_batch": rq.rt_batch,
               "rt_scene_info": rq.rt_scene_info}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rt_api.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(out[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)


def test_tuning_roundtrip_and_validation(rtlib):
    import paper_2305_07253_gb300 as rq
    prev = rq.rt_set_tuning(kernel=rq.KERNEL_SIMPLE, block=256, refill_min=4)
    try:
        t = rq.rt_get_tuning()
        assert (t.kernel, t.block, t.refill_min) == (rq.KERNEL_SIMPLE, 256, 4)
        for bad in (dict(block=48), dict(block=0), dict(refill_min=0), dict(refill_min=33), dict(kernel=7),
                    dict(grid_layout=5), dict(blocks_per_sm=-1), dict(refill_min_field=0), dict(bvh_width=4),
                    dict(order_bits=-1), dict(order_bits=6)):
            with pytest.raises(rq.RtError):
                rq.rt_set_tuning(**bad)
        assert rq.rt_get_tuning().block == 256  # a rejected call changes nothing
    finally:
        rq.rt_set_tuning(prev)


def test_argument_errors_without_a_gpu(rtlib):
    """Argument checks run on the host and return RT_ERR_INVALID_ARG with a message."""
    rtlib.rt_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    # null buffers
    rtlib.rt_scene_build.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_void_p]
    assert rtlib.rt_scene_build(None, 3, None, 1, None, ctypes.byref(out)) == 1
    assert b"null" in rtlib.rt_last_error()
    # grid with n < 2
    rtlib.rt_sdf_create.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]
    lo = (ctypes.c_float * 3)(0, 0, 0)
    hi = (ctypes.c_float * 3)(1, 1, 1)
    n = (ctypes.c_int32 * 3)(1, 4, 4)
    assert rtlib.rt_sdf_create(ctypes.c_void_p(256), 0, lo, hi, n, ctypes.byref(out)) == 1
    assert b"n[0]" in rtlib.rt_last_error()
    # misaligned grid pointer
    n2 = (ctypes.c_int32 * 3)(4, 4, 4)
    assert rtlib.rt_sdf_create(ctypes.c_void_p(258), 0, lo, hi, n2, ctypes.byref(out)) == 1
    # a valid wrap does not touch the device
    assert rtlib.rt_sdf_create(ctypes.c_void_p(256), 0, lo, hi, n2, ctypes.byref(out)) == 0
    rtlib.rt_sdf_destroy.argtypes = [ctypes.c_void_p]
    rtlib.rt_sdf_destroy(out)


PROBE_HEADER = os.path.join(ROOT, "include", "mem_probe.h")


def _declared_probe():
    src = re.sub(r"/\*.*?\*/", "", open(PROBE_HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"\b(mp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def probelib(rtlib):
    from paper_2305_07253_gb300 import mem_probe
    return mem_probe.lib()


def test_probe_library_exports_every_declared_symbol(probelib):
    from paper_2305_07253_gb300 import mem_probe
    names = _declared_probe()
    assert names == sorted(mem_probe.EXPORTS)
    assert not [n for n in names if not hasattr(probelib, n)]


def test_query_library_exports_no_probe(rtlib):
    """The memory-system probes live in their own library, not in the query ABI."""
    assert not [n for n in _declared() if "probe" in n]
    assert not hasattr(rtlib, "rt_gather_probe")


def test_probe_arguments_without_a_gpu(probelib):
    L = probelib
    buf, out = ctypes.c_void_p(4096), ctypes.c_void_p(8192)
    f = L.mp_random_gather
    assert f(None, 16, 4, 1, out, None) == 1 and b"null" in L.mp_last_error()
    assert f(ctypes.c_void_p(4112), 16, 4, 1, out, None) == 1 and b"32-byte" in L.mp_last_error()
    assert f(buf, 24, 4, 1, out, None) == 1 and b"power of two" in L.mp_last_error()
    assert f(buf, 16, 0, 1, out, None) == 1 and b"steps" in L.mp_last_error()
    assert f(buf, 16, 4, 0, out, None) == 1 and b"blocks" in L.mp_last_error()
    g = L.mp_l2_read
    assert g(ctypes.c_void_p(4100), 4096, 1, 1, out, None) == 1 and b"16-byte" in L.mp_last_error()
    assert g(buf, 4100, 1, 1, out, None) == 1 and b"multiple of 16" in L.mp_last_error()
    assert g(buf, 4096, 0, 1, out, None) == 1 and b"reps" in L.mp_last_error()
    h = L.mp_l1_read
    assert h(buf, 5000, 1, 1, out, None) == 1 and b"window" in L.mp_last_error()
    assert h(buf, 4096, 1, 0, out, None) == 1 and b"blocks" in L.mp_last_error()


def test_probe_binding_rejects_a_short_or_wrong_output():
    """The binding checks a caller's output tensor before the library is asked
    to write blocks x threads values into it."""
    import torch

    from paper_2305_07253_gb300 import mem_probe
    cells = torch.zeros(64, dtype=torch.float32)  # CPU tensor: refused before any device call
    with pytest.raises(ValueError):
        mem_probe.random_gather(cells, 4, 1)
    with pytest.raises(ValueError):
        mem_probe._out(torch.zeros(10, dtype=torch.float32), 128, torch.device("cpu"))
    with pytest.raises(ValueError):
        mem_probe._out(torch.zeros(256, dtype=torch.float64), 128, torch.device("cpu"))
    with pytest.raises(ValueError):
        mem_probe._out(torch.zeros(256, dtype=torch.float32)[::2], 128, torch.device("cpu"))


def test_bad_split_params_rejected(rtlib):
    import paper_2305_07253_gb300 as rq
    out = ctypes.c_void_p()
    lo = (ctypes.c_float * 3)(0, 0, 0)
    hi = (ctypes.c_float * 3)(1, 1, 1)
    n = (ctypes.c_int32 * 3)(4, 4, 4)
    rtlib.rt_sdf_create.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]
    assert rtlib.rt_sdf_create(ctypes.c_void_p(256), 0, lo, hi, n, ctypes.byref(out)) == 0
    rtlib.rt_trace_sdf.argtypes = [ctypes.c_void_p] * 6 + []
    rtlib.rt_trace_sdf.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p]
    rtlib.rt_last_error.restype = ctypes.c_char_p
    for bad in (rq.split_params(max_steps=0), rq.split_params(m_near=-1.0), rq.split_params(min_step_vox=0.0),
                rq.split_params(hit_eps_vox=float("nan"))):
        assert rtlib.rt_trace_sdf(out, ctypes.c_void_p(512), 4, ctypes.byref(bad), ctypes.c_void_p(1024), None) == 1
    # misaligned ray buffer
    good = rq.split_params()
    assert rtlib.rt_trace_sdf(out, ctypes.c_void_p(520), 4, ctypes.byref(good), ctypes.c_void_p(1024), None) == 1
    assert b"aligned" in rtlib.rt_last_error()
    # n = 0 is a no-op that succeeds without touching the device
    assert rtlib.rt_trace_sdf(out, None, 0, ctypes.byref(good), None, None) == 0
    rtlib.rt_sdf_destroy.argtypes = [ctypes.c_void_p]
    rtlib.rt_sdf_destroy(out)


def test_cascade_arguments_and_geometry_without_a_gpu(rtlib):
    """rt_cascade_create checks its arguments on the host, places every level
    where the checker's cascade places it, and a trace on a cascade without its
    cell copy is refused before any device work."""
    import numpy as np

    import oracle as O
    import paper_2305_07253_gb300 as rq
    rtlib.rt_last_error.restype = ctypes.c_char_p
    rtlib.rt_cascade_create.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]
    rtlib.rt_cascade_level.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    rtlib.rt_sdf_destroy.argtypes = [ctypes.c_void_p]
    out = ctypes.c_void_p()
    c3 = (ctypes.c_float * 3)(1.25, -0.5, 7.0)
    good = ctypes.c_void_p(256)
    assert rtlib.rt_cascade_create(good, 0, 0, 64, 0.1, c3, ctypes.byref(out)) == 1  # no levels
    assert rtlib.rt_cascade_create(good, 0, 9, 64, 0.1, c3, ctypes.byref(out)) == 1  # > RT_MAX_LEVELS
    assert rtlib.rt_cascade_create(good, 0, 5, 1, 0.1, c3, ctypes.byref(out)) == 1   # n < 2
    assert rtlib.rt_cascade_create(good, 0, 5, 64, 0.0, c3, ctypes.byref(out)) == 1  # h0 = 0
    assert rtlib.rt_cascade_create(ctypes.c_void_p(260), 0, 5, 64, 0.1, c3, ctypes.byref(out)) == 1
    far = (ctypes.c_float * 3)(1e6, 0, 0)
    assert rtlib.rt_cascade_create(good, 0, 5, 64, 0.1, far, ctypes.byref(out)) == 1
    assert b"2^22" in rtlib.rt_last_error()
    nanc = (ctypes.c_float * 3)(float("nan"), 0, 0)
    assert rtlib.rt_cascade_create(good, 0, 5, 64, 0.1, nanc, ctypes.byref(out)) == 1

    rng = np.random.default_rng(7)
    for _ in range(20):
        c = rng.uniform(-40, 40, size=3).astype(np.float32)
        n = int(rng.integers(2, 130))
        L = int(rng.integers(1, 9))
        h0 = np.float32(rng.uniform(0.01, 0.5))
        cc = (ctypes.c_float * 3)(*c.tolist())
        assert rtlib.rt_cascade_create(good, 0, L, n, float(h0), cc, ctypes.byref(out)) == 0
        ref = O.Cascade(c.astype(np.float64), float(h0), n, L, values=np.zeros((L, n, n, n)))
        for k in range(L):
            ilo = (ctypes.c_int32 * 3)()
            h = ctypes.c_float()
            assert rtlib.rt_cascade_level(out, k, ilo, ctypes.byref(h)) == 0
            want_ilo, want_h = ref.level(k)
            assert list(ilo) == want_ilo.tolist()
            assert h.value == np.float32(want_h)
        assert rtlib.rt_cascade_level(out, L, ilo, ctypes.byref(h)) == 1
        rtlib.rt_sdf_destroy(out)

    # a cascade is read through its cell copy: tracing before bake/prepare is refused
    assert rtlib.rt_cascade_create(good, 0, 3, 16, 0.25, c3, ctypes.byref(out)) == 0
    rtlib.rt_trace_sdf.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p]
    prm = rq.split_params()
    assert rtlib.rt_trace_sdf(out, ctypes.c_void_p(512), 4, ctypes.byref(prm), ctypes.c_void_p(1024), None) == 1
    assert b"cell copy" in rtlib.rt_last_error()
    # and rt_cascade_level on a single grid is refused
    lo = (ctypes.c_float * 3)(0, 0, 0)
    hi = (ctypes.c_float * 3)(1, 1, 1)
    n4 = (ctypes.c_int32 * 3)(4, 4, 4)
    single = ctypes.c_void_p()
    rtlib.rt_sdf_create.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]
    assert rtlib.rt_sdf_create(good, 0, lo, hi, n4, ctypes.byref(single)) == 0
    assert rtlib.rt_cascade_level(single, 0, ilo, ctypes.byref(h)) == 1
    rtlib.rt_sdf_destroy(single)
    rtlib.rt_sdf_destroy(out)
