"""Host-side tools of the benchmark and the input generators (no GPU)."""
import importlib.util
import os
import sys

import numpy as np

from synth import rays as R
from synth import scene as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    argv, sys.argv = sys.argv, ["bench.py"]
    try:
        spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        return mod
    finally:
        sys.argv = argv


def test_trace_hash_ignores_comments_but_not_code():
    b = _bench()
    src = 'int a = 1; // note\n/* block\n comment */ const char* s = "x // y /* z */";\n\nint b;\n'
    assert b._code_only(src) == 'int a = 1;\n const char* s = "x // y /* z */";\nint b;'
    assert b._code_only(src.replace("// note", "// other")) == b._code_only(src)
    assert b._code_only(src.replace("int b;", "int c;")) != b._code_only(src)
    assert len(b.trace_hash()) == 16


def test_mixed_frame_is_seeded_and_shaped_like_the_batching_workload():
    s = S.make_scene("tiny")
    a = R.mixed_frame(s, 0, 2.0)
    b = R.mixed_frame(s, 0, 2.0)
    c = R.mixed_frame(s, 1, 2.0)
    assert [x[0] for x in a] == ["primary", "ao", "gi", "shadow"]
    n_px = 1920 * 1080
    sizes = {name: rays.shape[0] for name, rays, _ in a}
    assert sizes["gi"] == n_px and n_px <= sizes["ao"] <= 4 * n_px and 500_000 <= sizes["shadow"] <= n_px
    for (_, ra, ka), (_, rb, kb) in zip(a, b):
        assert ka == kb and np.array_equal(ra, rb)
    assert not np.array_equal(a[2][1], c[2][1])
    assert a[3][2] == dict(mode=2, m_near=2.0, m_far=2.0, any_hit=True)
    for _, rays, _ in a:
        d = rays[:, 4:7].astype(np.float64)
        assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
        assert np.all(rays[:, 3] <= rays[:, 7])
