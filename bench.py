"""Benchmark of the combined ray query on the 1080p GI workload.

Workload (the paper's GI rays, Section 3 "GI & Shadow Rays"): the seeded
frame scene (20x6x20 m room, 400 subdivision-4 icospheres + 200 boxes =
2,050,412 triangles), a 256^3 float32 distance field baked on the device,
and 1920x1080 = 2,073,600 cosine-hemisphere GI rays with t_max = 30 m.  One
step = one rt_trace_combined call over all rays at the middle split setting
(m = 2 voxels); the pure techniques (m = inf: triangles only, m = 0: field
only) are timed the same way for the comparison the metric asks for.

Prints one JSON line.  `--impl reference` times the CPU checker instead (the
only place besides the CPU-baseline leg where this script runs it).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import rays as R  # noqa: E402
from synth import scene as S  # noqa: E402

METRIC = "combined-query rays/s vs BVH-only & SDF-only at 1080p GI; hit-t err vs FP64"
UNIT = "rays/s"
M_MIDDLE = 2.0
WORKLOAD = "frame-1080p-gi"
# the sources of the stage kernels: the measured DRAM traffic applies while they are unchanged
TRACE_SOURCES = ["paper_2305_07253_gb300/csrc/rt_trace.cu", "paper_2305_07253_gb300/csrc/rt_trace_dev.cuh",
                 "paper_2305_07253_gb300/csrc/rt_order.cu",
                 "paper_2305_07253_gb300/csrc/rt_internal.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other configurations (batching, precision, fit) and the AO / GI tables")
    ap.add_argument("--cpu-sample", type=int, default=1920 * 1080)
    ap.add_argument("--cpu-reps", type=int, default=3)
    ap.add_argument("--profile", action="store_true",
                    help="set up, then run only warmup+steps launches of the --only traces (for ncu); prints timings")
    ap.add_argument("--only", default="all", choices=["all", "combined", "bvh", "sdf"])
    ap.add_argument("--out", default="images", help="output folder of --workload ao-images / gi-images")
    ap.add_argument("--workload", default="frame", choices=["frame", "batching", "fit", "precision", "ao", "cascade", "ao-images", "gi-images", "dfbuild",
                             "gather"],
                    help="frame: the 1080p GI headline; batching: 8 frames of mixed primary/shadow/AO/GI "
                         "batches; fit: gradient fit of a noisy 128^3 grid; precision: float16 vs float32 "
                         "512^3 grid on the 8.2 M-triangle scene")
    ap.add_argument("--fit-steps", type=int, default=200)
    ap.add_argument("--frames", type=int, default=8)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---- seeded inputs of the extra measurements, made in spawned worker processes
def _gen_mixed_frame(f):
    return [(name, rays, kw) for name, rays, kw in R.mixed_frame(S.make_scene("frame"), f, M_MIDDLE)]


def _gen_fit_rays(n_pool, n_eval):
    s = S.make_scene("fit")
    margin = 2.0 * float((np.array(s.room) / (s.spec.grid_n - 1)).max())
    return R.free_space_rays(s, n_pool, 7, margin), R.free_space_rays(s, n_eval, 8, margin)


def _gen_precision_rays():
    return R.gi_rays(S.make_scene("precision"), 1920 * 1080, 7, 30.0)


def input_pool(jobs):
    """Start the input generators `jobs` = {name: (fn, args)} in a spawn pool;
    returns {name: future}."""
    import concurrent.futures as cf
    import multiprocessing as mp
    ex = cf.ProcessPoolExecutor(max_workers=min(len(jobs), max(1, (os.cpu_count() or 2) - 1)),
                                mp_context=mp.get_context("spawn"))
    futs = {name: ex.submit(fn, *a) for name, (fn, a) in jobs.items()}
    ex.shutdown(wait=False)
    return futs


def make_workload():
    s = S.make_scene("frame")
    rays = R.gi_rays(s, 1920 * 1080, 7, 30.0)
    return s, rays


def config_dict(s, n_rays, extra=None):
    c = {"workload": WORKLOAD, "scene": "frame", "n_tris": int(s.n_tris), "grid": [s.spec.grid_n] * 3,
         "grid_dtype": "f32", "rays": int(n_rays), "ray_kind": "cosine-hemisphere GI", "t_max_m": 30.0,
         "split": {"mode": "one split", "m": M_MIDDLE, "closest_hit": True},
         "l2": "inputs larger than L2 (working set > 500 MB: nodes, triangles, grid, rays, hits)"}
    if extra:
        c.update(extra)
    return c


def _code_only(src: str) -> str:
    """C++ source without its comments and blank lines (string literals kept)."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c == '"':  # string literal
            j = i + 1
            while j < n and src[j] != '"':
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            while i < n and src[i] != "\n":
                i += 1
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(line.rstrip() for line in "".join(out).splitlines() if line.strip())


def trace_hash():
    """Hash of the stage kernels' code (comments excluded): the measured DRAM
    traffic in profiles/traffic.json applies while it is unchanged."""
    h = hashlib.sha256()
    for f in TRACE_SOURCES:
        h.update(_code_only(open(os.path.join(ROOT, f)).read()).encode())
    return h.hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.rows = []
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max([num(r[2]) for r in rows if num(r[2]) is not None] or [0.0])}


def run_ours(args):
    import torch

    import paper_2305_07253_gb300 as rq

    from paper_2305_07253_gb300 import replicas

    rank, world, local = replicas.env()
    extras = rank == 0 and world == 1 and not args.no_extras and not args.profile
    torch.cuda.set_device(local)
    dist = None
    if replicas.init("nccl"):
        import torch.distributed as dist
    dev = torch.device("cuda", local)
    s, rays = make_workload()
    n_rays = rays.shape[0]
    n = s.spec.grid_n
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).to(dev), torch.from_numpy(s.tris).to(dev))
    grid = torch.empty((n, n, n), dtype=torch.float32, device=dev)
    sdf = rq.rt_sdf_create(grid, s.lo, s.hi)
    rq.rt_sdf_bake(scene, sdf, rq.BAKE_BVH)
    rays_d = torch.from_numpy(rays).to(dev)
    hits = torch.empty((n_rays, 6), dtype=torch.int32, device=dev)
    p_mid = rq.split_params(mode=rq.MODE_SPLIT1, m_near=M_MIDDLE)
    # the three forms of the paper's comparison: triangles only (HWRT-only), combined, field only
    p_bvh = rq.split_params(mode=rq.MODE_BVH)
    p_sdf = rq.split_params(mode=rq.MODE_SPLIT1, m_near=0.0)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def time_steps(p, K, W):
        for _ in range(W):
            rq.rt_trace_combined(scene, sdf, rays_d, p, hits)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            rq.rt_trace_combined(scene, sdf, rays_d, p, hits)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1) / K
        if dist is not None:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    K, W = args.steps, max(3, args.warmup)
    if args.profile:
        sel = {"combined": [("combined", p_mid)], "bvh": [("bvh", p_bvh)], "sdf": [("sdf", p_sdf)]}
        todo = sel.get(args.only, [("combined", p_mid), ("bvh", p_bvh), ("sdf", p_sdf)])
        out = {}
        for name, p in todo:
            out[name] = time_steps(p, args.steps, args.warmup)
        if rank == 0:
            print(json.dumps({"profile_ms_per_launch": out, "rays": n_rays}), flush=True)
        return
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    uuid = f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-") else (str(uuid) if uuid else None)

    # algorithmic bytes, from the counted variant and the hit records (untimed)
    counts, outcome = {}, {}
    for name, p in (("combined", p_mid), ("bvh", p_bvh), ("sdf", p_sdf)):
        h, c = rq.rt_trace_combined_counted(scene, sdf, rays_d, p)
        counts[name] = [int(x) for x in c.cpu().tolist()]
        tr = h[:, 4]
        outcome[name] = {"bvh_hits": int((tr == rq.TRACER_BVH).sum()), "sdf_hits": int((tr == rq.TRACER_SDF).sum())}
    step_bytes = 4 * 8  # eight float32 corners per march step

    def stage_bytes(name, stage):
        """Algorithmic bytes one launch of `stage` moves (reads of rays, nodes, triangles,
        grid cells and queue entries; writes of hit records and queue entries).  The query
        order (one kernel) reads each query's origin (16 B) and writes its 4-byte entry of
        the order, which the first stage reads."""
        nodes, tris, steps, _ = counts[name]
        n_bvh_hits = outcome[name]["bvh_hits"]
        q_in = 4 * n_rays if "order" in stage_ms.get(name, {}) else 0
        if stage == "order":
            return (16 + 4) * n_rays
        if "merge" in stage_ms.get(name, {}):
            # closest-hit split call, near and field stages side by side: the near stage lists
            # its hits (32 B each), the field stage reads every ray and writes every record,
            # the merge copies the near hits over their records
            if stage == "bvh_near":
                return 32 * n_rays + 64 * nodes + 48 * tris + 32 * n_bvh_hits + q_in
            if stage == "field_split":
                return 32 * n_rays + step_bytes * steps + 24 * n_rays
            if stage == "merge":
                return (32 + 24) * n_bvh_hits
            if stage == "bvh_near_rest":  # its queries' bytes are counted under bvh_near
                return 0
        if stage == "all":
            return 32 * n_rays + 24 * n_rays + 64 * nodes + 48 * tris + step_bytes * steps + q_in
        if stage == "bvh_full":
            return 32 * n_rays + 24 * n_rays + 64 * nodes + 48 * tris + q_in
        if stage == "field_full":
            return 32 * n_rays + 24 * n_rays + step_bytes * steps + q_in
        if stage == "bvh_near":  # all rays in; hits written; the rest queued
            fwd = n_rays - n_bvh_hits
            return 32 * n_rays + 64 * nodes + 48 * tris + 24 * n_bvh_hits + 8 * fwd + q_in
        if stage == "field_split" and name == "sdf":  # m = 0: no triangle stage, every ray in
            return 32 * n_rays + step_bytes * steps + 24 * n_rays + q_in
        if stage == "field_split":  # queued rays in; every record written here
            fwd = n_rays - n_bvh_hits
            return (8 + 32) * fwd + step_bytes * steps + 24 * fwd
        raise ValueError(stage)

    sampler = ClockSampler(uuid)
    ms_mid = time_steps(p_mid, K, W)
    clocks = sampler.stop()
    ms_bvh = time_steps(p_bvh, K, W)
    ms_sdf = time_steps(p_sdf, K, W)
    # per-kernel device times (events between the stage launches), untimed for the headline
    Kt = max(3, min(K, 30))
    stage_ms = {}
    for name, p in (("combined", p_mid), ("bvh", p_bvh), ("sdf", p_sdf)):
        acc = {}
        for _ in range(Kt):
            _, st = rq.rt_trace_combined_timed(scene, sdf, rays_d, p, hits)
            for sname, ms in st:
                acc.setdefault(sname, []).append(ms)
        stage_ms[name] = {k: statistics.mean(v) for k, v in acc.items()}
    # the same step with the one-thread-per-query kernel, for comparison
    prev = rq.rt_set_tuning(kernel=rq.KERNEL_SIMPLE)
    try:
        ms_simple = {name: time_steps(p, max(3, K // 4), W) for name, p in
                     (("combined", p_mid), ("bvh", p_bvh), ("sdf", p_sdf))}
    finally:
        rq.rt_set_tuning(prev)
    rq.rt_trace_combined(scene, sdf, rays_d, p_mid, hits)
    torch.cuda.synchronize()
    hits_mid = hits.cpu().numpy()
    # end to end through host buffers: pinned rays in, pinned hit records out
    rays_h = torch.from_numpy(rays).pin_memory()
    hits_h = torch.empty((n_rays, 6), dtype=torch.int32).pin_memory()
    Ke = max(3, min(K, 50))
    for _ in range(W):
        rq.trace_combined_from_host(scene, sdf, rays_h, p_mid, hits_h, rays_d, hits)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(Ke):
        rq.trace_combined_from_host(scene, sdf, rays_h, p_mid, hits_h, rays_d, hits)
    e1.record(stream)
    barrier()
    ms_e2e = e0.elapsed_time(e1) / Ke
    if dist is not None:
        t = torch.tensor([ms_e2e], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_e2e = float(t.item())

    value = world * n_rays / (ms_mid * 1e-3)
    peak, peak_kind = peaks()
    # the dominant kernel is the field stage, which carries the step's DRAM traffic; with the
    # near and field stages side by side the near stage's time stretches too, but it is served
    # from L1/L2 and its time is not its own
    comb = stage_ms["combined"]
    dom_stage = "field_split" if "field_split" in comb else max(comb.items(), key=lambda kv: kv[1])[0]
    dom_ms = comb[dom_stage]
    ab = stage_bytes("combined", dom_stage)
    achieved = ab / (dom_ms * 1e-3) / 1e9
    traffic = None
    tf = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tf):
        d = json.load(open(tf))
        if d.get("trace_hash") == trace_hash() and d.get("workload") == WORKLOAD:
            traffic = d.get("bytes_per_launch", {}).get(dom_stage)
    caches = cache_ceilings()
    kernel_names = {"bvh_near": "k_stage_bvh (near triangle sub-interval)",
                    "field_split": "k_stage_field (distance-field sub-interval)",
                    "bvh_full": "k_stage_bvh", "field_full": "k_stage_field", "all": "k_trace",
                    "order": "k_order_local (query order)", "merge": "k_merge_hits (near hits over the field's records)",
                    "bvh_near_rest": "k_stage_bvh (near sub-interval, second launch after the field stage)"}
    stages = {name: {st: {"ms": ms, "algorithmic_bytes": stage_bytes(name, st),
                          "GBps": stage_bytes(name, st) / (ms * 1e-3) / 1e9,
                          "frac_of_hbm": stage_bytes(name, st) / (ms * 1e-3) / 1e9 / peak,
                          "frac_of_l2_read": stage_bytes(name, st) / (ms * 1e-3) / 1e9 / caches["l2_read_GBps"]}
                     for st, ms in v.items()} for name, v in stage_ms.items()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_mid, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded procedural scene and rays)",
        "config": config_dict(s, n_rays),
        "parallelism": f"rays replicated per GPU x{world}" if world > 1 else "1 GPU",
        "tuning": rq.rt_get_tuning().as_dict(),
        "bvh_only": {"value": world * n_rays / (ms_bvh * 1e-3), "ms_per_step": ms_bvh},
        "sdf_only": {"value": world * n_rays / (ms_sdf * 1e-3), "ms_per_step": ms_sdf},
        "combined": {"value": value, "ms_per_step": ms_mid, "m": M_MIDDLE},
        "ordering_ok": bool(ms_bvh > ms_mid >= ms_sdf),
        "one_thread_per_query": {k: {"ms_per_step": v, "value": world * n_rays / (v * 1e-3)}
                                 for k, v in ms_simple.items()},
        "stages": stages,
        "work_counts": {k: {"nodes": v[0], "tris": v[1], "steps": v[2], "field_queries": v[3], **outcome[k]}
                        for k, v in counts.items()},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": kernel_names.get(dom_stage, dom_stage) + ", combined m=2"
                     + (", beside the near stage on the same SMs" if "merge" in comb else ""),
                     "algorithmic_bytes_per_launch": ab, "launch_ms": dom_ms, "peak_kind": f"of {peak_kind}",
                     "step": {"algorithmic_bytes": stage_bytes("combined", "all"),
                              "GBps": stage_bytes("combined", "all") / (ms_mid * 1e-3) / 1e9},
                     "random_gather": gather_ceiling(peak), "caches": caches},
        "e2e": {"value": world * n_rays / (ms_e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(rays.nbytes),
                "d2h_bytes_per_step": int(n_rays * 24), "ms_per_step": ms_e2e},
        "gpu_launches": K * len(stage_ms["combined"]),
        "clocks": clocks,
        "trace_hash": trace_hash(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"], line["hit_t_err_vs_fp64"] = cpu_baseline(s, rays, hits_mid, args.cpu_sample,
                                                                       args.cpu_reps, grid.cpu().numpy())
    if extras:
        # the other configurations and the paper's experiments, untimed for the headline.
        # Their host inputs are made first, in worker processes, and all of them before
        # any of these measurements: a busy host delays kernel launches, and the gap
        # would fall inside the device-timed intervals.
        del rays_h, hits_h
        t0 = time.perf_counter()
        jobs = {f"frame{f}": (_gen_mixed_frame, (f,)) for f in range(args.frames)}
        jobs["fit"] = (_gen_fit_rays, (2 * 1024 * 1024, 1024 * 1024))
        jobs["precision"] = (_gen_precision_rays, ())
        futs = input_pool(jobs)
        inputs = {k: f.result() for k, f in futs.items()}
        line["extras_input_seconds"] = time.perf_counter() - t0
        pool, evals = inputs.pop("fit")
        line["fit"] = extra_fit(rq, pool, evals, steps=args.fit_steps)
        del pool, evals
        line["ao"] = extra_ao(rq, scene, s, sdf256=sdf)
        line["gi_images"] = extra_gi_images(rq, scene, s, W=480, H=270, spp=8)
        frames = [inputs.pop(f"frame{f}") for f in range(args.frames)]
        line["batching"] = extra_batching(rq, scene, sdf, grid, frames)
        del frames
        torch.cuda.empty_cache()
        line["precision"] = extra_precision(rq, inputs.pop("precision"))
        line["extras_seconds"] = time.perf_counter() - t0
        line["success_conditions"] = {
            "ordering_bvh_gt_combined_ge_sdf": line["ordering_ok"],
            "combined_step_ge_0.4_of_roofline": bool(line["roofline"]["step"]["GBps"] / peak >= 0.4),
            "persistent_graph_beats_per_batch": line["batching"]["persistent_graph_beats_per_batch"],
            "f16_beats_per_batch": line["batching"]["f16_beats_per_batch"],
            "f16_beats_f32_at_m2_precision_scene": line["precision"]["f16_beats_f32_at_m2"],
            "fit_lowers_disagreement": line["fit"]["fit_lowers_disagreement"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def _oracle_world(s, sample_rays):
    import oracle as O
    n = s.spec.grid_n
    bvh = O.BVH(s.verts, s.tris)
    grid = O.Grid(s.lo, s.hi, [n, n, n], src=bvh)
    prm = O.make_params(mode=1, m_near=M_MIDDLE)
    # first pass evaluates the grid values the sample touches (the device grid
    # is baked before its timed region, so the timed CPU pass is the warm one)
    O.trace_combined(bvh, grid, sample_rays, prm, precision=64)
    return O, bvh, grid, prm


def fp64_gap(O, s, rays, g, o, grid_dev_h, ogrid):
    """Classify every difference between the device records (float path, the
    device's own bake) and the fp64 checker's (fp64 march on its fp64 bake):
      equal            same tracer; triangle: same primitive, t within 1e-4
                       relative; field: t within 1e-3 relative
      triangle_boundary a triangle hit on either side that lies within 1e-5 of
                       an edge, grazes (|n.d| < 1e-3), ties (fp64 t of the
                       device's triangle within 1e-4 of the checker's) or sits
                       within 1e-4 of a sub-interval end, in fp64
      field_near_tie   no triangle hit involved, and the fp64 march came within
                       one hit threshold eps_hit of the other outcome at some
                       step (its decision margin <= eps_hit): a near-tangent pass
                       by a surface, where the float march's samples (a few ulp
                       apart along the ray after many steps) may decide that
                       step the other way, a step-count flip
      field_other      anything else."""
    n = rays.shape[0]
    gt = g[:, 0].view(np.float32).astype(np.float64)
    gp = g[:, 1].astype(np.int64)
    gtr = g[:, 4].astype(np.int64)
    otr, ot, op = o["tracer"].astype(np.int64), o["t"], o["prim"].astype(np.int64)
    with np.errstate(invalid="ignore"):
        rel = np.abs(gt - ot) / np.maximum(1.0, np.abs(ot))
    equal = ((gtr == 0) & (otr == 0)) | ((gtr == 1) & (otr == 1) & (gp == op) & (rel <= 1e-4)) | \
        ((gtr == 2) & (otr == 2) & (rel <= 1e-3))
    vals, known = ogrid.export()
    bake_err = float(np.max(np.abs(grid_dev_h.reshape(-1)[known].astype(np.float64) - vals[known])))
    hmax = float(np.max((s.hi - s.lo) / (s.spec.grid_n - 1)))
    delta = 0.01 * float(np.min((s.hi - s.lo) / (s.spec.grid_n - 1)))  # eps_hit of the default step rule
    r64 = rays.astype(np.float64)
    t1 = np.minimum(np.maximum(r64[:, 3] + M_MIDDLE * hmax, r64[:, 3]), r64[:, 7])
    ends = np.stack([r64[:, 3], t1, r64[:, 7]], axis=1)

    def boundary(idx, prims, t_ref=None):
        if idx.size == 0:
            return np.zeros(0, dtype=bool)
        c = O.tri_check(s.verts, s.tris, rays[idx], prims)
        edge = np.abs(np.minimum(np.minimum(c["u"], c["v"]), 1 - c["u"] - c["v"])) < 1e-5
        graze = c["ndotd"] < 1e-3
        with np.errstate(invalid="ignore"):
            near_end = np.any(np.abs(ends[idx] - c["t"][:, None]) <= 1e-4 * np.maximum(1, np.abs(ends[idx])), axis=1)
            tie = np.zeros(idx.size, dtype=bool) if t_ref is None else \
                np.abs(c["t"] - t_ref) <= 1e-4 * np.maximum(1, np.abs(t_ref))
        return edge | graze | near_end | tie

    bad = ~equal
    tri_bound = np.zeros(n, dtype=bool)
    gi = np.nonzero(bad & (gtr == 1))[0]
    tri_bound[gi] |= boundary(gi, gp[gi], np.where(otr[gi] == 1, ot[gi], np.nan))
    oi = np.nonzero(bad & (otr == 1))[0]
    tri_bound[oi] |= boundary(oi, op[oi])
    fld = bad & ~((gtr == 1) | (otr == 1))
    near = fld & (o["margin"] <= delta)
    other = bad & ~tri_bound & ~near
    both_f = (gtr == 2) & (otr == 2)
    hist_edges = (1e-7, 1e-6, 1e-5, 1e-4, delta, 1e-3)
    hist = {f"<= {x:.3g} m": int((fld & (o["margin"] <= x)).sum()) for x in hist_edges}
    return {"rays": int(n), "equal": int(equal.sum()), "triangle_boundary": int((bad & tri_bound).sum()),
            "field_near_tie": int(near.sum()), "field_near_tie_tracer_flips": int((near & (gtr != otr)).sum()),
            "field_near_tie_both_field": int((near & both_f).sum()), "field_other": int(other.sum()),
            "eps_hit_m": delta, "device_bake_max_err_m": bake_err, "checker_samples_compared": int(known.sum()),
            "field_differences_by_fp64_margin": hist,
            "both_field_rel_dt_max": {"equal": float(rel[both_f & equal].max()) if (both_f & equal).any() else 0.0,
                                      "near_tie": float(rel[both_f & near].max()) if (both_f & near).any() else 0.0},
            "field_other_examples": [[int(i), int(gtr[i]), int(otr[i]), float(gt[i]), float(ot[i]),
                                      float(o["margin"][i])] for i in np.nonzero(other)[0][:5]]}


def cpu_baseline(s, rays, gpu_hits, sample, reps, grid_dev_h=None):
    idx = np.linspace(0, rays.shape[0] - 1, min(sample, rays.shape[0])).astype(np.int64)
    sr = rays[idx]
    O, bvh, grid, prm = _oracle_world(s, sr)
    cores = O.default_threads()
    times = []
    for _ in range(max(1, reps)):
        t0 = time.perf_counter()
        o = O.trace_combined(bvh, grid, sr, prm, precision=64, nthreads=cores)
        times.append(time.perf_counter() - t0)
    dt = statistics.median(times)
    g = gpu_hits[idx]
    gt = g[:, 0].view(np.float32).astype(np.float64)
    gtr = g[:, 4]
    err = {"bvh_resolved": _err_stats(gt, gtr, o, 1), "sdf_resolved": _err_stats(gt, gtr, o, 2)}
    err["tracer_agreement"] = float(np.mean(gtr == o["tracer"]))
    err["sample"] = f"{len(idx)} rays evenly spaced over the batch, fp64 checker, m={M_MIDDLE}"
    if grid_dev_h is not None:
        err["classified"] = fp64_gap(O, s, sr, g, o, grid_dev_h, grid)
    cb = {"value": len(idx) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
          "sample": f"{len(idx)} of {rays.shape[0]} GI rays (evenly spaced), fp64 combined query m={M_MIDDLE}, "
                    f"grid values evaluated before timing, median of {max(1, reps)} passes", "seconds": dt}
    return cb, err


def gather_ceiling(peak, K=10, W=2):
    """Rate of chains of dependent random 32-byte gathers over 2^24 cells (537 MB,
    beyond the L2), one chain per thread at the field stage's occupancy (12 blocks
    of 128 per SM), 64 gathers a chain: the access a march step makes, with no
    locality.  Context for the field stage's fraction of the copy bandwidth."""
    import torch

    from paper_2305_07253_gb300 import mem_probe
    n_cells, steps = 1 << 24, 64
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = sms * 12
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    cells = torch.rand(n_cells * 8, device="cuda", generator=g)
    out = torch.empty(blocks * 128, dtype=torch.float32, device="cuda")
    ms = _time_ms(lambda: mem_probe.random_gather(cells, steps, blocks, out), K, W)
    nbytes = blocks * 128 * steps * 32
    del cells, out
    gbps = nbytes / (ms * 1e-3) / 1e9
    return {"useful_GBps": gbps, "frac": gbps / peak, "bytes_per_launch": nbytes, "launch_ms": ms,
            "cells": n_cells, "chains": blocks * 128, "gathers_per_chain": steps}


def cache_ceilings(K=10, W=2):
    """Read bandwidth of the L2 (a 64 MiB buffer read 10 times over with
    coalesced 16-byte loads that bypass L1) and of the L1 (each block re-reading
    its own 64 KiB window 50 times, two blocks per SM): the ceilings of the
    triangle stages, whose node and triangle reads are mostly L1 and L2 hits."""
    import torch

    from paper_2305_07253_gb300 import mem_probe
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    l2_bytes, l2_reps, l2_blocks = 64 << 20, 10, sms * 8
    buf = torch.ones(l2_bytes // 4, dtype=torch.float32, device="cuda")
    out = torch.empty(l2_blocks * mem_probe.READ_BLOCK, dtype=torch.float32, device="cuda")
    ms_l2 = _time_ms(lambda: mem_probe.l2_read(buf, l2_reps, l2_blocks, out), K, W)
    window, l1_reps, l1_blocks = 64 << 10, 50, sms * 2
    out1 = torch.empty(l1_blocks * mem_probe.READ_BLOCK, dtype=torch.float32, device="cuda")
    ms_l1 = _time_ms(lambda: mem_probe.l1_read(buf, window, l1_reps, l1_blocks, out1), K, W)
    del buf, out, out1
    l2 = l2_bytes * l2_reps / (ms_l2 * 1e-3) / 1e9
    l1 = window * l1_blocks * l1_reps / (ms_l1 * 1e-3) / 1e9
    return {"l2_read_GBps": l2, "l1_read_GBps": l1,
            "l2": {"bytes": l2_bytes, "reps": l2_reps, "blocks": l2_blocks, "launch_ms": ms_l2},
            "l1": {"window_bytes": window, "reps": l1_reps, "blocks": l1_blocks, "launch_ms": ms_l1}}


def run_gather(args):
    """Only the memory-system probes (for a profiler): K timed launches after W."""
    import torch
    torch.cuda.set_device(0)
    peak, peak_kind = peaks()
    r = gather_ceiling(peak, K=args.steps, W=args.warmup)
    print(json.dumps({"metric": "dependent random 32-byte gathers, 537 MB", "value": r["useful_GBps"], "unit": "GB/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                      "dtype": "f32", "data": "synthetic", "peak_kind": f"of {peak_kind}", **r,
                      "caches": cache_ceilings(K=args.steps, W=args.warmup),
                      "config": {"workload": "gather-probe-537MB"}}), flush=True)


def run_reference(args):
    """The CPU checker (fp64, all host cores) on the benchmark's own workload:
    each step is one combined query (m = 2) over all 2,073,600 GI rays.  The
    grid values the rays touch are evaluated in a first, untimed pass (the
    device bakes its grid before its timed region too)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    s, rays = make_workload()
    O, bvh, grid, prm = _oracle_world(s, rays)
    cores = O.default_threads()
    for _ in range(args.warmup):
        O.trace_combined(bvh, grid, rays, prm, precision=64, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.trace_combined(bvh, grid, rays, prm, precision=64, nthreads=cores)
    dt = time.perf_counter() - t0
    v = args.steps * rays.shape[0] / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded procedural scene and rays)",
            "config": config_dict(s, rays.shape[0]), "parallelism": f"{cores} host threads",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"all {rays.shape[0]} GI rays per step, fp64 combined query m={M_MIDDLE}, "
                                       "grid values the rays touch evaluated before timing"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def extra_batching(rq, scene, sdf, grid, frames_np, reps=2, tune=True):
    """Batching configuration: len(frames_np) frames of mixed batches (primary,
    AO, GI, shadow; R.mixed_frame) on the frame scene, traced one call per
    batch, through rt_trace_batches, its CUDA graph, and with a float16 grid."""
    import torch

    from paper_2305_07253_gb300 import autotune

    dev = grid.device
    frames = [[(name, torch.from_numpy(r).to(dev), rq.split_params(**kw),
                torch.empty((r.shape[0], 6), dtype=torch.int32, device=dev)) for name, r, kw in fb]
              for fb in frames_np]
    n_total = sum(b[1].shape[0] for fb in frames for b in fb)
    sizes = [{b[0]: int(b[1].shape[0]) for b in fb} for fb in frames]

    def per_batch():
        for fb in frames:
            for _, rd, p, h in fb:
                rq.rt_trace_combined(scene, sdf, rd, p, h)

    def batched(sd=sdf):
        for fb in frames:
            rq.rt_trace_batches(scene, sd, [(rd, p, h) for _, rd, p, h in fb])

    rate = lambda ms: n_total / (ms * 1e-3)  # noqa: E731
    forms = {}
    forms["one_call_per_batch"] = _time_ms(per_batch, reps, warm=1)
    forms["batched"] = _time_ms(batched, reps, warm=1)
    default = rq.rt_get_tuning().as_dict()
    best, top = default, []
    prev = rq.rt_get_tuning()
    if tune:
        f0 = [(rd, p, h) for _, rd, p, h in frames[0]]
        best, results = autotune.autotune(lambda: rq.rt_trace_batches(scene, sdf, f0), reps=2, warmup=1)
        top = sorted(([r[1], r[0]] for r in results), key=lambda x: x[0])[:5]
        forms["batched_autotuned"] = _time_ms(batched, reps, warm=1)
    # the autotuner's pick for each batch kind of the first frame alone (one call per batch)
    per_kind = {}
    if tune:
        for name, rd, p, h in frames[0]:
            rq.rt_set_tuning(prev)
            ms_default = _time_ms(lambda: rq.rt_trace_combined(scene, sdf, rd, p, h), 3, warm=1)
            kbest, kres = autotune.autotune(lambda: rq.rt_trace_combined(scene, sdf, rd, p, h), reps=2, warmup=1,
                                            apply=False)
            per_kind[name] = {"rays": int(rd.shape[0]), "default_ms": ms_default,
                              "autotuned_ms": min(r[1] for r in kres), "pick": kbest}
        rq.rt_set_tuning(**best)
    graphs = []
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        for fb in frames:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=st):
                rq.rt_trace_batches(scene, sdf, [(rd, p, h) for _, rd, p, h in fb], stream=st)
            graphs.append(g)
    torch.cuda.current_stream().wait_stream(st)

    def replay():
        for g in graphs:
            g.replay()

    forms["batched_cuda_graph"] = _time_ms(replay, reps, warm=1)
    del graphs
    g16 = grid.half()
    sdf16 = rq.rt_sdf_create(g16, *_box(sdf))
    rq.rt_sdf_prepare(sdf16)
    forms["batched_f16_grid"] = _time_ms(lambda: batched(sdf16), reps, warm=1)
    rq.rt_set_tuning(prev)
    out = {"frames": len(frames), "rays_total": int(n_total), "batch_sizes_per_frame": sizes,
           "forms": {k: {"ms_total": v, "value": rate(v)} for k, v in forms.items()},
           "tuning_default": default, "tuning_autotuned": best, "autotune_top5": top,
           "autotune_per_kind": per_kind}
    out["persistent_graph_beats_per_batch"] = bool(forms["batched_cuda_graph"] < forms["one_call_per_batch"])
    out["f16_beats_per_batch"] = bool(forms["batched_f16_grid"] < forms["one_call_per_batch"])
    del g16, sdf16, frames
    return out


def _box(sdf):
    return sdf.lo, sdf.hi


def _frame_world(rq, dev):
    import torch
    s = S.make_scene("frame")
    n = s.spec.grid_n
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).to(dev), torch.from_numpy(s.tris).to(dev))
    grid = torch.empty((n, n, n), dtype=torch.float32, device=dev)
    sdf = rq.rt_sdf_create(grid, s.lo, s.hi)
    rq.rt_sdf_bake(scene, sdf, rq.BAKE_BVH)
    return s, scene, grid, sdf


def run_batching(args):
    import torch

    import paper_2305_07253_gb300 as rq

    futs = input_pool({f"frame{f}": (_gen_mixed_frame, (f,)) for f in range(args.frames)})
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    s, scene, grid, sdf = _frame_world(rq, dev)
    frames = [futs[f"frame{f}"].result() for f in range(args.frames)]
    out = extra_batching(rq, scene, sdf, grid, frames, reps=max(1, args.steps // 50))
    line = {"metric": "mixed-batch rays/s (primary, shadow, AO, GI per frame)",
            "value": out["forms"]["batched_cuda_graph"]["value"], "unit": UNIT, "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic (seeded procedural scene and rays)", "dtype": "f32",
            "config": {"workload": "frame-mixed-batches", "scene": "frame", "n_tris": int(s.n_tris),
                       "grid": [s.spec.grid_n] * 3}, "batching": out}
    print(json.dumps(line), flush=True)


def extra_fit(rq, pool_np, evals_np, steps=200, per=1024 * 1024):
    """Differentiation configuration: gradient fit of a noisy grid (102,532
    triangles, 128^3 float32 = exact bake + N(0, (0.5 voxel)^2) noise), `per`
    free-space rays a step drawn in turn from `pool_np`, loss = mean (t_field -
    t_triangles)^2 + 100 mean phi(p*)^2 at the triangle hit points, Adam (lr 0.02
    voxel) through the adjoint kernel.  Steps/s and the field-vs-triangles
    disagreement on `evals_np` before and after, and for the clean bake."""
    import torch

    from paper_2305_07253_gb300 import fit as F
    from synth import rng as RNG

    dev = torch.device("cuda", torch.cuda.current_device())
    s = S.make_scene("fit")
    n = s.spec.grid_n
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).to(dev), torch.from_numpy(s.tris).to(dev))
    clean = torch.empty((n, n, n), dtype=torch.float32, device=dev)
    sdf_clean = rq.rt_sdf_create(clean, s.lo, s.hi)
    rq.rt_sdf_bake(scene, sdf_clean)
    h = np.array(s.room) / (n - 1)
    h_min = float(h.min())
    noise = RNG.normal(s.seed, 501, n ** 3).astype(np.float32).reshape(n, n, n) * (0.5 * h_min)
    grid = clean + torch.from_numpy(noise).to(dev)
    sdf = rq.rt_sdf_create(grid, s.lo, s.hi)
    rq.rt_sdf_prepare(sdf)
    pool = torch.from_numpy(pool_np).to(dev)
    evals = torch.from_numpy(evals_np).to(dev)
    t_pool = rq.hit_fields(rq.rt_trace_bvh(scene, pool))["t"].clone()
    t_eval = rq.hit_fields(rq.rt_trace_bvh(scene, evals))["t"].clone()
    nb = max(1, pool.shape[0] // per)

    def batches(step):
        k = step % nb
        return pool[k * per:(k + 1) * per], t_pool[k * per:(k + 1) * per]

    before = F.disagreement(scene, sdf, evals, t_eval)
    before_c = F.disagreement(scene, sdf, evals, t_eval, m_near=M_MIDDLE)
    clean_d = F.disagreement(scene, sdf_clean, evals, t_eval)
    clean_c = F.disagreement(scene, sdf_clean, evals, t_eval, m_near=M_MIDDLE)
    lr, surface_weight = 0.02 * h_min, 100.0
    # warm-up on a copy (first-use costs of the optimiser and the gathers stay out of the timing)
    warm = grid.clone()
    F.fit_grid(scene, rq.rt_sdf_create(warm, s.lo, s.hi), batches, 3, lr=lr, surface_weight=surface_weight)
    del warm
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    hist = F.fit_grid(scene, sdf, batches, steps, lr=lr, log_every=20, surface_weight=surface_weight)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    after = F.disagreement(scene, sdf, evals, t_eval)
    after_c = F.disagreement(scene, sdf, evals, t_eval, m_near=M_MIDDLE)
    return {"n_tris": int(s.n_tris), "grid": [n, n, n], "rays_per_step": per, "steps": steps,
            "noise_sigma_m": 0.5 * h_min, "lr": lr, "surface_weight": surface_weight,
            "steps_per_s": steps / (ms * 1e-3), "ms_per_step": ms / steps,
            "disagreement_field_only": {"noisy_init": before, "fitted": after, "clean_bake": clean_d},
            "disagreement_combined_m2": {"noisy_init": before_c, "fitted": after_c, "clean_bake": clean_c},
            "fit_lowers_disagreement": bool(after["mean_abs"] < before["mean_abs"]),
            "loss_history": [[hh.step, hh.loss] for hh in hist]}


def run_fit(args):
    import torch

    import paper_2305_07253_gb300 as rq

    fut = input_pool({"fit": (_gen_fit_rays, (4 * 1024 * 1024, 1024 * 1024))})["fit"]
    torch.cuda.set_device(0)
    pool, evals = fut.result()
    out = extra_fit(rq, pool, evals, steps=args.fit_steps)
    line = {"metric": "gradient-fit steps/s and field-vs-triangle hit-t disagreement", "value": out["steps_per_s"],
            "unit": "steps/s", "n_gpus": 1, "steps": args.fit_steps, "higher_is_better": True,
            "data": "synthetic (seeded procedural scene and rays)", "dtype": "f32",
            "config": {"workload": "fit-noisy-grid"}, "fit": out}
    print(json.dumps(line), flush=True)


def _err_stats(gt, g_tr, o, tr):
    sel = (g_tr == tr) & (o["tracer"] == tr)
    r = np.abs(gt[sel] - o["t"][sel]) / np.maximum(1.0, np.abs(o["t"][sel]))
    return {"n": int(sel.sum()), "mean_rel": float(r.mean()) if r.size else 0.0,
            "p99_rel": float(np.quantile(r, 0.99)) if r.size else 0.0,
            "max_rel": float(r.max()) if r.size else 0.0}


def extra_precision(rq, rays, K=5, W=3, sample=16384):
    """Precision configuration: 8,201,612 triangles, a 512^3 grid baked in float32
    on the device and stored again in float16, 1080p GI rays: ms per step for
    m in {0, 2, inf} with each storage, and hit-t error against the fp64 checker
    (its own BVH and exact bake) per tracer segment on an evenly spaced sample."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    s = S.make_scene("precision")
    n = s.spec.grid_n
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).to(dev), torch.from_numpy(s.tris).to(dev))
    g32 = torch.empty((n, n, n), dtype=torch.float32, device=dev)
    sdf32 = rq.rt_sdf_create(g32, s.lo, s.hi)
    rq.rt_sdf_bake(scene, sdf32, rq.BAKE_BVH)
    g16 = g32.half()
    sdf16 = rq.rt_sdf_create(g16, s.lo, s.hi)
    rq.rt_sdf_prepare(sdf16)
    rd = torch.from_numpy(rays).to(dev)
    hits = torch.empty((rd.shape[0], 6), dtype=torch.int32, device=dev)
    idx = np.linspace(0, rays.shape[0] - 1, sample).astype(np.int64)
    timing, got = {}, {}
    for m in (0.0, M_MIDDLE, math.inf):
        p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=m)
        for name, sdf in (("f32", sdf32), ("f16", sdf16)):
            ms = _time_ms(lambda: rq.rt_trace_combined(scene, sdf, rd, p, hits), K, warm=W)
            got[(m, name)] = rq.rt_trace_combined(scene, sdf, rd, p).cpu().numpy()[idx]
            timing[f"m={m}/{name}"] = {"ms": ms, "rays_per_s": rays.shape[0] / (ms * 1e-3)}
    del sdf16, g16, sdf32, g32, scene
    torch.cuda.empty_cache()
    import oracle as O
    t0 = time.perf_counter()
    bvh = O.BVH(s.verts, s.tris)
    ogrid = O.Grid(s.lo, s.hi, [n, n, n], src=bvh)
    errs = {}
    for m in (0.0, M_MIDDLE, math.inf):
        o = O.trace_combined(bvh, ogrid, rays[idx], O.make_params(mode=1, m_near=m), precision=64)
        for name in ("f32", "f16"):
            g = got[(m, name)]
            gt, gtr = g[:, 0].view(np.float32).astype(np.float64), g[:, 4]
            errs[f"m={m}/{name}"] = {"bvh_resolved": _err_stats(gt, gtr, o, 1),
                                     "sdf_resolved": _err_stats(gt, gtr, o, 2),
                                     "tracer_agreement": float(np.mean(gtr == o["tracer"]))}
    return {"n_tris": int(s.n_tris), "grid": [n, n, n], "grid_bytes": {"f32": n ** 3 * 4, "f16": n ** 3 * 2},
            "rays": int(rays.shape[0]), "timing_ms": timing, "hit_t_err_vs_fp64": errs,
            "f16_beats_f32_at_m2": bool(timing[f"m={M_MIDDLE}/f16"]["ms"] < timing[f"m={M_MIDDLE}/f32"]["ms"]),
            "cpu_leg": {"sample": f"{sample} evenly spaced GI rays, fp64 checker with its own BVH and exact bake",
                        "seconds": time.perf_counter() - t0}}


def run_precision(args):
    import torch

    import paper_2305_07253_gb300 as rq

    fut = input_pool({"precision": (_gen_precision_rays, ())})["precision"]
    torch.cuda.set_device(0)
    out = extra_precision(rq, fut.result(), K=max(3, args.steps // 10), W=max(3, args.warmup))
    line = {"metric": "float16 vs float32 grid: rays/s and hit-t error vs fp64, per split setting",
            "value": out["timing_ms"][f"m={M_MIDDLE}/f16"]["rays_per_s"], "unit": UNIT, "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic (seeded procedural scene and rays)",
            "dtype": "f16 grid, f32 math", "config": {"workload": "precision-512"}, "precision": out}
    print(json.dumps(line), flush=True)


def extra_ao(rq, scene, s, sdf256=None, K=3, n_pts=1 << 18, spp=16):
    """Ambient occlusion with the three tracers (the numeric form of the paper's
    AO comparison, Section 3 "Occlusion Queries" and Fig. 2): n_pts camera-facing
    surface points, spp cosine rays each, t in [0, t_ao]; AO = share of a point's
    rays that reach t_ao unoccluded (harness.ambient_occlusion).  For each grid
    (the 256^3 frame grid and a coarse 64^3 one), t_ao and multiplier m: ms per
    call (default tuning, and one thread per query), and the AO error against
    triangles only (mean |dAO|, mean signed dAO, share of points off by > 0.1)."""
    import torch

    from paper_2305_07253_gb300 import harness as HN

    dev = torch.device("cuda", torch.cuda.current_device())
    p, nn = R.surface_points(s, n_pts, 31)
    bias = 1e-3 * s.diagonal
    out = {}
    for n in (s.spec.grid_n, 64):
        if n == s.spec.grid_n and sdf256 is not None:
            sdf, grid = sdf256, None
        else:
            grid = torch.empty((n, n, n), dtype=torch.float32, device=dev)
            sdf = rq.rt_sdf_create(grid, s.lo, s.hi)
            rq.rt_sdf_bake(scene, sdf, rq.BAKE_BVH)
        for t_ao in (0.5, 2.0, 10.0):
            rays = torch.from_numpy(R.ao_rays(p, nn, np.full(n_pts, spp, dtype=np.int64), 32, t_ao, bias)).to(dev)
            hits = torch.empty((rays.shape[0], 6), dtype=torch.int32, device=dev)
            ao_ref = None
            for m in (math.inf, 4.0, 2.0, 1.0, 0.0):
                prm = rq.split_params(mode=rq.MODE_SPLIT1, m_near=m)
                ms = _time_ms(lambda: rq.rt_trace_combined(scene, sdf, rays, prm, hits), K)
                prev = rq.rt_set_tuning(kernel=rq.KERNEL_SIMPLE)
                ms_simple = _time_ms(lambda: rq.rt_trace_combined(scene, sdf, rays, prm, hits), K)
                rq.rt_set_tuning(prev)
                ao = HN.ao_from_records(hits[:, 4], spp)
                if ao_ref is None:
                    ao_ref = ao.clone()
                d = ao - ao_ref
                out[f"grid={n}/t_ao={t_ao}/m={m}"] = {
                    "ms": ms, "ms_one_thread_per_query": ms_simple, "rays_per_s": rays.shape[0] / (ms * 1e-3),
                    "ao_mean": float(ao.mean()), "mean_abs_dAO": float(d.abs().mean()), "mean_dAO": float(d.mean()),
                    "share_off_0.1": float((d.abs() > 0.1).float().mean())}
            del rays, hits
        del sdf, grid
    return {"points": n_pts, "rays_per_point": spp, "grids": [s.spec.grid_n, 64], "table": out}


def run_ao(args):
    import torch

    import paper_2305_07253_gb300 as rq

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    s = S.make_scene("frame")
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).to(dev), torch.from_numpy(s.tris).to(dev))
    out = extra_ao(rq, scene, s, K=max(3, args.steps // 20))
    line = {"metric": "AO tracing time and AO error vs triangles-only, per AO distance and split multiplier",
            "value": out["table"][f"grid={s.spec.grid_n}/t_ao=2.0/m=2.0"]["rays_per_s"], "unit": UNIT, "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic (seeded procedural scene and rays)", "dtype": "f32",
            "config": {"workload": "frame-ao", "n_tris": int(s.n_tris)}, "ao": out}
    print(json.dumps(line), flush=True)


def _time_ms(fn, reps, warm=2):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_cascade(args):
    """The paper's distance-field set-up (Section 3, "Distance Field Generation"):
    camera-centred cascades of 5 levels, 64^3 with a 0.1 m finest voxel for the
    combined query and 128^3 with 0.05 m for field-only tracing, on the frame
    scene, each filled by the exact bake and by the paper's build
    (voxelisation, jump flooding, sweeps).  Reports: build times (also of the
    dense 256^3 grid); per form, 1080p GI tracing time (t_max 30 m; combined: one
    split, m = 2, t_1 from the voxel at the ray's origin) and agreement with
    triangles only; AO (t_ao = 2 m, 16 rays per point) time and error against
    triangles only; rolling updates as the camera moves one finest voxel per
    frame along each axis (Section 3)."""
    import torch

    import paper_2305_07253_gb300 as rq

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    s = S.make_scene("frame")
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).to(dev), torch.from_numpy(s.tris).to(dev))
    eye = np.asarray(s.camera.eye, dtype=np.float32)
    K = max(5, args.steps // 10)
    methods = {"exact": rq.BAKE_BVH, "jfa": rq.BAKE_JFA}
    forms = {"combined": (64, 0.1), "field_only": (128, 0.05)}
    cas = {}
    bake_ms = {}
    for mname, method in methods.items():
        for name, (n, h0) in forms.items():
            g = torch.empty((5, n, n, n), dtype=torch.float32, device=dev)
            sdf = rq.rt_cascade_create(g, h0, eye)
            bake_ms[f"{name}/{mname}"] = _time_ms(lambda: rq.rt_sdf_bake(scene, sdf, method), 3, warm=1)
            cas[(name, mname)] = (g, sdf)
        gd = torch.empty((256, 256, 256), dtype=torch.float32, device=dev)
        dense = rq.rt_sdf_create(gd, s.lo, s.hi)
        bake_ms[f"dense256/{mname}"] = _time_ms(lambda: rq.rt_sdf_bake(scene, dense, method), 3, warm=1)
        del dense, gd
    gi = torch.from_numpy(R.gi_rays(s, 1920 * 1080, 7, 30.0)).to(dev)
    p_pts, nn = R.surface_points(s, 1 << 18, 31)
    ao_rays = torch.from_numpy(R.ao_rays(p_pts, nn, np.full(1 << 18, 16, dtype=np.int64), 32, 2.0,
                                         1e-3 * s.diagonal)).to(dev)
    out = {"bake_ms": bake_ms, "gi": {}, "ao": {}}
    hits = torch.empty((gi.shape[0], 6), dtype=torch.int32, device=dev)
    ao_hits = torch.empty((ao_rays.shape[0], 6), dtype=torch.int32, device=dev)
    runs = {"bvh_only": (None, rq.split_params(mode=rq.MODE_BVH))}
    for mname in methods:
        runs[f"combined/{mname}"] = (cas[("combined", mname)][1], rq.split_params(mode=rq.MODE_SPLIT1, m_near=M_MIDDLE))
        runs[f"field_only/{mname}"] = (cas[("field_only", mname)][1], rq.split_params(mode=rq.MODE_SDF))
        runs[f"field_only_coarse/{mname}"] = (cas[("combined", mname)][1], rq.split_params(mode=rq.MODE_SDF))
    ref_t = ref_ao = None
    for name, (sdf, prm) in runs.items():
        ms = _time_ms(lambda: rq.rt_trace_combined(scene, sdf, gi, prm, hits), K)
        f = rq.hit_fields(hits)
        t = f["t"].double()
        if ref_t is None:
            ref_t = t.clone()
        both = torch.isfinite(t) & torch.isfinite(ref_t)
        rel = ((t - ref_t).abs() / ref_t.clamp(min=1e-6))[both]
        out["gi"][name] = {"ms": ms, "rays_per_s": gi.shape[0] / (ms * 1e-3),
                           "hit_agreement": float((torch.isfinite(t) == torch.isfinite(ref_t)).float().mean()),
                           "mean_rel_dt": float(rel.mean()) if rel.numel() else 0.0,
                           "share_rel_dt_above_1pct": float((rel > 0.01).float().mean()) if rel.numel() else 0.0}
        ms = _time_ms(lambda: rq.rt_trace_combined(scene, sdf, ao_rays, prm, ao_hits), K)
        ao = 1.0 - (ao_hits[:, 4] > 0).float().reshape(-1, 16).mean(dim=1)
        if ref_ao is None:
            ref_ao = ao.clone()
        d = ao - ref_ao
        out["ao"][name] = {"ms": ms, "mean_abs_dAO": float(d.abs().mean()), "mean_dAO": float(d.mean()),
                           "share_off_0.1": float((d.abs() > 0.1).float().mean())}
    # the split multiplier on the combined-mode cascade (Section 3: t_1 from the
    # voxel at the ray's start point), and the same split with the finest voxel
    # h0 instead: a query whose start point lies in level k is traced with
    # m * 2^-k, so that t_1 = t_min + m h0 exactly (h_k = h0 2^k)
    out["m_sweep"] = cascade_m_sweep(rq, scene, cas, gi, ao_rays, hits, ao_hits, K)
    # rolling updates: the camera walks one finest voxel per frame along x, y and z
    roll = {}
    for (name, mname), (g, sdf) in cas.items():
        h0 = forms[name][1]
        per_axis = {}
        for axis in range(3):
            rq.rt_cascade_recenter(scene, sdf, eye)
            c = eye.astype(np.float64) + 0.5 * h0  # mid-voxel: each step crosses one sample
            rq.rt_cascade_recenter(scene, sdf, c.astype(np.float32))
            times, moved = [], []
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            for f in range(24):
                c[axis] += h0
                e[0].record()
                moved.append(rq.rt_cascade_recenter(scene, sdf, c.astype(np.float32)))
                e[1].record()
                torch.cuda.synchronize()
                times.append(e[0].elapsed_time(e[1]))
            times = np.array(times)
            per_axis["xyz"[axis]] = {"mean_ms": float(times.mean()), "max_ms": float(times.max()),
                                     "median_ms": float(np.median(times)),
                                     "levels_moved_per_frame": float(np.mean(moved)), "frames": len(times)}
        roll[f"{name}/{mname}"] = per_axis
    out["rolling"] = roll
    line = {"metric": "cascaded distance field: GI and AO tracing, error vs triangles only, build and update cost",
            "value": out["gi"]["combined/exact"]["rays_per_s"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "data": "synthetic (seeded procedural scene and rays)", "dtype": "f32",
            "config": {"workload": "frame-cascade", "n_tris": int(s.n_tris), "levels": 5,
                       "combined": {"n": 64, "h0": 0.1}, "field_only": {"n": 128, "h0": 0.05},
                       "gi_rays": int(gi.shape[0]), "ao_rays": int(ao_rays.shape[0]), "m": M_MIDDLE},
            "cascade": out}
    print(json.dumps(line), flush=True)


def _start_levels(rq, sdf, rays):
    """Cascade level holding each query's start point o + t_min d (the finest
    whose closed box holds it; the coarsest otherwise), on the host."""
    r = rays.cpu().numpy().astype(np.float64)
    p = r[:, 0:3] + r[:, 3:4] * r[:, 4:7]
    lv = np.full(r.shape[0], sdf.levels - 1, dtype=np.int64)
    for k in range(sdf.levels - 2, -1, -1):
        lo, hi = (np.asarray(b, dtype=np.float64) for b in rq.rt_cascade_box(sdf, k))
        lv = np.where(np.all((p >= lo) & (p <= hi), axis=1), k, lv)
    return lv


def cascade_m_sweep(rq, scene, cas, gi, ao_rays, hits, ao_hits, K, spp=16):
    """Combined query on the 5 x 64^3 cascade for m in {0.5, 1, 2, 4}: GI and
    AO (t_ao 2 m) time and error against triangles only, with t_1 from the voxel
    at the start point (the paper's rule) and from the finest voxel."""
    import torch
    res = {}
    p_bvh = rq.split_params(mode=rq.MODE_BVH)
    ref = {}
    for name, rays, h in (("gi", gi, hits), ("ao", ao_rays, ao_hits)):
        ms = _time_ms(lambda: rq.rt_trace_combined(scene, None, rays, p_bvh, h), K)
        f = rq.hit_fields(h)
        ref[name] = (f["t"].double().clone(), (f["tracer"] > 0).clone())
        res[f"triangles_only/{name}_ms"] = ms
    for mname in ("exact", "jfa"):
        sdf = cas[("combined", mname)][1]
        groups = {}
        for name, rays in (("gi", gi), ("ao", ao_rays)):
            lv = _start_levels(rq, sdf, rays)
            order = np.argsort(lv, kind="stable")
            idx = torch.from_numpy(order).to(rays.device)
            bounds = np.searchsorted(lv[order], np.arange(sdf.levels + 1))
            groups[name] = (rays[idx].contiguous(), idx, bounds)
        for rule in ("start_voxel", "finest_voxel"):
            for m in (0.5, 1.0, 2.0, 4.0):
                for name, rays, h in (("gi", gi, hits), ("ao", ao_rays, ao_hits)):
                    if rule == "start_voxel":
                        prm = rq.split_params(mode=rq.MODE_SPLIT1, m_near=m)
                        fn = lambda: rq.rt_trace_combined(scene, sdf, rays, prm, h)  # noqa: E731
                        fn()
                        hh = h
                    else:
                        rs, idx, bounds = groups[name]
                        out_h = torch.empty_like(h)
                        specs = [(rs[bounds[k]:bounds[k + 1]], rq.split_params(mode=rq.MODE_SPLIT1, m_near=m * 2.0 ** -k),
                                  out_h[bounds[k]:bounds[k + 1]]) for k in range(sdf.levels) if bounds[k + 1] > bounds[k]]
                        fn = lambda: rq.rt_trace_batches(scene, sdf, specs)  # noqa: E731
                        fn()
                        hh = torch.empty_like(h)
                        hh[idx] = out_h
                    ms = _time_ms(fn, K)
                    f = rq.hit_fields(hh)
                    e = {"ms": ms, "speedup_vs_triangles": res[f"triangles_only/{name}_ms"] / ms}
                    if name == "gi":
                        t, rt = f["t"].double(), ref["gi"][0]
                        both = torch.isfinite(t) & torch.isfinite(rt)
                        rel = ((t - rt).abs() / rt.clamp(min=1e-6))[both]
                        e["mean_rel_dt"] = float(rel.mean())
                    else:
                        ao = 1.0 - (f["tracer"] > 0).double().reshape(-1, spp).mean(dim=1)
                        ao_ref = 1.0 - ref["ao"][1].double().reshape(-1, spp).mean(dim=1)
                        d = ao - ao_ref
                        e["mean_abs_dAO"] = float(d.abs().mean())
                        e["share_off_0.1"] = float((d.abs() > 0.1).double().mean())
                    res[f"{mname}/{rule}/m={m}/{name}"] = e
    return res


def _write_png(path, img):
    """8-bit greyscale PNG of a (h, w) array in [0, 1]."""
    import struct
    import zlib
    a = (np.clip(img, 0.0, 1.0) * 255.0 + 0.5).astype(np.uint8)
    h, w = a.shape
    raw = b"".join(b"\x00" + a[y].tobytes() for y in range(h))

    def chunk(tag, data):
        return struct.pack(">I", len(data)) + tag + data + struct.pack(">I", zlib.crc32(tag + data) & 0xffffffff)
    with open(path, "wb") as f:
        f.write(b"\x89PNG\r\n\x1a\n" + chunk(b"IHDR", struct.pack(">IIBBBBB", w, h, 8, 0, 0, 0, 0)) +
                chunk(b"IDAT", zlib.compress(raw, 6)) + chunk(b"IEND", b""))


def _pixels(W, H):
    """(row, column) of every primary ray (the rays come in 8x8 screen tiles)."""
    py, px = np.mgrid[0:H, 0:W]
    order = R._tile_order(px.ravel(), py.ravel(), W)
    return py.ravel()[order], px.ravel()[order]


def _visible(rq, scene, s, W, H):
    import torch
    prim_rays = R.primary_rays(s, W, H)
    f = rq.hit_fields(rq.rt_trace_bvh(scene, torch.from_numpy(prim_rays).cuda()))
    from paper_2305_07253_gb300 import harness as HN
    return HN.visible_points(prim_rays, f["t"].cpu().numpy().astype(np.float64), f["prim"].cpu().numpy(),
                             s.verts, s.tris)


def _image_fields(rq, scene, s):
    import torch
    dense = torch.empty((256, 256, 256), dtype=torch.float32, device="cuda")
    sdf_dense = rq.rt_sdf_create(dense, s.lo, s.hi)
    rq.rt_sdf_bake(scene, sdf_dense, rq.BAKE_BVH)
    cg = torch.empty((5, 64, 64, 64), dtype=torch.float32, device="cuda")
    sdf_c = rq.rt_cascade_create(cg, 0.1, np.asarray(s.camera.eye, dtype=np.float32))
    rq.rt_sdf_bake(scene, sdf_c, rq.BAKE_JFA)
    return (dense, sdf_dense), (cg, sdf_c)


def extra_ao_images(rq, scene, s, W=960, H=540, spp=16, t_ao=2.0, out_dir=None):
    """AO images (the image form of the paper's Fig. 2): per pixel the surface
    point the camera sees (primary rays, triangles), spp cosine rays to t_ao
    (harness.ambient_occlusion), with triangles only, the combined query (m = 2)
    and the field only, on the dense exact grid and on the paper's 5 x 64^3
    cascade built by its own method; per-pixel error against triangles only.
    With out_dir, writes the images and 4 x |dAO| error images as PNG."""
    from paper_2305_07253_gb300 import harness as HN
    x, nx, seen = _visible(rq, scene, s, W, H)
    pix_y, pix_x = _pixels(W, H)
    (_, sdf_dense), (_, sdf_c) = _image_fields(rq, scene, s)
    forms = {"triangles": (None, rq.split_params(mode=rq.MODE_BVH)),
             "combined_dense": (sdf_dense, rq.split_params(mode=rq.MODE_SPLIT1, m_near=M_MIDDLE)),
             "field_dense": (sdf_dense, rq.split_params(mode=rq.MODE_SDF)),
             "combined_cascade": (sdf_c, rq.split_params(mode=rq.MODE_SPLIT1, m_near=M_MIDDLE)),
             "field_cascade": (sdf_c, rq.split_params(mode=rq.MODE_SDF))}
    if out_dir:
        os.makedirs(out_dir, exist_ok=True)
    out, ref = {}, None
    for name, (sdf, prm) in forms.items():
        ao, _, _ = HN.ambient_occlusion(scene, sdf, prm, x, nx, spp, t_ao, 44, 1e-3 * s.diagonal)
        ao = ao.cpu().numpy()
        ao[~seen] = 1.0
        img = np.ones((H, W))
        img[pix_y, pix_x] = ao
        if out_dir:
            _write_png(os.path.join(out_dir, f"ao_{name}.png"), img)
        if ref is None:
            ref = img
        else:
            err = np.abs(img - ref)
            if out_dir:
                _write_png(os.path.join(out_dir, f"ao_err_{name}.png"), 4.0 * err)
            out[name] = {"mean_abs_dAO": float(err.mean()), "share_off_0.1": float((err > 0.1).mean())}
    return {"width": W, "height": H, "spp": spp, "t_ao": t_ao, "errors_vs_triangles": out}


def run_ao_images(args):
    import torch

    import paper_2305_07253_gb300 as rq

    torch.cuda.set_device(0)
    s = S.make_scene("frame")
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).cuda(), torch.from_numpy(s.tris).cuda())
    out = extra_ao_images(rq, scene, s, out_dir=args.out)
    print(json.dumps({"metric": "AO images vs triangles only", "config": {"workload": "frame-ao-images"},
                      "images": sorted(os.listdir(args.out)), "ao_images": out}), flush=True)


def extra_gi_images(rq, scene, s, W=960, H=540, spp=16, albedo=0.7, power=25.0, K=3, out_dir=None):
    """GI images (the image form of the paper's GI experiment, Section 3 "GI &
    Shadow Rays"): per pixel the surface point x the camera sees (primary rays,
    triangles, in every form) and its one-bounce radiance (harness.one_bounce):
    direct light from 4 point lights through shadow rays (two splits, any hit)
    and spp cosine GI rays (one split, closest hit, t_max 30 m) whose hit points
    are lit the same way; constant albedo.  Forms: triangles only, combined
    (m = 2) and field only, on the dense exact grid and on the paper's 5 x 64^3
    cascade.  Errors against triangles only per pixel, on 8 x 8 tile means and
    for the direct light alone, and the time of each form's queries.  With
    out_dir, writes tone-mapped images and 4 x error images as PNG."""
    import torch

    from paper_2305_07253_gb300 import harness as HN
    bias = 1e-3 * s.diagonal
    x, nx, seen = _visible(rq, scene, s, W, H)
    pix_y, pix_x = _pixels(W, H)
    lights = S.free_lights(s)
    V, Fi = s.verts.astype(np.float64), s.tris
    face_n = torch.from_numpy(np.cross(V[Fi[:, 1]] - V[Fi[:, 0]], V[Fi[:, 2]] - V[Fi[:, 0]])).cuda()
    face_n = face_n / face_n.norm(dim=1, keepdim=True).clamp(min=1e-30)
    (dense, sdf_dense), (cg, sdf_c) = _image_fields(rq, scene, s)
    lv_dense = [(dense, tuple(s.lo), tuple(s.hi))]
    lv_c = [(cg[k], *rq.rt_cascade_box(sdf_c, k)) for k in range(5)]
    gi_p = {"triangles": rq.split_params(mode=rq.MODE_BVH),
            "combined": rq.split_params(mode=rq.MODE_SPLIT1, m_near=M_MIDDLE),
            "field": rq.split_params(mode=rq.MODE_SDF)}
    sh_p = {"triangles": rq.split_params(mode=rq.MODE_BVH, any_hit=True),
            "combined": rq.split_params(mode=rq.MODE_SPLIT2, m_near=M_MIDDLE, m_far=M_MIDDLE, any_hit=True),
            "field": rq.split_params(mode=rq.MODE_SDF, any_hit=True)}
    forms = {"triangles": ("triangles", None, None), "combined_dense": ("combined", sdf_dense, lv_dense),
             "field_dense": ("field", sdf_dense, lv_dense), "combined_cascade": ("combined", sdf_c, lv_c),
             "field_cascade": ("field", sdf_c, lv_c)}
    if out_dir:
        os.makedirs(out_dir, exist_ok=True)

    def tiles(a):
        return a[:H // 8 * 8, :W // 8 * 8].reshape(H // 8, 8, W // 8, 8).mean(axis=(1, 3))

    def rel_err(a, b):
        m = b > 0
        r = np.abs(a - b)[m] / b[m]
        return {"mean_rel": float(r.mean()), "share_off_10pct": float((r > 0.1).mean())}

    out, ref, expo = {}, None, None
    for name, (kind, sdf, lv) in forms.items():
        res = HN.one_bounce(scene, sdf, gi_p[kind], sh_p[kind], x, nx, face_n, lv, lights, power, albedo, spp, 45,
                            bias)
        rad = res["radiance"].cpu().numpy()
        rad[~seen] = 0.0
        img = np.zeros((H, W))
        img[pix_y, pix_x] = rad
        dimg = np.zeros((H, W))
        dimg[pix_y, pix_x] = np.where(seen, res["direct"].cpu().numpy(), 0.0)
        if expo is None:
            expo = 1.0 / max(float(np.percentile(rad[seen], 90)), 1e-12)
        tone = 1.0 - np.exp(-expo * img)
        if out_dir:
            _write_png(os.path.join(out_dir, f"gi_{name}.png"), tone)
        r_x, gi, r_y = res["batches"]
        ms = (_time_ms(lambda: rq.rt_trace_combined(scene, sdf, r_x, sh_p[kind]), K) +
              _time_ms(lambda: rq.rt_trace_combined(scene, sdf, gi, gi_p[kind]), K) +
              _time_ms(lambda: rq.rt_trace_combined(scene, sdf, r_y, sh_p[kind]), K))
        entry = {"query_ms": ms, "rays": int(r_x.shape[0] + gi.shape[0] + r_y.shape[0])}
        if ref is None:
            ref, ref_tone, ref_direct = img, tone, dimg
        else:
            err = np.abs(tone - ref_tone)
            if out_dir:
                _write_png(os.path.join(out_dir, f"gi_err_{name}.png"), 4.0 * err)
            entry.update({"mean_abs_d_tone": float(err.mean()), "pixels": rel_err(img, ref),
                          "tiles_8x8": rel_err(tiles(img), tiles(ref)), "direct_only": rel_err(dimg, ref_direct)})
        out[name] = entry
        del res
    return {"width": W, "height": H, "spp": spp, "lights": int(lights.shape[0]), "albedo": albedo, "forms": out}


def run_gi_images(args):
    import torch

    import paper_2305_07253_gb300 as rq

    torch.cuda.set_device(0)
    s = S.make_scene("frame")
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).cuda(), torch.from_numpy(s.tris).cuda())
    out = extra_gi_images(rq, scene, s, K=max(3, args.steps // 40), out_dir=args.out)
    print(json.dumps({"metric": "GI images vs triangles only", "config": {"workload": "frame-gi-images"},
                      "images": sorted(os.listdir(args.out)), "gi_images": out}), flush=True)


def run_dfbuild(args):
    """The paper's field build (voxelisation, jump flooding, sweeps) of the
    combined-mode cascade, 5 x 64^3 with a 0.1 m finest voxel around the camera
    of the frame scene: --warmup untimed builds, then --steps timed ones."""
    import torch

    import paper_2305_07253_gb300 as rq

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    s = S.make_scene("frame")
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).to(dev), torch.from_numpy(s.tris).to(dev))
    g = torch.empty((5, 64, 64, 64), dtype=torch.float32, device=dev)
    sdf = rq.rt_cascade_create(g, 0.1, np.asarray(s.camera.eye, dtype=np.float32))
    ms = _time_ms(lambda: rq.rt_sdf_bake(scene, sdf, rq.BAKE_JFA), max(1, args.steps), warm=max(1, args.warmup))
    print(json.dumps({"metric": "field build time (voxelisation, jump flooding, sweeps)", "value": ms, "unit": "ms",
                      "higher_is_better": False, "config": {"workload": "frame-cascade-5x64-build",
                                                            "n_tris": int(s.n_tris)}}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batching":
        run_batching(args)
    elif args.workload == "fit":
        run_fit(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "ao":
        run_ao(args)
    elif args.workload == "cascade":
        run_cascade(args)
    elif args.workload == "ao-images":
        run_ao_images(args)
    elif args.workload == "gi-images":
        run_gi_images(args)
    elif args.workload == "gather":
        run_gather(args)
    elif args.workload == "dfbuild":
        run_dfbuild(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
