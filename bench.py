#!/usr/bin/env python
"""Rendering benchmark: sphere-traced rays/s and SDF queries/s at 1920x1080,
LOD 5, on the seeded CSG-64 scene (the paper's frame scope: ray/octree
traversal + sphere trace + normals), FP32 and BF16 decode.

One step = one frame: ray/octree traversal -> sphere trace -> normals over
2,073,600 rays already resident in HBM, as the library's frame renderer runs
it (two chunks of rays on two CUDA streams, so one chunk's stages overlap the
other's); the per-stage times come from the same frame run sequentially.
The L2 is flushed (a 256 MB write) between timed steps, outside the timed
events.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --workload batch     # many scenes per frame: per-scene calls vs one
                                         # persistent launch vs its CUDA graph
    python bench.py --workload train     # training steps (Eq. 4, LODs 1-5, 2^19 samples)

Under torchrun every rank renders its own frame (independent replicas, no
collective on the data path); rank 0 prints the whole-job throughput.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sphere-traced rays/s and SDF queries/s at 1080p LOD5, bf16 vs fp32, % roofline"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
CSRC = os.path.join(ROOT, "paper_2101_10994_gb300", "csrc")
KERNEL_SRC = {"k_traverse": ["traverse.cu", "nglod_internal.cuh"],
              "k_trace_f32": ["query.cu", "query_common.cuh", "trace_common.cuh", "nglod_internal.cuh"],
              "k_trace_bf16": ["trace_bf16.cu", "query_common.cuh", "trace_common.cuh", "tcgen05.cuh",
                               "nglod_internal.cuh"],
              "k_trace_warp_bf16": ["trace_bf16.cu", "query_common.cuh", "trace_common.cuh",
                                    "nglod_internal.cuh"]}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    # workload overrides, for profiling smaller cases only (the bench line
    # itself is always the 1920x1080 LOD 5 CSG-64 frame)
    p.add_argument("--width", type=int, default=1920)
    p.add_argument("--height", type=int, default=1080)
    p.add_argument("--decode", choices=["both", "all", "f32", "bf16", "fp8", "f32tc"], default="all")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--features", choices=["levels", "summed"], default="levels",
                   help="frame workload: per-level corner tables (Eq. 2's multi-level gather, the default) "
                        "or the summed corner table of the LOD (one 8-row gather per query)")
    p.add_argument("--workload", choices=["frame", "batch", "train"], default="frame",
                   help="frame: the 1080p LOD5 CSG-64 frame (default); batch: 32 seeded CSG scenes of "
                        "U{8..256} primitives at LOD U{3..6}, images U{128..1024} a side, BF16 decode; "
                        "train: Adam steps of Eq. 4 on the LOD 1-5 CSG-64 octree, 2^19 samples per batch")
    return p.parse_args()


def workload(width, height):
    from paper_2101_10994_gb300 import scenes as S
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    feats = S.readout_features(oc, sc)
    dec = S.readout_decoder(5)
    o, d, pix = S.camera_rays(width, height, tile=8)
    return dict(scene=sc, octree=oc, feats=feats, dec=dec, dec_lo=S.readout_decoder(4), o=o, d=d, lod=5, eps=1e-3,
                far=5.0,
                max_steps=128)


def bf16_available():
    from paper_2101_10994_gb300 import nglod as ng
    return hasattr(ng, "BF16_DECODE") and ng.BF16_DECODE


# ----------------------------------------------------------------------------
# replicas across ranks (torchrun): no collective on the data path, only the
# job's clock -- the slowest rank's time -- and the whole job's units
# ----------------------------------------------------------------------------
def max_over_ranks(value, device=None):
    """The largest value over the ranks of the process group (the value
    itself when no group is initialised)."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return world * units_per_rank / seconds


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def flops_per_query(in_dim, lod, decode):
    """Algorithmic flops of one SDF query: L levels x 8 corners x 32 channels
    of trilinear FMAs, the 128 x in_dim layer and the 128-wide output."""
    interp = 2 * 8 * 32 * lod
    layer1 = 2 * 128 * in_dim
    out = 2 * 128
    return interp, layer1, out


def measure_ceilings(dev, reps=5):
    """Hardware ceilings measured on this GPU with the library's probe kernels
    (include/nglod_probe.h), CUDA events, best of ``reps`` after a warm-up:
    L2 read bandwidth (a 40 MB buffer, well inside the L2, read 20 times with
    L2-only loads), L1 read bandwidth (each of 4 blocks per SM re-reading its
    own 32 KB window with the gathers' 32-byte read-only loads) and FP32 FMA
    throughput (8 independent chains per thread); the SM count from the
    device."""
    import torch

    from paper_2101_10994_gb300 import nglod as ng

    def best(fn):
        fn()
        ts, work = [], 0
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            work = fn()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        return work / min(ts)

    l2buf = torch.ones(40 << 20, dtype=torch.uint8, device=dev)
    sms = ng.device_sms()
    l1buf = torch.ones(sms * 4 * (32 << 10), dtype=torch.uint8, device=dev)
    out = {"sms": sms,
           "l2_read_GBps": best(lambda: ng.probe("l2", l2buf, passes=20)) / 1e9,
           "l1_read_GBps": best(lambda: ng.probe("l1", l1buf, passes=400, window_bytes=32 << 10)) / 1e9,
           "ffma_tflops": best(lambda: ng.probe("ffma", iters=4096)) / 1e12,
           "how": "probe kernels of include/nglod_probe.h, CUDA events, best of 5 after a warm-up: L2 = 40 MB "
                  "read 20x with ld.global.cg; L1 = 32 KB per block (4 blocks/SM) read 400x with "
                  "ld.global.nc.v8; FFMA = 8 chains x 16 x 4096 steps per thread, 8 x 256 threads per SM"}
    del l2buf, l1buf
    return out


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2101_10994_gb300 import nglod as ng
    from paper_2101_10994_gb300.frame import FrameRenderer, autotune_frame
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    W = workload(args.width, args.height)
    R = W["o"].shape[0]
    svo = ng.svo_build(W["octree"].keys)
    feats = ng.Features(W["feats"], "f32")
    dec = ng.DecoderDev.from_decoder(W["dec"])
    o = torch.from_numpy(W["o"]).to(dev)
    d = torch.from_numpy(W["d"]).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    modes = []
    if args.decode in ("both", "all", "f32"):
        modes.append("f32")
    if args.decode in ("both", "all", "bf16") and bf16_available():
        modes.append("bf16")
    summed = getattr(args, "features", "levels") == "summed"
    if summed:
        feats = feats.summed(svo, W["lod"])      # the frames below read the summed table
    if args.decode in ("all", "fp8") and bf16_available():
        modes.append("fp8")
        feats.set_fp8_bound(svo, W["lod"])
    if args.decode in ("all", "f32tc") and bf16_available():
        modes.append("f32tc")        # FP32-accurate decode on the tensor cores (three-term BF16 splits)
    dist = world > 1
    if dist:
        import torch.distributed as td

    def step(mode, out, ev):
        ev[0].record()
        lists = ng.svo_trace_rays(svo, o, d, W["lod"], t_range=False)
        ev[1].record()
        ng.sphere_trace(svo, feats, dec, o, d, lists, eps=W["eps"], far=W["far"], max_steps=W["max_steps"],
                        decode=mode, normals=False, out=out)
        ev[2].record()
        ng.trace_normals(svo, feats, dec, o, d, lists, out)
        ev[3].record()
        return lists

    results = {}
    configs = {}
    clock_info = None
    for mode in modes:
        out = dict(t=torch.empty(R, device=dev), hit=torch.empty(R, dtype=torch.uint8, device=dev),
                   steps=torch.empty(R, dtype=torch.int32, device=dev),
                   normal=torch.empty((R, 3), device=dev),
                   work=torch.empty(ng.lib().sphere_trace_workspace(R), dtype=torch.uint8, device=dev))
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
        wev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for _ in range(args.warmup):
            flush.zero_()
            step(mode, out, wev)
        torch.cuda.synchronize()
        if dist:
            td.barrier()
        torch.cuda.synchronize()
        queries = 0
        sampler = ClockSampler(local_rank)
        with sampler:
            t_wall = time.perf_counter()
            for k in range(args.steps):
                flush.zero_()
                step(mode, out, evs[k])
                queries += int(out["steps"].sum().item())
            torch.cuda.synchronize()
            t_wall = time.perf_counter() - t_wall
        if dist:
            td.barrier()
        torch.cuda.synchronize()
        trav = [e[0].elapsed_time(e[1]) for e in evs]
        trace = [e[1].elapsed_time(e[2]) for e in evs]
        norm = [e[2].elapsed_time(e[3]) for e in evs]
        total = sum(trav) + sum(trace) + sum(norm)           # ms over K steps
        ms_step = max_over_ranks(total, dev) / args.steps
        hits = int(out["hit"].sum().item())
        lists = step(mode, out, wev)
        sizes = lists.level_sizes()
        # the frame as the library's frame renderer runs it: the rays in chunks on as many
        # streams (traversal, trace and normals of one chunk overlap the others'), the chunk
        # count and the trace's CTAs per SM picked by its autotuner (untimed)
        fr, tune = autotune_frame(svo, feats, dec, o, d, W["lod"], eps=W["eps"], far=W["far"],
                                  max_steps=W["max_steps"], decode=mode, normals=True, flush=flush)
        for _ in range(args.warmup):
            flush.zero_()
            fr.frame()
        fr.check()
        fev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        if dist:
            td.barrier()
        torch.cuda.synchronize()
        with sampler:
            for k in range(args.steps):
                flush.zero_()
                fev[k][0].record()
                fr.frame()
                fev[k][1].record()
            torch.cuda.synchronize()
        fr.check()
        if dist:
            td.barrier()
        torch.cuda.synchronize()
        ms_seq = ms_step
        ms_step = max_over_ranks(sum(a.elapsed_time(b) for a, b in fev), dev) / args.steps
        assert torch.equal(fr.out["t"], out["t"]) and torch.equal(fr.out["normal"], out["normal"])
        chunks, ctas, tctas = len(fr.chunks), fr.ctas_per_sm, fr.trav_ctas_per_sm
        configs[mode] = (chunks, ctas, tctas)
        del fr
        results[mode] = dict(level_sizes=sizes, chunks=chunks, trace_ctas_per_sm=ctas, traversal_ctas_per_sm=tctas,
            schedule=f"{chunks} ray chunks on {chunks} streams, trace CTAs/SM {ctas or 'max'}, traversal "
                     f"CTAs/SM {tctas or 'max'} (autotuned)",
            autotune_ms_by_chunks_and_ctas=tune,
            ms_sequential=ms_seq, rays_per_s_sequential=job_rate(R, world, ms_seq * 1e-3),
            ms_per_step=ms_step, rays_per_s=job_rate(R, world, ms_step * 1e-3),
            queries_per_s=world * queries / args.steps / (sum(trace) / args.steps * 1e-3),
            ms_traverse=sum(trav) / args.steps, ms_trace=sum(trace) / args.steps,
            ms_normals=sum(norm) / args.steps, queries_per_frame=queries // args.steps,
            hit_pixels=hits, wall_s=t_wall)
        if clock_info is None or mode == "bf16":
            clock_info = sampler.summary()

    # ---- the traversal as the frame renderer runs it: staged lists (one launch, no tile scan or
    # placement), whole frame, CUDA events; decode-independent, so measured once ----
    if modes:
        Lc = ng.svo_trace_rays(svo, o, d, W["lod"], t_range=False)
        cap_st = int(Lc.voxel_id.numel() * 1.25) + 4096
        del Lc
        twork = torch.empty(ng.lib().svo_trace_rays_workspace(R, cap_st), dtype=torch.uint8, device=dev)
        tst = []
        for k in range(args.warmup + args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ng.svo_trace_rays_staged(svo, o, d, W["lod"], twork, cap_st)
            e1.record()
            torch.cuda.synchronize()
            if k >= args.warmup:
                tst.append(e0.elapsed_time(e1))
        ng._check(ng.lib().svo_trace_rays_check(twork.data_ptr(), W["lod"], None, None))
        results["traversal_staged"] = dict(
            ms_per_frame=max_over_ranks(sum(tst), dev) / args.steps, launches_per_frame=1,
            note="svo_trace_rays_staged_async: the frame renderer's traversal (each ray's entries left "
                 "where the traversal staged them)")
        del twork

    # ---- continuous LOD (Eq. 3): the same frame at L~ = lod - 0.5, BF16, frame renderer ----
    if "bf16" in modes and W["lod"] >= 2 and not summed:
        lt = W["lod"] - 0.5
        dlo = ng.DecoderDev.from_decoder(W["dec_lo"])
        fr, btune = autotune_frame(svo, feats, dlo, o, d, lt, eps=W["eps"], far=W["far"], max_steps=W["max_steps"],
                                   decode="bf16", normals=True, dec_hi=dec, flush=flush)
        bl = []
        for k in range(args.warmup + args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fr.frame()
            e1.record()
            e1.synchronize()
            if k >= args.warmup:
                bl.append(e0.elapsed_time(e1))
        fr.check()
        ms = max_over_ranks(statistics.mean(bl), dev)
        bch = len(fr.chunks)
        results["bf16_blend"] = dict(lod_tilde=lt, chunks=bch, trace_ctas_per_sm=fr.ctas_per_sm,
                                     traversal_ctas_per_sm=fr.trav_ctas_per_sm,
                                     schedule=f"{bch} ray chunks on {bch} streams, trace CTAs/SM "
                                              f"{fr.ctas_per_sm or 'max'} (autotuned)",
                                     autotune_ms_by_chunks_and_ctas=btune,
                                     ms_per_step=ms, rays_per_s=job_rate(R, world, ms * 1e-3),
                                     queries_per_frame=int(fr.out["steps"].sum().item()),
                                     hit_pixels=int(fr.out["hit"].sum().item()))
        del fr

    # ---- standalone sdf_query: 2^22 points uniform inside the target-level voxels ----
    from paper_2101_10994_gb300 import scenes as S
    xq = torch.from_numpy(S.points_in_voxels(W["octree"], W["lod"] + S.FIRST_FEATURE_DEPTH - 1, 1 << 22, 21)).to(dev)
    for qm in [m for m in ("f32", "bf16") if m in modes and not summed]:
        ql = []
        for k in range(args.warmup + args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ng.sdf_query(svo, feats, dec, xq, W["lod"], decode=qm)
            e1.record()
            e1.synchronize()
            if k >= args.warmup:
                ql.append(e0.elapsed_time(e1))
        ms = max_over_ranks(statistics.mean(ql), dev)
        results[f"sdf_query_{qm}"] = dict(points=int(xq.shape[0]), ms_per_call=ms,
                                          queries_per_s=world * xq.shape[0] / (ms * 1e-3))
    del xq

    # ---- the BF16 frame with FP16 corner features (half the gathered bytes) ----
    if "bf16" in modes and not summed:
        f16 = ng.Features(W["feats"], "f16")
        fr = FrameRenderer(svo, f16, dec, o, d, W["lod"], chunks=configs["bf16"][0], ctas_per_sm=configs["bf16"][1],
                           trav_ctas_per_sm=configs["bf16"][2], eps=W["eps"], far=W["far"],
                           max_steps=W["max_steps"], decode="bf16", normals=True)
        hl = []
        for k in range(args.warmup + args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fr.frame()
            e1.record()
            e1.synchronize()
            if k >= args.warmup:
                hl.append(e0.elapsed_time(e1))
        fr.check()
        ms = max_over_ranks(statistics.mean(hl), dev)
        results["bf16_f16features"] = dict(schedule="the BF16 frame's", chunks=configs["bf16"][0], ms_per_step=ms,
                                           rays_per_s=job_rate(R, world, ms * 1e-3),
                                           queries_per_frame=int(fr.out["steps"].sum().item()),
                                           hit_pixels=int(fr.out["hit"].sum().item()))
        del fr, f16

    # ---- the frames reading the summed corner table of the LOD (nglod_sum_features: z at
    # every corner of the LOD, so a query gathers 8 rows instead of 8 per level; built once per
    # feature set, its build timed apart).  Same rays, lists and decoders; the stage times come
    # from the sequential frame, the frame time from the autotuned renderer ----
    for sm_mode in [m for m in ("bf16", "f32") if m in modes and not summed]:
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        b0.record()
        fs = feats.summed(svo, W["lod"])
        b1.record()
        b1.synchronize()
        ms_build = b0.elapsed_time(b1)
        sout = dict(t=torch.empty(R, device=dev), hit=torch.empty(R, dtype=torch.uint8, device=dev),
                    steps=torch.empty(R, dtype=torch.int32, device=dev), normal=torch.empty((R, 3), device=dev),
                    work=torch.empty(ng.lib().sphere_trace_workspace(R), dtype=torch.uint8, device=dev))
        st_ms = []
        for k in range(args.warmup + args.steps):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record()
            lists = ng.svo_trace_rays(svo, o, d, W["lod"], t_range=False)
            ev[1].record()
            ng.sphere_trace(svo, fs, dec, o, d, lists, eps=W["eps"], far=W["far"], max_steps=W["max_steps"],
                            decode=sm_mode, normals=False, out=sout)
            ev[2].record()
            ng.trace_normals(svo, fs, dec, o, d, lists, sout)
            ev[3].record()
            ev[3].synchronize()
            if k >= args.warmup:
                st_ms.append([ev[i].elapsed_time(ev[i + 1]) for i in range(3)])
        ng.sphere_trace_status(sout)
        st_ms = [statistics.mean(v[i] for v in st_ms) for i in range(3)]
        fr, stune = autotune_frame(svo, fs, dec, o, d, W["lod"], eps=W["eps"], far=W["far"],
                                   max_steps=W["max_steps"], decode=sm_mode, normals=True, flush=flush)
        sl = []
        for k in range(args.warmup + args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fr.frame()
            e1.record()
            e1.synchronize()
            if k >= args.warmup:
                sl.append(e0.elapsed_time(e1))
        fr.check()
        assert torch.equal(fr.out["t"], sout["t"]) and torch.equal(fr.out["normal"], sout["normal"])
        ms = max_over_ranks(statistics.mean(sl), dev)
        sch = len(fr.chunks)
        q = int(sout["steps"].sum().item())
        results[f"{sm_mode}_summed"] = dict(
            chunks=sch, trace_ctas_per_sm=fr.ctas_per_sm, traversal_ctas_per_sm=fr.trav_ctas_per_sm,
            autotune_ms_by_chunks_and_ctas=stune,
            schedule=f"{sch} ray chunks on {sch} streams, trace CTAs/SM {fr.ctas_per_sm or 'max'} (autotuned)",
            ms_per_step=ms, rays_per_s=job_rate(R, world, ms * 1e-3),
            ms_traverse=float(st_ms[0]), ms_trace=float(st_ms[1]), ms_normals=float(st_ms[2]),
            ms_sequential=float(sum(st_ms)), queries_per_frame=q,
            queries_per_s=world * q / (float(st_ms[1]) * 1e-3),
            hit_pixels=int(sout["hit"].sum().item()),
            table_build_ms=ms_build, table_bytes=int(fs.tables[-1].numel() * 4),
            note="the summed table replaces the multi-level gather of Eq. 2 by the trilinear "
                 "interpolation of z's own corner values (the same function inside every voxel of the LOD)")
        del fr, fs, sout

    # ---- end to end through the public API with pinned host buffers: each chunk's
    # rays copied in and its t / hit / normals copied out on the chunk's stream ----
    mode = "bf16" if "bf16" in modes else modes[0]
    h_o = torch.from_numpy(W["o"]).pin_memory()
    h_d = torch.from_numpy(W["d"]).pin_memory()
    h_out = {"t": torch.empty(R, dtype=torch.float32).pin_memory(),
             "hit": torch.empty(R, dtype=torch.uint8).pin_memory(),
             "normal": torch.empty((R, 3), dtype=torch.float32).pin_memory()}
    # the renderer sizes its lists from the rays it is built on; every timed frame then
    # brings its rays in from the host buffers (the device copies are cleared first).
    # The schedule is tuned with the copies in (untimed): the one that hides them best
    # can differ from the device-only frame's
    fr, etune = autotune_frame(svo, feats, dec, o.clone(), d.clone(), W["lod"], host=((h_o, h_d), h_out),
                               eps=W["eps"], far=W["far"], max_steps=W["max_steps"], decode=mode, normals=True,
                               flush=flush)
    ech, ecta, etcta = len(fr.chunks), fr.ctas_per_sm, fr.trav_ctas_per_sm
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        fr.o.zero_()
        fr.d.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fr.frame(h_in=(h_o, h_d), h_out=h_out)
        e1.record()
        e1.synchronize()
        if k >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    fr.check()
    assert torch.equal(h_out["t"], fr.out["t"].cpu())
    e2e_ms_job = max_over_ranks(statistics.mean(e2e_ms), dev)
    e2e = dict(value=job_rate(R, world, e2e_ms_job * 1e-3), unit="rays/s",
               h2d_bytes_per_step=int(h_o.numel() * 4 + h_d.numel() * 4),
               d2h_bytes_per_step=int(sum(v.numel() * v.element_size() for v in h_out.values())),
               schedule=f"{ech} chunks on {ech} streams, trace CTAs/SM {ecta or 'max'}, traversal CTAs/SM "
                        f"{etcta or 'max'}, copies overlapped with the other chunks' work (autotuned with the copies)",
               autotune_ms_by_chunks_and_ctas=etune)
    svo.free()
    ceilings = measure_ceilings(dev)
    return W, results, clock_info, e2e, modes, ceilings


def source_hash(kernel):
    """Hash of the code a kernel is built from, comments left out (traffic
    taken from other code is dropped; a comment edit keeps it)."""
    h = hashlib.sha256()
    for f in KERNEL_SRC[kernel]:
        p = os.path.join(CSRC, f)
        if os.path.exists(p):
            code = re.sub(r"/\*.*?\*/", "", open(p).read(), flags=re.S)
            code = re.sub(r"//[^\n]*", "", code)
            h.update("\n".join(line.rstrip() for line in code.splitlines() if line.strip()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, tag=""):
    """The stored DRAM bytes per launch of ``kernel`` on the workload ``tag``
    ("" = the default frame, "@summed" = the summed-table frame)."""
    if os.path.exists(PROFILE_TRAFFIC):
        ent = json.load(open(PROFILE_TRAFFIC)).get(kernel + tag)
        if ent and ent.get("source_hash") == source_hash(kernel):
            return ent.get("dram_bytes_per_launch")
    return None


def traversal_bytes(W, sizes):
    """Algorithmic bytes of one frame's traversal as this design runs it
    (tiles of rays swept level by level on chip; the frame asks for no t
    ranges, which the tracers recompute): every ray read once (24 B) with
    its count written and read back and its CSR offset written (3 x 4 B);
    one node record (16 B) per ray/voxel pair Decide visits at depths
    0..D-1; every final entry (voxel id, 4 B) staged, read back and written
    to its final position (3 x 4 B)."""
    R = sizes[0]
    D = len(sizes) - 1
    H = sizes[D]
    visits = sum(sizes[:D])
    return 36 * R + 16 * visits + 12 * H


def cpu_model():
    """The host CPU's model name (Linux /proc/cpuinfo), for the CPU baseline."""
    try:
        for line in open("/proc/cpuinfo"):
            k, _, v = line.partition(":")
            if k.strip().lower() in ("model name", "cpu model", "hardware"):
                return v.strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def traversal_roofline(W, res, mode, peaks, staged=None):
    """The traversal (k_traverse + tile scan + placement, 3 launches) against
    HBM; it is issue-bound on the slab tests, so this fraction is low.
    staged: the renderer's one-launch form (staged lists), timed beside it."""
    hbm = peaks.get("hbm_gbs", 6800.0)
    nbytes = traversal_bytes(W, res["level_sizes"])
    sec = res["ms_traverse"] * 1e-3
    achieved = nbytes / sec / 1e9
    # the lower bound of any design: rays in, the final CSR lists (voxel ids) out
    sizes = res["level_sizes"]
    lower = 24 * sizes[0] + 4 * (sizes[0] + 1) + 4 * sizes[-1]
    traffic = profiled_traffic("k_traverse")
    return {"bound": "hbm", "kernel": "k_traverse", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic,
            "dram_frac": (traffic / sec / 1e9 / hbm) if traffic else None,
            "bytes_per_frame": nbytes, "launches_per_frame": 3,
            "ms_staged_lists": staged["ms_per_frame"] if staged else None,
            "lower_bound_bytes": lower, "lower_bound_frac": lower / sec / 1e9 / hbm,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback",
            "timing": "CUDA events around svo_trace_rays (3 launches + the H read-back)",
            "note": "issue-bound on the 8-child slab tests (ncu: ~71 % issue active, ALU pipe ~66 %); node records hit L1/L2"}


def trace_roofline(W, res, mode, peaks, levels=None, ceilings=None):
    """Dominant kernel = the sphere tracer (largest share of the frame in the
    launch list): its decode contraction against the tensor pipe (BF16) or
    its FP32 arithmetic against the CUDA cores (the measured FFMA ceiling);
    its feature gathers against the measured L1 and L2 read bandwidth."""
    ceilings = ceilings or {}
    levels = W["lod"] if levels is None else levels      # levels gathered per query (1: summed table)
    interp, layer1, outl = flops_per_query(W["dec"].in_dim, levels, mode)
    q = res["queries_per_frame"]
    sec = res["ms_trace"] * 1e-3
    # BF16 and three-term FP32: warp-level MMAs (k_trace_warp_bf16); FP8: tcgen05 (k_trace_bf16)
    kern = {"f32": "k_trace_f32", "fp8": "k_trace_bf16"}.get(mode, "k_trace_warp_bf16")
    if mode != "f32":
        tf = peaks.get("bf16_tflops", 1900.0)
        achieved = q * layer1 / sec / 1e12
        return {"bound": "tensor", "kernel": kern, "achieved": achieved, "peak": tf, "unit": "TFLOP/s",
                "frac": achieved / tf, "traffic": profiled_traffic(kern, "@summed" if levels == 1 else ""),
                "flops_per_query": layer1, "queries_per_launch": q,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops burst (of measured)",
                "note": "the kernel is bound by feature-gather latency (L1/L2), not by the 128x32 contraction"
                        + (" (decoded per warp with mma.sync m16n8k16, no CTA-wide tile)" if mode != "fp8" else ""),
                **gather_fracs(q, levels, sec, ceilings)}
    if "ffma_tflops" in ceilings:
        peak, src = ceilings["ffma_tflops"], "measured FFMA probe (of measured)"
    else:
        sms = ceilings.get("sms", 152)
        peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        src = f"{sms} SMs x 128 FP32 lanes x 2 flop x sm_max_mhz (nominal)"
    achieved = q * (interp + layer1 + outl) / sec / 1e12
    return {"bound": "alu", "kernel": kern, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": profiled_traffic(kern), "flops_per_query": interp + layer1 + outl,
            "queries_per_launch": q, "peak_source": src, **gather_fracs(q, levels, sec, ceilings)}


def gather_fracs(q, levels, sec, ceilings):
    """The gathers' requested bytes (8 corner rows of 32 FP32 channels per
    level per query) per second, as a fraction of the measured L1 and L2 read
    bandwidth (every request passes L1; what misses it is served by L2)."""
    gbps = q * 8 * 32 * 4 * levels / sec / 1e9
    out = {"gather_bytes_per_query": 8 * 32 * 4 * levels, "gather_GBps": gbps}
    if "l1_read_GBps" in ceilings:
        out["gather_frac_of_l1"] = gbps / ceilings["l1_read_GBps"]
        out["gather_frac_of_l2"] = gbps / ceilings["l2_read_GBps"]
    return out


# ----------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ----------------------------------------------------------------------------
def oracle_rate(W, budget_s, seed=0):
    """Oracle rays/s on a uniform random sample of the frame's rays sized to
    roughly ``budget_s`` seconds of CPU work (all host cores via OpenMP)."""
    import numpy as np

    from oracle.oracle import OracleSVO
    ora = OracleSVO(W["octree"].keys)
    R = W["o"].shape[0]
    rng = np.random.default_rng(seed)
    perm = rng.permutation(R)
    n = 256
    t = time.perf_counter()
    ora.sphere_trace(W["feats"], W["dec"], W["o"][perm[:n]], W["d"][perm[:n]], W["lod"], eps=W["eps"],
                     far=W["far"], max_steps=W["max_steps"])
    dt = time.perf_counter() - t
    n2 = int(min(R - n, max(256, n * (budget_s / max(dt, 1e-3)))))
    sel = perm[n:n + n2]
    t = time.perf_counter()
    ora.sphere_trace(W["feats"], W["dec"], W["o"][sel], W["d"][sel], W["lod"], eps=W["eps"], far=W["far"],
                     max_steps=W["max_steps"])
    dt = time.perf_counter() - t
    return n2 / dt, n2, dt


def run_reference(args):
    W = workload(args.width, args.height)
    R = W["o"].shape[0]
    from oracle import oracle
    oracle.build()
    cores = os.cpu_count()
    budget = max(1.0, min(20.0, 100.0 / max(1, args.steps + args.warmup)))
    rates, ns, dts = [], [], []
    for k in range(args.warmup + args.steps):
        rate, n, dt = oracle_rate(W, budget, seed=k)
        if k >= args.warmup:
            rates.append(rate)
            ns.append(n)
            dts.append(dt)
    v = statistics.mean(rates)
    # a step is the sampled rays of the frame: ms_per_step is the time those
    # took; the time the whole frame would take at that rate is separate
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "rays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(dts) * 1e3,
            "sample_rays_per_step": statistics.mean(ns), "sample_s_per_step": statistics.mean(dts),
            "projected_ms_per_frame": R / v * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "csg64_seed0_lod5_1920x1080", "lod": 5, "rays": R, "max_steps": 128,
                       "eps": 1e-3, "features": "f32 m=32, per-level tables (promoted to f64)",
                       "decoder": "32->128->1 readout-embedded", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "rays/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                             "sample": f"per step a uniform random sample of the 1920x1080 frame's rays "
                                       f"(~{budget:.0f} s of CPU work), FP64 oracle: brute-force traversal + "
                                       f"sphere trace + normals"},
            "e2e": {"value": v, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------------------
# batching: many scenes and images of uneven size per frame
# ----------------------------------------------------------------------------
def run_batch(args):
    from paper_2101_10994_gb300 import scenes as S
    items = S.batching_workload(32, seed=0, workers=min(16, os.cpu_count() or 1))
    import torch

    from paper_2101_10994_gb300 import batch as B
    from paper_2101_10994_gb300 import nglod as ng
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    decs = {}
    jobs = []
    for sc, oc, lod, w, h, feats in items:
        if lod not in decs:
            decs[lod] = ng.DecoderDev.from_decoder(S.readout_decoder(lod))
        o, d, _ = S.camera_rays(w, h, tile=8)
        svo = ng.svo_build(oc.keys)
        F = ng.Features(feats, "f32")
        if args.features == "summed":
            F = F.summed(svo, lod)       # each scene reads the summed corner table of its LOD
        jobs.append(B.Job(svo, F, decs[lod], lod, torch.from_numpy(o).to(dev), torch.from_numpy(d).to(dev)))
    R = sum(j.R for j in jobs)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn, n):
        ts = []
        for _ in range(n):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    def per_scene():
        B.per_scene_frame(jobs, decode="bf16")

    rnd = B.BatchRenderer(jobs, decode="bf16")
    best, tune = B.autotune(rnd, streams=[0, 2, 4, 8], reps=3)
    rnd.frame()
    rnd.check()
    rnd.capture()
    for _ in range(args.warmup):
        per_scene()
        rnd.frame()
        rnd.replay()
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    with sampler:
        ms_scene = timed(per_scene, args.steps)
        ms_batch = timed(rnd.frame, args.steps)
        ms_graph = timed(rnd.replay, args.steps)
    rnd.check()
    hits = sum(int(rnd.outputs(k)["hit"].sum().item()) for k in range(len(jobs)))
    line = {
        "metric": "batched sphere-traced rays/s (traversal + trace + normals), 32 scenes per frame",
        "value": R / (ms_graph * 1e-3), "unit": "rays/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "batch32_csg_u8-256_lod_u3-6_side_u128-1024_seed0", "rays": R,
                   "scenes": len(jobs), "decoder_groups": len(decs), "max_steps": 128, "eps": 1e-3,
                   "features": ("summed corner table of each scene's LOD, f32 m=32" if args.features == "summed"
                                else "f32 m=32, per-level tables"),
                   "l2": "flushed between steps (256 MB write)", "parallelism": "single GPU"},
        "schedules_ms": {"per_scene_calls": ms_scene, "persistent_launch": ms_batch, "graph_replay": ms_graph},
        "speedup_vs_per_scene": ms_scene / ms_graph,
        "autotune": {"best_ctas_per_sm": best[0], "best_traversal_streams": best[1],
                     "ms_by_ctas_per_sm_and_streams": tune},
        "hit_pixels": hits,
        "clocks": sampler.summary(),
        # per graph replay: the reset, the chunk order (keys, bucket scan, scatter) and the
        # persistent trace kernel; per job its staged traversal (1), its hit list in ray order
        # (counts, scan, placement: 3) and its normals (masked-sum operand, gradient: 2)
        "gpu_launches": args.steps * (5 + 6 * len(jobs)),
    }
    print(json.dumps(line))


# ----------------------------------------------------------------------------
# training: one Adam step of Eq. 4 over all LODs
# ----------------------------------------------------------------------------
def run_train(args):
    """One step = the fused prediction + residual + adjoint kernel per LOD
    (LODs 1..5 summed, Eq. 4) over a batch of 2^19 SDF samples (half near the
    surface, half uniform) and the Adam kernel over every parameter tensor;
    the adjoint's decoder contractions in FP32 on the CUDA cores, and (the
    reported value) in BF16 on the tensor cores."""
    from paper_2101_10994_gb300 import scenes as S
    import torch

    from paper_2101_10994_gb300 import nglod as ng
    from paper_2101_10994_gb300.train import Trainer
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    n = 1 << 19
    x_h, t_h = S.training_batch(sc, n, 17)
    x_p, t_p = torch.from_numpy(x_h).pin_memory(), torch.from_numpy(t_h).pin_memory()
    x, t = x_p.to(dev), t_p.to(dev)
    svo = ng.svo_build(oc.keys)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn, k):
        ts, out = [], None
        for _ in range(k):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), out

    loss_h = torch.empty(5, dtype=torch.float32).pin_memory()
    res = {}
    sampler = ClockSampler(0)
    for mma in ("f32", "bf16"):
        tr = Trainer(svo, S.init_features(oc, seed=0, sigma=0.01), [S.init_decoder(l, 32) for l in range(1, 6)],
                     mma=mma)
        first = tr.step(x, t).cpu().numpy()
        for _ in range(args.warmup):
            tr.step(x, t)
        torch.cuda.synchronize()

        def e2e_step():
            x.copy_(x_p, non_blocking=True)
            t.copy_(t_p, non_blocking=True)
            loss = tr.step(x, t)
            loss_h.copy_(loss, non_blocking=True)
            return loss

        with sampler:
            ms, last = timed(lambda: tr.step(x, t), args.steps)
            ms_e2e, _ = timed(e2e_step, args.steps)
        res[mma] = {"ms_per_step": ms, "samples_per_s": n / (ms * 1e-3), "e2e_samples_per_s": n / (ms_e2e * 1e-3),
                    "loss_first_step": [float(v) for v in first],
                    "loss_after": [float(v) for v in last.cpu().numpy()], "steps_taken": 2 + args.warmup + 2 * args.steps}
    nparam = len(tr.params)
    head = "bf16"
    ms = res[head]["ms_per_step"]
    line = {
        "metric": "SDF training samples/s (Eq. 4 over LODs 1-5: fused prediction + adjoint + Adam)",
        "value": n / (ms * 1e-3), "unit": "samples/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": head,
        "data": "synthetic",
        "config": {"workload": "train_csg64_seed0_lod1-5_2^19_samples", "samples": n, "lods": [1, 2, 3, 4, 5],
                   "features": "f32 m=32", "decoder": "32->128->1", "optimizer": "Adam lr 1e-3",
                   "adjoint": "bf16 tensor-core contractions, fp32 accumulation (fp32 CUDA-core adjoint in modes)",
                   "l2": "flushed between steps (256 MB write)", "parallelism": "single GPU"},
        "modes": res,
        "clocks": sampler.summary(),
        "e2e": {"value": res[head]["e2e_samples_per_s"], "unit": "samples/s", "h2d_bytes_per_step": int(n * 16),
                "d2h_bytes_per_step": 20},
        # per step: the point sort by cell (keys, three scan kernels, scatter: 5), one fused
        # adjoint kernel per LOD (5), one Adam kernel per parameter tensor
        "gpu_launches": args.steps * (5 + 5 + nparam),
    }
    print(json.dumps(line))


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    if args.workload == "batch":
        if rank == 0:
            run_batch(args)
        return
    if args.workload == "train":
        if rank == 0:
            run_train(args)
        return
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(local_rank)
        td.init_process_group("nccl")
    W, res, clocks, e2e, modes, ceilings = run_ours(args, rank, world, local_rank)
    if rank == 0:
        peaks = {}
        pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(pp):
            peaks = json.load(open(pp))
        head = "bf16" if "bf16" in res else list(res)[0]
        r = res[head]
        line = {
            "metric": METRIC, "value": r["rays_per_s"], "unit": "rays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": head,
            "data": "synthetic",
            "config": {"workload": f"csg64_seed0_lod5_{args.width}x{args.height}", "lod": 5,
                       "rays": int(W["o"].shape[0]), "max_steps": W["max_steps"], "eps": W["eps"],
                       "features": ("summed corner table of LOD 5, f32 m=32" if args.features == "summed"
                                    else "f32 m=32, per-level tables"),
                       "decoder": "32->128->1 readout-embedded",
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
            "queries_per_s": r["queries_per_s"],
            "modes": res,
            "roofline": trace_roofline(W, r, head, peaks, 1 if args.features == "summed" else None, ceilings),
            "traversal_roofline": traversal_roofline(W, r, head, peaks, res.get("traversal_staged")),
            "fp32_roofline": (trace_roofline(W, res["f32"], "f32", peaks, 1 if args.features == "summed" else None,
                                             ceilings) if "f32" in res else None),
            "ceilings": ceilings,
            "clocks": clocks,
            "e2e": e2e,
            # the library's kernels per timed frame: the sequential frame runs the CSR traversal
            # (tiles, tile scan, placement: 3), the ray-group order (keys, bucket scan, scatter: 3),
            # the tracer (1), the hit list in ray order (counts, scan, placement: 3) and the normals
            # (masked-sum operand, gradient: 2) = 12; each chunk of the renderer's frame the same
            # with the staged traversal (1) = 10; a blended chunk two operand builds and gradient
            # passes and the normalisation (13); the FP16-feature frame the renderer's frame once
            # more; each standalone sdf_query and the staged traversal one launch; each summed
            # table's timed build one
            "gpu_launches": args.steps * (sum(12 + 10 * res[m]["chunks"] for m in modes)
                                          + 13 * res.get("bf16_blend", {}).get("chunks", 0)
                                          + 10 * res.get("bf16_f16features", {}).get("chunks", 0)
                                          + sum(12 + 10 * res[k]["chunks"] for k in res if k.endswith("_summed"))
                                          + sum(k.startswith("sdf_query_") for k in res)
                                          + ("traversal_staged" in res))
                            + sum(k.endswith("_summed") for k in res),
        }
        if "bf16" in res and "f32" in res:
            line["bf16_speedup"] = res["f32"]["ms_per_step"] / res["bf16"]["ms_per_step"]
        if not args.no_cpu_baseline and world == 1:
            from oracle import oracle
            oracle.build()
            v, n, dt = oracle_rate(W, 15.0)
            line["cpu_baseline"] = {"value": v, "unit": "rays/s", "cores": os.cpu_count(), "kind": "oracle",
                                    "cpu": cpu_model(),
                                    "sample": f"{n} rays drawn uniformly from the frame, {dt:.1f} s, FP64 "
                                              f"brute-force traversal + sphere trace + normals"}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as td
        td.destroy_process_group()


if __name__ == "__main__":
    main()
