"""Batched rendering: many scenes and images of uneven size per frame.

Each job is one image of one scene at one LOD.  A frame enqueues every job's
traversal (svo_trace_rays_staged_async: one launch, each ray's list read
where the traversal staged it) and one persistent sphere-trace launch over
all jobs (sphere_trace_batch_run), with no host synchronisation, so the
whole frame is captured once in a CUDA graph and replayed.  The trace
kernel's residency (CTAs per SM) is chosen by a small autotuner that times
each candidate on the actual batch.
"""
from __future__ import annotations

import ctypes as C
import statistics

from . import nglod as ng


class Job:
    """One image: octree, features, the decoder of its LOD, and its rays."""

    def __init__(self, svo: ng.SVO, feats: ng.Features, dec: ng.DecoderDev, lod: int, o, d):
        self.svo, self.feats, self.dec, self.lod = svo, feats, dec, int(lod)
        self.o, self.d = o.contiguous(), d.contiguous()
        self.R = int(o.shape[0])


class BatchRenderer:
    def __init__(self, jobs, eps=1e-3, far=5.0, max_steps=128, decode="bf16", normals=True, ctas_per_sm=0,
                 headroom=1.25, stream=None, traversal_streams=4):
        import torch
        self.torch = torch
        self.jobs = jobs
        # the jobs' traversals are independent: they run on a few side streams
        # (forked from and joined back into the frame's stream, also under graph capture)
        self.stream_pool = [torch.cuda.Stream(device=jobs[0].o.device) for _ in range(max(0, traversal_streams))]
        self.tstreams = list(self.stream_pool)
        # the batched trace leaves the normals to frame(), which spreads the jobs'
        # normal kernels over the side streams
        self.normals = bool(normals)
        self.params = ng._TraceParams(eps, far, max_steps, 0, {"f32": ng.F32, "bf16": ng.BF16, "fp8": ng.FP8}[decode],
                                      0)
        self.decode = decode
        L = ng.lib()
        dev = jobs[0].o.device
        # sizing pass: one synchronous traversal per job fixes the list capacities
        self.bufs = []
        for j in jobs:
            lists = ng.svo_trace_rays(j.svo, j.o, j.d, j.lod, t_range=False)
            cap = max(int(lists.max_pairs * headroom) + 1024, j.R + 1024)
            tw = L.svo_trace_rays_workspace(j.R, cap)
            b = dict(cap=cap,
                     twork=torch.empty(tw, dtype=torch.uint8, device=dev),
                     ptrs=[C.c_void_p() for _ in range(3)],
                     swork=torch.empty(L.sphere_trace_workspace(j.R), dtype=torch.uint8, device=dev),
                     t=torch.empty(j.R, dtype=torch.float32, device=dev),
                     hit=torch.empty(j.R, dtype=torch.uint8, device=dev),
                     steps=torch.empty(j.R, dtype=torch.int32, device=dev),
                     normal=torch.empty((j.R, 3), dtype=torch.float32, device=dev) if normals else None)
            # the staged lists (views into twork, the same every frame): each
            # job's tracer reads a ray's entries where its traversal left them
            b["lists"] = ng.svo_trace_rays_staged(j.svo, j.o, j.d, j.lod, b["twork"], cap)
            self.bufs.append(b)
        self.ctas_per_sm = ctas_per_sm
        self.handle = None
        self._create(stream)
        self.graph = None

    def _create(self, stream=None):
        if self.handle:
            ng.lib().sphere_trace_batch_free(self.handle)
            self.handle = None
        arr = (ng._TraceJob * len(self.jobs))()
        for k, (j, b) in enumerate(zip(self.jobs, self.bufs)):
            arr[k].svo = j.svo.h.value
            arr[k].feats = j.feats.c()
            arr[k].dec = j.dec.c()
            arr[k].lod = j.lod
            arr[k].o, arr[k].d, arr[k].R = j.o.data_ptr(), j.d.data_ptr(), j.R
            # staged lists, no t ranges: the tracers recompute each entry's interval
            lists = b["lists"]
            arr[k].ray_offsets, arr[k].voxel_id, arr[k].t_range = (lists.ray_offsets.data_ptr(),
                                                                   lists.voxel_id.data_ptr(), None)
            arr[k].ray_counts = lists.ray_counts.data_ptr()
            arr[k].work, arr[k].work_bytes = b["swork"].data_ptr(), b["swork"].numel()
            arr[k].t_hit, arr[k].hit, arr[k].steps = b["t"].data_ptr(), b["hit"].data_ptr(), b["steps"].data_ptr()
            arr[k].normal = ng._ptr(b["normal"])
        h = C.c_void_p()
        ng._check(ng.lib().sphere_trace_batch_create(arr, len(self.jobs), C.byref(self.params), int(self.ctas_per_sm),
                                                     C.c_void_p(ng._stream(stream)), C.byref(h)))
        self.handle = h

    def free(self):
        if self.handle:
            ng.lib().sphere_trace_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def frame(self, stream=None):
        """Enqueues one frame: every job's traversal (spread over the
        traversal streams), then the batched trace on the frame's stream."""
        torch = self.torch
        L = ng.lib()
        main = stream if stream is not None else torch.cuda.current_stream()
        s = C.c_void_p(main.cuda_stream)
        if self.tstreams:
            start = torch.cuda.Event()
            start.record(main)
            for st in self.tstreams:
                st.wait_event(start)
        for i, (j, b) in enumerate(zip(self.jobs, self.bufs)):
            st = self.tstreams[i % len(self.tstreams)] if self.tstreams else main
            p = b["ptrs"]
            ng._check(L.svo_trace_rays_staged_async(j.svo.h, j.o.data_ptr(), j.d.data_ptr(), j.R, j.lod,
                                                    b["twork"].data_ptr(), b["twork"].numel(), b["cap"], 0,
                                                    C.byref(p[0]), C.byref(p[1]), C.byref(p[2]),
                                                    C.c_void_p(st.cuda_stream)))
        for st in self.tstreams:
            main.wait_stream(st)
        ng._check(L.sphere_trace_batch_run(self.handle, s))
        if self.normals:
            if self.tstreams:
                traced = torch.cuda.Event()
                traced.record(main)
                for st in self.tstreams:
                    st.wait_event(traced)
            for i, (j, b) in enumerate(zip(self.jobs, self.bufs)):
                st = self.tstreams[i % len(self.tstreams)] if self.tstreams else main
                fc, dc = j.feats.c(), j.dec.c()
                ng._check(L.trace_normals(j.svo.h, C.byref(fc), C.byref(dc), j.o.data_ptr(), j.d.data_ptr(), j.R,
                                          j.lod, b["swork"].data_ptr(), b["swork"].numel(), b["t"].data_ptr(),
                                          b["hit"].data_ptr(), b["normal"].data_ptr(), C.c_void_p(st.cuda_stream)))
            for st in self.tstreams:
                main.wait_stream(st)

    def check(self, stream=None):
        """Synchronises; raises if a traversal overflowed or a wait expired."""
        L = ng.lib()
        s = C.c_void_p(ng._stream(stream))
        stats = (C.c_int64 * 2)()
        for j, b in zip(self.jobs, self.bufs):
            ng._check(L.svo_trace_rays_check(b["twork"].data_ptr(), j.lod, stats, s))
        ng._check(L.sphere_trace_batch_status(self.handle, s))

    def capture(self):
        """Captures one frame in a CUDA graph (replay with replay())."""
        torch = self.torch
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.frame()          # warm: lazy kernel attributes are set outside the capture
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.frame()
        torch.cuda.synchronize()
        return self.graph

    def replay(self):
        self.graph.replay()

    def outputs(self, k):
        b = self.bufs[k]
        return dict(t=b["t"], hit=b["hit"], steps=b["steps"], normal=b["normal"])

    def time_frames(self, n=5, use_graph=False):
        torch = self.torch
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(n):
            e0.record()
            if use_graph:
                self.replay()
            else:
                self.frame()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)


def set_traversal_streams(renderer: BatchRenderer, n: int):
    """Spreads the jobs' traversals and normals over n side streams (0: the
    frame's own stream); n is capped by the renderer's stream pool, which
    grows on demand."""
    import torch
    while len(renderer.stream_pool) < n:
        renderer.stream_pool.append(torch.cuda.Stream(device=renderer.jobs[0].o.device))
    renderer.tstreams = renderer.stream_pool[:max(0, n)]
    renderer.graph = None


def autotune(renderer: BatchRenderer, candidates=None, streams=None, reps=3):
    """Picks the trace kernel's CTAs per SM (queries in flight per SM: 128
    per CTA) and the number of side streams for the jobs' traversals and
    normals, by timing every pair on the renderer's own batch; leaves the
    renderer configured with the best.  Returns ((ctas, streams), timings)
    with timings keyed "ctas/streams"."""
    cands = candidates or ([1, 2, 3] if renderer.decode == "f32" else [1, 2, 3, 4])
    scands = streams if streams is not None else [len(renderer.tstreams)]
    timings = {}
    for c in cands:
        renderer.ctas_per_sm = c
        renderer._create()
        for n in scands:
            set_traversal_streams(renderer, n)
            renderer.frame()
            renderer.check()
            timings[f"{c}/{n}"] = renderer.time_frames(reps)
    key = min(timings, key=timings.get)
    c, n = (int(v) for v in key.split("/"))
    renderer.ctas_per_sm = c
    renderer._create()
    set_traversal_streams(renderer, n)
    return (c, n), timings


def per_scene_frame(jobs, eps=1e-3, far=5.0, max_steps=128, decode="bf16", normals=True):
    """Reference schedule: each job traversed, traced and shaded by its own
    synchronous calls, one after another."""
    outs = []
    for j in jobs:
        lists = ng.svo_trace_rays(j.svo, j.o, j.d, j.lod)
        outs.append(ng.sphere_trace(j.svo, j.feats, j.dec, j.o, j.d, lists, eps=eps, far=far, max_steps=max_steps,
                                    decode=decode, normals=normals))
    return outs
