"""One image per frame with its stages overlapped across CUDA streams.

The rays of the image are split into a few consecutive chunks; each chunk's
traversal (svo_trace_rays_staged_async: one launch, the lists left where the
traversal staged them and read by each ray's first entry and count), sphere
trace and normals are enqueued on its own stream, so the tail of one chunk's trace -- the few long rays that
keep a persistent launch busy while most SMs idle -- overlaps the next
chunk's traversal and trace, and one chunk's normals overlap another's
trace.  No kernel waits for another; the chunks only share the GPU.  The
outputs are the single-pass frame's, bit for bit (rays are independent).

With host buffers, each chunk's rays are copied in and its results copied
out on the chunk's stream, so the copies overlap the other chunks' work.
"""
from __future__ import annotations

import ctypes as C

from . import nglod as ng


class FrameRenderer:
    def __init__(self, svo: ng.SVO, feats: ng.Features, dec: ng.DecoderDev, o, d, lod, chunks: int = 2,
                 eps: float = 1e-3, far: float = 5.0, max_steps: int = 128, decode: str = "bf16",
                 normals: bool = True, headroom: float = 1.25, dec_hi: ng.DecoderDev | None = None,
                 normal_mode: str = "analytic", fd_h: float = 1e-3, ctas_per_sm: int = 0,
                 trav_ctas_per_sm: int = 0, weights=None):
        """lod: an integer LOD, or a continuous L~ (Eq. 3) with dec = LOD floor(L~)'s decoder and
        dec_hi = LOD floor(L~) + 1's; rays then walk their lists at ceil(L~).
        ctas_per_sm / trav_ctas_per_sm: resident CTAs per SM of the persistent trace / traversal
        kernels (0: the most that fit); narrower launches leave room on each SM for the other
        chunks' kernels.  weights: relative chunk sizes (default equal); smaller first and last
        chunks shorten the stretches where only one chunk's stage runs."""
        import torch
        self.torch = torch
        self.lod_tilde = float(lod)
        self.blend = self.lod_tilde != int(self.lod_tilde)
        self.dec_hi = dec_hi
        if self.blend and dec_hi is None:
            raise ValueError("FrameRenderer: a fractional LOD needs dec_hi")
        lod = ng.blend_lists_lod(self.lod_tilde) if self.blend else int(lod)
        self.svo, self.feats, self.dec, self.lod = svo, feats, dec, int(lod)
        self.o, self.d = o.contiguous(), d.contiguous()
        self.R = R = int(self.o.shape[0])
        self.eps, self.far, self.max_steps, self.decode, self.normals = eps, far, max_steps, decode, normals
        self.nopt = dict(normal_mode=normal_mode, fd_h=fd_h)
        self.ctas_per_sm = int(ctas_per_sm)
        self.trav_ctas_per_sm = int(trav_ctas_per_sm)
        dev = self.o.device
        # chunk bounds on multiples of 128 rays (the traversal's tile)
        n = max(1, int(chunks))
        w = [1.0] * n if weights is None else [float(x) for x in weights]
        if len(w) != n or min(w) <= 0:
            raise ValueError("FrameRenderer: weights must be chunks positive numbers")
        cum = [sum(w[:i]) / sum(w) for i in range(n)]
        self.bounds = sorted(set([min(R, int(R * f) // 128 * 128) for f in cum] + [R]))
        if self.bounds[0] != 0:
            self.bounds = [0] + self.bounds
        self.out = dict(t=torch.empty(R, dtype=torch.float32, device=dev),
                        hit=torch.empty(R, dtype=torch.uint8, device=dev),
                        steps=torch.empty(R, dtype=torch.int32, device=dev),
                        normal=torch.empty((R, 3), dtype=torch.float32, device=dev) if normals else None)
        L = ng.lib()
        self.chunks = []
        for rs, re_ in zip(self.bounds[:-1], self.bounds[1:]):
            m = re_ - rs
            # sizing pass: the lists of this chunk fix its capacities
            lists = ng.svo_trace_rays(svo, self.o[rs:re_], self.d[rs:re_], self.lod, t_range=False)
            cap = int(lists.voxel_id.numel() * headroom) + 4096
            c = dict(rs=rs, n=m, cap=cap, stream=torch.cuda.Stream(device=dev),
                     twork=torch.empty(L.svo_trace_rays_workspace(m, cap), dtype=torch.uint8, device=dev),
                     swork=torch.empty(L.sphere_trace_workspace(m), dtype=torch.uint8, device=dev),
                     ptrs=[C.c_void_p() for _ in range(3)])
            # the staged lists (views into twork, the same every frame); no t
            # ranges: the tracers recompute each entry's interval
            c["lists"] = ng.svo_trace_rays_staged(svo, self.o[rs:re_], self.d[rs:re_], self.lod, c["twork"], cap,
                                                  self.trav_ctas_per_sm)
            c["outs"] = dict(t=self.out["t"][rs:re_], hit=self.out["hit"][rs:re_], steps=self.out["steps"][rs:re_],
                             normal=self.out["normal"][rs:re_] if normals else None, work=c["swork"])
            self.chunks.append(c)

    def _enqueue(self, c):
        L = ng.lib()
        st = c["stream"]
        rs, re_ = c["rs"], c["rs"] + c["n"]
        oo, dd = self.o[rs:re_], self.d[rs:re_]
        p = c["ptrs"]
        ng._check(L.svo_trace_rays_staged_async(self.svo.h, oo.data_ptr(), dd.data_ptr(), c["n"], self.lod,
                                                c["twork"].data_ptr(), c["twork"].numel(), c["cap"],
                                                self.trav_ctas_per_sm, C.byref(p[0]), C.byref(p[1]), C.byref(p[2]),
                                                C.c_void_p(st.cuda_stream)))
        if self.blend:
            ng.sphere_trace_blend(self.svo, self.feats, self.dec, self.dec_hi, oo, dd, c["lists"], self.lod_tilde,
                                  eps=self.eps, far=self.far, max_steps=self.max_steps, decode=self.decode,
                                  normals=self.normals, stream=st, out=c["outs"], ctas_per_sm=self.ctas_per_sm,
                                  **self.nopt)
        else:
            ng.sphere_trace(self.svo, self.feats, self.dec, oo, dd, c["lists"], eps=self.eps, far=self.far,
                            max_steps=self.max_steps, decode=self.decode, normals=self.normals, stream=st,
                            out=c["outs"], ctas_per_sm=self.ctas_per_sm, **self.nopt)

    def frame(self, h_in=None, h_out=None):
        """Enqueues one frame after the work already on the current stream,
        which waits for it.  h_in = (o, d) pinned host arrays to copy in, h_out
        = dict of pinned host tensors (t, hit, normal) to copy the results
        to, chunk by chunk on the chunks' streams."""
        torch = self.torch
        main = torch.cuda.current_stream()
        start = torch.cuda.Event()
        start.record(main)
        for c in self.chunks:
            st = c["stream"]
            st.wait_event(start)
            rs, re_ = c["rs"], c["rs"] + c["n"]
            with torch.cuda.stream(st):
                if h_in is not None:
                    self.o[rs:re_].copy_(h_in[0][rs:re_], non_blocking=True)
                    self.d[rs:re_].copy_(h_in[1][rs:re_], non_blocking=True)
                self._enqueue(c)
                if h_out is not None:
                    for k, v in h_out.items():
                        v[rs:re_].copy_(self.out[k][rs:re_], non_blocking=True)
        for c in self.chunks:
            main.wait_stream(c["stream"])

    def check(self):
        """Synchronises; raises if a chunk's lists outgrew their capacity or a
        bounded wait expired."""
        L = ng.lib()
        stats = (C.c_int64 * 2)()
        for c in self.chunks:
            s = C.c_void_p(c["stream"].cuda_stream)
            ng._check(L.svo_trace_rays_check(c["twork"].data_ptr(), self.lod, stats, s))
            ng._check(L.sphere_trace_status(c["swork"].data_ptr(), s))


def autotune_frame(svo: ng.SVO, feats: ng.Features, dec: ng.DecoderDev, o, d, lod, chunk_counts=(1, 2, 3, 4),
                   ctas=(0, 3, 2), trav_ctas=(0, 2), reps: int = 5, host=None, flush=None, **kw):
    """Times the frame renderer on these rays for every (chunk count, trace
    CTAs per SM, traversal CTAs per SM) triple -- narrower persistent
    launches leave room on each SM for the other chunks' kernels, so the
    chunks' stages share SMs instead of taking turns -- and returns the
    fastest renderer with the timings (ms per frame, keyed
    "chunks/trace ctas" for the widest traversal, "chunks/trace ctas/t<n>"
    for a traversal of n CTAs per SM).  host = (h_in, h_out): time frames
    that copy their rays in from and their results out to these pinned
    host buffers (the schedule that hides the copies best can differ).
    flush: a device buffer zeroed before every timed frame (larger than the
    L2, so each frame starts cold, as in a timed loop that flushes)."""
    import torch
    timings, best, best_ms = {}, None, float("inf")
    configs = [(n, c, t) for n in chunk_counts for c in ctas for t in (trav_ctas if n > 1 else (0,))]
    for n, c, t in configs:
        fr = FrameRenderer(svo, feats, dec, o, d, lod, chunks=n, ctas_per_sm=c, trav_ctas_per_sm=t, **kw)
        args = () if host is None else host
        for _ in range(2):
            fr.frame(*args)
        fr.check()
        ts = []
        for _ in range(reps):
            if flush is not None:
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fr.frame(*args)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        fr.check()
        ms = sorted(ts)[len(ts) // 2]
        timings[f"{n}/{c}/t{t}" if t else f"{n}/{c}"] = ms
        if ms < best_ms:
            best, best_ms = fr, ms
        else:
            del fr
    return best, timings
