"""Thin Python binding of libnglod (include/nglod.h) for torch CUDA tensors.

Argument marshalling only: every step of the rendering path runs in the CUDA
library.  The functions keep the C names (svo_build, svo_trace_rays,
sdf_query, sphere_trace, ...).  If libnglod.so is missing, or no CUDA device
is present, calls raise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnglod.so")

NGLOD_OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_NOT_SUPPORTED = range(7)
F32, F16, BF16, FP8, F32_SPLIT = 0, 1, 2, 3, 4
# decode names: "f32" CUDA cores; "bf16" / "fp8" tensor cores; "f32tc" tensor
# cores at FP32 accuracy (three-term BF16 splits, six products)
DECODES = {"f32": F32, "bf16": BF16, "fp8": FP8, "f32tc": F32_SPLIT}
BF16_DECODE = True          # the tensor-core (tcgen05) decode is built
FIRST_FEATURE_DEPTH = 3

EXPORTS = ["nglod_last_error", "svo_build", "svo_info", "svo_device_arrays", "svo_read_arrays", "svo_free",
           "svo_trace_rays_workspace", "svo_trace_rays", "sdf_query", "sphere_trace_workspace",
           "sphere_trace", "sphere_trace_status", "trace_normals", "svo_trace_rays_noalloc",
           "svo_trace_rays_sizes", "sdf_backward", "sdf_l2_backward", "nglod_adam_step",
           "nglod_features_absmax", "svo_trace_rays_async", "svo_trace_rays_check",
           "sphere_trace_batch_create", "sphere_trace_batch_run", "sphere_trace_batch_status",
           "sphere_trace_batch_free", "sdf_query_blend", "sphere_trace_blend", "nglod_lod_select",
           "trace_normals_fd", "sdf_backward_bf16", "sdf_l2_backward_bf16", "nglod_sort_points_workspace",
           "nglod_sort_points", "nglod_sum_features", "nglod_set_wait_polls", "svo_trace_rays_async_width",
           "svo_trace_rays_staged_async",
           # measurement probes (include/nglod_probe.h)
           "nglod_probe_l2_read", "nglod_probe_l1_read", "nglod_probe_ffma", "nglod_device_sms"]


class NglodError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[nglod status {code}] {msg}")
        self.code = code


class _Features(C.Structure):
    _fields_ = [("feats", C.c_void_p * 8), ("dtype", C.c_int), ("m", C.c_int), ("num_lods", C.c_int),
                ("fp8_z_absmax", C.c_float), ("summed_lod", C.c_int)]


class _Decoder(C.Structure):
    _fields_ = [("W1", C.c_void_p), ("b1", C.c_void_p), ("W2", C.c_void_p), ("b2", C.c_void_p),
                ("in_dim", C.c_int), ("hidden", C.c_int)]


class _TraceJob(C.Structure):
    _fields_ = [("svo", C.c_void_p), ("feats", _Features), ("dec", _Decoder), ("lod", C.c_int),
                ("o", C.c_void_p), ("d", C.c_void_p), ("R", C.c_int64), ("ray_offsets", C.c_void_p),
                ("voxel_id", C.c_void_p), ("t_range", C.c_void_p), ("work", C.c_void_p), ("work_bytes", C.c_size_t),
                ("t_hit", C.c_void_p), ("hit", C.c_void_p), ("steps", C.c_void_p), ("normal", C.c_void_p),
                ("ray_counts", C.c_void_p)]


class _TraceParams(C.Structure):
    _fields_ = [("eps", C.c_float), ("far_t", C.c_float), ("max_steps", C.c_int), ("osc_check", C.c_int),
                ("decode_dtype", C.c_int), ("want_normals", C.c_int), ("normal_mode", C.c_int),
                ("fd_h", C.c_float), ("ctas_per_sm", C.c_int), ("ray_counts", C.c_void_p)]

NORMALS = {"analytic": 0, "fd": 1}


_lib = None


def lib():
    """Loads libnglod.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2101_10994_gb300.build` (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        P, i64, i32, sz = C.c_void_p, C.c_int64, C.c_int, C.c_size_t
        L.nglod_last_error.restype = C.c_char_p
        L.svo_build.argtypes = [P, P, i32, P, P]
        L.svo_info.argtypes = [P, P, P, P]
        L.svo_device_arrays.argtypes = [P, i32, P, P]
        L.svo_read_arrays.argtypes = [P, i32, P, P, P]
        L.svo_free.argtypes = [P]
        L.svo_free.restype = None
        L.svo_trace_rays_workspace.restype = sz
        L.svo_trace_rays_workspace.argtypes = [i64, i64]
        L.svo_trace_rays.argtypes = [P, P, P, i64, i32, P, sz, i64, P, P, P, i64, P, P]
        L.sdf_query.argtypes = [P, P, P, P, i64, i32, i32, P, P, P, P]
        L.sphere_trace_workspace.restype = sz
        L.sphere_trace_workspace.argtypes = [i64]
        L.sphere_trace.argtypes = [P, P, P, P, P, i64, i32, P, P, P, P, P, sz, P, P, P, P, P]
        L.trace_normals.argtypes = [P, P, P, P, P, i64, i32, P, sz, P, P, P, P]
        L.trace_normals_fd.argtypes = [P, P, P, P, P, i64, i32, P, sz, P, P, C.c_float, P, P]
        L.sphere_trace_status.argtypes = [P, P]
        L.svo_trace_rays_sizes.argtypes = [P, P, i32, P]
        L.sdf_backward.argtypes = [P, P, P, P, i64, C.c_uint32, P, P, P, P, P, P, P, i32, P]
        L.sdf_l2_backward.argtypes = [P, P, P, P, P, i64, C.c_uint32, C.c_float, P, P, P, P, P, P, P]
        L.sdf_backward_bf16.argtypes = [P, P, P, P, i64, C.c_uint32, P, P, P, P, P, P, P]
        L.nglod_sort_points_workspace.restype = sz
        L.nglod_sort_points_workspace.argtypes = [i64, i32]
        L.nglod_sort_points.argtypes = [P, P, i64, i32, P, P, P, P, sz, P]
        L.sdf_l2_backward_bf16.argtypes = [P, P, P, P, P, i64, C.c_uint32, C.c_float, P, P, P, P, P, P, P]
        L.nglod_features_absmax.argtypes = [P, P, i32, P, P]
        L.nglod_sum_features.argtypes = [P, P, i32, P, P]
        L.svo_trace_rays_async.argtypes = [P, P, P, i64, i32, P, sz, i64, P, P, P, i64, P]
        L.svo_trace_rays_check.argtypes = [P, i32, P, P]
        L.svo_trace_rays_async_width.argtypes = [P, P, P, i64, i32, P, sz, i64, P, P, P, i64, i32, P]
        L.svo_trace_rays_staged_async.argtypes = [P, P, P, i64, i32, P, sz, i64, i32, P, P, P, P]
        L.sphere_trace_batch_create.argtypes = [P, i32, P, i32, P, P]
        L.sphere_trace_batch_run.argtypes = [P, P]
        L.sphere_trace_batch_status.argtypes = [P, P]
        L.sphere_trace_batch_free.argtypes = [P]
        L.sphere_trace_batch_free.restype = None
        L.sdf_query_blend.argtypes = [P, P, P, P, P, i64, C.c_float, i32, P, P]
        L.sphere_trace_blend.argtypes = [P, P, P, P, P, P, i64, C.c_float, P, P, P, P, P, sz, P, P, P, P, P]
        L.nglod_lod_select.argtypes = [C.c_float] * 5
        L.nglod_lod_select.restype = C.c_float
        L.nglod_adam_step.argtypes = [P, P, P, P, i64, C.c_float, C.c_float, C.c_float, C.c_float, i32, P]
        L.svo_trace_rays_noalloc.argtypes = [P, P, P, i64, i32, P, P, P, i64, P, P]
        L.nglod_set_wait_polls.argtypes = [i64]
        L.nglod_probe_l2_read.argtypes = [P, i64, i32, P, P, P]
        L.nglod_probe_l1_read.argtypes = [P, i64, i64, i32, P, P, P]
        L.nglod_probe_ffma.argtypes = [i64, P, P, P]
        L.nglod_device_sms.argtypes = [P]
        _lib = L
    return _lib


_probe_sink = None


def device_sms() -> int:
    """SMs of the current device (what the persistent launches are sized by)."""
    n = C.c_int(0)
    _check(lib().nglod_device_sms(C.byref(n)))
    return int(n.value)


def probe(kind: str, buf=None, passes: int = 20, window_bytes: int = 96 << 10, iters: int = 1 << 14,
          stream=None) -> int:
    """Enqueues one measurement-probe kernel (include/nglod_probe.h) and
    returns the bytes it reads ("l2", "l1") or the flops it executes
    ("ffma"); the caller times it with CUDA events."""
    import torch
    global _probe_sink
    if _probe_sink is None:
        _probe_sink = torch.zeros(4, dtype=torch.int32, device="cuda")
    sink = _probe_sink
    out = C.c_int64(0)
    s = C.c_void_p(_stream(stream))
    if kind == "l2":
        _check(lib().nglod_probe_l2_read(buf.data_ptr(), buf.numel() * buf.element_size(), passes, sink.data_ptr(),
                                         C.byref(out), s))
    elif kind == "l1":
        _check(lib().nglod_probe_l1_read(buf.data_ptr(), buf.numel() * buf.element_size(), window_bytes, passes,
                                         sink.data_ptr(), C.byref(out), s))
    elif kind == "ffma":
        _check(lib().nglod_probe_ffma(iters, sink.data_ptr(), C.byref(out), s))
    else:
        raise ValueError(kind)
    return int(out.value)


def set_wait_polls(polls: int):
    """Poll budget of every tensor-core kernel's per-tile MMA wait from now on
    (0: each such wait expires at once and the call reports ERR_TIMEOUT;
    negative: the default).  A testing hook for the expiry path."""
    _check(lib().nglod_set_wait_polls(int(polls)))


def _check(rc: int):
    if rc != NGLOD_OK:
        raise NglodError(rc, lib().nglod_last_error().decode())


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t) -> int:
    return 0 if t is None else t.data_ptr()


def _require_cuda(*tensors):
    for t in tensors:
        if t is not None and not t.is_cuda:
            raise ValueError("nglod operates on CUDA tensors only")


# ----------------------------------------------------------------------------
# Octree
# ----------------------------------------------------------------------------
class SVO:
    """Device octree built by svo_build; owns the C handle."""

    def __init__(self, handle: int, keys):
        self.h = C.c_void_p(handle)
        n = C.c_int(0)
        vox = (C.c_int64 * 16)()
        cor = (C.c_int64 * 16)()
        _check(lib().svo_info(self.h, C.byref(n), vox, cor))
        self.num_depths = n.value
        self.voxels = [vox[i] for i in range(self.num_depths)]
        self.corners = [cor[i] for i in range(self.num_depths - FIRST_FEATURE_DEPTH)]
        self.max_lod = self.num_depths - FIRST_FEATURE_DEPTH
        self._cap = {}

    def free(self):
        if self.h is not None and self.h.value:
            lib().svo_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def read_arrays(self, dp: int):
        """(node [V,4] int32, corners [V,8] int32, anc [V,8] int32) on the host.

        corners / anc are None for the structural depths 0..2."""
        V = self.voxels[dp]
        nb = np.empty((V, 4), np.int32)
        feat = dp >= FIRST_FEATURE_DEPTH
        cb = np.empty((V, 8), np.int32) if feat else None
        ab = np.empty((V, 8), np.int32) if feat else None
        _check(lib().svo_read_arrays(self.h, dp, nb.ctypes.data, cb.ctypes.data if feat else None,
                                     ab.ctypes.data if feat else None))
        return nb, cb, ab


def svo_build(keys_per_depth, stream=None) -> SVO:
    keys = [np.ascontiguousarray(k, dtype=np.uint64) for k in keys_per_depth]
    arr = (C.c_void_p * len(keys))(*[k.ctypes.data for k in keys])
    counts = np.array([k.shape[0] for k in keys], np.int64)
    out = C.c_void_p()
    _check(lib().svo_build(arr, counts.ctypes.data, len(keys), C.c_void_p(_stream(stream)), C.byref(out)))
    return SVO(out.value, keys)


# ----------------------------------------------------------------------------
# Parameters on the device
# ----------------------------------------------------------------------------
class Features:
    """Corner feature tables of LODs 1..L on the device (float32 or float16)."""

    def __init__(self, tables, dtype: str = "f32", device="cuda"):
        import torch
        tdt = {"f32": torch.float32, "f16": torch.float16}[dtype]
        self.dtype = dtype
        self.tables = [torch.as_tensor(np.asarray(t)).to(device=device, dtype=tdt).contiguous()
                       for t in tables]
        self.m = int(self.tables[0].shape[1])
        self.z_absmax = 0.0
        self.summed_lod = 0

    @classmethod
    def from_tensors(cls, tables):
        """A view on existing device tensors (FP32 or FP16 [C_l, 32], no copy)."""
        import torch
        f = cls.__new__(cls)
        f.tables = [t.contiguous() for t in tables]
        f.dtype = "f16" if f.tables[0].dtype == torch.float16 else "f32"
        f.m = int(f.tables[0].shape[1])
        f.z_absmax = 0.0
        f.summed_lod = 0
        return f

    def summed(self, svo, lod: int, stream=None) -> "Features":
        """The summed corner table of LOD ``lod`` (nglod_sum_features): per
        corner of that LOD, the sum over LODs 1..lod of the interpolated
        features there.  The returned Features serve sphere_trace (analytic
        normals) and trace_normals at that LOD with 8 row gathers per query."""
        import torch
        if getattr(self, "summed_lod", 0):
            raise ValueError("already a summed table")
        ref = self.tables[lod - 1]
        out = torch.empty((svo.corners[lod - 1], self.m), dtype=torch.float32, device=ref.device)
        fc = self.c()
        _check(lib().nglod_sum_features(svo.h, C.byref(fc), int(lod), out.data_ptr(),
                                        C.c_void_p(_stream(stream))))
        f = Features.__new__(Features)
        f.tables = [None] * (lod - 1) + [out]
        f.dtype = "f32"
        f.m = self.m
        f.z_absmax = 0.0
        f.summed_lod = int(lod)
        return f

    def set_fp8_bound(self, svo, lod: int, stream=None):
        """Computes the |z| bound the FP8 decode scales by (library reduction)."""
        out = C.c_float(0.0)
        fc = self.c()
        _check(lib().nglod_features_absmax(svo.h, C.byref(fc), int(lod), C.byref(out), C.c_void_p(_stream(stream))))
        self.z_absmax = float(out.value)
        return self.z_absmax

    def c(self) -> _Features:
        f = _Features()
        for i, t in enumerate(self.tables[:8]):
            f.feats[i] = t.data_ptr() if t is not None else None
        f.dtype = F32 if self.dtype == "f32" else F16
        f.m = self.m
        f.num_lods = len(self.tables)
        f.fp8_z_absmax = getattr(self, "z_absmax", 0.0)
        f.summed_lod = getattr(self, "summed_lod", 0)
        return f


class DecoderDev:
    """One LOD's decoder on the device (FP32 weights; b2 is a one-element
    device tensor, ``b2_t``, that the kernels read when they run)."""

    def __init__(self, W1, b1, W2, b2, device="cuda"):
        import torch
        self.h_W1 = np.ascontiguousarray(W1, np.float32)
        self.h_b1 = np.ascontiguousarray(b1, np.float32)
        self.h_W2 = np.ascontiguousarray(W2, np.float32)
        self.W1 = torch.from_numpy(self.h_W1).to(device)
        self.b1 = torch.from_numpy(self.h_b1).to(device)
        self.W2 = torch.from_numpy(self.h_W2).to(device)
        self.b2_t = torch.tensor([float(b2)], dtype=torch.float32, device=device)
        self.in_dim = int(self.h_W1.shape[1])
        self.hidden = int(self.h_W1.shape[0])

    @property
    def b2(self) -> float:
        """The current b2 (reads the device value: synchronises)."""
        return float(self.b2_t.item())

    @classmethod
    def from_decoder(cls, dec, device="cuda"):
        return cls(dec.W1, dec.b1, dec.W2, dec.b2, device)

    @classmethod
    def from_tensors(cls, W1, b1, W2, b2):
        """A view on existing FP32 device tensors (no copy).  ``b2``: a
        one-element FP32 device tensor (viewed, e.g. one entry of a
        per-LOD vector) or a float (uploaded)."""
        import torch
        d = cls.__new__(cls)
        d.W1, d.b1, d.W2 = W1.contiguous(), b1.contiguous(), W2.contiguous()
        if isinstance(b2, torch.Tensor):
            if b2.numel() != 1 or b2.dtype != torch.float32 or not b2.is_cuda:
                raise ValueError("b2 must be a one-element float32 CUDA tensor")
            d.b2_t = b2.reshape(1)
        else:
            d.b2_t = torch.tensor([float(b2)], dtype=torch.float32, device=W1.device)
        d.in_dim, d.hidden = int(W1.shape[1]), int(W1.shape[0])
        return d

    def c(self) -> _Decoder:
        d = _Decoder()
        d.W1, d.b1, d.W2 = self.W1.data_ptr(), self.b1.data_ptr(), self.W2.data_ptr()
        d.b2 = self.b2_t.data_ptr()
        d.in_dim, d.hidden = self.in_dim, self.hidden
        return d


# ----------------------------------------------------------------------------
# Calls
# ----------------------------------------------------------------------------
@dataclass
class RayLists:
    ray_offsets: object      # int32 [R + 1]
    voxel_id: object         # int32 [H]
    t_range: object          # float32 [H, 2], or None (not asked for: the tracers do not read it)
    max_pairs: int
    lod: int
    work: object = None      # the workspace the lists were built in
    # staged lists (svo_trace_rays_staged): ray_offsets is then each ray's
    # first entry [R] and ray_counts its entry count [R]
    ray_counts: object = None

    def level_sizes(self, stream=None):
        """Pairs kept by Decide at each depth 0..target (entry 0 = R)."""
        D = self.lod + FIRST_FEATURE_DEPTH - 1
        out = (C.c_int64 * (D + 1))()
        _check(lib().svo_trace_rays_sizes(self.work.data_ptr(), out, D + 1, C.c_void_p(_stream(stream))))
        return [int(v) for v in out]


def svo_trace_rays(svo: SVO, o, d, lod: int, stream=None, pair_capacity: int | None = None,
                   workspace=None, t_range: bool = True) -> RayLists:
    """Per-ray front-to-back voxel lists at LOD ``lod`` (CSR), with each
    entry's (t_enter, t_exit) unless ``t_range`` is False.

    Grows the intermediate-list capacity and retries when the library reports
    NGLOD_ERR_CAPACITY; the capacity that worked is remembered per (R, lod).
    """
    import torch
    _require_cuda(o, d)
    o = o.contiguous()
    d = d.contiguous()
    R = int(o.shape[0])
    key = (R, lod)
    cap = pair_capacity or svo._cap.get(key, max(1 << 20, 16 * R))
    L = lib()
    stats = (C.c_int64 * 2)()
    for _ in range(8):
        wbytes = L.svo_trace_rays_workspace(R, cap)
        if workspace is not None and workspace.numel() >= wbytes:
            work = workspace
        else:
            work = torch.empty(max(wbytes, 1), dtype=torch.uint8, device=o.device)
        offs = torch.empty(R + 1, dtype=torch.int32, device=o.device)
        vid = torch.empty(max(cap, 1), dtype=torch.int32, device=o.device)
        tr = torch.empty((max(cap, 1), 2), dtype=torch.float32, device=o.device) if t_range else None
        rc = L.svo_trace_rays(svo.h, o.data_ptr(), d.data_ptr(), R, lod, work.data_ptr(), wbytes, cap,
                              offs.data_ptr(), vid.data_ptr(), _ptr(tr), cap, stats,
                              C.c_void_p(_stream(stream)))
        if rc == ERR_CAPACITY:
            cap = int(max(2 * cap, 1.25 * max(stats[0], stats[1])))
            continue
        _check(rc)
        svo._cap[key] = cap
        H = int(stats[0])
        return RayLists(offs, vid[:H], tr[:H] if t_range else None, int(stats[1]), lod, work)
    raise NglodError(ERR_CAPACITY, "svo_trace_rays: capacity growth did not converge")


def svo_trace_rays_staged(svo: SVO, o, d, lod: int, work, pair_capacity: int, ctas_per_sm: int = 0,
                          stream=None) -> RayLists:
    """Enqueues the traversal without its placement pass (no host
    synchronisation): each ray's front-to-back entries stay where the
    traversal staged them in ``work`` (a uint8 tensor of at least
    svo_trace_rays_workspace(R, pair_capacity) bytes, 256-B aligned).
    Returns views into ``work``: ray_offsets = each ray's first entry,
    ray_counts = its count, voxel_id = the staging list.  Overflow is
    reported by svo_trace_rays_check on ``work``."""
    _require_cuda(o, d)
    import torch
    R = int(o.shape[0])
    first, cnt, vid = C.c_void_p(), C.c_void_p(), C.c_void_p()
    _check(lib().svo_trace_rays_staged_async(svo.h, o.data_ptr(), d.data_ptr(), R, lod, work.data_ptr(),
                                             work.numel(), int(pair_capacity), int(ctas_per_sm), C.byref(first),
                                             C.byref(cnt), C.byref(vid), C.c_void_p(_stream(stream))))
    base = work.data_ptr()

    def view(ptr, n):
        off = int(ptr.value or base) - base
        return work[off:off + 4 * n].view(torch.int32)
    return RayLists(view(first, R), view(vid, int(pair_capacity)), None, -1, lod, work, view(cnt, R))


def sdf_query(svo: SVO, feats: Features, dec: DecoderDev, x, lod: int, decode: str = "f32",
              grad: bool = False, deepest: bool = False, stream=None):
    import torch
    _require_cuda(x)
    x = x.contiguous()
    Q = int(x.shape[0])
    sdf = torch.empty(Q, dtype=torch.float32, device=x.device)
    dp = torch.empty(Q, dtype=torch.int8, device=x.device) if deepest else None
    g = torch.empty((Q, 3), dtype=torch.float32, device=x.device) if grad else None
    fc, dc = feats.c(), dec.c()
    _check(lib().sdf_query(svo.h, C.byref(fc), C.byref(dc), x.data_ptr(), Q, lod,
                           DECODES[decode], sdf.data_ptr(), _ptr(dp), _ptr(g),
                           C.c_void_p(_stream(stream))))
    out = [sdf]
    if deepest:
        out.append(dp)
    if grad:
        out.append(g)
    return out[0] if len(out) == 1 else tuple(out)


def sphere_trace(svo: SVO, feats: Features, dec: DecoderDev, o, d, lists: RayLists, eps: float = 1e-3,
                 far: float = 5.0, max_steps: int = 128, osc: bool = False, decode: str = "f32",
                 normals: bool = True, stream=None, out=None, normal_mode: str = "analytic", fd_h: float = 1e-3,
                 ctas_per_sm: int = 0):
    """Sphere-traces every ray through its voxel list; returns a dict of tensors.

    normal_mode "analytic" (gradient of the decoded SDF) or "fd" (central
    differences with step fd_h, supplementary Sec. A.4).  ctas_per_sm: the
    persistent trace's launch width (0: the most that fit)."""
    import torch
    _require_cuda(o, d)
    R = int(o.shape[0])
    dev = o.device
    if out is None:
        out = dict(t=torch.empty(R, dtype=torch.float32, device=dev),
                   hit=torch.empty(R, dtype=torch.uint8, device=dev),
                   steps=torch.empty(R, dtype=torch.int32, device=dev),
                   normal=torch.empty((R, 3), dtype=torch.float32, device=dev) if normals else None,
                   work=torch.empty(max(lib().sphere_trace_workspace(R), 1), dtype=torch.uint8, device=dev))
    p = _TraceParams(eps, far, max_steps, int(osc), DECODES[decode], int(normals),
                     NORMALS[normal_mode], fd_h, int(ctas_per_sm), _ptr(lists.ray_counts))
    fc, dc = feats.c(), dec.c()
    _check(lib().sphere_trace(svo.h, C.byref(fc), C.byref(dc), o.data_ptr(), d.data_ptr(), R, lists.lod,
                              C.byref(p), lists.ray_offsets.data_ptr(), lists.voxel_id.data_ptr(),
                              _ptr(lists.t_range), out["work"].data_ptr(), out["work"].numel(),
                              out["t"].data_ptr(), out["hit"].data_ptr(), _ptr(out["steps"]),
                              _ptr(out["normal"]), C.c_void_p(_stream(stream))))
    out["hit_voxel"] = out["work"][256:256 + 4 * R].view(torch.int32)
    return out


def trace_normals(svo: SVO, feats: Features, dec: DecoderDev, o, d, lists: RayLists, out, stream=None,
                  normal_mode: str = "analytic", fd_h: float = 1e-3):
    """Normals of the hits of the preceding sphere_trace call that filled ``out``."""
    R = int(o.shape[0])
    if out.get("normal") is None:
        import torch
        out["normal"] = torch.empty((R, 3), dtype=torch.float32, device=o.device)
    fc, dc = feats.c(), dec.c()
    args = (svo.h, C.byref(fc), C.byref(dc), o.data_ptr(), d.data_ptr(), R, lists.lod, out["work"].data_ptr(),
            out["work"].numel(), out["t"].data_ptr(), out["hit"].data_ptr())
    if NORMALS[normal_mode]:
        _check(lib().trace_normals_fd(*args, fd_h, out["normal"].data_ptr(), C.c_void_p(_stream(stream))))
    else:
        _check(lib().trace_normals(*args, out["normal"].data_ptr(), C.c_void_p(_stream(stream))))
    return out


def sphere_trace_status(out, stream=None):
    """Raises if the sphere_trace that filled ``out`` hit an expired wait."""
    _check(lib().sphere_trace_status(out["work"].data_ptr(), C.c_void_p(_stream(stream))))


# ----------------------------------------------------------------------------
# Continuous LOD (level blending, Eq. 3) and LOD selection
# ----------------------------------------------------------------------------
def lod_select(distance: float, d_near: float, d_far: float, lod_near: float, lod_far: float) -> float:
    """Continuous LOD moving linearly with the distance to the object."""
    return float(lib().nglod_lod_select(distance, d_near, d_far, lod_near, lod_far))


def blend_lists_lod(lod_tilde: float) -> int:
    """The LOD whose ray lists sphere_trace_blend walks: ceil(L~)."""
    import math
    return int(math.ceil(float(np.float32(lod_tilde))))


def sdf_query_blend(svo: SVO, feats: Features, dec_lo: DecoderDev, dec_hi: DecoderDev | None, x, lod_tilde: float,
                    decode: str = "f32", stream=None):
    import torch
    _require_cuda(x)
    x = x.contiguous()
    Q = int(x.shape[0])
    out = torch.empty(Q, dtype=torch.float32, device=x.device)
    fc, lo = feats.c(), dec_lo.c()
    hi = (dec_hi or dec_lo).c()
    _check(lib().sdf_query_blend(svo.h, C.byref(fc), C.byref(lo), C.byref(hi), x.data_ptr(), Q, lod_tilde,
                                 DECODES[decode], out.data_ptr(),
                                 C.c_void_p(_stream(stream))))
    return out


def sphere_trace_blend(svo: SVO, feats: Features, dec_lo: DecoderDev, dec_hi: DecoderDev | None, o, d,
                       lists: RayLists, lod_tilde: float, eps: float = 1e-3, far: float = 5.0, max_steps: int = 128,
                       osc: bool = False, decode: str = "f32", normals: bool = True, stream=None, out=None,
                       normal_mode: str = "analytic", fd_h: float = 1e-3, ctas_per_sm: int = 0):
    """Sphere-traces the Eq. 3 blend; ``lists`` must be at LOD ceil(L~)."""
    import torch
    _require_cuda(o, d)
    if lists.lod != blend_lists_lod(lod_tilde):
        raise ValueError("sphere_trace_blend: lists must be traced at LOD ceil(lod_tilde)")
    R = int(o.shape[0])
    dev = o.device
    if out is None:
        out = dict(t=torch.empty(R, dtype=torch.float32, device=dev),
                   hit=torch.empty(R, dtype=torch.uint8, device=dev),
                   steps=torch.empty(R, dtype=torch.int32, device=dev),
                   normal=torch.empty((R, 3), dtype=torch.float32, device=dev) if normals else None,
                   work=torch.empty(max(lib().sphere_trace_workspace(R), 1), dtype=torch.uint8, device=dev))
    p = _TraceParams(eps, far, max_steps, int(osc), DECODES[decode], int(normals),
                     NORMALS[normal_mode], fd_h, int(ctas_per_sm), _ptr(lists.ray_counts))
    fc, lo = feats.c(), dec_lo.c()
    hi = (dec_hi or dec_lo).c()
    _check(lib().sphere_trace_blend(svo.h, C.byref(fc), C.byref(lo), C.byref(hi), o.data_ptr(), d.data_ptr(), R,
                                    lod_tilde, C.byref(p), lists.ray_offsets.data_ptr(), lists.voxel_id.data_ptr(),
                                    _ptr(lists.t_range), out["work"].data_ptr(), out["work"].numel(),
                                    out["t"].data_ptr(), out["hit"].data_ptr(), _ptr(out["steps"]),
                                    _ptr(out["normal"]), C.c_void_p(_stream(stream))))
    out["hit_voxel"] = out["work"][256:256 + 4 * R].view(torch.int32)
    return out


def new_grads(svo: SVO, decs, device="cuda"):
    """Zeroed gradient buffers matching the features and decoders."""
    import torch
    return dict(feats=[torch.zeros((c, 32), dtype=torch.float32, device=device) for c in svo.corners],
                W1=[torch.zeros_like(d.W1) for d in decs], b1=[torch.zeros_like(d.b1) for d in decs],
                W2=[torch.zeros_like(d.W2) for d in decs],
                b2=torch.zeros(len(decs), dtype=torch.float32, device=device))


def sdf_backward(svo: SVO, feats: Features, decs, x, lods, grad_sdf, grads=None, grad_x=None, stream=None,
                 deterministic: bool = False, mma: str = "f32"):
    """Accumulates the gradients of sum_i grad_sdf[i] . sdf_{lods[i]}(x) into ``grads``.

    ``decs`` lists every LOD's decoder (index lod - 1); ``lods`` the
    increasing LODs whose outputs carry gradient (rows of ``grad_sdf``).
    ``deterministic``: exact fixed-point sums, bit-identical between runs.
    ``mma="bf16"``: the decoder's contractions on the tensor cores (BF16
    operands, FP32 accumulation; no grad_x, not deterministic)."""
    _require_cuda(x, grad_sdf)
    x = x.contiguous()
    grad_sdf = grad_sdf.contiguous()
    Q = int(x.shape[0])
    if grads is None:
        grads = new_grads(svo, decs, x.device)
    mask = 0
    for l in lods:
        mask |= 1 << (int(l) - 1)
    dec_arr = (_Decoder * len(decs))(*[d.c() for d in decs])
    fc = feats.c()
    P = C.c_void_p

    def parr(ts):
        return (P * len(ts))(*[t.data_ptr() for t in ts])

    if mma == "bf16":
        if grad_x is not None or deterministic:
            raise ValueError("sdf_backward: the BF16 tensor-core adjoint has no grad_x or deterministic mode")
        _check(lib().sdf_backward_bf16(svo.h, C.byref(fc), dec_arr, x.data_ptr(), Q, mask, grad_sdf.data_ptr(),
                                       parr(grads["feats"]), parr(grads["W1"]), parr(grads["b1"]), parr(grads["W2"]),
                                       grads["b2"].data_ptr(), C.c_void_p(_stream(stream))))
        return grads
    _check(lib().sdf_backward(svo.h, C.byref(fc), dec_arr, x.data_ptr(), Q, mask, grad_sdf.data_ptr(),
                              parr(grads["feats"]), parr(grads["W1"]), parr(grads["b1"]), parr(grads["W2"]),
                              grads["b2"].data_ptr(), _ptr(grad_x), int(bool(deterministic)),
                              C.c_void_p(_stream(stream))))
    return grads


def sdf_l2_backward(svo: SVO, feats: Features, decs, x, target, lods, loss_scale: float, grads, loss=None,
                    stream=None, mma: str = "f32"):
    """Gradients of loss_scale * sum_L sum_q (sdf_L(x_q) - target_q)^2 (Eq. 4), accumulated into ``grads``.

    ``mma="bf16"``: the decoder's contractions on the tensor cores (BF16 operands, FP32 accumulation)."""
    _require_cuda(x, target)
    mask = 0
    for l in lods:
        mask |= 1 << (int(l) - 1)
    dec_arr = (_Decoder * len(decs))(*[d.c() for d in decs])
    fc = feats.c()
    P = C.c_void_p

    def parr(ts):
        return (P * len(ts))(*[t.data_ptr() for t in ts])

    fn = lib().sdf_l2_backward_bf16 if mma == "bf16" else lib().sdf_l2_backward
    _check(fn(svo.h, C.byref(fc), dec_arr, x.data_ptr(), target.data_ptr(), int(x.shape[0]),
              mask, float(loss_scale), _ptr(loss), parr(grads["feats"]), parr(grads["W1"]),
              parr(grads["b1"]), parr(grads["W2"]), grads["b2"].data_ptr(), C.c_void_p(_stream(stream))))
    return grads


def sort_points(x, extra=None, depth: int = 7, out=None, stream=None):
    """Points (and one float per point) reordered by the Morton code of their
    depth-``depth`` octree cell; returns (x_sorted, extra_sorted, perm).
    ``out``: a dict of reusable buffers (x, extra, perm, work)."""
    import torch
    _require_cuda(x)
    x = x.contiguous()
    Q = int(x.shape[0])
    dev = x.device
    o = out if out is not None else {}
    if o.get("x") is None or o["x"].shape[0] != Q:
        o["x"] = torch.empty((Q, 3), dtype=torch.float32, device=dev)
        o["extra"] = torch.empty(Q, dtype=torch.float32, device=dev)
        o["perm"] = torch.empty(Q, dtype=torch.int32, device=dev)
        o["work"] = torch.empty(max(1, lib().nglod_sort_points_workspace(Q, depth)), dtype=torch.uint8, device=dev)
    if o["work"].numel() < lib().nglod_sort_points_workspace(Q, depth):
        o["work"] = torch.empty(lib().nglod_sort_points_workspace(Q, depth), dtype=torch.uint8, device=dev)
    e = extra.contiguous() if extra is not None else None
    _check(lib().nglod_sort_points(x.data_ptr(), _ptr(e), Q, int(depth), o["x"].data_ptr(),
                                   o["extra"].data_ptr() if e is not None else None, o["perm"].data_ptr(),
                                   o["work"].data_ptr(), o["work"].numel(), C.c_void_p(_stream(stream))))
    return o["x"], (o["extra"] if e is not None else None), o["perm"]


def adam_step(param, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """In-place Adam update of one FP32 tensor (grad is zeroed)."""
    _check(lib().nglod_adam_step(param.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), param.numel(),
                                 float(lr), float(beta1), float(beta2), float(eps), int(step),
                                 C.c_void_p(_stream(stream))))
