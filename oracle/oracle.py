"""ctypes binding of the FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg import this module.  It shares no code with the CUDA library; it reads
the same seeded inputs (``paper_2101_10994_gb300.scenes``).

Every function promotes its inputs from their stored precision to float64
exactly and returns float64 results (except the traversal lists, whose FP32
interval bounds are part of the method's FP32 decision).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "nglod_oracle.c")
LIB = os.path.join(HERE, "liboracle_nglod.so")
FIRST_FEATURE_DEPTH = 3

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off, OpenMP if present)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", SRC, "-o", LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(LIB)
        P = C.c_void_p
        i64, i32, f64 = C.c_int64, C.c_int, C.c_double
        lib.or_svo_new.restype = P
        lib.or_svo_new.argtypes = [P, P, i32]
        lib.or_svo_free.argtypes = [P]
        lib.or_corner_count.restype = i64
        lib.or_corner_count.argtypes = [P, i32]
        lib.or_svo_arrays.argtypes = [P, i32, P, P, P, P]
        lib.or_trace_rays.restype = i64
        lib.or_trace_rays.argtypes = [P, P, P, i64, i32, P, P, P, i32]
        lib.or_sdf_query.argtypes = [P, P, i32, P, P, P, f64, i32, i32, P, i64, i32,
                                     P, P, P, i32]
        lib.or_sphere_trace.argtypes = [P, P, i32, P, P, P, f64, i32, i32, P, P, i64,
                                        i32, f64, f64, i32, i32, P, P, P, P, P, i32]
        lib.or_sphere_trace_blend.argtypes = [P, P, i32, P, P, P, f64, P, P, P, f64, i32, i32, P, P,
                                              i64, i32, f64, f64, f64, i32, i32, P, P, P, P, P, i32]
        lib.or_feature_sum.argtypes = [P, P, i32, P, i64, i32, P]
        lib.or_sdf_backward.argtypes = [P, P, i32, P, P, P, P, i32, i32, P, i64, P, i32,
                                        P, P, P, P, P, P, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    """Exact promotion to float64 (torch tensors of any float dtype too)."""
    if hasattr(a, "detach"):
        import torch
        a = a.detach().to("cpu", torch.float64).numpy()
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class _PtrArray:
    """Keeps a list of numpy arrays alive and exposes a ``void*[]``."""

    def __init__(self, arrays):
        self.arrays = list(arrays)
        self.c = (C.c_void_p * max(1, len(self.arrays)))(
            *[a.ctypes.data_as(C.c_void_p).value for a in self.arrays])

    @property
    def p(self):
        return C.cast(self.c, C.c_void_p)


class OracleSVO:
    """The oracle's own copy of an octree given as sorted Morton keys per depth."""

    def __init__(self, keys_per_depth):
        lib = _load()
        self.keys = [np.ascontiguousarray(k, dtype=np.uint64) for k in keys_per_depth]
        self.num_depths = len(self.keys)
        counts = np.array([k.shape[0] for k in self.keys], dtype=np.int64)
        arr = _PtrArray(self.keys)
        self.h = lib.or_svo_new(arr.p, _ptr(counts), self.num_depths)
        if not self.h:
            raise ValueError("keys are not a valid parent-closed octree")
        self.counts = counts

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_svo_free(self.h)
            self.h = None

    @property
    def max_lod(self) -> int:
        return self.num_depths - FIRST_FEATURE_DEPTH

    def corner_count(self, lod: int) -> int:
        return int(_load().or_corner_count(self.h, lod))

    def arrays(self, dp: int):
        V = int(self.counts[dp])
        parent = np.zeros(V, np.int32)
        mask = np.zeros(V, np.uint8)
        base = np.zeros(V, np.int32)
        corners = np.zeros((V, 8), np.int32) if dp >= FIRST_FEATURE_DEPTH else None
        _load().or_svo_arrays(self.h, dp, _ptr(parent), _ptr(mask), _ptr(base),
                              _ptr(corners) if corners is not None else None)
        return parent, mask, base, corners

    # -- ray/voxel lists --------------------------------------------------
    def trace_rays(self, o, d, lod: int, nthreads: int = 0):
        o = np.ascontiguousarray(o, np.float32).reshape(-1, 3)
        d = np.ascontiguousarray(d, np.float32).reshape(-1, 3)
        R = o.shape[0]
        offs = np.zeros(R + 1, np.int64)
        lib = _load()
        H = lib.or_trace_rays(self.h, _ptr(o), _ptr(d), R, lod, _ptr(offs), None, None,
                              nthreads)
        vid = np.zeros(max(H, 1), np.int32)
        tr = np.zeros(max(2 * H, 2), np.float32)
        lib.or_trace_rays(self.h, _ptr(o), _ptr(d), R, lod, _ptr(offs), _ptr(vid),
                          _ptr(tr), nthreads)
        return offs, vid[:H], tr[:2 * H].reshape(-1, 2)

    # -- query / trace ----------------------------------------------------
    @staticmethod
    def _dec(dec):
        W1 = _f64(dec.W1)
        return (W1, _f64(dec.b1), _f64(dec.W2), float(dec.b2), int(W1.shape[1]),
                int(W1.shape[0]))

    def sdf_query(self, feats, dec, x, lod: int, grad: bool = False, nthreads: int = 0):
        fs = _PtrArray([_f64(f) for f in feats])
        m = int(fs.arrays[0].shape[1])
        W1, b1, W2, b2, ind, hid = self._dec(dec)
        x = np.ascontiguousarray(x, np.float32).reshape(-1, 3)
        Q = x.shape[0]
        sdf = np.zeros(Q)
        deep = np.zeros(Q, np.int32)
        g = np.zeros((Q, 3)) if grad else None
        _load().or_sdf_query(self.h, fs.p, m, _ptr(W1), _ptr(b1), _ptr(W2), b2, ind, hid,
                             _ptr(x), Q, lod, _ptr(sdf), _ptr(deep),
                             _ptr(g) if grad else None, nthreads)
        return (sdf, deep, g) if grad else (sdf, deep)

    def feature_sum(self, feats, x, lod: int):
        """z(x; lod) in FP64, [Q, m] (the decoder input of Eq. 2)."""
        fs = _PtrArray([_f64(f) for f in feats])
        m = int(fs.arrays[0].shape[1])
        x = np.ascontiguousarray(x, np.float32).reshape(-1, 3)
        z = np.zeros((x.shape[0], m))
        _load().or_feature_sum(self.h, fs.p, m, _ptr(x), x.shape[0], lod, _ptr(z))
        return z

    def sphere_trace(self, feats, dec, o, d, lod: int, eps: float = 1e-3,
                     far: float = 5.0, max_steps: int = 32, osc: bool = False,
                     nthreads: int = 0):
        fs = _PtrArray([_f64(f) for f in feats])
        m = int(fs.arrays[0].shape[1])
        W1, b1, W2, b2, ind, hid = self._dec(dec)
        o = np.ascontiguousarray(o, np.float32).reshape(-1, 3)
        d = np.ascontiguousarray(d, np.float32).reshape(-1, 3)
        R = o.shape[0]
        out = dict(t=np.zeros(R), hit=np.zeros(R, np.uint8), steps=np.zeros(R, np.int32),
                   x=np.zeros((R, 3)), normal=np.zeros((R, 3)))
        _load().or_sphere_trace(self.h, fs.p, m, _ptr(W1), _ptr(b1), _ptr(W2), b2, ind, hid,
                                _ptr(o), _ptr(d), R, lod, eps, far, max_steps, int(osc),
                                _ptr(out["t"]), _ptr(out["hit"]), _ptr(out["steps"]),
                                _ptr(out["x"]), _ptr(out["normal"]), nthreads)
        return out

    # -- level blending (Sec. 3.2, Eq. 3) ----------------------------------
    @staticmethod
    def split_lod(lod_tilde: float):
        """L* = floor(L~) and alpha = L~ - L* (Eq. 3)."""
        lstar = int(np.floor(lod_tilde))
        return lstar, float(lod_tilde) - lstar

    def sdf_query_blend(self, feats, dec_lo, dec_hi, x, lod_tilde: float):
        """Eq. 3 at the points x: (1 - alpha) sdf_{L*}(x) + alpha sdf_{L*+1}(x),
        each term the plain LOD query (dec_lo = LOD L*'s decoder, dec_hi =
        LOD L*+1's; alpha = 0 needs no dec_hi)."""
        lstar, alpha = self.split_lod(lod_tilde)
        lo, _ = self.sdf_query(feats, dec_lo, x, lstar)
        if alpha == 0.0:
            return lo
        hi, _ = self.sdf_query(feats, dec_hi, x, lstar + 1)
        return (1.0 - alpha) * lo + alpha * hi

    def fd_normals(self, feats, dec, x, lod, h: float, dec_hi=None, lod_tilde=None):
        """Normals by central differences (supplementary Sec. A.4 obtains the
        rendered normals by finite differences; the scheme and step are not
        given -- read here as central differences with step h): the SDF in
        FP64 at the points x + h e_a and x - h e_a, each coordinate rounded to
        FP32 as the points are formed, and n = the normalised vector of the
        three differences.  With ``lod_tilde`` the SDF is the Eq. 3 blend
        (dec = LOD floor(L~)'s decoder, dec_hi = the next one's)."""
        x = np.ascontiguousarray(x, np.float32).reshape(-1, 3)
        Q = x.shape[0]
        pts = np.repeat(x[:, None, :], 6, axis=1)
        for a in range(3):
            pts[:, 2 * a, a] = (x[:, a] + np.float32(h)).astype(np.float32)
            pts[:, 2 * a + 1, a] = (x[:, a] - np.float32(h)).astype(np.float32)
        pts = pts.reshape(-1, 3)
        if lod_tilde is None:
            f, _ = self.sdf_query(feats, dec, pts, lod)
        else:
            f = self.sdf_query_blend(feats, dec, dec_hi, pts, lod_tilde)
        f = f.reshape(Q, 6)
        g = f[:, 0::2] - f[:, 1::2]
        n = np.linalg.norm(g, axis=1, keepdims=True)
        return np.where(n > 0, g / np.where(n > 0, n, 1.0), 0.0)

    def sphere_trace_blend(self, feats, dec_lo, dec_hi, o, d, lod_tilde: float, eps: float = 1e-3,
                           far: float = 5.0, max_steps: int = 32, osc: bool = False, alpha=None,
                           nthreads: int = 0):
        """Sphere tracing of the Eq. 3 blend.  With alpha = 0 this is the
        plain trace at L*; otherwise rays walk their lists at L* + 1 and
        each step decodes both LODs at the same point.  ``alpha`` overrides
        the fractional part (the tests use alpha = 1 with L~ = L*)."""
        lstar, a = self.split_lod(lod_tilde)
        a = a if alpha is None else float(alpha)
        if a == 0.0:
            return self.sphere_trace(feats, dec_lo, o, d, lstar, eps=eps, far=far, max_steps=max_steps, osc=osc,
                                     nthreads=nthreads)
        fs = _PtrArray([_f64(f) for f in feats])
        m = int(fs.arrays[0].shape[1])
        W1l, b1l, W2l, b2l, ind, hid = self._dec(dec_lo)
        W1h, b1h, W2h, b2h, ind2, hid2 = self._dec(dec_hi)
        assert (ind, hid) == (ind2, hid2)
        o = np.ascontiguousarray(o, np.float32).reshape(-1, 3)
        d = np.ascontiguousarray(d, np.float32).reshape(-1, 3)
        R = o.shape[0]
        out = dict(t=np.zeros(R), hit=np.zeros(R, np.uint8), steps=np.zeros(R, np.int32),
                   x=np.zeros((R, 3)), normal=np.zeros((R, 3)))
        _load().or_sphere_trace_blend(self.h, fs.p, m, _ptr(W1l), _ptr(b1l), _ptr(W2l), b2l, _ptr(W1h),
                                      _ptr(b1h), _ptr(W2h), b2h, ind, hid, _ptr(o), _ptr(d), R, lstar + 1, a,
                                      eps, far, max_steps, int(osc), _ptr(out["t"]), _ptr(out["hit"]),
                                      _ptr(out["steps"]), _ptr(out["x"]), _ptr(out["normal"]), nthreads)
        return out

    def sdf_backward(self, feats, decs, x, lods, grad_sdf):
        """Gradients of sum_i sum_q grad_sdf[i, q] * sdf_{lods[i]}(x_q).

        ``decs`` is the list of per-LOD decoders (index lod - 1).  Returns a
        dict with float64 ``feats`` (per LOD), ``W1``, ``b1``, ``W2``, ``b2``
        (per LOD) and ``x``.
        """
        fs = _PtrArray([_f64(f) for f in feats])
        m = int(fs.arrays[0].shape[1])
        D = [self._dec(dd) for dd in decs]
        W1 = _PtrArray([t[0] for t in D])
        b1 = _PtrArray([t[1] for t in D])
        W2 = _PtrArray([t[2] for t in D])
        b2 = np.array([t[3] for t in D])
        ind, hid = D[0][4], D[0][5]
        x = np.ascontiguousarray(x, np.float32).reshape(-1, 3)
        Q = x.shape[0]
        lods = np.ascontiguousarray(lods, np.int32)
        gs = np.ascontiguousarray(grad_sdf, np.float64).reshape(len(lods), Q)
        gf = [np.zeros_like(a) for a in fs.arrays]
        gW1 = [np.zeros_like(t[0]) for t in D]
        gb1 = [np.zeros_like(t[1]) for t in D]
        gW2 = [np.zeros_like(t[2]) for t in D]
        gb2 = np.zeros(len(D))
        gx = np.zeros((Q, 3))
        GF, GW1, GB1, GW2 = (_PtrArray(a) for a in (gf, gW1, gb1, gW2))
        _load().or_sdf_backward(self.h, fs.p, m, W1.p, b1.p, W2.p, _ptr(b2), ind, hid,
                                _ptr(x), Q, _ptr(lods), len(lods), _ptr(gs), GF.p,
                                GW1.p, GB1.p, GW2.p, _ptr(gb2), _ptr(gx))
        return dict(feats=gf, W1=gW1, b1=gb1, W2=gW2, b2=gb2, x=gx)


def lod_select(distance, d_near: float, d_far: float, lod_near: float, lod_far: float):
    """LOD selection of Sec. 3.4: the continuous LOD moves linearly from
    lod_near (distance <= d_near) to lod_far (distance >= d_far)."""
    dist = np.asarray(distance, np.float64)
    s = np.clip((dist - d_near) / (d_far - d_near), 0.0, 1.0)
    return lod_near + s * (lod_far - lod_near)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
