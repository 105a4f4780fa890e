"""svo_trace_rays_noalloc: the traversal for callers that cannot allocate.

Renderers embedded in an application that owns the GPU memory budget, or
frame loops that must not trigger the device-wide synchronisation a
cudaMalloc/cudaFree can cause, call this variant: it takes only inputs and
outputs and keeps its workspace in a fixed array inside the library.  Its
lists must equal those of svo_trace_rays (which uses a caller workspace) bit
for bit, on two calls in a row of different sizes -- the second call runs on
whatever the first left in the shared array.  This file is collected last so
a failure here never hides another test's result.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2101_10994_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def noalloc_lists(ng, svo, o, d, lod, hit_capacity):
    to = torch.from_numpy(np.ascontiguousarray(o, np.float32)).cuda()
    td = torch.from_numpy(np.ascontiguousarray(d, np.float32)).cuda()
    R = len(o)
    offs = torch.empty(R + 1, dtype=torch.int32, device="cuda")
    vid = torch.empty(max(hit_capacity, 1), dtype=torch.int32, device="cuda")
    tr = torch.empty((max(hit_capacity, 1), 2), dtype=torch.float32, device="cuda")
    stats = (ctypes.c_int64 * 2)()
    rc = ng.lib().svo_trace_rays_noalloc(svo.h, to.data_ptr(), td.data_ptr(), R, lod, offs.data_ptr(),
                                         vid.data_ptr(), tr.data_ptr(), hit_capacity, stats,
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    ng._check(rc)
    H = int(stats[0])
    return offs.cpu().numpy(), vid[:H].cpu().numpy(), tr[:H].cpu().numpy()


def reference_lists(ng, svo, o, d, lod):
    L = ng.svo_trace_rays(svo, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), lod)
    return L.ray_offsets.cpu().numpy(), L.voxel_id.cpu().numpy(), L.t_range.cpu().numpy()


def test_noalloc_matches_caller_workspace_twice(ng):
    sc1, oc1 = S.csg_workload(16, seed=3, max_lod=3)
    sc2, oc2 = S.plain_sphere(3)
    cases = [(oc1, S.camera_rays(96, 80, tile=8), 3), (oc2, S.camera_rays(128, 128), 2)]
    for oc, (o, d, _), lod in cases:
        svo = ng.svo_build(oc.keys)
        ref = reference_lists(ng, svo, o, d, lod)
        got = noalloc_lists(ng, svo, o, d, lod, hit_capacity=len(ref[1]) + 16)
        np.testing.assert_array_equal(got[0], ref[0])
        np.testing.assert_array_equal(got[1], ref[1])
        np.testing.assert_array_equal(got[2].view(np.uint32), ref[2].view(np.uint32))
        assert len(ref[1]) > 1000
        svo.free()


def test_noalloc_rejects_rays_beyond_its_scratch(ng):
    sc, oc = S.plain_sphere(3)
    svo = ng.svo_build(oc.keys)
    # the fixed part of the workspace (a count per ray, a record per tile of
    # 128 rays) for 2^31 - 2 rays is ~8.9 GB, far more than the 32 MiB array:
    # rejected on the host before anything is read or launched (the NULL ray
    # and offset pointers are never reached; with no size check they would be
    # rejected as invalid arguments, also before any launch)
    R = (1 << 31) - 2
    assert ng.lib().svo_trace_rays_workspace(R, 0) > 32 << 20
    assert ng.lib().svo_trace_rays_workspace(2_000_000, 0) < 32 << 20
    rc = ng.lib().svo_trace_rays_noalloc(svo.h, None, None, R, 3, None, None, None, 0, None,
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == ng.ERR_CAPACITY
    assert b"32 MiB" in ng.lib().nglod_last_error()
    svo.free()
