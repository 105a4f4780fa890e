"""svo_trace_rays (Algorithm 1 on the GPU) vs the oracle's brute-force lists:
bit-exact voxel ids, order and FP32 (t_enter, t_exit) bits."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2101_10994_gb300 import scenes as S

from traverse_paths import pairs_by_depth, tile_paths

pytestmark = pytest.mark.gpu


def gpu_lists(ng, svo, o, d, lod, **kw):
    to = torch.from_numpy(np.ascontiguousarray(o, np.float32)).cuda()
    td = torch.from_numpy(np.ascontiguousarray(d, np.float32)).cuda()
    L = ng.svo_trace_rays(svo, to, td, lod, **kw)
    return (L.ray_offsets.cpu().numpy().astype(np.int64), L.voxel_id.cpu().numpy(),
            L.t_range.cpu().numpy(), L)


def assert_same_lists(g, o):
    np.testing.assert_array_equal(g[0], o[0])
    np.testing.assert_array_equal(g[1], o[1])
    np.testing.assert_array_equal(g[2].view(np.uint32), o[2].view(np.uint32))


@pytest.mark.parametrize("lod", [1, 2, 3])
def test_plain_sphere_128(ng, oracle_mod, lod):
    sc, oc = S.plain_sphere(3)
    svo = ng.svo_build(oc.keys)
    ora = oracle_mod.OracleSVO(oc.keys)
    o, d, _ = S.camera_rays(128, 128)
    assert_same_lists(gpu_lists(ng, svo, o, d, lod), ora.trace_rays(o, d, lod))


def test_axis_aligned_view_and_ties(ng, oracle_mod):
    # eye on the z axis: many rays run exactly along octree centre planes
    sc, oc = S.csg_workload(16, seed=2, max_lod=3)
    svo = ng.svo_build(oc.keys)
    ora = oracle_mod.OracleSVO(oc.keys)
    o, d, _ = S.camera_rays(65, 65, eye=(0.0, 0.0, 2.5))
    assert_same_lists(gpu_lists(ng, svo, o, d, 3), ora.trace_rays(o, d, 3))
    dense = S.full_octree(4)
    svo2 = ng.svo_build(dense.keys)
    ora2 = oracle_mod.OracleSVO(dense.keys)
    ys = np.linspace(-1, 1, 17)
    oo = np.array([[-3.0, y, z] for y in ys for z in ys], np.float32)
    dd = np.tile(np.array([[1.0, 0.0, 0.0]], np.float32), (len(oo), 1))
    assert_same_lists(gpu_lists(ng, svo2, oo, dd, 2), ora2.trace_rays(oo, dd, 2))


def test_degenerate_rays_and_empty(ng, oracle_mod):
    sc, oc = S.plain_sphere(3)
    svo = ng.svo_build(oc.keys)
    ora = oracle_mod.OracleSVO(oc.keys)
    o = np.array([[np.nan, 0, 0], [-3, 0.1, 0.1], [-3, 0.1, 0.1], [-3, 5.0, 0.1], [0.3, 0.05, 0.05],
                  [0.0, 0.0, 0.0], [3, 3, 3], [-2, 0.2, 0.1]], np.float32)
    d = np.array([[1, 0, 0], [0, 0, 0], [np.nan, 0, 0], [1, 0, 0], [0, 0, 1], [1, 1e-39, 0],
                  [1, 0, 0], [1, 1e-30, -1e-30]], np.float32)
    assert_same_lists(gpu_lists(ng, svo, o, d, 3), ora.trace_rays(o, d, 3))
    g = gpu_lists(ng, svo, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), 2)
    assert g[0].tolist() == [0] and g[1].size == 0


def test_capacity_growth(ng, oracle_mod):
    sc, oc = S.csg_workload(16, seed=4, max_lod=3)
    svo = ng.svo_build(oc.keys)
    ora = oracle_mod.OracleSVO(oc.keys)
    o, d, _ = S.camera_rays(64, 48)
    to = torch.from_numpy(o).cuda()
    td = torch.from_numpy(d).cuda()
    with pytest.raises(ng.NglodError) as e:
        import ctypes
        L = ng.lib()
        cap = 64
        work = torch.empty(L.svo_trace_rays_workspace(len(o), cap), dtype=torch.uint8, device="cuda")
        offs = torch.empty(len(o) + 1, dtype=torch.int32, device="cuda")
        vid = torch.empty(cap, dtype=torch.int32, device="cuda")
        tr = torch.empty((cap, 2), dtype=torch.float32, device="cuda")
        stats = (ctypes.c_int64 * 2)()
        ng._check(L.svo_trace_rays(svo.h, to.data_ptr(), td.data_ptr(), len(o), 3, work.data_ptr(),
                                   work.numel(), cap, offs.data_ptr(), vid.data_ptr(), tr.data_ptr(), cap,
                                   stats, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    assert e.value.code == ng.ERR_CAPACITY
    # the binding grows the capacity and the result is exact
    assert_same_lists(gpu_lists(ng, svo, o, d, 3, pair_capacity=64), ora.trace_rays(o, d, 3))


def test_full_size_1080p_lod5_sampled(ng, oracle_mod):
    # the benchmark's workload: CSG-64, LOD 5, 1920x1080, in its launch setup
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    svo = ng.svo_build(oc.keys)
    o, d, _ = S.camera_rays(1920, 1080, tile=8)
    g = gpu_lists(ng, svo, o, d, 5)
    ora = oracle_mod.OracleSVO(oc.keys)
    rng = np.random.default_rng(0)
    hit_rays = np.nonzero(np.diff(g[0]) > 0)[0]
    pick = np.concatenate([rng.choice(hit_rays, 300, replace=False), rng.choice(len(o), 100, replace=False)])
    offs, vid, tr = ora.trace_rays(o[pick], d[pick], 5)
    for n, r in enumerate(pick):
        a, b = g[0][r], g[0][r + 1]
        np.testing.assert_array_equal(g[1][a:b], vid[offs[n]:offs[n + 1]])
        np.testing.assert_array_equal(g[2][a:b].view(np.uint32), tr[offs[n]:offs[n + 1]].view(np.uint32))
    # invariants over every ray: CSR monotone, ids in range, t_enter <= t_exit
    assert np.all(np.diff(g[0]) >= 0) and g[0][-1] == len(g[1])
    assert g[1].min() >= 0 and g[1].max() < oc.counts()[7]
    assert np.all(g[2][:, 0] <= g[2][:, 1])
    # the frame renderer's variant (no t ranges): identical CSR lists
    L2 = ng.svo_trace_rays(svo, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), 5, t_range=False)
    np.testing.assert_array_equal(L2.ray_offsets.cpu().numpy(), g[0])
    np.testing.assert_array_equal(L2.voxel_id.cpu().numpy(), g[1])


def test_dense_grid_frontier_overflow_path(ng, oracle_mod):
    # every voxel of a dense depth-6 grid is occupied: a ray crossing the cube
    # meets ~100-190 voxels per level, so 128 rays overflow the on-chip
    # frontier and the traversal continues those tiles in chunks of rays;
    # the lists must still equal the brute-force ones bit for bit
    dense = S.full_octree(6)
    svo = ng.svo_build(dense.keys)
    ora = oracle_mod.OracleSVO(dense.keys)
    rng = np.random.default_rng(9)
    n = 300
    o = np.tile(np.array([[-2.5, 0.05, -0.1]], np.float32), (n, 1)) + rng.uniform(-0.3, 0.3, (n, 3)).astype(np.float32)
    tgt = rng.uniform(-0.6, 0.6, (n, 3))
    d = (tgt - o).astype(np.float64)
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    assert tile_paths(pairs_by_depth(ora, o, d, 6), 6) == ["chunks", "chunks", "whole"]
    g = gpu_lists(ng, svo, o, d, 4)
    assert np.diff(g[0]).mean() > 60
    assert_same_lists(g, ora.trace_rays(o, d, 4))
    sizes = g[3].level_sizes()
    assert sizes[-1] == len(g[1]) and sizes[0] == n


def test_dense_grid_every_overflow_path(ng, oracle_mod):
    # rays near the cube's main diagonal cross ~3 x 2^dp voxels per depth: the
    # first tile overflows early, and one of its chunks overflows again
    # further down (its rays then run from the root over halving ranges); the
    # second continues in chunks; the third (rays running along one edge of
    # the cube) fits whole.  Lists bit-exact, and every depth's pair count (each
    # counted once whatever the path) equal to the brute-force list lengths.
    dense = S.full_octree(6)
    svo = ng.svo_build(dense.keys)
    ora = oracle_mod.OracleSVO(dense.keys)
    rng = np.random.default_rng(1)
    o = np.full((256, 3), -2.0, np.float32) + rng.uniform(-0.2, 0.2, (256, 3)).astype(np.float32)
    d = rng.uniform(-0.2, 0.2, (256, 3)) - o
    o2 = np.tile(np.array([[-2.0, 0.97, 0.97]], np.float32), (70, 1))
    d2 = np.stack([np.ones(70), rng.uniform(-0.01, 0.01, 70), rng.uniform(-0.01, 0.01, 70)], 1)
    o = np.concatenate([o, o2])
    d = np.concatenate([d, d2])
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    P = pairs_by_depth(ora, o, d, 6)
    assert tile_paths(P, 6) == ["halving", "chunks", "whole"]
    g = gpu_lists(ng, svo, o, d, 4)
    assert_same_lists(g, ora.trace_rays(o, d, 4))
    sizes = g[3].level_sizes()
    assert sizes[0] == len(o)
    assert sizes[3:] == [int(v) for v in P.sum(0)[3:]]
    # without t ranges (the kernel variant the frame renderer runs): the same
    # lists and level sizes on every path
    L2 = ng.svo_trace_rays(svo, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), 4, t_range=False)
    assert L2.t_range is None
    np.testing.assert_array_equal(L2.ray_offsets.cpu().numpy(), g[0])
    np.testing.assert_array_equal(L2.voxel_id.cpu().numpy(), g[1])
    assert L2.level_sizes() == sizes
    # staged (no placement pass): each ray's entries where the traversal
    # staged them -- the same entries on every path, the same level sizes
    assert_staged_lists(ng, svo, o, d, 4, L2)
    svo.free()


def assert_staged_lists(ng, svo, o, d, lod, L):
    """svo_trace_rays_staged: ray by ray equal to the CSR lists L, with the
    same level sizes and status, and a trace over them bit-identical to one
    over L."""
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    cap = int(L.voxel_id.numel()) + 1024
    work = torch.empty(ng.lib().svo_trace_rays_workspace(len(o), cap), dtype=torch.uint8, device="cuda")
    St = ng.svo_trace_rays_staged(svo, to, td, lod, work, cap)
    stats = (C.c_int64 * 2)()
    ng._check(ng.lib().svo_trace_rays_check(work.data_ptr(), lod, stats, None))
    assert stats[0] == L.voxel_id.numel()
    assert St.level_sizes() == L.level_sizes()
    offs = L.ray_offsets.long()
    cnt = St.ray_counts.long()
    assert torch.equal(cnt, offs[1:] - offs[:-1])
    H = int(offs[-1])
    start = torch.repeat_interleave(St.ray_offsets.long(), cnt)
    within = torch.arange(H, device="cuda") - torch.repeat_interleave(offs[:-1], cnt)
    assert torch.equal(St.voxel_id[start + within], L.voxel_id)
    return St


def test_staged_lists_and_trace(ng, oracle_mod):
    # the 1080p-style camera on the CSG scene (tiles staged whole) and a
    # trace over the staged lists: every output bit-identical to CSR lists
    sc, oc = S.csg_workload(16, seed=2, max_lod=4)
    svo = ng.svo_build(oc.keys)
    o, d, _ = S.camera_rays(320, 200, tile=8)
    L = ng.svo_trace_rays(svo, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), 4, t_range=False)
    St = assert_staged_lists(ng, svo, o, d, 4, L)
    F = ng.Features(S.readout_features(oc, sc))
    D = ng.DecoderDev.from_decoder(S.readout_decoder(4))
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    for decode in ("f32", "bf16"):
        a = ng.sphere_trace(svo, F, D, to, td, L, decode=decode, normals=True)
        b = ng.sphere_trace(svo, F, D, to, td, St, decode=decode, normals=True)
        assert int(a["hit"].sum()) > 1000
        for k in ("t", "hit", "steps", "normal"):
            assert torch.equal(a[k], b[k]), (decode, k)
    # a capacity below the entries is reported, not overrun
    small = 64
    work = torch.empty(ng.lib().svo_trace_rays_workspace(len(o), small), dtype=torch.uint8, device="cuda")
    ng.svo_trace_rays_staged(svo, to, td, 4, work, small)
    stats = (C.c_int64 * 2)()
    assert ng.lib().svo_trace_rays_check(work.data_ptr(), 4, stats, None) == ng.ERR_CAPACITY
    # after an overflow every list a reader sees is whole: the rays whose
    # lists did not fit get none (misses), the others trace as before
    half = int(L.voxel_id.numel()) // 2
    work = torch.empty(ng.lib().svo_trace_rays_workspace(len(o), half), dtype=torch.uint8, device="cuda")
    Sh = ng.svo_trace_rays_staged(svo, to, td, 4, work, half)
    assert ng.lib().svo_trace_rays_check(work.data_ptr(), 4, stats, None) == ng.ERR_CAPACITY
    cnt, first = Sh.ray_counts.long(), Sh.ray_offsets.long()
    full = (L.ray_offsets[1:] - L.ray_offsets[:-1]).long()
    kept = cnt > 0
    assert torch.all(first[kept] + cnt[kept] <= half)
    assert torch.equal(cnt[kept], full[kept]) and 0 < int(kept.sum()) < int((full > 0).sum())
    a = ng.sphere_trace(svo, F, D, to, td, L, decode="bf16", normals=True)
    b = ng.sphere_trace(svo, F, D, to, td, Sh, decode="bf16", normals=True)
    ng.sphere_trace_status(b)
    for k in ("t", "hit", "steps", "normal"):
        assert torch.equal(a[k][kept], b[k][kept]), k
    assert int(b["hit"][~kept].sum()) == 0
    # the CSR lists of an overflowed asynchronous traversal are empty
    R = len(o)
    work = torch.empty(ng.lib().svo_trace_rays_workspace(R, 2 * int(L.voxel_id.numel())), dtype=torch.uint8,
                       device="cuda")
    offs = torch.full((R + 1,), 7, dtype=torch.int32, device="cuda")
    vid = torch.empty(half, dtype=torch.int32, device="cuda")
    ng._check(ng.lib().svo_trace_rays_async(svo.h, to.data_ptr(), td.data_ptr(), R, 4, work.data_ptr(), work.numel(),
                                            2 * int(L.voxel_id.numel()), offs.data_ptr(), vid.data_ptr(), None,
                                            half, None))
    assert ng.lib().svo_trace_rays_check(work.data_ptr(), 4, stats, None) == ng.ERR_CAPACITY
    assert int(offs.abs().sum()) == 0
    svo.free()


def test_async_width_rejects_bad_width(ng):
    import ctypes as C
    sc, oc = S.plain_sphere(3)
    svo = ng.svo_build(oc.keys)
    o, d, _ = S.camera_rays(16, 16)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    L = ng.lib()
    R, cap = len(o), 1 << 14
    work = torch.empty(L.svo_trace_rays_workspace(R, cap), dtype=torch.uint8, device="cuda")
    offs = torch.empty(R + 1, dtype=torch.int32, device="cuda")
    vid = torch.empty(cap, dtype=torch.int32, device="cuda")
    tr = torch.empty((cap, 2), dtype=torch.float32, device="cuda")
    for w in (-1, 5):
        rc = L.svo_trace_rays_async_width(svo.h, to.data_ptr(), td.data_ptr(), R, 3, work.data_ptr(), work.numel(),
                                          cap, offs.data_ptr(), vid.data_ptr(), tr.data_ptr(), cap, w,
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == ng.ERR_INVALID_ARG
    svo.free()
