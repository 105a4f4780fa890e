"""Bounded tensor-core waits run out without faulting or hanging the GPU.

Every tcgen05 kernel waits for each tile's MMA with a poll budget; on
expiry it raises its status word, waits for the MMA in flight (default
budget), frees its tensor memory and returns, and the call reports
NGLOD_ERR_TIMEOUT.  nglod_set_wait_polls(0) makes the per-tile wait expire
at once, so this is a device-side wait with a short limit, made to run out
by the test.  For each tcgen05 call: the expired call reports
NGLOD_ERR_TIMEOUT and names itself in nglod_last_error, and the same call
with the default budget right after is bit-identical to a clean run (no
state of the expired call leaks into the next one).  The BF16 and
three-term FP32 tracers decode with warp-level MMAs, which complete in the
issuing warp: they have no device wait, and a zero budget leaves their
results unchanged.
"""
import numpy as np
import pytest
import torch

from paper_2101_10994_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene(ng):
    sc, oc = S.csg_workload(16, seed=5, max_lod=4)
    svo = ng.svo_build(oc.keys)
    feats = S.readout_features(oc, sc)
    o, d, _ = S.camera_rays(160, 120, tile=8)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    lists = ng.svo_trace_rays(svo, to, td, 4)
    yield dict(sc=sc, oc=oc, svo=svo, feats=feats, F=ng.Features(feats), o=to, d=td, lists=lists,
               dec=ng.DecoderDev.from_decoder(S.readout_decoder(4)))
    svo.free()


@pytest.fixture
def expire(ng):
    """Sets the per-tile MMA wait budget to 0 for the duration of a block and
    always restores the default."""
    class _Expire:
        def __enter__(self):
            ng.set_wait_polls(0)

        def __exit__(self, *exc):
            ng.set_wait_polls(-1)
    yield _Expire()
    ng.set_wait_polls(-1)


def same(a, b):
    a, b = a.cpu(), b.cpu()
    if a.dtype.is_floating_point:
        a, b = a.view(torch.int32), b.view(torch.int32)
    return torch.equal(a, b)


@pytest.mark.parametrize("decode", ["fp8"])
def test_sphere_trace_timeout(ng, scene, expire, decode):
    if decode == "fp8":
        scene["F"].set_fp8_bound(scene["svo"], 4)
    args = (scene["svo"], scene["F"], scene["dec"], scene["o"], scene["d"], scene["lists"])
    kw = dict(eps=1e-3, max_steps=128, decode=decode, normals=True)
    clean = ng.sphere_trace(*args, **kw)
    ng.sphere_trace_status(clean)
    clean = {k: v.clone() for k, v in clean.items() if k in ("t", "hit", "steps", "normal")}
    assert int(clean["hit"].sum()) > 500
    with expire:
        out = ng.sphere_trace(*args, **kw)
        with pytest.raises(ng.NglodError) as e:
            ng.sphere_trace_status(out)
    assert e.value.code == ng.ERR_TIMEOUT
    assert "sphere_trace" in str(e.value) and "expired" in str(e.value)
    again = ng.sphere_trace(*args, out=out, **kw)
    ng.sphere_trace_status(again)
    for k in clean:
        assert same(again[k], clean[k]), k


@pytest.mark.parametrize("decode", ["bf16", "f32tc"])
def test_warp_tracers_have_no_wait(ng, scene, expire, decode):
    from paper_2101_10994_gb300 import batch as B
    args = (scene["svo"], scene["F"], scene["dec"], scene["o"], scene["d"], scene["lists"])
    kw = dict(eps=1e-3, max_steps=128, decode=decode, normals=True)
    clean = ng.sphere_trace(*args, **kw)
    ng.sphere_trace_status(clean)
    clean = {k: v.clone() for k, v in clean.items() if k in ("t", "hit", "steps", "normal")}
    assert int(clean["hit"].sum()) > 500
    rnd = None
    if decode == "bf16":
        rnd = B.BatchRenderer([B.Job(scene["svo"], scene["F"], scene["dec"], 4, scene["o"], scene["d"])],
                              decode="bf16")
    with expire:
        out = ng.sphere_trace(*args, **kw)
        ng.sphere_trace_status(out)
        if rnd is not None:
            rnd.frame()
            rnd.check()
    for k in clean:
        assert same(out[k], clean[k]), k
        if rnd is not None:
            assert same(rnd.outputs(0)[k], clean[k]), k
    if rnd is not None:
        rnd.free()


def test_sdf_query_timeout(ng, scene, expire):
    x = torch.from_numpy(np.concatenate([S.points_in_voxels(scene["oc"], 6, 3000, 1),
                                         S.uniform_points(500, 2)])).cuda()
    clean = ng.sdf_query(scene["svo"], scene["F"], scene["dec"], x, 4, decode="bf16")
    with expire:
        with pytest.raises(ng.NglodError) as e:
            ng.sdf_query(scene["svo"], scene["F"], scene["dec"], x, 4, decode="bf16")
    assert e.value.code == ng.ERR_TIMEOUT and "sdf_query" in str(e.value)
    assert same(ng.sdf_query(scene["svo"], scene["F"], scene["dec"], x, 4, decode="bf16"), clean)


def test_blend_timeout(ng, scene, expire):
    lo = ng.DecoderDev.from_decoder(S.readout_decoder(3))
    x = torch.from_numpy(S.points_in_voxels(scene["oc"], 6, 2000, 4)).cuda()
    clean = ng.sdf_query_blend(scene["svo"], scene["F"], lo, scene["dec"], x, 3.5, decode="bf16")
    with expire:
        with pytest.raises(ng.NglodError) as e:
            ng.sdf_query_blend(scene["svo"], scene["F"], lo, scene["dec"], x, 3.5, decode="bf16")
    assert e.value.code == ng.ERR_TIMEOUT and "sdf_query_blend" in str(e.value)
    assert same(ng.sdf_query_blend(scene["svo"], scene["F"], lo, scene["dec"], x, 3.5, decode="bf16"), clean)


def test_batch_timeout(ng, scene, expire):
    # the FP8 batch decode runs on tcgen05
    from paper_2101_10994_gb300 import batch as B
    scene["F"].set_fp8_bound(scene["svo"], 4)
    jobs = [B.Job(scene["svo"], scene["F"], scene["dec"], 4, scene["o"], scene["d"]),
            B.Job(scene["svo"], scene["F"], scene["dec"], 4, scene["o"][:777].contiguous(),
                  scene["d"][:777].contiguous())]
    rnd = B.BatchRenderer(jobs, decode="fp8")
    rnd.frame()
    rnd.check()
    clean = [{k: v.clone() for k, v in rnd.outputs(i).items()} for i in range(len(jobs))]
    with expire:
        rnd.frame()
        with pytest.raises(ng.NglodError) as e:
            rnd.check()
    assert e.value.code == ng.ERR_TIMEOUT and "sphere_trace_batch" in str(e.value)
    rnd.frame()
    rnd.check()
    for i in range(len(jobs)):
        for k, v in rnd.outputs(i).items():
            assert same(v, clean[i][k]), (i, k)
    rnd.free()


def test_tc_backward_timeout(ng, scene, expire):
    svo, oc, sc = scene["svo"], scene["oc"], scene["sc"]
    decs = [ng.DecoderDev.from_decoder(S.init_decoder(l, 32)) for l in range(1, 5)]
    x = torch.from_numpy(S.points_in_voxels(oc, 6, 4096, 7)).cuda()
    target = torch.from_numpy(S.scene_sdf(sc, x.cpu().numpy()).astype(np.float32)).cuda()

    def run():
        grads = ng.new_grads(svo, decs)
        loss = torch.zeros(4, dtype=torch.float32, device="cuda")
        ng.sdf_l2_backward(svo, scene["F"], decs, x, target, [2, 4], 1.0 / 4096, grads, loss, mma="bf16")
        torch.cuda.synchronize()
        return grads, loss

    with expire:
        with pytest.raises(ng.NglodError) as e:
            run()
    assert e.value.code == ng.ERR_TIMEOUT and "sdf_l2_backward_bf16" in str(e.value)
    # atomics make the FP32 sums' rounding order vary between runs, so the
    # recovered call is compared with a clean one within a relative 1e-5
    g1, l1 = run()
    g2, l2 = run()
    assert torch.allclose(l1, l2, rtol=1e-5, atol=0)
    for key in ("W1", "b1", "W2"):
        for a, b in zip(g1[key], g2[key]):
            assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * float(b.abs().max()) + 1e-12), key
    assert torch.allclose(g1["b2"], g2["b2"], rtol=1e-4, atol=1e-9)
