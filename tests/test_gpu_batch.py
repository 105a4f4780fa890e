"""Batched multi-scene tracing (one persistent launch over many images of
uneven size, traversals enqueued without host synchronisation, the frame
captured in a CUDA graph) against per-image calls.

The batched path runs the same per-ray arithmetic as sphere_trace (the
stepping rules of Sec. 3.4 / A.4) and differs only in which CTA takes which
ray, so every output -- hit mask, hit depth, step count, normal, and the
traversal lists (staged; the same entries ray by ray) -- must be
bit-identical to the per-image calls.  Per-image
sphere_trace itself is checked against the oracle elsewhere; one job here is
also checked against the oracle directly.
"""
import numpy as np
import pytest
import torch

from paper_2101_10994_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def make_jobs(ng, items, decode, in_dim=32, fdt="f32"):
    from paper_2101_10994_gb300 import batch as B
    decs = {}
    jobs = []
    for sc, oc, lod, w, h, feats in items:
        svo = ng.svo_build(oc.keys)
        if fdt == "f16":
            feats = [f.astype(np.float16) for f in feats]
        F = ng.Features(feats, fdt)
        if lod not in decs:                          # one decoder per LOD, shared by its scenes
            decs[lod] = ng.DecoderDev.from_decoder(S.readout_decoder(lod, in_dim=in_dim))
        o, d, _ = S.camera_rays(w, h, tile=8)
        jobs.append(B.Job(svo, F, decs[lod], lod, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()))
    if decode == "fp8":
        # one z bound per decoder group (the batch scales a group by the
        # largest bound of its members), so set every member to that bound
        for lod in decs:
            members = [j for j in jobs if j.lod == lod]
            b = max(j.feats.set_fp8_bound(j.svo, lod) for j in members)
            for j in members:
                j.feats.z_absmax = b
    return jobs


def per_job(ng, j, decode):
    lists = ng.svo_trace_rays(j.svo, j.o, j.d, j.lod)
    out = ng.sphere_trace(j.svo, j.feats, j.dec, j.o, j.d, lists, eps=1e-3, far=5.0, max_steps=128,
                          decode=decode, normals=True)
    ng.sphere_trace_status(out)
    return lists, out


def assert_same(r, lists, ref, bufs=None):
    for k in ("t", "hit", "steps", "normal"):
        a, b = r[k].cpu(), ref[k].cpu()
        assert torch.equal(a.view(torch.uint8) if a.dtype == torch.float32 else a,
                           b.view(torch.uint8) if b.dtype == torch.float32 else b), k
    if bufs is not None:
        # the job's staged lists hold, ray by ray, the CSR lists' entries
        St = bufs["lists"]
        offs = lists.ray_offsets.long()
        cnt = St.ray_counts.long()
        assert torch.equal(cnt, offs[1:] - offs[:-1])
        start = torch.repeat_interleave(St.ray_offsets.long(), cnt)
        within = torch.arange(int(offs[-1]), device=cnt.device) - torch.repeat_interleave(offs[:-1], cnt)
        assert torch.equal(St.voxel_id[start + within], lists.voxel_id)


@pytest.fixture(scope="module")
def items():
    # 6 scenes, 8..64 primitives, LOD 2..4, images 40..200 a side (ragged tiles)
    return S.batching_workload(6, seed=3, min_prims=8, max_prims=64, min_lod=2, max_lod=4,
                               min_side=40, max_side=200)


@pytest.mark.parametrize("decode", ["f32", "bf16", "fp8"])
def test_batch_equals_per_job(ng, items, decode):
    from paper_2101_10994_gb300 import batch as B
    jobs = make_jobs(ng, items, decode)
    assert len({j.lod for j in jobs}) >= 2 and len({j.lod for j in jobs}) < len(jobs)   # groups of several jobs
    rnd = B.BatchRenderer(jobs, decode=decode)
    rnd.frame()
    rnd.check()
    for k, j in enumerate(jobs):
        lists, ref = per_job(ng, j, decode)
        assert int(ref["hit"].sum()) > 0
        assert_same(rnd.outputs(k), lists, ref, rnd.bufs[k])
    rnd.free()


def test_batch_f16_features_in35(ng, items):
    from paper_2101_10994_gb300 import batch as B
    jobs = make_jobs(ng, items[:4], "bf16", in_dim=35, fdt="f16")
    rnd = B.BatchRenderer(jobs, decode="bf16")
    rnd.frame()
    rnd.check()
    for k, j in enumerate(jobs):
        lists, ref = per_job(ng, j, "bf16")
        assert_same(rnd.outputs(k), lists, ref)


def test_batch_graph_replay_and_autotune(ng, items):
    from paper_2101_10994_gb300 import batch as B
    jobs = make_jobs(ng, items, "bf16")
    rnd = B.BatchRenderer(jobs, decode="bf16")
    best, timings = B.autotune(rnd, streams=[0, 2], reps=2)
    assert best[0] in (1, 2, 3, 4) and best[1] in (0, 2)
    assert set(timings) == {f"{c}/{n}" for c in (1, 2, 3, 4) for n in (0, 2)}
    rnd.frame()
    rnd.check()
    first = [{k: v.clone() for k, v in rnd.outputs(i).items()} for i in range(len(jobs))]
    rnd.capture()
    for i in range(len(jobs)):
        for v in rnd.outputs(i).values():
            v.fill_(7)
    for _ in range(3):
        rnd.replay()
    torch.cuda.synchronize()
    rnd.check()
    for i in range(len(jobs)):
        for k, v in rnd.outputs(i).items():
            assert torch.equal(v, first[i][k]), (i, k)
    rnd.free()


def test_batch_one_job_vs_oracle(ng, oracle_mod, items):
    from paper_2101_10994_gb300 import batch as B
    sc, oc, lod, w, h, feats = items[0]
    jobs = make_jobs(ng, [items[0], items[1]], "f32")
    rnd = B.BatchRenderer(jobs, decode="f32")
    rnd.frame()
    rnd.check()
    o, d, _ = S.camera_rays(w, h, tile=8)
    sel = np.random.default_rng(0).choice(len(o), min(800, len(o)), replace=False)
    ora = oracle_mod.OracleSVO(oc.keys)
    ref = ora.sphere_trace(feats, S.readout_decoder(lod), o[sel], d[sel], lod, eps=1e-3, far=5.0, max_steps=128)
    g = {k: v.cpu().numpy()[sel] for k, v in rnd.outputs(0).items()}
    gh, rh = g["hit"].astype(bool), ref["hit"].astype(bool)
    assert int((gh != rh).sum()) <= 1
    both = gh & rh
    assert both.sum() > 50
    assert np.abs(g["t"][both] - ref["t"][both]).max() <= 1e-3
    rnd.free()


def test_batch_rejects_mixed_in_dim(ng, items):
    from paper_2101_10994_gb300 import batch as B
    jobs = make_jobs(ng, items[:2], "f32")
    jobs[1].dec = ng.DecoderDev.from_decoder(S.readout_decoder(jobs[1].lod, in_dim=35))
    with pytest.raises(ng.NglodError):
        B.BatchRenderer(jobs, decode="f32")


def test_batch_tiny_jobs_padding(ng, items):
    # jobs of 1 and 33 rays between larger ones of the same decoder group: each
    # job's queue range is padded to 32-ray chunks, and the padding must start
    # no ray and disturb no neighbour
    from paper_2101_10994_gb300 import batch as B
    sc, oc, lod, w, h, feats = items[0]
    tiny = [(sc, oc, lod, 1, 1, feats), (sc, oc, lod, 11, 3, feats)]
    jobs = make_jobs(ng, [items[0]] + tiny + [items[0]], "bf16")
    assert len({j.lod for j in jobs}) == 1
    rnd = B.BatchRenderer(jobs, decode="bf16")
    rnd.frame()
    rnd.check()
    for k, j in enumerate(jobs):
        lists, ref = per_job(ng, j, "bf16")
        assert_same(rnd.outputs(k), lists, ref, rnd.bufs[k])
    rnd.free()


def test_batch_full_workload_equals_per_scene(ng):
    # the benchmark's batching workload (32 seeded CSG scenes, LOD 3..6,
    # images 128..1024 a side) in its timed configuration (autotuned trace
    # width and side streams, CUDA-graph replay): every output bit-identical
    # to the per-scene calls (whose parity with the oracle is tested above);
    # one job's sampled pixels also against the oracle
    import os
    from paper_2101_10994_gb300 import batch as B
    items = S.batching_workload(32, seed=0, workers=min(16, os.cpu_count() or 1))
    jobs = make_jobs(ng, items, "bf16")
    rnd = B.BatchRenderer(jobs, decode="bf16")
    B.autotune(rnd, streams=[0, 8], reps=1)
    rnd.frame()
    rnd.check()
    rnd.capture()
    rnd.replay()
    torch.cuda.synchronize()
    rnd.check()
    for k, j in enumerate(jobs):
        lists, ref = per_job(ng, j, "bf16")
        assert_same(rnd.outputs(k), lists, ref)
    rnd.free()


@pytest.mark.parametrize("decode", ["f32", "bf16"])
def test_batch_summed_tables_equal_per_job(ng, items, decode):
    # every other job reads the summed corner table of its LOD: the batch
    # takes each job's gather depth from that job's tables
    from paper_2101_10994_gb300 import batch as B
    jobs = make_jobs(ng, items, decode)
    for k, j in enumerate(jobs):
        if k % 2 == 0:
            j.feats = j.feats.summed(j.svo, j.lod)
    rnd = B.BatchRenderer(jobs, decode=decode)
    rnd.frame()
    rnd.check()
    for k, j in enumerate(jobs):
        lists, ref = per_job(ng, j, decode)
        assert_same(rnd.outputs(k), lists, ref)
    # FD normals leave the hit voxel: a batch whose own normals are FD ones
    # refuses summed tables
    rnd.params.want_normals, rnd.params.normal_mode, rnd.params.fd_h = 1, ng.NORMALS["fd"], 1e-3
    with pytest.raises(ng.NglodError, match="summed"):
        rnd._create()
    rnd.free()
