"""A frame traced as chunks on several CUDA streams (FrameRenderer) equals the
single-pass frame output for output: rays are independent, so splitting them
changes only which launch handles which ray."""
import numpy as np
import pytest
import torch

from paper_2101_10994_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def assert_staged_equal(staged, L):
    """Ray by ray, the staged lists (first entry, count, staging list) equal
    the CSR lists L of svo_trace_rays, entry for entry."""
    offs = L.ray_offsets.long()
    cnt = staged.ray_counts.long()
    assert torch.equal(cnt, offs[1:] - offs[:-1])
    H = int(offs[-1])
    start = torch.repeat_interleave(staged.ray_offsets.long(), cnt)
    within = torch.arange(H, device=cnt.device) - torch.repeat_interleave(offs[:-1], cnt)
    assert torch.equal(staged.voxel_id[start + within], L.voxel_id)


@pytest.mark.parametrize("decode,chunks", [("bf16", 2), ("f32", 3), ("fp8", 2)])
def test_chunked_frame_equals_single_pass(ng, decode, chunks):
    from paper_2101_10994_gb300.frame import FrameRenderer
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(S.readout_features(oc, sc))
    if decode == "fp8":
        F.set_fp8_bound(svo, 5)
    D = ng.DecoderDev.from_decoder(S.readout_decoder(5))
    o, d, _ = S.camera_rays(640, 360, tile=8)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    lists = ng.svo_trace_rays(svo, to, td, 5)
    ref = ng.sphere_trace(svo, F, D, to, td, lists, decode=decode, normals=True)
    fr = FrameRenderer(svo, F, D, to, td, 5, chunks=chunks, decode=decode)
    assert len(fr.chunks) == chunks
    # uneven chunk sizes change only the schedule
    fw = FrameRenderer(svo, F, D, to, td, 5, chunks=chunks, decode=decode, weights=list(range(1, chunks + 1)))
    sizes = [c["n"] for c in fw.chunks]
    assert sum(sizes) == len(o) and sizes == sorted(sizes)
    fw.frame()
    fw.check()
    for k in ("t", "hit", "steps", "normal"):
        assert torch.equal(fw.out[k], ref[k]), k
    with pytest.raises(ValueError):
        FrameRenderer(svo, F, D, to, td, 5, chunks=chunks, decode=decode, weights=[1.0] * (chunks + 1))
    for _ in range(2):                     # a second frame reuses every buffer
        fr.frame()
        fr.check()
        for k in ("t", "hit", "steps", "normal"):
            assert torch.equal(fr.out[k], ref[k]), k
    # narrower traversal and trace launches change only the schedule
    fn = FrameRenderer(svo, F, D, to, td, 5, chunks=chunks, decode=decode, ctas_per_sm=2, trav_ctas_per_sm=1)
    fn.frame()
    fn.check()
    for k in ("t", "hit", "steps", "normal"):
        assert torch.equal(fn.out[k], ref[k]), k
    for c in fn.chunks:                    # and the staged lists hold those of svo_trace_rays
        n = c["n"]
        L = ng.svo_trace_rays(svo, to[c["rs"]:c["rs"] + n], td[c["rs"]:c["rs"] + n], 5)
        assert_staged_equal(c["lists"], L)
    # rays and results through pinned host buffers, copied chunk by chunk
    h_in = (torch.from_numpy(o).pin_memory(), torch.from_numpy(d).pin_memory())
    h_out = {"t": torch.empty(len(o)).pin_memory(), "hit": torch.empty(len(o), dtype=torch.uint8).pin_memory(),
             "normal": torch.empty((len(o), 3)).pin_memory()}
    fr.o.zero_()
    fr.frame(h_in, h_out)
    torch.cuda.synchronize()
    fr.check()
    assert torch.equal(h_out["t"], ref["t"].cpu()) and torch.equal(h_out["normal"], ref["normal"].cpu())
    assert torch.equal(h_out["hit"], ref["hit"].cpu())
    svo.free()


def test_chunked_blended_frame_equals_single_pass(ng):
    from paper_2101_10994_gb300.frame import FrameRenderer
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(S.readout_features(oc, sc))
    D4, D5 = ng.DecoderDev.from_decoder(S.readout_decoder(4)), ng.DecoderDev.from_decoder(S.readout_decoder(5))
    o, d, _ = S.camera_rays(480, 270, tile=8)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    lists = ng.svo_trace_rays(svo, to, td, ng.blend_lists_lod(4.5))
    ref = ng.sphere_trace_blend(svo, F, D4, D5, to, td, lists, 4.5, decode="bf16", normals=True)
    fr = FrameRenderer(svo, F, D4, to, td, 4.5, chunks=2, decode="bf16", dec_hi=D5)
    fr.frame()
    fr.check()
    for k in ("t", "hit", "steps", "normal"):
        assert torch.equal(fr.out[k], ref[k]), k
    svo.free()


@pytest.mark.parametrize("decode", ["bf16", "f32"])
def test_trace_width_and_frame_autotune(ng, decode):
    # the persistent trace's launch width changes no output; the frame
    # autotuner returns a renderer whose frame equals the single pass
    from paper_2101_10994_gb300.frame import autotune_frame
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(S.readout_features(oc, sc))
    D = ng.DecoderDev.from_decoder(S.readout_decoder(5))
    o, d, _ = S.camera_rays(400, 300, tile=8)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    lists = ng.svo_trace_rays(svo, to, td, 5)
    ref = ng.sphere_trace(svo, F, D, to, td, lists, decode=decode, normals=True)
    for c in (1, 2, 3, 4):
        got = ng.sphere_trace(svo, F, D, to, td, lists, decode=decode, normals=True, ctas_per_sm=c)
        for k in ("t", "hit", "steps", "normal"):
            assert torch.equal(got[k], ref[k]), (c, k)
    with pytest.raises(ng.NglodError) as e:
        ng.sphere_trace(svo, F, D, to, td, lists, decode=decode, ctas_per_sm=5)
    assert e.value.code == ng.ERR_INVALID_ARG
    fr, timings = autotune_frame(svo, F, D, to, td, 5, chunk_counts=(1, 2), ctas=(0, 2), reps=2, decode=decode)
    assert set(timings) == {"1/0", "1/2", "2/0", "2/2", "2/0/t2", "2/2/t2"}
    fr.frame()
    fr.check()
    for k in ("t", "hit", "steps", "normal"):
        assert torch.equal(fr.out[k], ref[k]), k
    # tuned with the host copies in: the frames it times copy rays in and
    # results out, and the returned renderer's copies equal the single pass
    h_in = (torch.from_numpy(o).pin_memory(), torch.from_numpy(d).pin_memory())
    h_out = {"t": torch.empty(len(o)).pin_memory(), "hit": torch.empty(len(o), dtype=torch.uint8).pin_memory(),
             "normal": torch.empty((len(o), 3)).pin_memory()}
    fh, th = autotune_frame(svo, F, D, to.clone(), td.clone(), 5, chunk_counts=(1, 2), ctas=(0,), reps=2,
                            decode=decode, host=(h_in, h_out))
    assert set(th) == {"1/0", "2/0", "2/0/t2"}
    fh.o.zero_()
    fh.frame(h_in, h_out)
    torch.cuda.synchronize()
    fh.check()
    assert torch.equal(h_out["t"], ref["t"].cpu()) and torch.equal(h_out["normal"], ref["normal"].cpu())
    svo.free()
