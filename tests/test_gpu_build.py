"""svo_build on the GPU vs the oracle's own octree arrays (bit-exact):
packed coordinates, parent, child mask, first child, 8 corner ids per voxel,
corner counts and the ancestor table; malformed octrees are rejected."""
import numpy as np
import pytest

from paper_2101_10994_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["sphere3", "csg16_4", "csg64_5"])
def test_build_matches_oracle(ng, oracle_mod, which):
    if which == "sphere3":
        sc, oc = S.plain_sphere(3)
    elif which == "csg16_4":
        sc, oc = S.csg_workload(16, seed=1, max_lod=4)
    else:
        sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    svo = ng.svo_build(oc.keys)
    ora = oracle_mod.OracleSVO(oc.keys)
    assert svo.voxels == oc.counts()
    assert svo.corners == [ora.corner_count(l) for l in range(1, oc.max_lod + 1)]
    assert svo.corners == oc.corner_counts()
    for dp in range(oc.max_depth + 1):
        node, corners, anc = svo.read_arrays(dp)
        parent, mask, base, ocorners = ora.arrays(dp)
        i, j, k = S.morton_decode(oc.keys[dp])
        np.testing.assert_array_equal(node[:, 0], (i | (j << 10) | (k << 20)).astype(np.int32))
        np.testing.assert_array_equal(node[:, 3], parent)
        np.testing.assert_array_equal(node[:, 2], mask.astype(np.int32))
        has_child = mask != 0
        np.testing.assert_array_equal(node[has_child, 1], base[has_child])
        if dp >= S.FIRST_FEATURE_DEPTH:
            np.testing.assert_array_equal(corners, ocorners)
            # ancestors by walking the oracle's parent arrays
            exp = np.full((len(parent), 8), -1, np.int64)
            cur = np.arange(len(parent))
            for dd in range(dp, S.FIRST_FEATURE_DEPTH - 1, -1):
                exp[:, dd - S.FIRST_FEATURE_DEPTH] = cur
                cur = ora.arrays(dd)[0][cur]
            np.testing.assert_array_equal(anc, exp.astype(np.int32))
    svo.free()


def test_build_rejects_malformed(ng):
    sc, oc = S.plain_sphere(2)
    keys = [k.copy() for k in oc.keys]
    bad = [k.copy() for k in keys]
    bad[4] = np.concatenate([bad[4], [np.uint64(8 ** 4 - 1)]])     # parent missing
    with pytest.raises(ng.NglodError) as e:
        ng.svo_build(bad)
    assert e.value.code == ng.ERR_INVALID_ARG
    bad = [k.copy() for k in keys]
    bad[3] = bad[3][::-1].copy()                                   # not sorted
    with pytest.raises(ng.NglodError):
        ng.svo_build(bad)
    bad = [k.copy() for k in keys]
    bad[0] = np.array([1], np.uint64)                              # bad root
    with pytest.raises(ng.NglodError):
        ng.svo_build(bad)
    with pytest.raises(ng.NglodError):
        ng.svo_build(keys[:3])                                     # no feature depth
