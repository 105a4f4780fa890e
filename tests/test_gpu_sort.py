"""nglod_sort_points: a permutation of the points whose depth-d Morton cell
keys (computed here in NumPy with the same FP32 cell rule) never decrease."""
import numpy as np
import pytest
import torch

from paper_2101_10994_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def keys(x, depth):
    q = ((x.astype(np.float32) + np.float32(1.0)) * np.float32(2 ** (depth - 1))).astype(np.float32)
    hi = 2 ** depth - 1
    with np.errstate(invalid="ignore"):
        c = np.where(q >= 0, np.where(q < hi, np.floor(np.nan_to_num(q, nan=0.0)), hi), 0).astype(np.int64)
    return S.morton_encode(c[:, 0], c[:, 1], c[:, 2])


@pytest.mark.parametrize("depth,n", [(7, 100_003), (5, 4097), (1, 33)])
def test_sort_points_is_sorted_permutation(ng, depth, n):
    rng = np.random.default_rng(depth)
    x = rng.uniform(-1.0, 1.0, (n, 3)).astype(np.float32)
    x[:5] = [[1.0, 1.0, 1.0], [-1.0, -1.0, -1.0], [2.0, -3.0, 0.5], [np.nan, 0.0, 0.0], [0.0, 0.0, 0.0]]
    e = rng.normal(size=n).astype(np.float32)
    xo, eo, perm = ng.sort_points(torch.from_numpy(x).cuda(), torch.from_numpy(e).cuda(), depth)
    xo, eo, perm = xo.cpu().numpy(), eo.cpu().numpy(), perm.cpu().numpy()
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert np.array_equal(xo.view(np.uint32), x[perm].view(np.uint32))
    assert np.array_equal(eo, e[perm])
    k = keys(xo, depth)
    assert np.all(np.diff(k) >= 0)


def test_sort_points_rejects_bad_depth(ng):
    x = torch.zeros((10, 3), device="cuda")
    for d in (0, 8):
        with pytest.raises(ng.NglodError) as e:
            ng.sort_points(x, None, d)
        assert e.value.code == ng.ERR_INVALID_ARG
