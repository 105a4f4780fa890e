"""Input generators: the training-sample mixes (Sec. 3.3 sampling)."""
import numpy as np

from paper_2101_10994_gb300 import scenes as S


def test_training_mixes():
    sc, _ = S.csg_workload(16, seed=1, max_lod=3)
    n = 2000
    x, t = S.training_batch(sc, n, 3)
    assert x.shape == (n, 3) and x.dtype == np.float32 and t.dtype == np.float32
    assert np.median(np.abs(t[: n // 2])) < 0.02 < np.median(np.abs(t[n // 2:]))
    x2, t2 = S.training_batch(sc, n, 3, mix="paper")
    k = 2 * n // 5
    assert np.abs(t2[:k]).max() < 1e-6                      # on the surface
    assert 1e-4 < np.median(np.abs(t2[k:2 * k])) < 0.02     # near it (sigma 0.01)
    assert np.median(np.abs(t2[2 * k:])) > 0.05             # uniform in the cube
    # targets are the exact scene SDF at the float32 points
    np.testing.assert_allclose(t2, S.scene_sdf(sc, x2.astype(np.float64)).astype(np.float32))
