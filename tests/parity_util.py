"""Comparison rules shared by the sphere-trace parity tests (test code only).

Two effects make a handful of rays differ between a correct GPU trace and
the FP64 oracle, and both are accounted for here instead of being skipped:

* ReLU kinks.  Inside a voxel the decoded SDF of Eq. 2 is smooth except on
  the kink surfaces pre_h = 0 of the hidden units, where its gradient jumps.
  At a point within rounding of a kink the GPU's ReLU mask (FP32, or the one
  the tensor-core decode recorded) may lie on the other side than the
  oracle's FP64 one, and the GPU normal is then the gradient of the
  neighbouring piece.  The oracle evaluates that piece a step of KINK_STEP
  away: a kink plane with unit normal nu is crossed by one of the six axis
  steps whenever it lies within KINK_STEP * max_a |nu_a| >= KINK_STEP / sqrt(3)
  of x, far more than the rounding of any mask.  Every hit is compared with
  the nearest of the seven oracle normals (x and x +- KINK_STEP e_a), and
  the number that needed a one-sided normal is reported.
* Stop-test straddles.  The stop rule d < eps (supplementary Sec. A.4) is a
  comparison: when the oracle's distance at a step lies within the GPU's
  decode error of eps, the two sides may stop one step apart, which moves t
  by about one step.  A ray is a straddle when the oracle's own distance at
  either side's stopping point lies within that bound of eps.  Every other
  ray must meet the hit-depth tolerance; straddles are counted and bounded.
"""
import numpy as np

from paper_2101_10994_gb300 import scenes as S

KINK_STEP = 5e-5
# FP32 positions: the two sides accumulate t in FP32 / FP64, so their points
# at the same step differ by up to a few ulps of t per step (128 steps at
# t ~ 3: ~2e-5); the distance moves by |grad d| times that
POSITION_SLACK = 5e-5


def voxel_lo(oc, D, vox):
    """Low corner and edge length of target-depth voxels ``vox``."""
    i, j, k = S.morton_decode(oc.keys[D][vox])
    s = 2.0 / (1 << D)
    return np.stack([-1 + i * s, -1 + j * s, -1 + k * s], axis=1), s


def min_normal_angle(unit, x, n_gpu, step=KINK_STEP):
    """(angle to the oracle normal at x, angle to the nearest of the normals at
    x and x +- step e_a), both in degrees.  ``unit`` maps points to the
    oracle's unit normals (evaluated in the GPU's voxel)."""
    cands = [unit(x)]
    for a in range(3):
        for sgn in (-1.0, 1.0):
            xs = x.copy()
            xs[:, a] += sgn * step
            cands.append(unit(xs))
    ang = np.stack([np.degrees(np.arccos(np.clip((n_gpu * c).sum(1), -1.0, 1.0))) for c in cands], axis=1)
    return ang[:, 0], ang.min(axis=1)


def oracle_distance(ora, feats, dec, lod):
    """x -> the oracle's distance at the FP32 points x (the plain LOD query)."""
    return lambda x: ora.sdf_query(feats, dec, np.asarray(x, np.float32), lod)[0]


def straddles(dist, eps, bound, x_a, x_b):
    """True where the oracle distance ``dist`` at x_a or at x_b lies within
    ``bound`` (+ POSITION_SLACK) of eps; x_a / x_b may hold NaN rows (no
    point)."""
    out = np.zeros(len(x_a), bool)
    for x in (x_a, x_b):
        ok = np.all(np.isfinite(x), axis=1)
        if ok.any():
            dd = dist(x[ok])
            b = bound[ok] if np.ndim(bound) else bound
            out[np.flatnonzero(ok)] |= np.abs(dd - eps) <= b + POSITION_SLACK
    return out


def hit_points(o, d, t, hit):
    """FP64 points o + t d of the hit rays, NaN rows elsewhere."""
    x = o.astype(np.float64) + np.asarray(t, np.float64)[:, None] * d.astype(np.float64)
    x[~hit.astype(bool)] = np.nan
    return x
