"""Which of the tiled traversal's three paths each tile of a ray set takes
(test code only, used to show that a test's inputs reach a path).

The GPU traversal sweeps tiles of TILE_RAYS consecutive rays level by level
with an on-chip frontier of FRONTIER_CAP pairs per buffer:
* "whole": every frontier of the tile fits;
* "chunks": the frontier after some Decide at depth dp would not fit, so the
  tile continues from the decided depth-dp pairs in chunks of whole rays,
  each fitting one of two buffers of F = min(cap, (2 cap - n) / 2) pairs
  (n = the kept pairs) with at most F children at depth dp + 1 (F / 2 when
  deeper frontiers follow);
* "halving": a chunk overflowed further down, and its rays and the tile's
  later ones were run from the root over halving ray ranges.
The number of pairs of a ray at depth dp is the length of its depth-dp list
(hierarchical culling loses nothing, so the traversal keeps exactly the
voxels whose own slab test hits); depths below 3 never overflow a tile.
"""
import numpy as np

TILE_RAYS = 128
FRONTIER_CAP = 4096


def pairs_by_depth(ora, o, d, D):
    """[R, D + 1] pairs per ray at depths 0..D (depths 1, 2 left 0: they
    never decide a path) from the oracle's lists."""
    P = np.zeros((len(o), D + 1), np.int64)
    P[:, 0] = 1
    for dp in range(3, D + 1):
        offs, _, _ = ora.trace_rays(o, d, dp - 2)
        P[:, dp] = np.diff(offs)
    return P


def tile_paths(P, D, cap=FRONTIER_CAP, tile=TILE_RAYS):
    """Path label of every tile of the ray set with per-depth pairs P."""
    out = []
    for t0 in range(0, len(P), tile):
        T = P[t0:t0 + tile]
        nr = len(T)
        fail = next((dp for dp in range(0, D - 1) if T[:, dp + 1].sum() > cap), None)
        if fail is None:
            out.append("whole")
            continue
        dp = fail
        n = int(T[:, dp].sum())
        F = min(cap, (2 * cap - n) // 2)
        budget = F if dp + 2 == D else F // 2
        bounds, acc, pairs, first, start_pairs = [0], 0, 0, 0, 0
        for r in range(nr):
            c, pc = int(T[r, dp + 1]), int(T[r, dp])
            if r > first and (acc + c > budget or pairs + pc - start_pairs > F):
                bounds.append(r)
                first, acc, start_pairs = r, 0, pairs
            acc += c
            pairs += pc
        bounds.append(nr)
        label = "chunks"
        for a, b in zip(bounds[:-1], bounds[1:]):
            if any(T[a:b, l + 1].sum() > F for l in range(dp + 1, D - 1)):
                label = "halving"
                break
        out.append(label)
    return out
