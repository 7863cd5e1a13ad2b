"""Pins of the oracle's tile binning: 64-bit (tile, depth) keys, stable sort
order and per-tile ranges (the tile-based rasterizer the paper builds on,
Sec. 4 implementation note)."""
import numpy as np
import pytest

import oracle
from paper_2412_04469_gb300 import synthetic as S


def brute(depth, rect, tx, ty):
    pairs = []
    e = 0
    for i in range(depth.size):
        x0, y0, x1, y1 = (int(v) for v in rect[:, i])
        bits = int(np.float32(depth[i]).view(np.uint32))
        for yy in range(y0, y1):
            for xx in range(x0, x1):
                pairs.append((((yy * tx + xx) << 32) | bits, e, i))
                e += 1
    pairs.sort()
    keys = np.array([p[0] for p in pairs], np.uint64)
    vals = np.array([p[2] for p in pairs], np.uint32)
    ranges = np.zeros((tx * ty, 2), np.uint32)
    tiles = keys >> np.uint64(32)
    for t in range(tx * ty):
        ranges[t] = [(tiles < t).sum(), (tiles <= t).sum()]
    return keys, vals, ranges


@pytest.mark.parametrize("n,tx,ty,seed", [(0, 3, 2, 0), (1, 1, 1, 1), (7, 4, 3, 2), (64, 5, 4, 3),
                                          (300, 9, 7, 4), (500, 2, 2, 5)])
def test_matches_brute_force(n, tx, ty, seed):
    depth, rect = S.make_bin_inputs(n, tx, ty, seed)
    k, v, r = oracle.bin_sort(depth, rect, tx, ty)
    bk, bv, br = brute(depth, rect, tx, ty)
    assert np.array_equal(k, bk) and np.array_equal(v, bv) and np.array_equal(r, br)


def test_invariants_and_ties():
    depth, rect = S.make_bin_inputs(400, 6, 5, 9, tie_frac=0.6)
    k, v, r = oracle.bin_sort(depth, rect, 6, 5)
    area = np.maximum(rect[2] - rect[0], 0) * np.maximum(rect[3] - rect[1], 0)
    assert k.size == area.sum()
    assert np.all(np.diff(k.astype(np.float64)) >= 0) and np.all(k[1:] >= k[:-1])
    assert r[0, 0] == 0 and r[-1, 1] == k.size and np.all(r[1:, 0] == r[:-1, 1])
    # stable: equal keys keep Gaussian index order
    same = k[1:] == k[:-1]
    assert same.any() and np.all(v[1:][same] > v[:-1][same])
    # every pair sits in its tile's range and belongs to a rect covering it
    for t in range(30):
        ids = v[r[t, 0]:r[t, 1]]
        xx, yy = t % 6, t // 6
        assert np.all((rect[0, ids] <= xx) & (xx < rect[2, ids]) & (rect[1, ids] <= yy) & (yy < rect[3, ids]))
