"""Pins of the adaptive-mask oracle (Sec. 3.3, App. B): the box dilation, the
tile mask and the masked L1 loss against brute force and closed forms, and
the dynamic-only rendering's pixels against the union of the dynamic
Gaussians' alpha >= 1/255 footprints computed pixel by pixel."""
import numpy as np
import pytest

import oracle
from paper_2412_04469_gb300 import synthetic as S


def _dilate_brute(m, k):
    H, W = m.shape
    out = np.zeros_like(m, bool)
    for y in range(H):
        for x in range(W):
            for yy in range(H):
                for xx in range(W):
                    if m[yy, xx] and yy - k // 2 <= y <= yy + k // 2 - 1 and xx - k // 2 <= x <= xx + k // 2 - 1:
                        out[y, x] = True
    return out


@pytest.mark.parametrize("k,seed", [(2, 0), (4, 1), (6, 2), (48, 3)])
def test_dilate_matches_brute_force(k, seed):
    rng = np.random.default_rng(seed)
    m = rng.uniform(size=(9, 13)) < 0.06
    assert np.array_equal(oracle.dilate(m, k), _dilate_brute(m, k))


def test_dilate_special_cases():
    assert not oracle.dilate(np.zeros((5, 7), bool), 4).any()
    assert oracle.dilate(np.ones((5, 7), bool), 4).all()
    m = np.zeros((60, 70), bool)
    m[0, 0] = True                                      # corner: the window reaches 23 right and down of it
    d = oracle.dilate(m, 48)
    assert d[:24, :24].all() and not d[24:, :].any() and not d[:, 24:].any()
    m = np.zeros((60, 70), bool)
    m[30, 40] = True                                    # interior: 48 x 48 square from (x-24, y-24)
    d = oracle.dilate(m, 48)
    ys, xs = np.nonzero(d)
    assert (ys.min(), ys.max(), xs.min(), xs.max()) == (6, 53, 16, 63) and d.sum() == 48 * 48


def test_tile_mask_matches_brute_force():
    rng = np.random.default_rng(4)
    m = rng.uniform(size=(37, 50)) < 0.01
    got = oracle.tile_mask(m)
    TX, TY = 4, 3
    want = [m[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16].any() for ty in range(TY) for tx in range(TX)]
    assert list(got) == want


def test_masked_l1_loss_closed_forms():
    img = np.array([[[0.5, 0.2], [0.9, 0.0]]])          # C = 1, 2 x 2
    tgt = np.array([[[0.1, 0.2], [1.0, 0.3]]])
    mask = np.array([[True, True], [False, True]])
    loss, g = oracle.masked_l1_loss(img, tgt, mask)
    assert loss == pytest.approx((0.4 + 0.0 + 0.3) / 3)
    assert np.allclose(g, np.array([[[1 / 3, 0.0], [0.0, -1 / 3]]]))
    full, gf = oracle.masked_l1_loss(img, tgt, np.ones((2, 2), bool))
    ref, gr = oracle.l1_loss(img, tgt)
    assert full == pytest.approx(ref) and np.allclose(gf, gr)
    zl, zg = oracle.masked_l1_loss(img, tgt, np.zeros((2, 2), bool))
    assert zl == 0.0 and not zg.any()


def test_dynamic_pixels_are_the_union_of_dynamic_footprints():
    n, deg, W, H = 60, 0, 48, 40
    A = S.make_scene(n, deg, 6).astype(np.float64)
    A[7:10] += 0.4
    cam = S.make_camera(W, H, 60.0)
    proj = oracle.project(A, cam, deg, blur=0.3)
    flags = np.random.default_rng(2).uniform(size=n) < 0.3
    got = oracle.dynamic_pixels(proj, flags)
    ys, xs = np.mgrid[0:H, 0:W]
    want = np.zeros((H, W), bool)
    for i in np.nonzero(flags)[0]:
        x0, y0, x1, y1 = proj["rect"][:, i]
        if x1 <= x0 or y1 <= y0:
            continue
        dx = xs + 0.5 - proj["mean2d"][0, i]
        dy = ys + 0.5 - proj["mean2d"][1, i]
        a, b, c = proj["conic"][:, i]
        power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
        alpha = np.minimum(0.99, proj["opac"][i] * np.exp(power))
        inside = (xs >= 16 * x0) & (xs < 16 * x1) & (ys >= 16 * y0) & (ys < 16 * y1)
        want |= inside & (power <= 0) & (alpha >= 1 / 255)
    assert want.any() and not want.all()
    assert np.array_equal(got, want)
    assert not oracle.dynamic_pixels(proj, np.zeros(n, bool)).any()
    d = np.array([[0.0, 0.001 / 50, 0.0011 / 50, 0.0, 0.0006 / 50], [0.0, 0.0, 0.0, 0.0011 / 20, 0.0008 / 20]])
    assert np.array_equal(oracle.dynamic_flags(d, 100, 40), [False, False, True, True, False])   # NDC: x W/2, y H/2
    assert oracle.dynamic_flags(np.array([[0.0006 / 50], [0.00081 / 20]]), 100, 40)[0]               # |(6, 8.1)| e-4 > 1e-3
