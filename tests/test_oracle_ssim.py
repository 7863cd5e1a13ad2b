"""Pins of the D-SSIM oracle (Eq. 3's structural term): the window filter
against scipy's Gaussian filter with zero padding, the SSIM map against
closed forms (identical images, constant images inside and at a corner where
the zero padding creates variance) and a pure-Python brute force, and its
gradient against central differences and the zero at identical images."""
import numpy as np
import pytest
from scipy import ndimage

import oracle


def test_window_filter_is_a_zero_padded_gaussian_filter():
    rng = np.random.default_rng(0)
    a = rng.uniform(size=(23, 31))
    want = ndimage.gaussian_filter(a, sigma=1.5, mode="constant", cval=0.0, truncate=5 / 1.5)   # radius 5
    got = oracle.window_filter(a, oracle.ssim_window())
    assert np.allclose(got, want, rtol=0, atol=1e-14)
    assert oracle.ssim_window().sum() == pytest.approx(1.0, abs=1e-15)


def test_window_filter_adjoint_is_its_transpose():
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal((17, 9)), rng.standard_normal((17, 9))
    w = oracle.ssim_window()
    lhs = (oracle.window_filter(a, w) * b).sum()
    rhs = (a * oracle.window_filter_adjoint(b, w)).sum()
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_identical_images():
    rng = np.random.default_rng(2)
    x = rng.uniform(size=(3, 20, 14))
    assert np.allclose(oracle.ssim_map(x, x), 1.0, rtol=0, atol=1e-13)
    loss, g = oracle.dssim_loss(x, x)
    assert abs(loss) < 1e-13
    assert np.abs(g).max() < 1e-15          # SSIM <= 1 with equality at x = y: a maximum


def test_constant_images_closed_forms():
    a, b = 0.3, 0.7
    H, W = 24, 30
    x, y = np.full((1, H, W), a), np.full((1, H, W), b)
    S = oracle.ssim_map(x, y)[0]
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    # away from the border the window sees a constant: no variance
    assert np.allclose(S[5:-5, 5:-5], (2 * a * b + c1) / (a * a + b * b + c1), rtol=1e-13)
    # at a corner the window keeps a share s of its mass (scipy's filter of ones),
    # so mu = a s, E[x^2] = a^2 s: variance a^2 s (1 - s), covariance a b s (1 - s)
    s = ndimage.gaussian_filter(np.ones((H, W)), 1.5, mode="constant", truncate=5 / 1.5)[0, 0]
    assert 0.35 < s < 0.45                  # (1/2 + half the centre tap)^2
    v = s * (1 - s)
    want = ((2 * a * b * s * s + c1) * (2 * a * b * v + c2)) / (((a * a + b * b) * s * s + c1) * ((a * a + b * b) * v + c2))
    assert S[0, 0] == pytest.approx(want, rel=1e-13)
    assert S[0, 0] == pytest.approx(S[-1, -1], rel=1e-13)


def test_ssim_map_matches_brute_force():
    rng = np.random.default_rng(3)
    C, H, W = 2, 7, 6
    x, y = rng.uniform(size=(C, H, W)), rng.uniform(size=(C, H, W))
    w = oracle.ssim_window()
    got = oracle.ssim_map(x, y)
    for c in range(C):
        for py in range(H):
            for px in range(W):
                mx = my = exx = eyy = exy = 0.0
                for i in range(11):
                    for j in range(11):
                        qy, qx = py + i - 5, px + j - 5
                        if 0 <= qy < H and 0 <= qx < W:
                            u, v = x[c, qy, qx], y[c, qy, qx]
                            mx += w[i, j] * u
                            my += w[i, j] * v
                            exx += w[i, j] * u * u
                            eyy += w[i, j] * v * v
                            exy += w[i, j] * u * v
                num = (2 * mx * my + 1e-4) * (2 * (exy - mx * my) + 9e-4)
                den = (mx * mx + my * my + 1e-4) * ((exx - mx * mx) + (eyy - my * my) + 9e-4)
                assert got[c, py, px] == pytest.approx(num / den, rel=1e-12)
    assert np.array_equal(got, oracle.ssim_map(y, x)) or np.allclose(got, oracle.ssim_map(y, x), rtol=1e-14)


def test_dssim_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    C, H, W = 2, 14, 12
    x, y = rng.uniform(size=(C, H, W)), rng.uniform(size=(C, H, W))
    loss, g = oracle.dssim_loss(x, y)
    assert loss == pytest.approx(1.0 - oracle.ssim_map(x, y).mean(), rel=1e-14)
    h = 1e-6
    pts = [(0, 0, 0), (1, 13, 11), (0, 6, 5), (1, 0, 7), (0, 9, 0), (1, 4, 4), (0, 13, 2)]
    for c, py, px in pts:
        xp, xm = x.copy(), x.copy()
        xp[c, py, px] += h
        xm[c, py, px] -= h
        fd = (oracle.dssim_loss(xp, y)[0] - oracle.dssim_loss(xm, y)[0]) / (2 * h)
        assert g[c, py, px] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_masked_dssim():
    rng = np.random.default_rng(5)
    C, H, W = 2, 13, 11
    x, y = rng.uniform(size=(C, H, W)), rng.uniform(size=(C, H, W))
    full = oracle.dssim_loss(x, y)
    ones = oracle.dssim_loss(x, y, np.ones((H, W), bool))
    assert ones[0] == full[0] and np.array_equal(ones[1], full[1])
    assert oracle.dssim_loss(x, y, np.zeros((H, W), bool))[0] == 0.0
    m = rng.uniform(size=(H, W)) < 0.3
    loss, g = oracle.dssim_loss(x, y, m)
    assert loss == pytest.approx(1.0 - oracle.ssim_map(x, y)[:, m].mean(), rel=1e-14)
    h = 1e-6
    for c, py, px in [(0, 0, 0), (1, 6, 5), (0, 12, 10), (1, 3, 9)]:
        xp, xm = x.copy(), x.copy()
        xp[c, py, px] += h
        xm[c, py, px] -= h
        fd = (oracle.dssim_loss(xp, y, m)[0] - oracle.dssim_loss(xm, y, m)[0]) / (2 * h)
        assert g[c, py, px] == pytest.approx(fd, rel=1e-6, abs=1e-10)
