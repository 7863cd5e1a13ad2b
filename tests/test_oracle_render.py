"""Pins of the oracle's compositing (Eq. 2, Sec. 3.1) and its adjoint."""
import math

import numpy as np
import pytest

import oracle
from paper_2412_04469_gb300 import synthetic as S
from tests._golden import load


def splats(W, H, means, sig, opac, rgb, depth):
    """Directly built 2D records (isotropic footprints, rects covering the image)."""
    n = len(opac)
    sig = np.broadcast_to(np.asarray(sig, float), (n,))
    TX, TY = (W + 15) // 16, (H + 15) // 16
    return dict(mean2d=np.asarray(means, float).T.copy(),
                conic=np.stack([1 / sig ** 2, np.zeros(n), 1 / sig ** 2]),
                opac=np.asarray(opac, float), rgb=np.asarray(rgb, float).T.copy(),
                depth=np.asarray(depth, float), radius=np.full(n, 3, np.int32),
                rect=np.tile(np.array([[0], [0], [TX], [TY]], np.int32), (1, n)),
                fragile=np.zeros(n, np.int32), frag_rect=np.zeros((4, n), np.int32), width=W, height=H)


def test_single_gaussian_footprint_and_pixel_centre():
    W, H, sig, o = 40, 36, 4.0, 0.8
    c = np.array([0.3, 0.6, 0.9])
    pr = splats(W, H, [(20.5, 17.5)], sig, [o], [c], [1.0])
    img, T, last, _ = oracle.render_fwd(pr)
    v, u = np.mgrid[0:H, 0:W]
    r2 = (u + 0.5 - 20.5) ** 2 + (v + 0.5 - 17.5) ** 2
    a = np.minimum(0.99, o * np.exp(-r2 / (2 * sig ** 2)))
    a = np.where(a >= 1 / 255, a, 0.0)
    assert np.allclose(img, c[:, None, None] * a[None], atol=1e-15)
    assert np.allclose(T, 1 - a, atol=1e-15)
    assert img[0, 17, 20] == pytest.approx(0.3 * o)      # pixel (20, 17) samples the mean exactly
    # the footprint ends where alpha crosses 1/255: radius sig sqrt(2 ln(255 o))
    rr = sig * math.sqrt(2 * math.log(255 * o))
    inside = r2 < rr ** 2 * (1 - 1e-9)
    assert np.all(last[inside] == 1) and np.all(last[r2 > rr ** 2 * (1 + 1e-9)] == 0)


def test_alpha_cap():
    pr = splats(16, 16, [(8.5, 8.5)], 3.0, [1.0], [(1, 1, 1)], [1.0])
    img, T, _, _ = oracle.render_fwd(pr)
    assert img[0, 8, 8] == 0.99 and T[8, 8] == pytest.approx(0.01)
    r_cap = 3.0 * math.sqrt(2 * math.log(1 / 0.99))     # o G >= 0.99 inside this radius
    v, u = np.mgrid[0:16, 0:16]
    r2 = (u + 0.5 - 8.5) ** 2 + (v + 0.5 - 8.5) ** 2
    assert np.all(img[0][r2 < r_cap ** 2] == 0.99)


def test_two_gaussians_by_hand_and_depth_order():
    g = load("composite_hand.txt")
    # both centred on pixel (4, 4) with huge footprints, so alpha = opacity there
    pr = splats(16, 16, [(4.5, 4.5), (4.5, 4.5)], 1e6, [0.5, 0.25], [(1, 0, 0), (0, 1, 0)], [1.0, 2.0])
    img, T, last, _ = oracle.render_fwd(pr)
    assert np.allclose([*img[:, 4, 4], T[4, 4]], g["ORDER_AB"], atol=1e-9)
    assert last[4, 4] == 2
    pr["depth"] = np.array([2.0, 1.0])
    img, T, last, _ = oracle.render_fwd(pr)
    assert np.allclose([*img[:, 4, 4], T[4, 4]], g["ORDER_BA"], atol=1e-9)


def test_background_and_termination():
    g = load("composite_hand.txt")
    n = 20
    pr = splats(16, 16, [(8.5, 8.5)] * n, 1e6, [0.5] * n, [(1, 1, 1)] * n, np.arange(1, n + 1, dtype=float))
    img, T, last, _ = oracle.render_fwd(pr, bg=(0.0, 0.5, 1.0))
    k = int(g["STACK_LAST"][0])
    assert last[8, 8] == k and T[8, 8] == pytest.approx(g["STACK_T"][0], rel=1e-6)
    Tk = 0.5 ** k
    assert img[:, 8, 8] == pytest.approx([1 - Tk, 1 - Tk + 0.5 * Tk, 1 - Tk + Tk], rel=1e-6)


def _scene(n, W, H, seed, degree=0, grow=0.0, cam_eye=(0.0, 0.0, 4.0)):
    A = S.make_scene(n, degree, seed).astype(np.float64)
    A[7:10] += grow
    cam = S.make_camera(W, H, 60.0, eye=cam_eye)
    return A, oracle.OracleCamera.of(cam)


def test_transmittance_invariants_random_scene():
    A, oc = _scene(2000, 128, 128, 0)
    pr = oracle.project(A, oc, 0)
    img, T, last, _ = oracle.render_fwd(pr)
    assert T.min() >= 1e-4 and T.max() <= 1.0
    assert np.all(img >= 0) and np.all(img <= 1.0 + 1e-12)
    assert np.all(T[last == 0] == 1.0)


def brute_pixelwise(pr, W, H, bg):
    """Per pixel, every visible Gaussian whose rect holds the pixel's tile,
    sorted by (depth, index), composited with Eq. 2 in pure Python."""
    n = pr["opac"].size
    img = np.zeros((3, H, W))
    T_all = np.zeros((H, W))
    for v in range(H):
        for u in range(W):
            tx, ty = u // 16, v // 16
            lst = sorted((pr["depth"][i], i) for i in range(n)
                         if pr["rect"][0, i] <= tx < pr["rect"][2, i] and pr["rect"][1, i] <= ty < pr["rect"][3, i])
            T, C = 1.0, np.zeros(3)
            for _, i in lst:
                dx, dy = u + 0.5 - pr["mean2d"][0, i], v + 0.5 - pr["mean2d"][1, i]
                a, b, c = pr["conic"][:, i]
                pw = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
                if pw > 0:
                    continue
                al = min(0.99, pr["opac"][i] * math.exp(pw))
                if al < 1 / 255:
                    continue
                if T * (1 - al) < 1e-4:
                    break
                C += pr["rgb"][:, i] * al * T
                T *= 1 - al
            img[:, v, u] = C + T * np.asarray(bg)
            T_all[v, u] = T
    return img, T_all


@pytest.mark.parametrize("n,W,H,seed", [(40, 32, 32, 1), (64, 33, 17, 2)])
def test_brute_force_tiny_scenes(n, W, H, seed):
    A, oc = _scene(n, W, H, seed, grow=1.2)
    pr = oracle.project(A, oc, 0)
    bg = (0.1, 0.2, 0.3)
    img, T, _, _ = oracle.render_fwd(pr, bg=bg)
    bimg, bT = brute_pixelwise(pr, W, H, bg)
    assert np.abs(img - bimg).max() < 1e-13 and np.abs(T - bT).max() < 1e-13


def brute_all_gaussians(pr, W, H, bg):
    """Per pixel, every visible Gaussian -- no tile-rect membership test --
    sorted by (depth, index) and composited with Eq. 2; also returns, per
    pixel, the Gaussians it composited whose rect misses the pixel's tile."""
    vis = [i for i in range(pr["opac"].size) if pr["radius"][i] > 0]
    order = sorted(vis, key=lambda i: (pr["depth"][i], i))
    img = np.zeros((3, H, W))
    T_all = np.zeros((H, W))
    outside = {}
    for v in range(H):
        for u in range(W):
            tx, ty = u // 16, v // 16
            T, C = 1.0, np.zeros(3)
            for i in order:
                dx, dy = u + 0.5 - pr["mean2d"][0, i], v + 0.5 - pr["mean2d"][1, i]
                a, b, c = pr["conic"][:, i]
                pw = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
                if pw > 0:
                    continue
                al = min(0.99, pr["opac"][i] * math.exp(pw))
                if al < 1 / 255:
                    continue
                if T * (1 - al) < 1e-4:
                    break
                r = pr["rect"][:, i]
                if not (r[0] <= tx < r[2] and r[1] <= ty < r[3]):
                    outside.setdefault((v, u), []).append(i)
                C += pr["rgb"][:, i] * al * T
                T *= 1 - al
            img[:, v, u] = C + T * np.asarray(bg)
            T_all[v, u] = T
    return img, T_all, outside


# A pixel outside a Gaussian's rect lies more than r = ceil(3 sqrt(lambda_max))
# from its centre along x or y, so its Mahalanobis distance exceeds 3 and
# alpha < o e^(-4.5): only an opacity above e^4.5 / 255 reaches 1/255 there.
OPAC_BEYOND_RECT = math.exp(4.5) / 255


@pytest.mark.parametrize("seed", [5, 6])
def test_rect_only_drops_alpha_beyond_three_sigma(seed):
    W, H, bg = 48, 40, (0.1, 0.2, 0.3)
    A, oc = _scene(60, W, H, seed, grow=1.0)
    pr = oracle.project(A, oc, 0)                         # rects from the 3-sigma radius
    vis = np.nonzero(pr["radius"] > 0)[0]
    v, u = np.mgrid[0:H, 0:W]
    for i in vis:                                         # every pixel outside the rect: power < -4.5
        r = pr["rect"][:, i]
        out = ~((r[0] <= u // 16) & (u // 16 < r[2]) & (r[1] <= v // 16) & (v // 16 < r[3]))
        dx, dy = u + 0.5 - pr["mean2d"][0, i], v + 0.5 - pr["mean2d"][1, i]
        a, b, c = pr["conic"][:, i]
        pw = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
        assert not out.any() or pw[out].max() < -4.5
    img, T, _, _ = oracle.render_fwd(pr, bg=bg)
    bimg, bT, outside = brute_all_gaussians(pr, W, H, bg)
    differ = (np.abs(img - bimg).max(axis=0) > 1e-13) | (np.abs(T - bT) > 1e-13)
    for pix in zip(*np.nonzero(differ)):                  # explained by a Gaussian composited from outside its rect
        assert pix in outside
    for ids in outside.values():
        assert all(pr["opac"][i] > OPAC_BEYOND_RECT for i in ids)
    assert (pr["opac"][vis] > OPAC_BEYOND_RECT).any()


@pytest.mark.parametrize("o,differs", [(0.99, True), (0.34, False)])
def test_rect_cut_off_hand_case(o, differs):
    """sigma = 4 at x = 28: r = 12 and the rect's first tile column is 1
    (pixels 16..47).  Column 15's pixel centres are at least 12.5 = 3.125
    sigma away, where alpha <= o e^(-4.88): 0.0075 for o = 0.99 (composited
    without the rect), 0.0026 < 1/255 for o = 0.34 (no difference anywhere)."""
    W, H = 64, 32
    pr = splats(W, H, [(28.0, 16.0)], 4.0, [o], [(1.0, 0.5, 0.25)], [1.0])
    r = 12
    TX, TY = (W + 15) // 16, (H + 15) // 16
    pr["rect"] = np.array([[max(0, (28 - r) // 16)], [max(0, (16 - r) // 16)],
                           [min(TX, (28 + r + 15) // 16)], [min(TY, (16 + r + 15) // 16)]], np.int32)
    assert list(pr["rect"][:, 0]) == [1, 0, 3, 2]
    img, T, _, _ = oracle.render_fwd(pr)
    bimg, bT, outside = brute_all_gaussians(pr, W, H, (0.0, 0.0, 0.0))
    assert np.all(img[:, :, 16:48] == bimg[:, :, 16:48])  # inside the rect's columns: identical
    assert (np.abs(img - bimg).max() > 0) == differs
    if differs:
        r2 = 12.5 ** 2 + 0.5 ** 2                         # pixel (15, 16)'s centre from the mean
        assert img[0, 16, 15] == 0.0 and bimg[0, 16, 15] == pytest.approx(o * math.exp(-r2 / 32), rel=1e-12)
        assert o > OPAC_BEYOND_RECT


def _fd_scene(seed):
    A, oc = _scene(24, 32, 32, seed, degree=0, grow=1.0)
    pr = oracle.project(A, oc, 0, eps_g=1e-5)
    return pr


@pytest.mark.parametrize("seed", [3, 4])
def test_backward_matches_finite_differences(seed):
    pr = _fd_scene(seed)
    bg = (0.2, 0.1, 0.4)
    _, _, last0, frag = oracle.render_fwd(pr, bg=bg, eps=1e-4, eps_d=1e-6)
    rng = np.random.default_rng(seed)
    Wt = rng.standard_normal((3, 32, 32)) * (frag == 0)[None]   # no weight on pixels near a threshold
    g = oracle.render_bwd(pr, Wt, bg=bg)

    def f(q):
        img, _, last, _ = oracle.render_fwd(q, bg=bg)
        return (Wt * img).sum(), last

    h = 1e-7
    vis = np.nonzero(pr["radius"] > 0)[0]
    checked = 0
    for key, gk in (("mean2d", "d_mean2d"), ("conic", "d_conic"), ("opac", "d_opac"), ("rgb", "d_rgb")):
        arr = pr[key] if pr[key].ndim == 2 else pr[key][None]
        grad = g[gk] if g[gk].ndim == 2 else g[gk][None]
        for row in range(arr.shape[0]):
            for i in vis:
                step = h * max(1.0, abs(arr[row, i]))
                qp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in pr.items()}
                qm = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in pr.items()}
                (qp[key] if qp[key].ndim == 2 else qp[key][None])[row, i] += step
                (qm[key] if qm[key].ndim == 2 else qm[key][None])[row, i] -= step
                fp, lp = f(qp)
                fm, lm = f(qm)
                if not (np.array_equal(lp, last0) and np.array_equal(lm, last0)):
                    continue     # the step crossed a threshold somewhere: not differentiable here
                fd = (fp - fm) / (2 * step)
                assert fd == pytest.approx(grad[row, i], rel=1e-5, abs=1e-6), (key, row, i)
                checked += 1
    assert checked > 0.9 * 9 * vis.size


@pytest.mark.parametrize("seed,grow", [(5, 0.8), (6, 1.4)])
def test_tight_rects_render_identically(seed, grow):
    """Limiting tile lists to the tiles the alpha >= 1/255 ellipse reaches
    drops only pairs every pixel skips: same image, T and adjoint in FP64."""
    A, oc = _scene(300, 64, 48, seed, degree=1, grow=grow)
    A[10] += np.linspace(-6, 4, A.shape[1])          # include Gaussians with o < 1/255
    plain = oracle.project(A, oc, 1)
    tight = oracle.project(A, oc, 1, tight=True)
    area = lambda r: np.maximum(r[2] - r[0], 0) * np.maximum(r[3] - r[1], 0)
    ne = area(tight["rect"]) > 0                                  # non-empty tight rects lie inside
    t, p = tight["rect"][:, ne], plain["rect"][:, ne]
    assert np.all(t[0] >= p[0]) and np.all(t[1] >= p[1]) and np.all(t[2] <= p[2]) and np.all(t[3] <= p[3])
    assert area(tight["rect"]).sum() < 0.9 * area(plain["rect"]).sum()
    assert np.all(area(tight["rect"])[plain["opac"] < 0.99 / 255] == 0)
    i1, T1, _, _ = oracle.render_fwd(plain, bg=(0.1, 0.2, 0.3))
    i2, T2, _, _ = oracle.render_fwd(tight, bg=(0.1, 0.2, 0.3))
    assert np.array_equal(i1, i2) and np.array_equal(T1, T2)
    d = S.make_image(64, 48, seed) - 0.5
    g1 = oracle.render_bwd(plain, d, bg=(0.1, 0.2, 0.3))
    g2 = oracle.render_bwd(tight, d, bg=(0.1, 0.2, 0.3))
    for k in g1:
        assert np.array_equal(g1[k], g2[k]), k


def test_tight_rect_closed_form():
    W, H, f, z, sig = 256, 256, 100.0, 2.0, 0.1
    cam = oracle.OracleCamera(np.eye(3), np.zeros(3), f, f, W / 2, H / 2, W, H, 0.2, np.zeros(3))
    Ahat = np.zeros((14, 1))
    Ahat[0:3, 0] = [0.3, -0.2, z]
    Ahat[3, 0] = 1.0
    Ahat[7:10, 0] = math.log(sig)
    Ahat[10, 0] = 0.0                                  # o = 1/2
    r = oracle.project(Ahat, cam, 0, blur=0.0, tight=True)
    s2 = (f * sig / z) ** 2                            # isotropic footprint, Sigma'_xx = Sigma'_yy
    k = 2 * math.log(255 * 0.5) + 0.01
    h = math.sqrt(1.01 * k * s2) + 0.01
    mx, my = f * 0.3 / z + W / 2, f * -0.2 / z + H / 2
    assert list(r["rect"][:, 0]) == [math.floor((mx - h) / 16), math.floor((my - h) / 16),
                                     math.floor((mx + h) / 16) + 1, math.floor((my + h) / 16) + 1]


def test_magnitude_sums_bound_and_equal_without_sign_changes():
    """The adjoint's magnitude sums (the bound floating-point summation keeps
    to): never below an entry's magnitude on a random scene; equal to it for
    one Gaussian over a black background under a positive upstream gradient,
    where no term of the conic's diagonal, the opacity or the colour changes
    sign; far above it where an antisymmetric upstream gradient cancels."""
    pr = _fd_scene(3)
    rng = np.random.default_rng(3)
    g = oracle.render_bwd(pr, rng.standard_normal((3, 32, 32)), bg=(0.2, 0.1, 0.4), magnitudes=True)
    for k in ("d_mean2d", "d_conic", "d_opac", "d_rgb"):
        assert np.all(g["mag"][k] >= np.abs(g[k]) * (1 - 1e-12)), k
    W = H = 32
    pr1 = splats(W, H, [(15.7, 16.2)], 3.0, [0.7], [(0.3, 0.6, 0.9)], [1.0])
    g1 = oracle.render_bwd(pr1, np.ones((3, H, W)), magnitudes=True)
    m = g1["mag"]
    assert m["d_conic"][0, 0] == pytest.approx(abs(g1["d_conic"][0, 0]), rel=1e-12)
    assert m["d_conic"][2, 0] == pytest.approx(abs(g1["d_conic"][2, 0]), rel=1e-12)
    assert m["d_opac"][0] == pytest.approx(abs(g1["d_opac"][0]), rel=1e-12)
    assert np.allclose(m["d_rgb"][:, 0], np.abs(g1["d_rgb"][:, 0]), rtol=1e-12)
    # upstream +1 left of the mean, -1 right of it: the x-moment terms cancel
    pr2 = splats(W, H, [(16.0, 16.0)], 3.0, [0.7], [(0.3, 0.6, 0.9)], [1.0])
    d = np.where(np.arange(W)[None, None, :] < 16, 1.0, -1.0) * np.ones((3, H, W))
    g2 = oracle.render_bwd(pr2, d, magnitudes=True)
    assert abs(g2["d_conic"][0, 0]) < 1e-9 * g2["mag"]["d_conic"][0, 0]
    assert g2["mag"]["d_conic"][0, 0] > 0
