"""Pins of the oracle's FP32-fragility classifier, the part of the oracle that
decides which pixels the GPU parity tests compare (Eq. 1-2 and the readings of
the cited rasterizer: alpha threshold 1/255, cap 0.99, termination at 1e-4,
tile rect of the 3-sigma radius, near plane, determinant sign, tight rect of
the alpha >= 1/255 ellipse).

Two kinds of pins.  (1) Hand cases: a decision placed at 0.5 eps from its
threshold must be flagged, with the documented bit and nothing else; the same
decision at 3 eps must not be.  (2) Flip cases: the same scene is built on
both sides of the threshold (so that the decision really flips) and rendered;
every pixel whose result changes must be flagged on both sides, and only the
documented tile band of a rect edge may be flagged by that Gaussian.
"""
import math

import numpy as np
import pytest

import oracle

EPS_A, EPS_D, EPS_G = 2e-5, 1e-6, 2e-6
W = H = 256                           # 16 x 16 tiles
F = 100.0
BIT_NEAR, BIT_RADIUS, BIT_RECT, BIT_DET, BIT_OPAC = 1, 2, 4, 8, 16
EDGE_X0, EDGE_Y0, EDGE_X1, EDGE_Y1 = 32, 64, 128, 256


def _cam(near=0.2):
    return oracle.OracleCamera(np.eye(3), np.zeros(3), F, F, W / 2, H / 2, W, H, near, np.zeros(3))


def _gauss(p, sig=None, logscale=None, quat=(1, 0, 0, 0), opac=0.9):
    A = np.zeros((14, 1))
    A[0:3, 0] = p
    A[3:7, 0] = quat
    A[7:10, 0] = [math.log(sig)] * 3 if logscale is None else logscale
    A[10, 0] = math.log(opac / (1 - opac))
    A[11:14, 0] = 0.3                  # SH DC: some colour
    return A


def _proj(A, near=0.2, tight=False, blur=0.0):
    return oracle.project(A, _cam(near), 0, blur=blur, eps_g=EPS_G, tight=tight)


Z, SIG = 4.0, 0.8                     # projected sigma F SIG / Z = 20 px, radius 61


def _x_for_mean(mx, z=Z):
    return (mx - W / 2) * z / F


def _edge_scene(which, rel):
    """One Gaussian (o = 0.9, projected sigma ~20 px) whose rect edge `which`
    ((m - r)/16 for x0 and y0, (m + r + 15)/16 for x1 and y1) lies at the
    integer k times (1 + rel); the other three edges lie far from integers.
    The radius depends slightly on the position (through J), so the mean is
    solved for the radius it gets."""
    k = {"x0": 3, "y0": 2, "x1": 13, "y1": 12}[which]
    edge = k * (1 + rel)
    rad = 61
    for _ in range(4):
        if which == "x0":
            mx, my = 16 * edge + rad, 16 * 7.3 + 5.0
        elif which == "y0":
            mx, my = 16 * 7.3 + 5.0, 16 * edge + rad
        elif which == "x1":
            mx, my = 16 * edge - rad - 15, 16 * 7.3 + 5.0
        else:
            mx, my = 16 * 7.3 + 5.0, 16 * edge - rad - 15
        A = _gauss([_x_for_mean(mx), _x_for_mean(my), Z], SIG)
        pr = _proj(A)
        if pr["radius"][0] == rad:
            break
        rad = int(pr["radius"][0])
    assert pr["radius"][0] == rad
    assert pr["mean2d"][:, 0] == pytest.approx([mx, my], abs=1e-9)
    return A, pr


@pytest.mark.parametrize("which,bit", [("x0", EDGE_X0), ("y0", EDGE_Y0), ("x1", EDGE_X1), ("y1", EDGE_Y1)])
def test_rect_edge_on_an_integer_is_flagged_alone(which, bit):
    for rel in (0.5 * EPS_G, -0.5 * EPS_G):
        _, pr = _edge_scene(which, rel)
        assert pr["fragile"][0] == BIT_RECT | bit, (which, rel, pr["fragile"][0])
        r, fr = pr["rect"][:, 0], pr["frag_rect"][:, 0]
        assert list(fr) == [max(r[0] - 1, 0), max(r[1] - 1, 0), min(r[2] + 1, 16), min(r[3] + 1, 16)]
    for rel in (3 * EPS_G, -3 * EPS_G):
        _, pr = _edge_scene(which, rel)
        assert pr["fragile"][0] == 0 and not pr["frag_rect"][:, 0].any(), (which, rel)


def test_rect_edge_far_from_an_integer_is_not_flagged():
    for mx, my in ((100.3, 131.7), (57.25, 170.5), (200.9, 90.1)):
        pr = _proj(_gauss([_x_for_mean(mx), _x_for_mean(my), Z], SIG))
        assert pr["radius"][0] > 0 and pr["fragile"][0] == 0


def test_radius_ceil_on_an_integer_flags_all_four_edges():
    # on the axis Sigma' = s^2 I exactly (blur 0): lambda_max = s^2 + sqrt(0.1),
    # r = 3 sqrt(lambda_max); place r at 20 (1 +- 0.5 eps) and at 3 eps
    for rel, flagged in ((0.5 * EPS_G, True), (-0.5 * EPS_G, True), (3 * EPS_G, False), (-3 * EPS_G, False)):
        r3 = 20.0 * (1 + rel)
        s = math.sqrt((r3 / 3) ** 2 - math.sqrt(0.1))
        pr = _proj(_gauss([0, 0, Z], s * Z / F))
        want = BIT_RADIUS | EDGE_X0 | EDGE_Y0 | EDGE_X1 | EDGE_Y1 if flagged else 0
        assert pr["fragile"][0] == want, (rel, pr["fragile"][0])
        assert pr["radius"][0] == (21 if rel > 0 else 20)


def test_near_plane_decision_is_flagged_on_both_sides():
    near = 0.2
    for rel, visible in ((0.5 * EPS_G, True), (-0.5 * EPS_G, False)):
        pr = _proj(_gauss([0.0023, 0.0041, near * (1 + rel)], 0.01), near=near)
        assert pr["fragile"][0] == BIT_NEAR, pr["fragile"][0]
        assert (pr["radius"][0] > 0) == visible
        assert pr["frag_rect"][:, 0].any()          # a culled fragile Gaussian keeps its footprint
    for rel in (3 * EPS_G, -3 * EPS_G):
        pr = _proj(_gauss([0.0023, 0.0041, near * (1 + rel)], 0.01), near=near)
        assert pr["fragile"][0] == 0


def test_opacity_bound_of_the_tight_rect_is_flagged():
    # tight rects: k = 2 ln(255 o) + 0.01 <= 0 empties the rect; flagged when |k| <= 10 eps
    for dk, flagged in ((5 * EPS_G, True), (-5 * EPS_G, True), (30 * EPS_G, False), (-30 * EPS_G, False)):
        o = math.exp((dk - 0.01) / 2) / 255
        pr = _proj(_gauss([0.1, 0.05, Z], SIG, opac=o), tight=True)
        assert bool(pr["fragile"][0] & BIT_OPAC) == flagged, (dk, pr["fragile"][0])
        assert (pr["radius"][0] > 0) == (dk > 0)


def test_nearly_singular_covariance_flags_the_determinant():
    c, s = math.cos(math.pi / 8), math.sin(math.pi / 8)      # 45 degrees about z: b != 0
    sig = 0.83                                                # radius 63, away from an integer
    needle = _gauss([0, 0, Z], logscale=[math.log(sig), -40.0, -40.0], quat=(c, 0, 0, s))
    assert _proj(needle)["fragile"][0] == BIT_DET
    flat = _gauss([0, 0, Z], logscale=[math.log(sig), math.log(0.3 * sig), -40.0], quat=(c, 0, 0, s))
    assert _proj(flat)["fragile"][0] == 0


@pytest.mark.parametrize("which", ["x0", "x1", "y0", "y1"])
def test_flipping_a_rect_edge_changes_only_flagged_pixels_in_the_band(which):
    """Both sides of the edge's integer: the rect gains or loses one column (or
    row) of tiles.  Every pixel that changes is flagged on both sides, and the
    Gaussian flags only the documented band -- the tile column (row) on each
    side of the edge, rows (columns) y0 - 1 .. y1 -- where it reaches
    alpha >= (1 - eps)/255."""
    out = {}
    for rel in (0.5 * EPS_G, -0.5 * EPS_G):
        A, pr = _edge_scene(which, rel)
        img, T, last, frag = oracle.render_fwd(pr, eps=EPS_A, eps_d=EPS_D)
        out[rel] = (pr, img, frag)
    (pa, ia, fa), (pb, ib, fb) = out[0.5 * EPS_G], out[-0.5 * EPS_G]
    k = {"x0": 0, "y0": 1, "x1": 2, "y1": 3}[which]
    assert pa["rect"][k, 0] != pb["rect"][k, 0]               # the decision really flips
    # the mean moves by 1e-4 - 4e-4 px between the two sides: every pixel
    # moves continuously by < 1e-5, and where the Gaussian's alpha lies within
    # 1e-3 of 1/255 it may cross the threshold (an alpha decision, pinned
    # above); a tile that gains or loses the Gaussian jumps by at least its
    # alpha >= 1/255 times its colour
    v, u = np.mgrid[0:H, 0:W]

    def alpha(pr):
        mx, my = pr["mean2d"][:, 0]
        a, b, c = pr["conic"][:, 0]
        dx, dy = u + 0.5 - mx, v + 0.5 - my
        return pr["opac"][0] * np.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy)

    near_thr = (np.abs(alpha(pa) * 255 - 1) < 1e-3) | (np.abs(alpha(pb) * 255 - 1) < 1e-3)
    changed = (np.abs(ia - ib).max(axis=0) > 1e-4) & ~near_thr
    assert changed.sum() > 50
    assert np.all(fa[changed] & 8) and np.all(fb[changed] & 8)
    # the band of each side
    for pr, frag in ((pa, fa), (pb, fb)):
        x0, y0, x1, y1 = pr["rect"][:, 0]
        reach = alpha(pr) >= (1 - EPS_A) / 255
        tx, ty = u // 16, v // 16
        iny, inx = (ty >= y0 - 1) & (ty <= y1), (tx >= x0 - 1) & (tx <= x1)
        band = {"x0": iny & ((tx == x0 - 1) | (tx == x0)), "x1": iny & ((tx == x1 - 1) | (tx == x1)),
                "y0": inx & ((ty == y0 - 1) | (ty == y0)), "y1": inx & ((ty == y1 - 1) | (ty == y1))}[which]
        assert np.array_equal((frag & 8) != 0, band & reach)
        # pixels the Gaussian reaches elsewhere in its rect are not flagged
        inside = (tx >= x0) & (tx < x1) & (ty >= y0) & (ty < y1) & reach & ~band
        assert inside.sum() > 1000 and not np.any(frag[inside] & 8)


def splats(means, sig, opac, depth, rgb=None):
    """Directly built 2D records: isotropic footprints, rects over the whole
    256 x 256 image, no projection fragility."""
    n = len(opac)
    rgb = np.full((n, 3), 0.5) if rgb is None else np.asarray(rgb, float)
    return dict(mean2d=np.asarray(means, float).T.copy(),
                conic=np.stack([np.full(n, 1 / sig ** 2), np.zeros(n), np.full(n, 1 / sig ** 2)]),
                opac=np.asarray(opac, float), rgb=rgb.T.copy(), depth=np.asarray(depth, float),
                radius=np.full(n, 3, np.int32), rect=np.tile(np.array([[0], [0], [16], [16]], np.int32), (1, n)),
                fragile=np.zeros(n, np.int32), frag_rect=np.zeros((4, n), np.int32), width=W, height=H)


def _pixel(pr, u=100, v=60):
    img, T, last, frag = oracle.render_fwd(pr, eps=EPS_A, eps_d=EPS_D)
    return img[:, v, u], T[v, u], last[v, u], frag[v, u]


def test_alpha_near_the_threshold_is_flagged():
    # a flat footprint centred on the pixel: alpha = o exactly there
    for o, flag, drawn in ((1 / 255 * (1 + 0.5 * EPS_A), 1, True), (1 / 255 * (1 - 0.5 * EPS_A), 1, False),
                           (1 / 255 * (1 + 3 * EPS_A), 0, True), (1 / 255 * (1 - 3 * EPS_A), 0, False)):
        _, T, last, fr = _pixel(splats([(100.5, 60.5)], 1e6, [o], [1.0]))
        assert fr == flag and (last == 1) == drawn, (o, fr, last)


def test_alpha_near_the_cap_is_flagged():
    for rel, flag in ((0.5 * EPS_A, 1), (-0.5 * EPS_A, 1), (3 * EPS_A, 0), (-3 * EPS_A, 0)):
        col, T, last, fr = _pixel(splats([(100.5, 60.5)], 1e6, [0.99 * (1 + rel)], [1.0]))
        assert fr == flag and last == 1, (rel, fr)
        assert T == pytest.approx(1 - min(0.99, 0.99 * (1 + rel)), rel=1e-12)


def _t3():
    t = 1.0
    for _ in range(3):
        t *= 1.0 - 0.9
    return t


def test_termination_product_near_the_bound_is_flagged():
    # three layers of alpha 0.9 leave T3 ~ 1e-3; a fourth of 1 - 1e-4 (1 + d) / T3
    # makes T (1 - alpha) = 1e-4 (1 + d): kept for d > 0, the stop for d < 0
    for d, flag, n_drawn in ((0.5 * EPS_A, 2, 4), (-0.5 * EPS_A, 2, 3), (3 * EPS_A, 0, 4), (-3 * EPS_A, 0, 3)):
        a4 = 1 - 1e-4 * (1 + d) / _t3()
        pr = splats([(100.5, 60.5)] * 4, 1e6, [0.9, 0.9, 0.9, a4], [1.0, 2.0, 3.0, 4.0])
        _, T, last, fr = _pixel(pr)
        assert fr == flag and last == n_drawn, (d, fr, last)


def test_termination_margin_is_separate_from_the_alpha_margin():
    # eps_t alone governs the termination flag; eps alone the alpha flags
    d = 0.5 * EPS_A
    a4 = 1 - 1e-4 * (1 + d) / _t3()
    pr = splats([(100.5, 60.5)] * 4, 1e6, [0.9, 0.9, 0.9, a4], [1.0, 2.0, 3.0, 4.0])
    assert oracle.render_fwd(pr, eps=EPS_A / 10, eps_t=EPS_A, eps_d=EPS_D)[3][60, 100] == 2
    assert oracle.render_fwd(pr, eps=EPS_A, eps_t=EPS_A / 10, eps_d=EPS_D)[3][60, 100] == 0
    pr = splats([(100.5, 60.5)], 1e6, [1 / 255 * (1 + 0.5 * EPS_A)], [1.0])
    assert oracle.render_fwd(pr, eps=EPS_A, eps_t=0.0, eps_d=EPS_D)[3][60, 100] == 1
    assert oracle.render_fwd(pr, eps=EPS_A / 10, eps_t=1.0, eps_d=EPS_D)[3][60, 100] == 0


def test_near_equal_depths_of_consecutive_contributors_are_flagged():
    for rel, flag in ((0.5 * EPS_D, 4), (3 * EPS_D, 0)):
        pr = splats([(100.5, 60.5)] * 2, 1e6, [0.5, 0.5], [1.0, 1.0 * (1 + rel)])
        _, _, last, fr = _pixel(pr)
        assert fr == flag and last == 2, (rel, fr)
    # depths both sides share (the GPU's own FP32 values) order alike: eps_d < 0 flags no tie
    pr = splats([(100.5, 60.5)] * 2, 1e6, [0.5, 0.5], [1.0, 1.0])
    img, T, last, frag = oracle.render_fwd(pr, eps=EPS_A, eps_d=-1.0)
    assert frag[60, 100] == 0 and last[60, 100] == 2
    assert _pixel(pr)[3] == 4
    # equal-depth non-contributors do not count: the second is below 1/255
    pr = splats([(100.5, 60.5)] * 2, 1e6, [0.5, 0.001], [1.0, 1.0])
    assert _pixel(pr)[3] == 0


@pytest.mark.parametrize("case", ["alpha_min", "alpha_max", "t_min"])
def test_flipping_a_compositing_decision_changes_only_flagged_pixels(case):
    """A random background scene plus one flat Gaussian whose decision sits
    at +-0.5 eps from its threshold on every pixel it reaches: the two renders
    differ only on flagged pixels (and do differ)."""
    rng = np.random.default_rng(5)
    nb = 40
    means = rng.uniform(0, 256, size=(nb, 2))
    base_o = rng.uniform(0.05, 0.6, nb)
    order = rng.permutation(nb) + 2.0
    imgs, frags = [], []
    for s in (0.5, -0.5):
        if case == "t_min":
            lay = [0.9, 0.9, 0.9, 1 - 1e-4 * (1 + s * EPS_A) / _t3()]
            pr = splats([(128.5, 128.5)] * 4, 1e6, lay, [1.0, 2.0, 3.0, 4.0])
        else:
            o = (1 / 255) if case == "alpha_min" else 0.99
            pr = splats(np.vstack([means, [(128.5, 128.5)]]), 20.0,
                        np.concatenate([base_o, [o * (1 + s * EPS_A)]]), np.concatenate([order, [1.0]]))
            pr["conic"][:, -1] = [1e-12, 0, 1e-12]            # flat: the same alpha on every pixel
        img, T, last, frag = oracle.render_fwd(pr, eps=EPS_A, eps_d=EPS_D)
        imgs.append(img)
        frags.append(frag)
    changed = np.any(imgs[0] != imgs[1], axis=0)
    assert changed.any()
    assert np.all(frags[0][changed] != 0) and np.all(frags[1][changed] != 0)
