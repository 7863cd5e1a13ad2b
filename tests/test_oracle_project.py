"""Pins of the oracle's EWA projection and SH colour (Eq. 1, Sec. 3.1)."""
import math

import numpy as np
import pytest

import oracle
from paper_2412_04469_gb300 import synthetic as S


def _cam(W=64, H=48, f=50.0, R=None, t=None, campos=None, near=0.2):
    R = np.eye(3) if R is None else R
    t = np.zeros(3) if t is None else t
    campos = -R.T @ t if campos is None else campos
    return oracle.OracleCamera(R, t, f, f, W / 2, H / 2, W, H, near, campos)


def _one(p, quat=(1, 0, 0, 0), logscale=(0, 0, 0), logit_o=0.0, sh=None, degree=0):
    K = (degree + 1) ** 2
    A = np.zeros((11 + 3 * K, 1))
    A[0:3, 0] = p
    A[3:7, 0] = quat
    A[7:10, 0] = logscale
    A[10, 0] = logit_o
    if sh is not None:
        A[11:, 0] = np.asarray(sh).reshape(-1)
    return A


@pytest.mark.parametrize("blur", [0.0, 0.3])
def test_isotropic_on_axis(blur):
    f, z, sig = 50.0, 3.0, 0.05
    cam = _cam(f=f)
    r = oracle.project(_one([0, 0, z], quat=(0.3, -0.2, 0.5, 0.1), logscale=[math.log(sig)] * 3), cam, 0, blur=blur)
    v = (f * sig / z) ** 2 + blur
    assert r["mean2d"][:, 0] == pytest.approx([32.0, 24.0], abs=1e-12)
    assert r["conic"][:, 0] == pytest.approx([1 / v, 0.0, 1 / v], rel=1e-12, abs=1e-14)
    assert r["radius"][0] == math.ceil(3 * math.sqrt(v + math.sqrt(0.1)))
    assert r["depth"][0] == z
    assert r["opac"][0] == 0.5


def test_off_axis_jacobian():
    f, x, z, sig = 50.0, 0.6, 2.0, 0.1
    cam = _cam(W=200, H=100, f=f)
    r = oracle.project(_one([x, 0, z], logscale=[math.log(sig)] * 3), cam, 0, blur=0.0)
    a = sig ** 2 * f ** 2 / z ** 2 * (1 + x ** 2 / z ** 2)   # J = [[f/z, 0, -f x/z^2], [0, f/z, 0]]
    c = sig ** 2 * f ** 2 / z ** 2
    assert r["mean2d"][:, 0] == pytest.approx([f * x / z + 100, 50], abs=1e-12)
    assert r["conic"][:, 0] == pytest.approx([1 / a, 0, 1 / c], rel=1e-12, abs=1e-14)


def test_jacobian_clamp():
    f, W, z, sig = 50.0, 64, 1.0, 0.5   # large enough to reach the image from off screen
    lim = 1.3 * 0.5 * W / f
    x = 1.5   # x/z = 1.5 > lim = 0.832; the mean still uses x/z
    cam = _cam(W=W, H=64, f=f)
    r = oracle.project(_one([x, 0.0, z], logscale=[math.log(sig)] * 3), cam, 0, blur=0.0)
    a = sig ** 2 * f ** 2 / z ** 2 * (1 + lim ** 2)
    assert 1 / r["conic"][0, 0] == pytest.approx(a, rel=1e-12)
    assert r["mean2d"][0, 0] == pytest.approx(f * x / z + W / 2, abs=1e-12)


def test_rotated_anisotropic_fixes_quaternion_convention():
    f, z, th = 40.0, 2.0, 0.7
    s1, s2, s3 = 0.2, 0.05, 0.1
    cam = _cam(f=f)
    q = (math.cos(th / 2), 0, 0, math.sin(th / 2))          # rotation by +th about z, (w, x, y, z)
    r = oracle.project(_one([0, 0, z], quat=q, logscale=np.log([s1, s2, s3])), cam, 0, blur=0.0)
    c, s = math.cos(th), math.sin(th)
    k = (f / z) ** 2
    a, b, cc = k * (s1 ** 2 * c * c + s2 ** 2 * s * s), k * (s1 ** 2 - s2 ** 2) * c * s, k * (s1 ** 2 * s * s + s2 ** 2 * c * c)
    det = a * cc - b * b
    assert r["conic"][:, 0] == pytest.approx([cc / det, -b / det, a / det], rel=1e-12)
    # unnormalised quaternions give the same result
    r2 = oracle.project(_one([0, 0, z], quat=np.array(q) * 3.7, logscale=np.log([s1, s2, s3])), cam, 0, blur=0.0)
    assert np.allclose(r2["conic"], r["conic"], rtol=1e-13)


def test_look_at_camera_convention():
    cam = S.make_camera(128, 128, 60.0, eye=(0.0, 0.0, 4.0))
    f = cam.fx
    A = np.concatenate([_one([0, 0, 0]), _one([1, 0, 0]), _one([0, 1, 0])], axis=1)
    r = oracle.project(A, cam, 0, blur=0.0)
    assert r["depth"] == pytest.approx([4, 4, 4], abs=1e-6)
    assert r["mean2d"][:, 0] == pytest.approx([64, 64], abs=1e-5)
    assert r["mean2d"][:, 1] == pytest.approx([64 + f / 4, 64], abs=1e-5)    # world +x to the right
    assert r["mean2d"][:, 2] == pytest.approx([64, 64 - f / 4], abs=1e-5)    # world +y up in the image


def test_culling_and_rect():
    cam = _cam(W=64, H=48, f=50.0, near=0.2)
    A = np.concatenate([_one([0, 0, 0.19]), _one([0, 0, -1.0]), _one([5.0, 0, 1.0]),
                        _one([0.1, 0.05, 1.0], logscale=[math.log(0.02)] * 3)], axis=1)
    r = oracle.project(A, cam, 0, blur=0.3)
    assert list(r["radius"][:3]) == [0, 0, 0]                   # near plane, behind, off screen
    assert np.all(r["rect"][:, :3] == 0)
    mx, my, rad = 50 * 0.1 + 32, 50 * 0.05 + 24, r["radius"][3]
    v = (50 * 0.02) ** 2 + 0.3
    assert rad == math.ceil(3 * math.sqrt(v + math.sqrt(0.1)))
    exp = [max(0, math.floor((mx - rad) / 16)), max(0, math.floor((my - rad) / 16)),
           min(4, math.floor((mx + rad + 15) / 16)), min(3, math.floor((my + rad + 15) / 16))]
    assert list(r["rect"][:, 3]) == exp


def test_sh_colour():
    cam = _cam(f=50.0)
    c0, c1 = 0.5 / math.sqrt(math.pi), math.sqrt(3 / (4 * math.pi))
    sh = np.zeros((4, 3))
    sh[0] = [0.2, -0.4, -3.0]     # DC
    sh[3] = [0.5, 0.0, 0.0]       # k = 3: Y_{1,+1} ~ x
    sh[1] = [0.0, 0.7, 0.0]       # k = 1: Y_{1,-1} ~ y
    p = np.array([0.6, 0.0, 0.8])  # direction from the camera centre (origin) = p
    r = oracle.project(_one(p, sh=sh, degree=1), cam, 1, blur=0.3)
    exp = [0.5 + c0 * 0.2 + c1 * 0.6 * 0.5, 0.5 - c0 * 0.4, 0.0]   # blue clamps at 0
    assert r["rgb"][:, 0] == pytest.approx(exp, abs=1e-14)


@pytest.mark.parametrize("blur,degree", [(0.3, 3), (0.0, 1)])
def test_backward_matches_finite_differences(blur, degree):
    rng = np.random.default_rng(11 + degree)
    n = 12
    cam = S.make_camera(96, 64, 60.0, eye=(1.0, 0.5, 4.0))
    A = S.make_scene(n, degree, seed=5).astype(np.float64)
    A[7:10] += 1.0       # larger Gaussians
    A[0, 0] = 2.6        # one Gaussian past the Jacobian clamp in x
    oc = oracle.OracleCamera.of(cam)
    r = oracle.project(A, oc, degree, blur=blur)
    assert r["radius"].min() > 0
    W = {k: rng.standard_normal(r[k].shape) for k in ("mean2d", "conic", "opac", "rgb")}
    W["conic"] *= 0.01

    def f(Ax):
        q = oracle.project(Ax, oc, degree, blur=blur)
        return sum((W[k] * q[k]).sum() for k in W)

    dA = oracle.project_bwd(A, oc, degree, W["mean2d"], W["conic"], W["opac"], W["rgb"], blur=blur)
    h = 1e-6
    for plane in range(A.shape[0]):
        for i in range(n):
            Ap = A.copy(); Ap[plane, i] += h
            Am = A.copy(); Am[plane, i] -= h
            fd = (f(Ap) - f(Am)) / (2 * h)
            assert fd == pytest.approx(dA[plane, i], rel=2e-5, abs=1e-6), (plane, i)
