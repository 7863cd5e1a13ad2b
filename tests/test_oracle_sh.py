"""Pins of the oracle's real spherical-harmonic basis (SH colour of Sec. 3.1)."""
import math

import numpy as np
import pytest

import oracle


def _unit(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_orthonormal_on_sphere():
    # Gauss-Legendre in z times a uniform grid in phi integrates polynomials of
    # degree <= 6 on the sphere exactly.
    z, wz = np.polynomial.legendre.leggauss(8)
    nphi = 16
    phi = 2 * math.pi * np.arange(nphi) / nphi
    Z, PH = np.meshgrid(z, phi, indexing="ij")
    r = np.sqrt(1 - Z ** 2)
    dirs = np.stack([r * np.cos(PH), r * np.sin(PH), Z], -1).reshape(-1, 3)
    w = (wz[:, None] * np.full(nphi, 2 * math.pi / nphi)[None, :]).reshape(-1)
    Y = oracle.sh_basis(3, dirs)
    gram = (Y * w[:, None]).T @ Y
    assert np.abs(gram - np.eye(16)).max() < 1e-12


def test_axis_values_fix_order_and_sign():
    c1 = math.sqrt(3 / (4 * math.pi))
    Y = oracle.sh_basis(1, np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]]))
    assert Y[0, 0] == pytest.approx(0.5 / math.sqrt(math.pi), abs=1e-15)
    # k = l^2 + l + m: k=1 is m=-1 (y), k=2 is m=0 (z), k=3 is m=+1 (x); positive signs
    assert np.allclose(Y[:, 1:], [[0, 0, c1], [c1, 0, 0], [0, c1, 0]], atol=1e-15)
    Y2 = oracle.sh_basis(2, np.array([[0, 0, 1.0]]))
    assert Y2[0, 6] == pytest.approx(0.5 * math.sqrt(5 / math.pi), abs=1e-14)   # Y_20 on the pole


def test_matches_scipy_spherical_harmonics():
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(3)
    d = _unit(rng, 50)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = oracle.sh_basis(3, d)
    for l in range(4):
        for m in range(-l, l + 1):
            cplx = sp.sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                ref = math.sqrt(2) * (-1) ** m * cplx.real
            elif m < 0:
                ref = math.sqrt(2) * (-1) ** m * cplx.imag
            else:
                ref = cplx.real
            assert np.abs(Y[:, l * l + l + m] - ref).max() < 1e-12, (l, m)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    d = _unit(rng, 10) * 1.0
    Y, dY = oracle.sh_basis(3, d, grad=True)
    h = 1e-6
    for e in range(3):
        dp = d.copy(); dp[:, e] += h
        dm = d.copy(); dm[:, e] -= h
        fd = (oracle.sh_basis(3, dp) - oracle.sh_basis(3, dm)) / (2 * h)
        assert np.abs(fd - dY[:, :, e]).max() < 1e-8
