"""Pins of the oracle's residual decode and gate (Eq. 4-8, Sec. 3.2)."""
import numpy as np
import pytest

import oracle
from paper_2412_04469_gb300.synthetic import DecoderLayout
from tests._golden import load

TAU, G0, G1 = 0.3, -0.5, 1.01   # N3DV row of the gate hyper-parameter table (App. B)


def _hand_layout():
    return DecoderLayout([3], [2], [3])


def test_hand_example_eq5():
    g = load("decode_hand.txt")
    lay = _hand_layout()
    n = 2
    prev = np.zeros((11, n))
    lat = g["LHAT"].reshape(3, n)
    out, gate, lreg = oracle.decode(prev, lat, g["D"], np.zeros((3, n)), np.zeros(n), lay, TAU, G0, G1)
    r = g["R"].reshape(n, 2).T    # fixture lists r per Gaussian
    assert np.array_equal(out[3:5], r)
    assert np.all(out[:3] == 0) and np.all(out[5:] == 0)


def test_gate_closed_forms():
    g = load("decode_hand.txt")
    lay = _hand_layout()
    x0, x1 = -G0 / (G1 - G0), (1 - G0) / (G1 - G0)
    thr0 = TAU * np.log(x0 / (1 - x0))   # below this log alpha the stretched gate is <= 0
    thr1 = TAU * np.log(x1 / (1 - x1))   # above it the stretched gate is >= 1
    la = np.array([0.0, thr0 - 1e-9, thr0 - 5.0, thr0 + 1e-3, thr1 + 1e-9, thr1 + 5, g["LA_HALF"][0]])
    n = la.size
    lp = np.ones((3, n))
    out, gate, lreg = oracle.decode(np.zeros((11, n)), np.zeros((3, n)), np.zeros(6), lp, la, lay, TAU, G0, G1)
    assert gate[0] == pytest.approx(g["GATE0"][0], abs=1e-15)
    assert gate[1] == 0.0 and gate[2] == 0.0 and gate[3] > 0.0
    assert gate[4] == 1.0 and gate[5] == 1.0
    assert np.array_equal(out[0], gate) and np.array_equal(out[2], gate)   # dp = g l_p
    # L_reg of Eq. 8 is a sum of sigmoids; at LA_HALF the term is exactly 1/2
    _, _, l_half = oracle.decode(np.zeros((11, 1)), np.zeros((3, 1)), np.zeros(6), np.zeros((3, 1)),
                                 g["LA_HALF"], lay, TAU, G0, G1)
    assert l_half == pytest.approx(0.5, abs=1e-14)
    ref = sum(1 / (1 + np.exp(-(v - TAU * np.log(-G0 / G1)))) for v in la)
    assert lreg == pytest.approx(ref, rel=1e-14)


def test_rounding_half_even_and_saturation():
    lay = DecoderLayout([3], [1], [1])
    vals = np.array([0.5, 1.5, 2.5, -0.5, -1.5, 127.6, 200.0, -128.4, -300.0, 0.49999997])
    exp = np.array([0, 2, 2, 0, -2, 127, 127, -128, -128, 0], float)
    n = vals.size
    out, _, _ = oracle.decode(np.zeros((11, n)), vals[None, :], np.array([1.0]), np.zeros((3, n)),
                              np.zeros(n), lay, TAU, G0, G1)
    assert np.array_equal(out[3], exp)


def test_adds_to_previous_attributes():
    rng = np.random.default_rng(0)
    lay = DecoderLayout.default(sh_degree=0, latent=4)
    n = 5
    prev = rng.standard_normal((14, n))
    zero = oracle.decode(prev, np.zeros((lay.n_latent, n)), rng.standard_normal(lay.n_dec),
                         np.zeros((3, n)), np.full(n, -10.0), lay, TAU, G0, G1)[0]
    assert np.array_equal(zero, prev)    # Eq. 4 with R_t = 0


def _rand_problem(rng, n, lay):
    prev = rng.standard_normal((11 + 3, n))
    lat = rng.standard_normal((lay.n_latent, n)) * 2
    dec = rng.standard_normal(lay.n_dec) * 0.1
    lp = rng.standard_normal((3, n)) * 0.1
    la = rng.uniform(-0.6, 0.6, n)      # inside the open interval where 0 < g~ < 1
    return prev, lat, dec, lp, la


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    lay = DecoderLayout([3, 7, 10, 11], [4, 3, 1, 3], [3, 2, 2, 4])
    n = 6
    prev, lat, dec, lp, la = _rand_problem(rng, n, lay)
    W = rng.standard_normal((14, n))
    c_reg = 0.37

    def f(lat_, dec_, lp_, la_):
        out, _, lreg = oracle.decode(prev, lat_, dec_, lp_, la_, lay, TAU, G0, G1, round_latents=False)
        return (W * out).sum() + c_reg * lreg

    d_lat, d_dec, d_lp, d_la = oracle.decode_bwd(lat, dec, lp, la, lay, TAU, G0, G1, W, c_reg,
                                                 round_latents=False)
    h = 1e-6
    for name, x, g in (("lat", lat, d_lat), ("dec", dec, d_dec), ("lp", lp, d_lp), ("la", la, d_la)):
        flat = x.reshape(-1)
        for j in range(flat.size):
            xp = flat.copy(); xp[j] += h
            xm = flat.copy(); xm[j] -= h
            args = {"lat": lat, "dec": dec, "lp": lp, "la": la}
            args[name] = xp.reshape(x.shape); fp = f(args["lat"], args["dec"], args["lp"], args["la"])
            args[name] = xm.reshape(x.shape); fm = f(args["lat"], args["dec"], args["lp"], args["la"])
            fd = (fp - fm) / (2 * h)
            assert fd == pytest.approx(g.reshape(-1)[j], rel=1e-6, abs=1e-8), (name, j)


def test_backward_ste_and_gate_clamp():
    rng = np.random.default_rng(2)
    lay = DecoderLayout([3], [2], [2])
    n = 4
    lat = rng.standard_normal((2, n))
    dec = rng.standard_normal(4)
    la = np.array([-5.0, 5.0, 0.0, 0.1])   # g clamped to 0, to 1, open, open
    d_out = rng.standard_normal((14, n))
    d_lat, d_dec, d_lp, d_la = oracle.decode_bwd(lat, dec, np.ones((3, n)), la, lay, TAU, G0, G1, d_out)
    D = dec.reshape(2, 2)
    assert np.allclose(d_lat, D.T @ d_out[3:5], atol=1e-15)      # STE: identity through rounding
    lint = np.rint(lat)
    assert np.allclose(d_dec.reshape(2, 2), d_out[3:5] @ lint.T, atol=1e-14)
    assert d_la[0] == 0.0 and d_la[1] == 0.0 and d_la[2] != 0.0


def test_skip_mask_excludes_gaussians():
    rng = np.random.default_rng(3)
    lay = DecoderLayout([3, 7], [4, 3], [2, 3])
    n = 8
    prev, lat, dec, lp, la = _rand_problem(rng, n, lay)
    d_out = rng.standard_normal((14, n))
    skip = np.array([0, 1, 0, 0, 1, 1, 0, 0], np.uint8)
    full = oracle.decode_bwd(lat, dec, lp, la, lay, TAU, G0, G1, d_out, 0.1, skip=skip)
    keep = skip == 0
    sub = oracle.decode_bwd(lat[:, keep], dec, lp[:, keep], la[keep], lay, TAU, G0, G1, d_out[:, keep], 0.1)
    assert np.allclose(full[1], sub[1], rtol=1e-13, atol=1e-15)
    for a, b in ((full[0], sub[0]), (full[2], sub[2])):
        assert np.all(a[:, ~keep] == 0) and np.allclose(a[:, keep], b)
    assert np.all(full[3][~keep] == 0) and np.allclose(full[3][keep], sub[3])
