"""Pins of the oracle's loss, Eq. 9-10 score/gate initialisation, Adam and
static-skip MLP; plus an end-to-end finite-difference check of the whole
decode -> project -> composite chain."""
import math

import numpy as np
import pytest

import oracle
from paper_2412_04469_gb300 import synthetic as S
from paper_2412_04469_gb300.synthetic import DecoderLayout

TAU, G0, G1 = 0.3, -0.5, 1.01


def test_l1_closed_form():
    img = np.array([[[0.5, 0.2], [0.1, 0.9]]] * 3)
    tgt = np.array([[[0.4, 0.2], [0.3, 0.5]]] * 3)
    loss, g = oracle.l1_loss(img, tgt)
    assert loss == pytest.approx((0.1 + 0 + 0.2 + 0.4) / 4)
    assert np.array_equal(g[0], np.array([[1, 0], [-1, 1]]) / 12)


def test_gate_init_median_rule_and_round_trip():
    d = np.array([[3.0, 1.0, 2.0, 0.0], [0.0, 0.0, 0.0, 0.0]])
    la, nrm, med = oracle.gate_init(d, TAU, G0, G1, nonzero_median=False)
    assert med == 1.0                                   # lower median of (0, 1, 2, 3)
    p = 1 / (1 + np.exp(-(la - TAU * math.log(-G0 / G1))))
    assert p == pytest.approx([0.75, 0.5, 2 / 3, 1e-6], rel=1e-9)
    la0, _, med0 = oracle.gate_init(np.array([[0.0, 0.0, 5.0], [0.0, 0.0, 0.0]]), TAU, G0, G1, nonzero_median=False)
    p0 = 1 / (1 + np.exp(-(la0 - TAU * math.log(-G0 / G1))))
    assert med0 == 0.0 and p0 == pytest.approx([1e-6, 1e-6, 1 - 1e-6], rel=1e-9)
    # median over the non-zero scores only: (1, 2, 3) -> 2; zero scores get p = 0 (clamped)
    la2, _, med2 = oracle.gate_init(d, TAU, G0, G1)
    p2 = 1 / (1 + np.exp(-(la2 - TAU * math.log(-G0 / G1))))
    assert med2 == 2.0 and p2 == pytest.approx([0.6, 1 / 3, 0.5, 1e-6], rel=1e-9)
    assert oracle.gate_init(np.zeros((2, 3)), TAU, G0, G1)[2] == 0.0


def test_viewspace_score_linearity_and_zero():
    A = S.make_scene(150, 0, 3).astype(np.float64)
    A[7:10] += 0.8
    cams = S.make_arc_cameras(2, 48, 32, arc_deg=40)
    projs = [oracle.project(A, c, 0) for c in cams]
    I_prev = [S.make_image(48, 32, 1 + v) for v in range(2)]
    I_new = [S.make_image(48, 32, 11 + v) for v in range(2)]
    d = oracle.viewspace_score(projs, I_new, I_prev)
    # Eq. 9 is linear in the target: one backward of 2 (I_prev - I_new) / (3 H W) per view
    lin = sum(oracle.render_bwd(p, 2 * (ip - inew) / ip.size)["d_mean2d"]
              for p, inew, ip in zip(projs, I_new, I_prev)) / 2
    assert np.abs(d - lin).max() <= 1e-9 * max(1.0, np.abs(lin).max())   # the two terms cancel
    assert np.abs(d).max() > 0
    assert np.all(oracle.viewspace_score(projs, I_prev, I_prev) == 0)


def test_adam_closed_form_steps():
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = np.array([1.0, 1.0, 1.0]), np.zeros(3), np.zeros(3)
    lr, eps = 0.01, 1e-8
    for step in (1, 2):
        p, m, v = oracle.adam_step(p, g, m, v, step, lr, eps=eps)
    # constant gradient: bias-corrected moments are g and g^2 at every step
    assert p == pytest.approx(1.0 - 2 * lr * g / (np.abs(g) + eps), rel=1e-12)
    p2, m2, v2 = oracle.adam_step(p, g, m, v, 3, lr, mask=np.array([0, 1, 0]))
    assert p2[1] == p[1] and m2[1] == m[1] and v2[1] == v[1] and p2[0] != p[0]


def _mlp_params(rng, scale=0.3):
    return {"W1": rng.standard_normal((64, 16)) * scale, "b1": rng.standard_normal(64) * 0.1,
            "W2": rng.standard_normal((64, 64)) * scale / 2, "b2": rng.standard_normal(64) * 0.1,
            "W3": rng.standard_normal((1, 64)) * scale, "b3": rng.standard_normal(1) * 0.1}


def test_mlp_hand_example_and_bce():
    P = {k: np.zeros_like(v) for k, v in _mlp_params(np.random.default_rng(0)).items()}
    P["W1"][0, 0] = 2.0; P["b1"][0] = -1.0          # h1_0 = relu(2 x0 - 1)
    P["W2"][3, 0] = 1.5                            # h2_3 = relu(1.5 h1_0)
    P["W3"][0, 3] = -1.0; P["b3"][0] = 0.25        # logit = 0.25 - h2_3
    X = np.zeros((2, 16)); X[0, 0] = 1.0; X[1, 0] = 0.2
    z, _ = oracle.mlp_forward(X, P)
    assert z == pytest.approx([0.25 - 1.5, 0.25])
    loss, dz = oracle.bce_loss(np.zeros(4), np.array([0, 1, 1, 0]))
    assert loss == pytest.approx(math.log(2)) and dz == pytest.approx([0.125, -0.125, -0.125, 0.125])


def test_mlp_backward_finite_differences():
    rng = np.random.default_rng(5)
    P = _mlp_params(rng)
    X = rng.standard_normal((9, 16))
    y = (rng.uniform(size=9) > 0.5).astype(float)

    def f(Q):
        return oracle.bce_loss(oracle.mlp_forward(X, Q)[0], y)[0]

    z, cache = oracle.mlp_forward(X, P)
    g = oracle.mlp_backward(oracle.bce_loss(z, y)[1], P, cache)
    h = 1e-6
    for k in P:
        flat = P[k].reshape(-1)
        for j in rng.choice(flat.size, size=min(flat.size, 25), replace=False):
            Qp = {kk: vv.copy() for kk, vv in P.items()}; Qp[k].reshape(-1)[j] += h
            Qm = {kk: vv.copy() for kk, vv in P.items()}; Qm[k].reshape(-1)[j] -= h
            fd = (f(Qp) - f(Qm)) / (2 * h)
            assert fd == pytest.approx(g[k].reshape(-1)[j], rel=1e-5, abs=1e-9), (k, j)


@pytest.mark.parametrize("n,W,H,grow", [(16, 32, 32, 1.0), (500, 64, 64, 0.5)])
def test_chain_decode_project_render_finite_differences(n, W, H, grow):
    """Eq. 11's reconstruction term through Eq. 2, Eq. 1 and Eq. 4-8: the chained
    oracle adjoints equal central differences of the forward chain, on a tiny
    scene and on the 500-Gaussian 64 x 64 slice (20 sampled parameters of each
    kind)."""
    rng = np.random.default_rng(8)
    deg = 1
    lay = DecoderLayout.default(sh_degree=deg, latent=3)
    prev = S.make_scene(n, deg, 21).astype(np.float64)
    prev[7:10] += grow
    res = S.make_residuals(n, lay, 21)
    lat = res.lat.astype(np.float64)
    dec = rng.standard_normal(lay.n_dec) * 0.02
    lp = rng.standard_normal((3, n)) * 0.01
    la = rng.uniform(-0.5, 0.5, n)
    oc = oracle.OracleCamera.of(S.make_camera(W, H, 60.0, eye=(0.5, 0.3, 4.0)))
    bg = (0.1, 0.1, 0.1)
    c_reg = 0.01

    def forward(lat_, dec_, lp_, la_):
        A, _, lreg = oracle.decode(prev, lat_, dec_, lp_, la_, lay, TAU, G0, G1, round_latents=False)
        pr = oracle.project(A, oc, deg, eps_g=1e-5)
        img, _, last, frag = oracle.render_fwd(pr, bg=bg, eps=1e-4, eps_d=1e-6)
        return A, pr, img, lreg, last, frag

    A, pr, img, lreg, last0, frag = forward(lat, dec, lp, la)
    Wt = rng.standard_normal(img.shape) * (frag == 0)[None]
    g2 = oracle.render_bwd(pr, Wt, bg=bg)
    dA = oracle.project_bwd(A, oc, deg, g2["d_mean2d"], g2["d_conic"], g2["d_opac"], g2["d_rgb"])
    d_lat, d_dec, d_lp, d_la = oracle.decode_bwd(lat, dec, lp, la, lay, TAU, G0, G1, dA, c_reg,
                                                 round_latents=False)
    h = 1e-6
    checked = nonzero = 0
    for name, x, gx in (("lat", lat, d_lat), ("dec", dec, d_dec), ("lp", lp, d_lp), ("la", la, d_la)):
        flat = x.reshape(-1)
        for j in rng.choice(flat.size, size=min(flat.size, 20), replace=False):
            vals = []
            for s in (1, -1):
                xx = flat.copy(); xx[j] += s * h
                args = {"lat": lat, "dec": dec, "lp": lp, "la": la, name: xx.reshape(x.shape)}
                _, _, im, lr, last, _ = forward(args["lat"], args["dec"], args["lp"], args["la"])
                vals.append(((Wt * im).sum() + c_reg * lr, np.array_equal(last, last0)))
            if not (vals[0][1] and vals[1][1]):
                continue
            fd = (vals[0][0] - vals[1][0]) / (2 * h)
            assert fd == pytest.approx(gx.reshape(-1)[j], rel=1e-4, abs=1e-7), (name, j)
            checked += 1
            nonzero += abs(gx.reshape(-1)[j]) > 1e-5
    assert checked >= 60 and nonzero >= 40


def test_skip_features_hand_example():
    # two Gaussians: |d| = (5, 0) -> lower median of (0, 5) is 0 -> p = (1, 0)
    score = np.array([[3.0, 0.0], [4.0, 0.0]])
    prev = np.zeros((14, 2))
    prev[0:3, 0] = [0.1, 0.2, 0.3]
    prev[7:10, 1] = [-3.0, -1.0, -5.0]
    prev[10] = [0.0, 100.0]
    X = oracle.skip_features(score, prev, np.array([0.5, 0.0]), np.array([TAU * math.log(-G0 / G1), 0.0]),
                             np.array([[0.01, 0.0], [0.0, 0.0], [0.0, 0.0]]), TAU, G0, G1, nonzero_median=False)
    assert list(X[0]) == [1.0, 0.0] and list(X[1]) == [0.0, 0.0]
    assert X[2, 0] == pytest.approx(0.6) and X[3, 0] == pytest.approx(0.8) and X[2, 1] == 0.0
    assert list(X[4:7, 0]) == [0.1, 0.2, 0.3]
    assert list(X[7]) == [0.5, 0.0] and X[8, 0] == pytest.approx(0.5)
    assert X[9, 0] == 0.5 and X[9, 1] == pytest.approx(1.0)
    assert list(X[10:13, 1]) == [0.0, 1.0, -1.0]
    assert X[13, 0] == pytest.approx(0.5) and X[13, 1] == 0.0
    assert list(X[14]) == [0.0, 1.0] and list(X[15]) == [1.0, 1.0]
    # a positive median switches on the log-ratio feature
    X2 = oracle.skip_features(np.array([[1.0, 2.0, 4.0], [0.0, 0.0, 0.0]]), np.zeros((14, 3)), np.zeros(3),
                              np.zeros(3), np.zeros((3, 3)), TAU, G0, G1, nonzero_median=False)
    assert X2[0] == pytest.approx([1 / 3, 0.5, 2 / 3])
    assert X2[1] == pytest.approx(np.log(np.array([0.5, 1.0, 2.0]) + 1e-6) / 4)
