"""GPU parity of the viewspace gradient difference (Eq. 9), gate
initialisation (Eq. 10) and the static-skip MLP kernels against the oracle,
through the C ABI, on seeded inputs; and the skip's in-iteration un-skipping
of composited Gaussians against plain training."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2412_04469_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

TAU, G0, G1 = 0.3, -0.5, 1.01
EPS_A, EPS_D, EPS_G = 2e-5, 1e-6, 2e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_04469_gb300 import build
    build.build()


def B():
    from paper_2412_04469_gb300 import binding
    return binding


def up(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def planes(a, stride):
    t = torch.zeros((a.shape[0], stride), device="cuda")
    t[:, :a.shape[1]] = up(a)
    return t


def close(got, ref, rtol=1e-4, floor_frac=0.05, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = max(np.abs(ref).max(), 1e-30)
    err = np.abs(got - ref) / np.maximum(np.abs(ref), floor_frac * scale)
    assert float(err.max()) <= rtol, f"{what}: max scaled error {float(err.max()):.3e} > {rtol:.1e}"


def test_viewspace_score_and_gate_init_match_oracle():
    from paper_2412_04469_gb300.pipeline import Rasterizer
    n, deg, W, H, V = 1500, 1, 96, 64, 2
    A = S.make_scene(n, deg, 7)
    A[7:10] += 0.6
    cams = S.make_arc_cameras(V, W, H, arc_deg=30)
    I_prev = [S.make_image(W, H, 20 + v) for v in range(V)]
    I_new = [S.make_image(W, H, 40 + v) for v in range(V)]
    projs = [oracle.project(A.astype(np.float64), c, deg, blur=0.3, eps_g=EPS_G, tight=True) for c in cams]
    for v in range(V):                       # no upstream gradient on pixels near an FP32-flippable decision
        frag = oracle.render_fwd(projs[v], eps=EPS_A, eps_d=EPS_D)[3] != 0
        I_new[v][:, frag] = I_prev[v][:, frag]
    Sd = (n + 31) // 32 * 32
    attrs = planes(A, Sd)
    r = Rasterizer(n, Sd, deg, W, H, 1 << 20)
    score = torch.zeros((2, Sd), device="cuda")
    for v, cam in enumerate(cams):
        c = B().make_camera(cam)
        r.project(attrs, c, 0.3)
        r.bin_sort(sync=True)
        r.render_fwd(c, (0, 0, 0))
        B().qn_image_loss(3 * W * H, up(I_prev[v]), up(I_new[v]), 1.0, True, r.loss, r.d_img)
        r.render_bwd(c, (0, 0, 0))
        B().qn_viewspace_accum(n, Sd, r.d_splats, 1.0 / V, score)
    norms = torch.zeros(n, device="cuda")
    med = torch.zeros(1, device="cuda")
    la = torch.zeros(n, device="cuda")
    B().qn_gate_init(n, Sd, score, B().make_gate(TAU, G0, G1), norms, med, la)
    torch.cuda.synchronize()
    d_ref = oracle.viewspace_score(projs, I_new, I_prev)
    close(score.cpu().numpy()[:, :n], d_ref, what="score d_t")
    la_ref, nrm_ref, med_ref = oracle.gate_init(d_ref, TAU, G0, G1)
    close(norms.cpu().numpy(), nrm_ref, what="norms")
    assert float(med.item()) == pytest.approx(med_ref, rel=1e-4)
    # log alpha = logit(p) + c is steep near p = 0 and 1: compare p itself
    shift = TAU * math.log(-G0 / G1)
    p_gpu = 1 / (1 + np.exp(-(la.cpu().numpy().astype(np.float64) - shift)))
    p_ref = 1 / (1 + np.exp(-(la_ref - shift)))
    close(p_gpu, p_ref, floor_frac=0.01, what="gate probability")


@pytest.mark.parametrize("nonzero", [False, True])
def test_gate_init_median_edge_cases(nonzero):
    n = 6
    cases = ((np.array([[3.0, 1.0, 2.0, 0.0, 5.0, 4.0], [0.0] * 6]), 3.0 if nonzero else 2.0),
             (np.zeros((2, 6)), 0.0))
    for d, med_ref in cases:
        score = planes(d, 8)
        norms, med, la = torch.zeros(n, device="cuda"), torch.zeros(1, device="cuda"), torch.zeros(n, device="cuda")
        B().qn_gate_init(n, 8, score, B().make_gate(TAU, G0, G1), norms, med, la, nonzero_median=nonzero)
        torch.cuda.synchronize()
        la_ref, _, m = oracle.gate_init(d, TAU, G0, G1, nonzero_median=nonzero)
        assert m == med_ref and float(med.item()) == med_ref
        assert np.allclose(la.cpu().numpy(), la_ref, atol=2e-4)


def test_skip_features_match_oracle():
    n, deg = 2000, 1
    rng = np.random.default_rng(3)
    A = S.make_scene(n, deg, 3)
    score = rng.standard_normal((2, n)).astype(np.float32) * np.exp(rng.normal(-9, 2, n)).astype(np.float32)
    gate = np.where(rng.uniform(size=n) < 0.7, 0.0, rng.uniform(size=n)).astype(np.float32)
    la = rng.normal(-1, 2, n).astype(np.float32)
    lp = (rng.standard_normal((3, n)) * 0.01).astype(np.float32)
    Sd = 2016
    sc = planes(score, Sd)
    norms, med, lad = torch.zeros(n, device="cuda"), torch.zeros(1, device="cuda"), torch.zeros(n, device="cuda")
    gp = B().make_gate(TAU, G0, G1)
    B().qn_gate_init(n, Sd, sc, gp, norms, med, lad)
    X = torch.zeros((16, Sd), device="cuda")
    for pst in (None, (rng.uniform(size=n) < 0.5).astype(np.uint8)):
        B().qn_skip_features(n, Sd, A.shape[0], sc, med, planes(A, Sd), up(gate), up(la), planes(lp, Sd), gp, X,
                             prev_static=None if pst is None else up(pst, torch.uint8))
        torch.cuda.synchronize()
        ref = oracle.skip_features(score, A, gate, la, lp, TAU, G0, G1, prev_static=pst)
        got = X.cpu().numpy()[:, :n]
        for f in range(16):
            close(got[f], ref[f], floor_frac=0.01, what=f"feature {f}")


def test_skip_labels_zero_residual():
    n, S_ = 7, 8
    gate = np.array([0, 0, 0, 0.3, 0, 1.0, 0], np.float32)
    lat = np.zeros((3, n), np.float32)
    lat[:, 1] = [0.4, -0.49, 0.5]          # rounds to (0, 0, 0): half to even
    lat[2, 2] = 1.5                        # rounds to 2
    lat[0, 6] = -0.51                      # rounds to -1
    labels = torch.zeros(n, device="cuda", dtype=torch.uint8)
    B().qn_skip_labels(n, S_, 3, up(gate), planes(lat, S_), labels)
    torch.cuda.synchronize()
    assert list(labels.cpu().numpy()) == [1, 1, 0, 0, 1, 0, 0]
    # with composited marks: a Gaussian that received an image gradient is not static
    hit = torch.zeros(n, device="cuda", dtype=torch.uint8)
    B().qn_or_marks(n, up(np.array([0, 1, 0, 0, 0, 0, 0], np.uint8), torch.uint8), hit)
    B().qn_or_marks(n, up(np.array([0, 0, 0, 1, 2, 0, 0], np.uint8), torch.uint8), hit)
    assert list(hit.cpu().numpy()) == [0, 1, 0, 1, 1, 0, 0]
    B().qn_skip_labels(n, S_, 3, up(gate), planes(lat, S_), labels, hit=hit)
    torch.cuda.synchronize()
    assert list(labels.cpu().numpy()) == [1, 0, 0, 0, 0, 0, 0]


def _mlp_params(seed):
    rng = np.random.default_rng(seed)
    flat = np.concatenate([rng.standard_normal(1024) * 0.3, rng.standard_normal(64) * 0.1,
                           rng.standard_normal(4096) * 0.15, rng.standard_normal(64) * 0.1,
                           rng.standard_normal(64) * 0.3, rng.standard_normal(1) * 0.1]).astype(np.float32)
    flat = S.to_bf16_values(flat)
    P = {"W1": flat[0:1024].reshape(64, 16).astype(np.float64), "b1": flat[1024:1088].astype(np.float64),
         "W2": flat[1088:5184].reshape(64, 64).astype(np.float64), "b2": flat[5184:5248].astype(np.float64),
         "W3": flat[5248:5312].reshape(1, 64).astype(np.float64), "b3": flat[5312:5313].astype(np.float64)}
    return flat, P


def _flat(g):
    return np.concatenate([g["W1"].reshape(-1), g["b1"], g["W2"].reshape(-1), g["b2"], g["W3"].reshape(-1), g["b3"]])


@pytest.mark.parametrize("n", [1, 33, 5000])
def test_skip_mlp_forward_and_backward_match_oracle(n):
    flat, P = _mlp_params(n)
    rng = np.random.default_rng(n + 1)
    X = rng.standard_normal((16, n)).astype(np.float32)
    y = (rng.uniform(size=n) < 0.8).astype(np.uint8)
    Sd = (n + 31) // 32 * 32
    Xd = planes(X, Sd)
    pb = up(S.bf16_bits(flat).view(np.int16), torch.int16).view(torch.bfloat16)
    logits = torch.zeros(n, device="cuda")
    skip = torch.zeros(n, device="cuda", dtype=torch.uint8)
    B().qn_skip_mlp_fwd(n, Sd, Xd, pb, 0.9, logits, skip)
    dP = torch.zeros(B().QN_MLP_PARAMS, device="cuda")
    loss = torch.zeros(1, device="cuda")
    part = torch.zeros(B().QN_MLP_BWD_BLOCKS * (B().QN_MLP_PARAMS + 1), device="cuda")
    B().qn_skip_mlp_bwd(n, Sd, Xd, up(y, torch.uint8), pb, dP, loss, part)
    torch.cuda.synchronize()
    z_ref, cache = oracle.mlp_forward(X.T, P)
    close(logits.cpu().numpy(), z_ref, floor_frac=0.01, what="logits")
    thr = math.log(0.9 / 0.1)
    far = np.abs(z_ref - thr) > 1e-3
    assert np.array_equal(skip.cpu().numpy()[far], (z_ref > thr)[far].astype(np.uint8))
    l_ref, dz = oracle.bce_loss(z_ref, y)
    assert float(loss.item()) == pytest.approx(l_ref, rel=1e-4)
    g_ref = _flat(oracle.mlp_backward(dz, P, cache))
    close(dP.cpu().numpy(), g_ref, what="MLP parameter gradient")


def test_unskip_within_iteration_matches_plain_for_composited():
    """Every Gaussian marked skipped, one iteration with unskip: exactly the
    Gaussians some pixel composites are un-skipped, and they -- with the
    shared decoders -- take the update plain training gives them (the
    forward marks them, they are un-skipped before the compositing adjoint,
    and the adjoint, which drops the Gaussians left skipped, and every later
    stage run with the mask); the others stay frozen at their initial
    values."""
    from paper_2412_04469_gb300.pipeline import QueenFrame, Rasterizer, training_iteration
    from paper_2412_04469_gb300.synthetic import DecoderLayout
    n, deg, W, H = 3000, 1, 160, 120
    lay = DecoderLayout.default(sh_degree=deg, latent=8)
    prev = S.make_scene(n, deg, 12)
    res = S.make_residuals(n, lay, 12)
    cam = B().make_camera(S.make_camera(W, H, 60.0, eye=(0.4, 0.3, 4.0)))
    tgt = up(S.make_image(W, H, 12))
    arms = {}
    for mode in ("plain", "unskip"):
        f = QueenFrame(prev, deg, lay, res.lat, res.dec, res.lp, res.log_alpha)
        r = Rasterizer(n, f.S, deg, W, H, 1)
        f.decode()                                    # A_t of every column, reused for the skipped ones
        r.size_for_views(f.attrs, [cam], f.hp.blur)
        skip = torch.ones(f.S, device="cuda", dtype=torch.uint8) if mode == "unskip" else None
        la0 = f.log_alpha.clone()
        training_iteration(f, r, cam, tgt, skip, unskip=mode == "unskip", mark=True)
        torch.cuda.synchronize()
        arms[mode] = (f, r, skip, la0)
    fp, rp, _, _ = arms["plain"]
    fu, ru, sk, la0 = arms["unskip"]
    hit = ru.composited[:n].bool()
    assert torch.equal(rp.composited[:n], ru.composited[:n])
    assert 100 < int(hit.sum()) < n                   # some composited, some not
    assert torch.equal(sk[:n].bool(), ~hit)           # exactly the composited ones un-skipped
    h = hit.cpu().numpy()
    for name, a, b in (("latents", fp.lat, fu.lat), ("position residuals", fp.lp, fu.lp)):
        close(b[:, :n].cpu().numpy()[:, h], a[:, :n].cpu().numpy()[:, h], rtol=1e-6, floor_frac=1e-3, what=name)
        moved = (b[:, :n][:, hit] != planes(res.lat if name == "latents" else res.lp, fu.S)[:, :n][:, hit])
        assert moved.any(), name
    close(fu.log_alpha[:n].cpu().numpy()[h], fp.log_alpha[:n].cpu().numpy()[h], rtol=1e-6, floor_frac=1e-3,
          what="log alpha")
    close(fu.dec.cpu().numpy(), fp.dec.cpu().numpy(), rtol=1e-6, floor_frac=1e-3, what="decoders")
    frozen = ~hit
    assert torch.equal(fu.lat[:, :n][:, frozen], planes(res.lat, fu.S)[:, :n][:, frozen])
    assert torch.equal(fu.lp[:, :n][:, frozen], planes(res.lp, fu.S)[:, :n][:, frozen])
    assert torch.equal(fu.log_alpha[:n][frozen], la0[:n][frozen])
