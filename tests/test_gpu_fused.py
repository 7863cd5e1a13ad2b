"""The fused kernels of the training iteration against the kernels they
replace and the oracle: qn_decode_project (Eq. 4-8 then Eq. 1 on a tile
staged in shared memory) against qn_decode_residuals + qn_project, and
qn_decode_project_bwd (A_t rebuilt in shared memory, then the projection and
decode adjoints) against qn_project_bwd + qn_decode_residuals_bwd.  They run
the same operations in the same order, so A_t, the records, the rects, the
gate, d_lat, d_lp and d_log_alpha match bit for bit; the decoder gradient is
the same sum in another order.  Sizes span ragged last tiles, n = 1, every SH
degree, the paper's N3DV decoder layout (latent widths 6/8/3/8/4), skip
masks and the stochastic gate."""
import numpy as np
import pytest
import torch

import oracle
from paper_2412_04469_gb300 import synthetic as S
from paper_2412_04469_gb300.synthetic import DecoderLayout

pytestmark = pytest.mark.gpu
TAU, G0, G1 = 0.3, -0.5, 1.01


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_04469_gb300 import build
    build.build()


def up(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def close(got, ref, rtol=1e-4, floor_frac=1e-2, what=""):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    if ref.size == 0:
        return
    den = np.maximum(np.abs(ref), floor_frac * max(np.abs(ref).max(), 1e-30))
    err = np.abs(got - ref) / den
    assert err.max() <= rtol, f"{what}: {err.max():.3e}"


def _setup(n, deg, seed, layout, noise=False, W=160, H=120):
    from paper_2412_04469_gb300 import binding as B
    from paper_2412_04469_gb300.pipeline import HParams, QueenFrame, Rasterizer, n3dv_hparams
    prev = S.make_scene(n, deg, seed)
    res = S.make_residuals(n, layout, seed)
    hp = n3dv_hparams() if layout.n_cat == 5 else HParams()
    hp.gate_noise = noise
    f = QueenFrame(prev, deg, layout, res.lat, res.dec, res.lp, res.log_alpha, hp=hp)
    r = Rasterizer(n, f.S, deg, W, H, 1)
    cam = S.make_camera(W, H, 60.0, eye=(0.3, -0.2, 4.0))
    return B, f, r, B.make_camera(cam), cam, prev, res


CASES = [  # n, sh degree, seed, layout, noise
    (2000, 3, 0, "default", False),
    (130, 1, 1, "default", False),       # ragged last tile (130 = 2 x 64 + 2)
    (1, 0, 2, "default", False),
    (777, 2, 3, "n3dv", False),          # the paper's layout: the general (any width) path
    (900, 3, 4, "default", True),        # stochastic gate
]


def _layout(name, deg):
    return DecoderLayout.paper_n3dv(sh_degree=deg) if name == "n3dv" else DecoderLayout.default(sh_degree=deg, latent=8)


@pytest.mark.parametrize("n,deg,seed,lay,noise", CASES)
def test_decode_project_equals_decode_then_project(n, deg, seed, lay, noise):
    B, f, r, c, cam, prev, res = _setup(n, deg, seed, _layout(lay, deg), noise)
    skip = up((np.arange(f.S) % 5 == 1).astype(np.uint8), torch.uint8)
    # the two-kernel path (the gate noise of the same step for both)
    f.decode(train=True)
    r.project(f.attrs, c, f.hp.blur)
    torch.cuda.synchronize()
    sp0, rc0, gate0, lreg0 = r.splats.clone(), r.rects.clone(), f.gate.clone(), float(f.lreg.item())
    A0 = f.attrs.clone()
    # the fused call draws the gate noise of the same Adam step again: the same noise
    r.splats.fill_(7.0)
    r.rects.fill_(7)
    f.gate.fill_(7.0)
    f.attrs.fill_(7.0)
    f.decode_project(r, c)
    torch.cuda.synchronize()
    assert torch.equal(r.splats[:n], sp0[:n]) and torch.equal(r.rects[:n], rc0[:n])
    assert torch.equal(f.gate[:n], gate0[:n]) and torch.equal(f.attrs[:, :n], A0[:, :n])
    assert float(f.lreg.item()) == pytest.approx(lreg0, rel=1e-5)
    # with a skip mask: the skipped keep their gate entries and add nothing to lreg
    f.gate.fill_(7.0)
    f.decode_project(r, c, skip=skip)
    torch.cuda.synchronize()
    sk = skip[:n].bool()
    assert torch.equal(r.splats[:n], sp0[:n])
    assert torch.all(f.gate[:n][sk] == 7.0) and torch.equal(f.gate[:n][~sk], gate0[:n][~sk])
    # against the oracle: decode then project (the tolerance of test_gpu_parity)
    if not noise:
        A, _, _ = oracle.decode(prev.astype(np.float64), res.lat, res.dec, res.lp, res.log_alpha,
                                _layout(lay, deg), TAU, G0, G1)
        pr = oracle.project(A, cam, deg, blur=f.hp.blur, eps_g=2e-6, tight=True)
        vis = np.nonzero((pr["radius"] > 0) & (pr["fragile"] == 0))[0]
        sp = r.splats[:n].cpu().numpy()
        close(sp[vis, 0:2].T, pr["mean2d"][:, vis], what="mean2d")
        close(sp[vis, 4:7].T, pr["conic"][:, vis], what="conic")
        close(sp[vis, 8:11].T, pr["rgb"][:, vis], what="rgb")


@pytest.mark.parametrize("n,deg,seed,lay,noise", CASES)
def test_decode_project_bwd_equals_project_bwd_then_decode_bwd(n, deg, seed, lay, noise):
    B, f, r, c, cam, prev, res = _setup(n, deg, seed, _layout(lay, deg), noise)
    rng = np.random.default_rng(seed)
    f.decode_project(r, c)                       # A_t into attrs, this step's gate noise drawn
    d = rng.standard_normal((n, 12)).astype(np.float32)
    d[:, [3, 7, 11]] = 0.0
    d[:, 4:7] *= 0.01
    r.d_splats[:n] = up(d)
    for skip in (up((np.arange(f.S) % 3 == 2).astype(np.uint8), torch.uint8), None):   # unmasked last
        r.project_bwd(f.attrs, c, f.hp.blur, f.d_attrs, skip)
        f.decode_bwd(skip)
        torch.cuda.synchronize()
        ref = [f.d_lat[:, :n].clone(), f.d_lp[:, :n].clone(), f.d_log_alpha[:n].clone(), f.d_dec.clone()]
        for t in (f.d_lat, f.d_lp, f.d_log_alpha, f.d_dec):
            t.fill_(7.0)
        f.decode_project_bwd(r, c, skip)
        torch.cuda.synchronize()
        got = [f.d_lat[:, :n], f.d_lp[:, :n], f.d_log_alpha[:n], f.d_dec]
        for name, a, b in zip(("d_lat", "d_lp", "d_log_alpha"), got[:3], ref[:3]):
            assert torch.equal(a, b), name
        close(got[3].cpu().numpy(), ref[3].cpu().numpy(), floor_frac=0.01, what="d_dec")   # another summation order
    # against the oracle (the unmasked call above, no noise): the projection
    # adjoint at the GPU's A_t, then the decode adjoint
    if not noise:
        d64 = d.astype(np.float64)
        dA = oracle.project_bwd(f.attrs[:, :n].cpu().numpy().astype(np.float64), cam, deg, d64[:, 0:2].T,
                                d64[:, 4:7].T, d64[:, 2], d64[:, 8:11].T, blur=f.hp.blur)
        want = oracle.decode_bwd(res.lat, res.dec, res.lp, res.log_alpha, _layout(lay, deg), TAU, G0, G1, dA,
                                 f.d_lreg)
        close(f.d_lat[:, :n].cpu().numpy(), want[0], floor_frac=0.01, what="d_lat (oracle)")
        close(f.d_dec.cpu().numpy(), want[1], floor_frac=0.01, what="d_dec (oracle)")
        close(f.d_lp[:, :n].cpu().numpy(), want[2], floor_frac=0.01, what="d_lp (oracle)")
        close(f.d_log_alpha[:n].cpu().numpy(), want[3], floor_frac=0.01, what="d_log_alpha (oracle)")


def test_fused_training_iteration_matches_two_kernel_iteration():
    """A whole training iteration with the fused forward equals the same
    iteration with the separate kernels bit for bit: records, every gradient
    and Adam's update.  With the fused adjoint too, every per-Gaussian array
    still matches bit for bit; the decoder gradient (another summation order)
    and the decoders after Adam's step agree to rounding.  Lists formed in
    the compositing forward (the default) or written by the binning give the
    same iteration bit for bit."""
    from paper_2412_04469_gb300.pipeline import training_iteration
    n, deg = 3000, 3
    outs = []
    for fused, fused_bwd, lazy in ((False, False, True), (True, False, True), (True, True, True),
                                   (True, False, False)):
        B, f, r, c, cam, prev, res = _setup(n, deg, 5, DecoderLayout.default(sh_degree=deg, latent=8))
        f.hp.fused, f.hp.fused_bwd, f.hp.lazy_lists = fused, fused_bwd, lazy
        f.decode()
        r.size_for_views(f.attrs, [c], f.hp.blur)
        tgt = up(S.make_image(160, 120, 5))
        training_iteration(f, r, c, tgt)
        torch.cuda.synchronize()
        outs.append((r.splats[:n].clone(), r.d_splats[:n].clone(), f.d_lat[:, :n].clone(), f.d_lp[:, :n].clone(),
                     f.d_log_alpha[:n].clone(), f.d_dec.clone(), f.lat[:, :n].clone(), f.dec.clone()))
    a, b, fb, written = outs
    names = ("splats", "d_splats", "d_lat", "d_lp", "d_log_alpha", "d_dec", "lat", "dec")
    for k, name in enumerate(names):
        assert torch.equal(a[k], b[k]), name
        assert torch.equal(written[k], b[k]), name
    for k, name in enumerate(names):
        if name in ("d_dec", "dec"):
            close(fb[k].cpu().numpy(), a[k].cpu().numpy(), floor_frac=0.01, what=name)
        else:
            assert torch.equal(fb[k], a[k]), name
