"""The D-SSIM term of Eq. 3 on the GPU (qn_dssim_loss) against the oracle:
loss and image gradient on images from 1 x 1 to the full 1352 x 1014, both
unrelated images (SSIM near 0) and near-identical smooth ones (SSIM near 1,
where the gradient's terms cancel most), with and without a pixel mask; the
call adds to the loss and gradient it is given, and repeats bit for bit."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


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


def _images(C, H, W, kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "random":
        return rng.uniform(size=(C, H, W)).astype(np.float32), rng.uniform(size=(C, H, W)).astype(np.float32)
    # smooth target (noise blurred by a 5 x 5 box) and a slightly perturbed rendering
    t = rng.uniform(size=(C, H + 4, W + 4))
    t = sum(t[:, i:i + H, j:j + W] for i in range(5) for j in range(5)) / 25.0
    x = np.clip(t + 0.02 * rng.standard_normal((C, H, W)), 0, 1)
    return x.astype(np.float32), t.astype(np.float32)


def _run(x, y, w, mask=None, loss0=0.0, d0=None):
    C, H, W = x.shape
    ws = torch.zeros(B().qn_dssim_workspace_size(W, H, C), device="cuda", dtype=torch.uint8)
    loss = torch.full((1,), loss0, device="cuda")
    d = up(d0) if d0 is not None else torch.zeros((C, H, W), device="cuda")
    pm = cnt = None
    if mask is not None:
        pm = up(mask.astype(np.uint8), torch.uint8)
        cnt = torch.tensor([int(mask.sum())], device="cuda", dtype=torch.int32)
    B().qn_dssim_loss(W, H, C, up(x), up(y), w, loss, d, ws, pm, cnt)
    torch.cuda.synchronize()
    return float(loss.item()), d.cpu().numpy().astype(np.float64)


def _close(got, ref, rtol=1e-4, floor=0.05, what=""):
    err = np.abs(got - ref) / np.maximum(np.abs(ref), floor * np.abs(ref).max())
    assert err.max() <= rtol, f"{what}: {err.max():.3e}"


@pytest.mark.parametrize("C,H,W", [(1, 1, 1), (3, 3, 5), (3, 17, 33), (3, 61, 97), (3, 112, 160), (2, 40, 300)])
@pytest.mark.parametrize("kind", ["random", "smooth"])
def test_dssim_matches_oracle(C, H, W, kind):
    x, y = _images(C, H, W, kind, H * W + C)
    w = 0.2
    loss, d = _run(x, y, w)
    ref_l, ref_g = oracle.dssim_loss(x, y)
    assert loss == pytest.approx(w * ref_l, rel=1e-4, abs=1e-6)
    _close(d, w * ref_g, what=f"{kind} {C}x{H}x{W}")


def test_dssim_full_size():
    x, y = _images(3, 1014, 1352, "smooth", 7)
    loss, d = _run(x, y, 0.2)
    ref_l, ref_g = oracle.dssim_loss(x, y)
    assert loss == pytest.approx(0.2 * ref_l, rel=1e-4)
    _close(d, 0.2 * ref_g, what="1352x1014")


@pytest.mark.parametrize("frac", [0.0, 0.3, 1.0])
def test_dssim_masked(frac):
    C, H, W = 3, 70, 90
    x, y = _images(C, H, W, "smooth", 11)
    mask = np.random.default_rng(12).uniform(size=(H, W)) < frac
    loss, d = _run(x, y, 0.5, mask)
    ref_l, ref_g = oracle.dssim_loss(x, y, mask)
    if frac == 0.0:
        assert loss == 0.0 and not d.any()
        return
    assert loss == pytest.approx(0.5 * ref_l, rel=1e-4, abs=1e-6)
    _close(d, 0.5 * ref_g, what=f"mask {frac}")


def test_dssim_accumulates_and_repeats():
    C, H, W = 3, 50, 70
    x, y = _images(C, H, W, "random", 3)
    d0 = np.random.default_rng(4).standard_normal((C, H, W)).astype(np.float32)
    l1, g1 = _run(x, y, 0.25, loss0=1.5, d0=d0)
    l2, g2 = _run(x, y, 0.25, loss0=1.5, d0=d0)
    assert l1 == l2 and np.array_equal(g1, g2)
    l0, g0 = _run(x, y, 0.25)
    assert l1 == pytest.approx(1.5 + l0, rel=1e-6)
    assert np.allclose(g1, d0 + g0, rtol=0, atol=1e-6)
