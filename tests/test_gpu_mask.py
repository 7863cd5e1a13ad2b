"""Adaptive masked training (Sec. 3.3, App. B) on the GPU against the
oracle: the dilation (bit-exact), the dynamic-only rendering's pixels, the
masked loss, and a masked iteration's gradient, which must equal the full
compositing adjoint fed the masked loss's upstream image."""
import numpy as np
import pytest
import torch

import oracle
from paper_2412_04469_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

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


def _score(n, Sd, W, H, seed, frac):
    """d_t planes [2][Sd] in pixel units whose NDC norm is 10 t_d for a
    fraction frac of the Gaussians and t_d / 2 for the rest, in random
    directions (both far from the threshold, so FP32 and FP64 agree)."""
    rng = np.random.default_rng(seed)
    m = np.where(rng.uniform(size=n) < frac, 10.0, 0.5) * oracle.MASK_T_D
    th = rng.uniform(0, 2 * np.pi, n)
    out = np.zeros((2, Sd), np.float32)
    out[0, :n] = m * np.cos(th) / (W / 2)
    out[1, :n] = m * np.sin(th) / (H / 2)
    return out


@pytest.mark.parametrize("W,H,k,density", [(97, 61, 48, 0.002), (160, 112, 48, 0.0), (1352, 1014, 48, 0.0005),
                                           (33, 17, 2, 0.05), (64, 48, 10, 0.02)])
def test_dilate_mask_matches_oracle(W, H, k, density):
    from paper_2412_04469_gb300.pipeline import ViewMask
    rng = np.random.default_rng(W + H)
    last = np.where(rng.uniform(size=(H, W)) < density, rng.integers(1, 100, size=(H, W)), 0).astype(np.uint32)
    vm = ViewMask.empty(W, H)
    tmp = torch.zeros((H, W), device="cuda", dtype=torch.uint8)
    B().qn_dilate_mask(W, H, up(last.view(np.int32), torch.int32), k, tmp, vm.pixel, vm.tiles, vm.count)
    torch.cuda.synchronize()
    want = oracle.dilate(last > 0, k)
    assert np.array_equal(vm.pixel.cpu().numpy().astype(bool), want)
    assert np.array_equal(vm.tiles.cpu().numpy().astype(bool), oracle.tile_mask(want))
    assert int(vm.count.item()) == int(want.sum())


def test_dynamic_only_rendering_matches_oracle():
    from paper_2412_04469_gb300.pipeline import Rasterizer
    n, deg, W, H = 3000, 1, 128, 96
    A = S.make_scene(n, deg, 12)
    A[7:10] += 0.3
    Sd = (n + 31) // 32 * 32
    score = _score(n, Sd, W, H, 3, 0.2)
    attrs = torch.zeros((A.shape[0], Sd), device="cuda")
    attrs[:, :n] = up(A)
    cam = S.make_camera(W, H, 60.0)
    r = Rasterizer(n, Sd, deg, W, H, 1 << 20)
    r.project(attrs, B().make_camera(cam), 0.3)
    B().qn_select_rects(n, Sd, r.rects, up(score), W / 2, H / 2, oracle.MASK_T_D, r.rects_sel)
    r.bin_sort(sync=True, rects=r.rects_sel)
    r.render_fwd(B().make_camera(cam), (0, 0, 0))
    torch.cuda.synchronize()
    got = r.last.cpu().numpy() > 0
    flags = oracle.dynamic_flags(score[:, :n], W, H)
    assert 0.1 < flags.mean() < 0.3
    proj = oracle.project(A.astype(np.float64), cam, deg, blur=0.3, eps_g=EPS_G, tight=True)
    want = oracle.dynamic_pixels(proj, flags)
    p = dict(proj)
    rect = proj["rect"].copy()
    rect[:, ~flags] = 0
    p["rect"] = rect
    frag = oracle.render_fwd(p, eps=EPS_A, eps_d=EPS_D)[3] != 0
    # no pixel saturates in this sparse rendering, so every list Gaussian is
    # tested and more pixels lie near some alpha = 1/255 boundary
    assert frag.mean() < 0.05
    assert want.any() and np.array_equal(got[~frag], want[~frag])


@pytest.mark.parametrize("mse", [False, True])
def test_masked_loss_matches_oracle(mse):
    from paper_2412_04469_gb300.pipeline import ViewMask
    W, H = 70, 45
    rng = np.random.default_rng(9)
    img, tgt = S.make_image(W, H, 1), S.make_image(W, H, 2)
    pm = rng.uniform(size=(H, W)) < 0.3
    vm = ViewMask.empty(W, H)
    vm.pixel.copy_(up(pm.astype(np.uint8), torch.uint8))
    vm.count.fill_(int(pm.sum()))
    loss = torch.zeros(1, device="cuda")
    d = torch.zeros((3, H, W), device="cuda")
    B().qn_masked_image_loss(W * H, 3, up(img), up(tgt), vm.pixel, vm.count, 1.0, mse, loss, d)
    torch.cuda.synchronize()
    if mse:
        dd = img.astype(np.float64) - tgt
        m = np.broadcast_to(pm[None], dd.shape)
        ref_l, ref_g = float((dd[m] ** 2).mean()), np.where(m, 2 * dd, 0.0) / m.sum()
    else:
        ref_l, ref_g = oracle.masked_l1_loss(img, tgt, pm)
    assert float(loss.item()) == pytest.approx(ref_l, rel=1e-5)
    assert np.allclose(d.cpu().numpy(), ref_g, rtol=1e-6, atol=0)
    vm.count.fill_(0)
    B().qn_masked_image_loss(W * H, 3, up(img), up(tgt), vm.pixel, vm.count, 1.0, mse, loss, d)
    torch.cuda.synchronize()
    assert float(loss.item()) == 0.0 and not d.any()


def test_masked_iteration_gradient_equals_full_adjoint_with_masked_upstream():
    from paper_2412_04469_gb300.pipeline import Rasterizer, ViewMask
    n, deg, W, H = 6000, 1, 200, 150
    A = S.make_scene(n, deg, 14)
    A[7:10] += 0.4
    Sd = (n + 31) // 32 * 32
    attrs = torch.zeros((A.shape[0], Sd), device="cuda")
    attrs[:, :n] = up(A)
    cam = B().make_camera(S.make_camera(W, H, 60.0))
    tgt = up(S.make_image(W, H, 5))
    score = up(_score(n, Sd, W, H, 4, 0.05))
    r = Rasterizer(n, Sd, deg, W, H, 1 << 21)
    vm = ViewMask.empty(W, H)
    r.build_mask(attrs, cam, 0.3, score, vm)
    torch.cuda.synchronize()
    assert 0 < int(vm.tiles.sum().item()) < vm.tiles.numel()
    # masked: inactive tiles emptied, masked loss
    r.project(attrs, cam, 0.3)
    r.bin_sort(sync=True)
    r.mask_ranges(vm)
    r.render_fwd(cam, (0, 0, 0), ranges=r.ranges_masked)
    r.masked_loss_grad(tgt, vm)
    r.render_bwd(cam, (0, 0, 0), ranges=r.ranges_masked)
    torch.cuda.synchronize()
    g_masked = r.d_splats.clone()
    loss_masked = float(r.loss.item())
    # full: every tile composited, the same masked loss as upstream
    r.render_fwd(cam, (0, 0, 0))
    r.masked_loss_grad(tgt, vm)
    r.render_bwd(cam, (0, 0, 0))
    torch.cuda.synchronize()
    assert torch.equal(r.d_splats, g_masked)
    assert float(r.loss.item()) == loss_masked
    assert g_masked.abs().sum() > 0
