"""The torch.autograd.Function wrappers over the C ABI, on the 500-Gaussian
64 x 64 slice of the streaming configuration: their gradients against the
oracle's analytic gradient and against central finite differences of the
forward (FP64, converged: steps h and h/10 agree), and bit-for-bit
reproducibility of a whole training iteration (every gradient reduction runs
in a fixed order)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2412_04469_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

TAU, G0, G1 = 0.3, -0.5, 1.01
EPS_A, EPS_D, EPS_G = 2e-5, 1e-6, 2e-6
N, DEG, W, H = 500, 1, 64, 64


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_04469_gb300 import build
    build.build()


def _setup(seed):
    from paper_2412_04469_gb300 import binding as B
    from paper_2412_04469_gb300.autograd import DecodeArgs, RasterArgs
    from paper_2412_04469_gb300.pipeline import Rasterizer
    lay = S.DecoderLayout.default(sh_degree=DEG, latent=4)
    A = S.make_scene(N, DEG, seed)
    A[7:10] += 0.8
    res = S.make_residuals(N, lay, seed)
    res.lp *= 5
    res.log_alpha[:] = np.random.default_rng(seed).uniform(-0.8, 0.8, N).astype(np.float32)
    Sd = (N + 31) // 32 * 32
    cam = S.make_camera(W, H, 60.0, eye=(0.3, 0.2, 4.0))
    rast = Rasterizer(N, Sd, DEG, W, H, 1 << 18)
    rargs = RasterArgs(rast, B.make_camera(cam), 0.3, (0.0, 0.0, 0.0))
    dargs = DecodeArgs(N, Sd, A.shape[0], B.make_layout(lay), B.make_gate(TAU, G0, G1))

    def planes(a):
        t = torch.zeros((a.shape[0], Sd), device="cuda")
        t[:, :N] = torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
        return t
    return lay, A, res, cam, planes, rargs, dargs, Sd


def _weights(seed, proj):
    """Seeded upstream weights, zero on pixels whose result an FP32-flippable
    decision could change."""
    frag = oracle.render_fwd(proj, eps=EPS_A, eps_d=EPS_D)[3] != 0
    return (S.make_image(W, H, seed) - 0.5) * (frag == 0)[None]


def _close(got, ref, floor=0.05, rtol=1e-4, what=""):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    err = np.abs(got - ref) / np.maximum(np.abs(ref), floor * np.abs(ref).max())
    assert err.max() <= rtol, f"{what}: {err.max():.3e}"


def _converged_fd(f, x0, idx, hs):
    """Central differences at steps hs (descending); returns the last one when
    the last two agree within 1e-3 relative, else None (a kink nearby)."""
    out = []
    for i in idx:
        vals = []
        for h in hs:
            xp, xm = x0.copy(), x0.copy()
            xp.reshape(-1)[i] += h
            xm.reshape(-1)[i] -= h
            vals.append((f(xp) - f(xm)) / (2 * h))
        ok = abs(vals[-1] - vals[-2]) <= 1e-3 * max(abs(vals[-1]), 1e-12)
        out.append(vals[-1] if ok else None)
    return out


def test_project_rasterize_function_gradients():
    from paper_2412_04469_gb300.autograd import Project, Rasterize
    lay, A, res, cam, planes, rargs, dargs, Sd = _setup(2)
    A64 = A.astype(np.float64)
    proj = oracle.project(A64, cam, DEG, blur=0.3, eps_g=EPS_G, tight=True)
    wn = _weights(5, proj)
    attrs = planes(A).requires_grad_(True)
    img = Rasterize.apply(Project.apply(attrs, rargs), rargs)
    (img * torch.from_numpy(wn.astype(np.float32)).cuda()).sum().backward()
    got = attrs.grad[:, :N].cpu().numpy()
    g2 = oracle.render_bwd(proj, wn)
    ref = oracle.project_bwd(A64, cam, DEG, g2["d_mean2d"], g2["d_conic"], g2["d_opac"], g2["d_rgb"])
    for name, sl in (("position", slice(0, 3)), ("rotation", slice(3, 7)), ("scale", slice(7, 10)),
                     ("opacity", slice(10, 11)), ("sh", slice(11, None))):
        _close(got[sl], ref[sl], what=name)

    def f(Ax):
        return float((oracle.render_fwd(oracle.project(Ax, cam, DEG, blur=0.3, tight=True))[0] * wn).sum())

    rng = np.random.default_rng(1)
    idx = [p * N + c for p in (0, 1, 3, 7, 10, 11) for c in rng.choice(N, 6, replace=False)]
    fd = _converged_fd(f, A64, idx, (1e-4, 1e-5))
    checked = 0
    for i, v in zip(idx, fd):
        if v is None:
            continue
        g = got.reshape(-1)[i]
        assert abs(v - g) <= 1e-3 * max(abs(v), 0.05 * np.abs(got).max()), (i, v, g)
        checked += 1
    assert checked >= 25


def test_decode_gate_function_gradients():
    from paper_2412_04469_gb300.autograd import DecodeGate, Project, Rasterize
    lay, A, res, cam, planes, rargs, dargs, Sd = _setup(4)
    At, _, _ = oracle.decode(A.astype(np.float64), res.lat, res.dec, res.lp, res.log_alpha, lay, TAU, G0, G1)
    proj = oracle.project(At, cam, DEG, blur=0.3, eps_g=EPS_G, tight=True)
    wn = _weights(6, proj)
    prev, lat, dec = planes(A), planes(res.lat), torch.from_numpy(res.dec).cuda()
    lp = planes(res.lp).requires_grad_(True)
    la = torch.zeros(Sd, device="cuda")
    la[:N] = torch.from_numpy(res.log_alpha).cuda()
    la.requires_grad_(True)
    out, lreg = DecodeGate.apply(prev, lat, dec, lp, la, dargs)
    img = Rasterize.apply(Project.apply(out, rargs), rargs)
    ((img * torch.from_numpy(wn.astype(np.float32)).cuda()).sum() + 0.01 * lreg.sum()).backward()
    g_lp, g_la = lp.grad[:, :N].cpu().numpy(), la.grad[:N].cpu().numpy()
    g2 = oracle.render_bwd(proj, wn)
    dA = oracle.project_bwd(At, cam, DEG, g2["d_mean2d"], g2["d_conic"], g2["d_opac"], g2["d_rgb"])
    _, _, r_lp, r_la = oracle.decode_bwd(res.lat, res.dec, res.lp, res.log_alpha, lay, TAU, G0, G1, dA, 0.01)
    _close(g_lp, r_lp, what="d lp")
    _close(g_la, r_la, what="d log alpha")

    def f_of(lp_x, la_x):
        Ax, _, lr = oracle.decode(A.astype(np.float64), res.lat, res.dec, lp_x, la_x, lay, TAU, G0, G1)
        im = oracle.render_fwd(oracle.project(Ax, cam, DEG, blur=0.3, tight=True))[0]
        return float((im * wn).sum() + 0.01 * lr)

    rng = np.random.default_rng(3)
    lp0, la0 = res.lp.astype(np.float64), res.log_alpha.astype(np.float64)
    i_lp = [d * N + c for d in range(3) for c in rng.choice(N, 6, replace=False)]
    i_la = list(rng.choice(N, 15, replace=False))
    fd_lp = _converged_fd(lambda x: f_of(x, la0), lp0, i_lp, (1e-4, 1e-5))
    fd_la = _converged_fd(lambda x: f_of(lp0, x), la0, i_la, (1e-4, 1e-5))
    checked = 0
    for idx, fds, g in ((i_lp, fd_lp, g_lp), (i_la, fd_la, g_la)):
        for i, v in zip(idx, fds):
            if v is None:
                continue
            gi = g.reshape(-1)[i]
            assert abs(v - gi) <= 1e-3 * max(abs(v), 0.05 * np.abs(g).max()), (i, v, gi)
            checked += 1
    assert checked >= 20


def test_training_iteration_is_reproducible():
    from paper_2412_04469_gb300 import binding as B
    from paper_2412_04469_gb300.pipeline import QueenFrame, Rasterizer, training_iteration
    n, deg, Wd, Hd = 3000, 1, 96, 80
    lay = S.DecoderLayout.default(sh_degree=deg, latent=8)
    prev = S.make_scene(n, deg, 8)
    res = S.make_residuals(n, lay, 8)
    cam = B.make_camera(S.make_camera(Wd, Hd, 60.0))
    tgt = torch.from_numpy(S.make_image(Wd, Hd, 3)).cuda()
    outs = []
    for _ in range(2):
        f = QueenFrame(prev, deg, lay, res.lat, res.dec, res.lp, res.log_alpha)
        r = Rasterizer(n, f.S, deg, Wd, Hd, 1 << 20)
        for _ in range(3):
            training_iteration(f, r, cam, tgt)
        torch.cuda.synchronize()
        outs.append([t.clone() for t in (f.lat, f.dec, f.lp, f.log_alpha, r.d_splats, f.d_dec, r.loss)])
    for a, b in zip(*outs):
        assert torch.equal(a, b)
