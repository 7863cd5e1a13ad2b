"""The whole path at the benchmark's full sizes -- 300k Gaussians at 1352 x 1014
and 1M at 1920 x 1080, SH degree 3, set up by bench.py's own setup (same
buffers, capacities and launch configuration as the timed step) -- against
the oracle on sampled outputs the oracle computes one by one: the decode of
sampled Gaussians, the projection of sampled Gaussians, the rendered pixels
and last contributors of sampled tiles (corner and ragged-edge tiles
included), the compositing adjoint and gather for an upstream image gradient
that lives on those tiles only (every per-Gaussian gradient is then the
oracle's sum over the sampled tiles), and the projection and decode adjoints
of all Gaussians fed the oracle's upstream gradients.

The compositing is compared twice.  First against the oracle fed the GPU's
own FP32 records and rects (the same tile lists, so only the alpha and
termination decisions can flip: at most 0.1% of the sampled pixels
excluded), then against the oracle's own FP64 projection, where every
projection decision within 2e-6 of flipping must also be excluded (at 60-90
Gaussians per pixel, a large share of the pixels)."""
import os
import sys

import numpy as np
import pytest
import torch

import oracle
from tests._oracle_fed import proj_from_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EPS_A, EPS_D, EPS_G = 2e-5, 1e-6, 2e-6
TAU, G0, G1 = 0.3, -0.5, 1.01
GRAD_FLOOR = 0.01
MAX_FRAGILE_FED = 0.001
EPS_A_FED, EPS_T_FED = 5e-6, 2e-5     # margins of the fed leg (see test_gpu_parity.py)
# a gradient entry that cancels is kept by FP32 only to a multiple of u times
# the sum of its terms' magnitudes (the oracle's magnitude sums); 512 ulps as
# in test_gpu_parity.py
KMAG = 512 * 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_04469_gb300 import build
    build.build()


def up(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def close(got, ref, rtol=1e-4, floor_frac=1e-2, what="", mag=None):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    if ref.size == 0:
        return
    den = np.maximum(np.abs(ref), floor_frac * np.abs(ref).max())
    err = np.abs(got - ref) / den
    tol = rtol * den if mag is None else np.maximum(rtol * den, KMAG * np.asarray(mag, np.float64))
    ratio = np.abs(got - ref) / tol
    at = np.unravel_index(ratio.argmax(), ratio.shape)
    nrm = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    extra = "" if mag is None else f", {int((rtol * den < tol).sum())} entries under the magnitude bound"
    print(f"  {what}: worst {err.max():.3e} of the {floor_frac:g} floor (bar {rtol:.1e}), worst "
          f"{ratio.max():.3f} of its bound, norm-wise {nrm:.2e}{extra}")
    assert ratio.max() <= 1.0, (f"{what}: {ratio.max():.3f} of its bound at {at}: got {got[at]:.9g} "
                                f"ref {ref[at]:.9g} den {den[at]:.3g}")


def close_grads(gs, ref, tag=""):
    m = ref["mag"]
    close(gs[:, 0:2].T, ref["d_mean2d"], floor_frac=GRAD_FLOOR, what="d_mean2d" + tag, mag=m["d_mean2d"])
    close(gs[:, 2], ref["d_opac"], floor_frac=GRAD_FLOOR, what="d_opacity" + tag, mag=m["d_opac"])
    close(gs[:, 4:7].T, ref["d_conic"], floor_frac=GRAD_FLOOR, what="d_conic" + tag, mag=m["d_conic"])
    close(gs[:, 8:11].T, ref["d_rgb"], floor_frac=GRAD_FLOOR, what="d_rgb" + tag, mag=m["d_rgb"])


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


@pytest.mark.parametrize("name", ["full", "large"])
def test_full_size_path_on_sampled_outputs(name):
    bench = _bench()
    frame, rast, ccams, _, _, lay, prev, res, cams = bench.setup(name, quick=True)
    n, deg, W, H, V, L = bench.WORKLOADS[name]
    hp = frame.hp
    cam, c = cams[0], ccams[0]
    bg = hp.bg
    # GPU forward, as the training step issues it
    frame.decode()
    rast.project(frame.attrs, c, hp.blur)
    P = rast.bin_sort(sync=True)
    assert 0 < P <= rast.capacity
    rast.render_fwd(c, bg)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    # decode and projection of sampled Gaussians
    A_ref, gate_ref, _ = oracle.decode(prev.astype(np.float64), res.lat, res.dec, res.lp, res.log_alpha, lay, TAU,
                                       G0, G1)
    idx = np.sort(rng.choice(n, 4000, replace=False))
    got_A = frame.attrs[:, :n].cpu().numpy()
    close(got_A[:3, idx], A_ref[:3, idx], what="decoded position")
    close(got_A[3:, idx] - prev[3:, idx], A_ref[3:, idx] - prev[3:, idx].astype(np.float64), rtol=2e-3,
          what="decoded residual")
    proj = oracle.project(A_ref, cam, deg, blur=hp.blur, eps_g=EPS_G, tight=True)
    sp = rast.splats[:n].cpu().numpy()
    vis = idx[(proj["radius"][idx] > 0) & (proj["fragile"][idx] == 0)]
    close(sp[vis, 0:2].T, proj["mean2d"][:, vis], what="mean2d")
    close(sp[vis, 4:7].T, proj["conic"][:, vis], what="conic")
    close(sp[vis, 8:11].T, proj["rgb"][:, vis], what="rgb")
    # sampled tiles: corners, the ragged last column and row, and random ones
    TX, TY = (W + 15) // 16, (H + 15) // 16
    tiles = {0, TX - 1, (TY - 1) * TX, TY * TX - 1, (TY // 2) * TX + TX // 2}
    tiles |= set(rng.choice(TX * TY, 11, replace=False).tolist())
    tiles = np.array(sorted(tiles))
    insample = np.zeros((H, W), bool)
    for t in tiles:
        ty, tx = divmod(int(t), TX)
        insample[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = True
    gimg, gT, glast = rast.img.cpu().numpy(), rast.T_final.cpu().numpy(), rast.last.cpu().numpy()
    # leg 1: the oracle composites the GPU's own FP32 projection, on the
    # sampled tiles and 240 more (a rate of ~0.05% needs ~60k pixels to be
    # told from the 0.1% bar)
    tiles_f = np.array(sorted(set(tiles.tolist()) | set(rng.choice(TX * TY, 240, replace=False).tolist())))
    ins_f = np.zeros((H, W), bool)
    for t in tiles_f:
        ty, tx = divmod(int(t), TX)
        ins_f[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = True
    pf = proj_from_gpu(rast.splats.cpu().numpy(), rast.rects.cpu().numpy(), n, W, H)
    img_f, T_f, last_f, frag_f = oracle.render_fwd(pf, bg, eps=EPS_A_FED, eps_t=EPS_T_FED, eps_d=-1.0,
                                                   tiles=tiles_f)
    insample_all, insample = insample, ins_f
    ok_f = insample & (frag_f == 0)
    excluded = 1.0 - ok_f.sum() / insample.sum()
    print(f"[{name}] fed the GPU projection: {excluded:.5f} of {int(insample.sum())} sampled pixels excluded")
    assert excluded <= MAX_FRAGILE_FED, excluded
    close(gimg[:, ok_f], img_f[:, ok_f], what="image (fed)")
    close(gT[ok_f], T_f[ok_f], what="T_final (fed)")
    assert np.array_equal(glast[ok_f], last_f[ok_f])
    d_img_f = (rng.uniform(size=(3, H, W)) - 0.5) * ok_f[None]
    rast.d_img.copy_(up(d_img_f))
    rast.render_bwd(c, bg)
    torch.cuda.synchronize()
    gf = oracle.render_bwd(pf, d_img_f, bg, tiles=tiles_f, magnitudes=True)
    assert (np.abs(gf["d_rgb"]).max(axis=0) > 0).sum() >= 500
    gs = rast.d_splats[:n].cpu().numpy()
    close_grads(gs, gf, " (fed)")
    # leg 2: the oracle's own FP64 projection, on the 16 sampled tiles
    insample = insample_all
    img, T, last, frag = oracle.render_fwd(proj, bg, eps=EPS_A, eps_d=EPS_D, tiles=tiles)
    ok = insample & (frag == 0)
    # at this density (60-90 Gaussians per pixel, footprints of ~50 tiles)
    # Gaussians with a projection decision within 2e-6 of flipping reach many
    # pixels, so this leg compares fewer of them (leg 1 covers the rest)
    print(f"[{name}] FP64 projection: {1 - ok.sum() / insample.sum():.4f} of the sampled pixels excluded")
    assert ok.sum() >= max(1000, 0.3 * insample.sum()), (int(ok.sum()), int(insample.sum()))
    close(gimg[:, ok], img[:, ok], what="image")
    close(gT[ok], T[ok], what="T_final")
    # last contributor: identity of the Gaussian, from each side's own lists
    ranges = rast.ranges.cpu().numpy().astype(np.int64)
    vals = rast.vals.cpu().numpy().astype(np.int64)
    lg = rast.last.cpu().numpy().astype(np.int64)
    v, u = np.nonzero(ok)
    t_of = (v // 16) * TX + (u // 16)
    ids_g = np.where(lg[v, u] > 0, vals[np.maximum(ranges[t_of, 0] + lg[v, u] - 1, 0)], -1)
    vis_all = np.nonzero(proj["radius"] > 0)[0]
    ids_o = np.full(v.size, -1, np.int64)
    for t in tiles:
        ty, tx = divmod(int(t), TX)
        r = proj["rect"][:, vis_all]
        m = vis_all[(r[0] <= tx) & (tx < r[2]) & (r[1] <= ty) & (ty < r[3])]
        lst = m[np.lexsort((m, proj["depth"][m]))]
        sel = t_of == t
        lo = last[v[sel], u[sel]].astype(np.int64)
        ids_o[sel] = np.where(lo > 0, lst[np.maximum(lo - 1, 0)] if lst.size else -1, -1)
    assert np.array_equal(ids_g, ids_o)
    # the compositing adjoint and gather for an upstream gradient on the
    # sampled, non-fragile pixels
    d_img = (rng.uniform(size=(3, H, W)) - 0.5) * ok[None]
    rast.d_img.copy_(up(d_img))
    rast.render_bwd(c, bg)
    torch.cuda.synchronize()
    g2 = oracle.render_bwd(proj, d_img, bg, tiles=tiles, magnitudes=True)
    touched = np.abs(g2["d_mean2d"]).max(axis=0) > 0
    assert touched.sum() >= 500 and (gate_ref[touched] > 0).sum() >= 10     # enough Gaussians and open gates
    gs = rast.d_splats[:n].cpu().numpy()
    close_grads(gs, g2)
    # the projection and decode adjoints, each fed the same inputs on both
    # sides: the projection adjoint the GPU's decoded A_t and the oracle's
    # upstream gradient rounded to FP32, the decode adjoint that projection
    # adjoint (as the binning and the compositing are compared: the adjoint
    # of a needle-like Gaussian is sensitive to the FP32 rounding of A_t)
    rec = np.zeros((n, 12), np.float32)
    rec[:, 0:2] = g2["d_mean2d"].T
    rec[:, 2] = g2["d_opac"]
    rec[:, 4:7] = g2["d_conic"].T
    rec[:, 8:11] = g2["d_rgb"].T
    rast.d_splats[:n] = up(rec)
    rast.project_bwd(frame.attrs, c, hp.blur, frame.d_attrs)
    torch.cuda.synchronize()
    r64 = rec.astype(np.float64)
    dA = oracle.project_bwd(got_A.astype(np.float64), cam, deg, r64[:, 0:2].T, r64[:, 4:7].T, r64[:, 2],
                            r64[:, 8:11].T, blur=hp.blur)
    # needle-like Gaussians included: the kernel forms dL/dSigma' in the
    # eigenbasis of the projected covariance, so the flat bar holds for them
    A_, B_, C_ = proj["conic"]
    tr, dt = A_ + C_, A_ * C_ - B_ * B_
    disc = np.sqrt(np.maximum(tr * tr / 4 - dt, 0.0))
    kappa = np.where(dt > 0, (tr / 2 + disc) / np.maximum(tr / 2 - disc, 1e-30), 1.0)
    print(f"  touched Gaussians: {int(touched.sum())}, largest condition number {kappa[touched].max():.0f}")
    got = frame.d_attrs[:, :n].cpu().numpy()
    for k in range(dA.shape[0]):        # each attribute plane against its own 1% floor
        if 3 <= k <= 6:
            continue
        if np.abs(dA[k]).max() == 0.0:
            assert not got[k].any(), k
        else:
            close(got[k], dA[k], floor_frac=GRAD_FLOOR, what=f"d_attrs plane {k}")
    # the rotation gradient is a 4-vector tangent to the unit quaternion:
    # compared per Gaussian as a vector (a component that is small in this
    # frame carries the rounding of the large ones)
    nq = np.linalg.norm(dA[3:7], axis=0)
    eq = np.linalg.norm(got[3:7] - dA[3:7], axis=0) / np.maximum(nq, GRAD_FLOOR * nq.max())
    print(f"  d_attrs rotation (per Gaussian, norm-wise): worst {eq.max():.3e} at {eq.argmax()}")
    assert eq.max() <= 1e-4, (eq.max(), int(eq.argmax()))
    frame.d_attrs[:, :n] = up(dA)
    frame.decode_bwd()
    torch.cuda.synchronize()
    want = oracle.decode_bwd(res.lat, res.dec, res.lp, res.log_alpha, lay, TAU, G0, G1, dA, frame.d_lreg)
    close(frame.d_lat[:, :n].cpu().numpy(), want[0], floor_frac=GRAD_FLOOR, what="d_lat")
    close(frame.d_dec.cpu().numpy(), want[1], floor_frac=GRAD_FLOOR, what="d_dec")
    close(frame.d_lp[:, :n].cpu().numpy(), want[2], floor_frac=GRAD_FLOOR, what="d_lp")
    close(frame.d_log_alpha[:n].cpu().numpy(), want[3], floor_frac=GRAD_FLOOR, what="d_log_alpha")


@pytest.mark.parametrize("name", ["full", "large"])
def test_full_size_lists_formed_in_the_forward_equal_the_written_lists(name):
    """At the benchmark's sizes, the training iteration's binning (no pair
    lists written) and forward (each tile's list formed from the chunk masks)
    give the written-list forward's image, transmittance and last contributors
    bit for bit, write every list position the adjoint reads with the written
    list's value, and so give the same adjoint bit for bit."""
    bench = _bench()
    frame, rast, ccams, targets, _, lay, prev, res, cams = bench.setup(name, quick=True)
    hp = frame.hp
    c, bg = ccams[0], hp.bg
    frame.decode()
    rast.project(frame.attrs, c, hp.blur)
    out = []
    for lazy in (False, True):
        rast.vals.fill_(-1)
        rast.bin_sort(sync=True, lazy=lazy, list_max=hp.list_max)
        rast.render_fwd(c, bg, mark=True, order=False)
        rast.photometric_loss(targets[0], hp.lambda_dssim)
        rast.d_splats.zero_()
        rast.render_bwd(c, bg, marks=True)
        torch.cuda.synchronize()
        out.append((rast.img.clone(), rast.T_final.clone(), rast.last.clone(), rast.composited.clone(),
                    rast.vals.clone(), rast.d_splats.clone()))
    (i0, t0, l0, m0, v0, g0), (i1, t1, l1, m1, v1, g1) = out
    assert torch.equal(i0, i1) and torch.equal(t0, t1) and torch.equal(l0, l1) and torch.equal(m0, m1)
    assert torch.equal(g0, g1)
    TX, TY = rast.TX, rast.TY
    pad = torch.zeros((TY * 16, TX * 16), dtype=torch.long, device="cuda")
    pad[:rast.H, :rast.W] = l0.long()
    vm = pad.view(TY, 16, TX, 16).amax(dim=(1, 3)).reshape(-1).cpu().numpy()
    beg = rast.ranges[:, 0].cpu().numpy().astype(np.int64)
    w0, w1 = v0.cpu().numpy(), v1.cpu().numpy()
    need = np.zeros(w0.size, bool)
    for t in np.nonzero(vm)[0]:
        need[beg[t]:beg[t] + vm[t]] = True
    written = w1 != -1
    assert written[need].all() and np.array_equal(w1[written], w0[written])
    print(f"  {name}: {int(written.sum())} of {int(rast.n_pairs.item())} list positions written by the forward")
