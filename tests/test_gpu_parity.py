"""GPU parity: every C-ABI entry point against the FP64 oracle on the same
seeded inputs.  Integer work (keys, order, ranges, last contributor) is
compared bit for bit; floating point within the stated tolerances.

Pixels whose result hinges on a decision that FP32 rounding can flip (an
alpha within EPS_A of 1/255 or 0.99, T within EPS_A of 1e-4, contributors
within EPS_D relative depth, or a projection decision within EPS_G) are
flagged by the oracle, excluded, counted and bounded; their upstream
gradient is set to zero so the adjoints are compared on the rest.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2412_04469_gb300 import synthetic as S
from tests._oracle_fed import proj_from_gpu
from paper_2412_04469_gb300.synthetic import DecoderLayout

pytestmark = pytest.mark.gpu

EPS_A, EPS_D, EPS_G = 2e-5, 1e-6, 2e-6
# fed the GPU's own FP32 projection, both sides evaluate alpha from the same
# records: the GPU's exponent (a few FP32 roundings of terms up to |log2(255)|)
# and ex2.approx (2^-22) leave alpha within ~3e-6 relative, so the alpha
# decisions take a 5e-6 margin; the termination product accumulates the
# error of every (1 - alpha) in front and keeps 2e-5
EPS_A_FED, EPS_T_FED = 5e-6, 2e-5
# gradients downstream of a projection each side computes itself (FP32 on the
# GPU, FP64 in the oracle): the GPU's adjoint runs at its FP32-rounded records
# (a mean of ~1000 px to 6e-5 px), and a first moment sum s dx whose terms
# cancel moves with them; measured worst 1.2e-4 of the 1% floor.  Fed the same
# FP32 records (the *_fed tests), the adjoints hold RTOL.
RTOL_GRAD_PROJ64 = 2e-4
# FP32 keeps a gradient entry that cancels only to a multiple of u times the
# sum of its terms' magnitudes: each term carries the roundings of T rebuilt
# through the contributors behind it (~2.5 per contributor, stacks up to
# ~150 deep) and of b, and the sum those of the gather's tiles; 512 ulps
# covers that
KMAG = 512 * 2.0 ** -24
# the rotation gradient of needle-like Gaussians (17:1 axes, kappa ~ 300):
# forming Sigma', its eigenbasis and the axes' coordinates in it each leave
# an FP32 error of ~kappa eps there (measured worst 5.5e-4 in an FP32
# emulation of the kernel's arithmetic; 4e-6 with those steps in FP64)
RTOL_NEEDLE_ROT = 2e-3
RTOL = 1e-4          # FP32 images, 2D records, gradients (relative, see `close`)
GRAD_FLOOR = 0.01    # gradients, like values: entries below 1% of the array's largest compare absolutely
RTOL_BF16 = 2e-3     # decoder outputs
MAX_FRAGILE = 0.005  # fraction of excluded pixels, oracle projecting in FP64
MAX_FRAGILE_FED = 0.001  # fraction of excluded pixels, oracle fed the GPU's FP32 projection
TAU, G0, G1 = 0.3, -0.5, 1.01


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


def stride_of(n):
    return max(4, (n + 31) // 32 * 32)


def close(got, ref, rtol=RTOL, floor_frac=1e-2, what="", mag=None):
    """|got - ref| <= rtol * max(|ref|, floor_frac * max|ref|) elementwise: relative
    for entries above floor_frac of the array's largest, absolute below.

    Values (images, projected records) and gradients (GRAD_FLOOR) both use
    floor_frac = 1%: 1e-4 relative above it, 1e-6 of the array's largest
    magnitude below it.  mag (the oracle's magnitude sums of a gradient's
    entries): an entry may also differ by up to KMAG ulps of its magnitude sum,
    the most FP32 evaluation and summation of an entry that cancels can keep;
    KMAG is above rtol / 2^-24 divided by a few, so the bound only matters
    for entries that cancel by more than about 3x."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if ref.size == 0:
        return 0.0
    scale = max(np.abs(ref).max(), 1e-30)
    den = np.maximum(np.abs(ref), floor_frac * scale)
    tol = rtol * den
    if mag is not None:
        tol = np.maximum(tol, KMAG * np.asarray(mag, np.float64))
    ratio = np.abs(got - ref) / tol
    worst = float((np.abs(got - ref) / den).max())
    at = np.unravel_index(ratio.argmax(), ratio.shape)
    assert ratio.max() <= 1.0, (f"{what}: error {ratio.max():.3f} of its bound at {at} (scaled error "
                                f"{np.abs(got - ref)[at] / den[at]:.3e}, bar {rtol:.1e})")
    return worst


def close_grads(g, ref, rtol=RTOL, what=""):
    """A compositing adjoint's per-Gaussian records g [n][12] against the
    oracle's gradients (called with magnitudes=True), each array at rtol of
    the 1% floor or KMAG ulps of an entry's magnitude sum."""
    m = ref["mag"]
    close(g[:, 0:2].T, ref["d_mean2d"], rtol, GRAD_FLOOR, what + "d_mean2d", m["d_mean2d"])
    close(g[:, 2], ref["d_opac"], rtol, GRAD_FLOOR, what + "d_opacity", m["d_opac"])
    close(g[:, 4:7].T, ref["d_conic"], rtol, GRAD_FLOOR, what + "d_conic", m["d_conic"])
    close(g[:, 8:11].T, ref["d_rgb"], rtol, GRAD_FLOOR, what + "d_rgb", m["d_rgb"])


def gpu_raster(A, cam, deg, blur, bg=(0.0, 0.0, 0.0), keep_keys=False, tight=True):
    from paper_2412_04469_gb300.pipeline import Rasterizer
    n = A.shape[1]
    Sd = stride_of(n)
    r = Rasterizer(n, Sd, deg, cam.width, cam.height, 1, keep_keys=keep_keys, tight_rects=tight)
    c = B().make_camera(cam)
    attrs = planes(A, Sd)
    r.project(attrs, c, blur)
    r.bin_sort(sync=False)
    torch.cuda.synchronize()
    P = int(r.n_pairs.item())
    r.set_capacity(P + 16)
    assert r.bin_sort(sync=True) == P
    r.render_fwd(c, bg)
    torch.cuda.synchronize()
    return r, c, attrs


def oracle_last_ids(proj, last, W, H):
    """Gaussian index of each pixel's last contributor from the oracle's lists."""
    TX, TY = (W + 15) // 16, (H + 15) // 16
    vis = np.nonzero(proj["radius"] > 0)[0]
    out = np.full((H, W), -1, np.int64)
    for ty in range(TY):
        for tx in range(TX):
            r = proj["rect"][:, vis]
            m = vis[(r[0] <= tx) & (tx < r[2]) & (r[1] <= ty) & (ty < r[3])]
            lst = m[np.lexsort((m, proj["depth"][m]))]
            blk = last[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16]
            ids = np.where(blk > 0, lst[np.maximum(blk - 1, 0)] if lst.size else -1, -1)
            out[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = ids
    return out


def gpu_last_ids(r, W, H):
    last = r.last.cpu().numpy().astype(np.int64)
    ranges = r.ranges.cpu().numpy().astype(np.int64)
    vals = r.vals.cpu().numpy().astype(np.int64)
    TX = (W + 15) // 16
    v, u = np.mgrid[0:H, 0:W]
    start = ranges[(v // 16) * TX + (u // 16), 0]
    return np.where(last > 0, vals[np.maximum(start + last - 1, 0)], -1)


SCENES = [  # n, W, H, sh degree, blur, seed
    (2000, 128, 128, 0, 0.3, 0),     # the small plain config: 2,000 Gaussians, 128 x 128
    (900, 97, 61, 3, 0.3, 1),        # SH degree 3, ragged tiles
    (64, 17, 33, 1, 0.0, 2),         # tiny, no blur, partial tiles
    (700, 80, 72, 2, 0.3, 3),        # SH degree 2 (the paper's N3DV setting)
]


def _scene(n, W, H, deg, seed):
    A = S.make_scene(n, deg, seed)
    cam = S.make_camera(W, H, 60.0, eye=(0.4, 0.3, 4.0))
    return A, cam


# ---------------------------------------------------------------- projection
@pytest.mark.parametrize("n,W,H,deg,blur,seed", SCENES)
def test_project_matches_oracle(n, W, H, deg, blur, seed):
    A, cam = _scene(n, W, H, deg, seed)
    r, _, _ = gpu_raster(A, cam, deg, blur)
    sp = r.splats.cpu().numpy()[:n]
    rc = r.rects.cpu().numpy()[:n]
    ref = oracle.project(A.astype(np.float64), cam, deg, blur=blur, eps_g=EPS_G, tight=True)
    ok = ref["fragile"] == 0
    assert (~ok).mean() < 0.01
    vis_ref = ref["radius"] > 0
    vis_gpu = (rc[:, 2] > rc[:, 0]) & (rc[:, 3] > rc[:, 1])
    assert np.array_equal(vis_ref[ok], vis_gpu[ok])
    assert np.array_equal(rc[ok].T, ref["rect"][:, ok])
    m = ok & vis_ref
    close(sp[m, 0:2].T, ref["mean2d"][:, m], what="mean2d")
    close(sp[m, 2], ref["opac"][m], what="opacity")
    close(sp[m, 3], ref["depth"][m], what="depth")
    close(sp[m, 4:7].T, ref["conic"][:, m], what="conic")
    close(sp[m, 8:11].T, ref["rgb"][:, m], what="rgb")


@pytest.mark.parametrize("n,W,H,deg,blur,seed", SCENES)
def test_project_bwd_matches_oracle(n, W, H, deg, blur, seed):
    A, cam = _scene(n, W, H, deg, seed)
    A[7:10] += 0.5
    r, c, attrs = gpu_raster(A, cam, deg, blur)
    rng = np.random.default_rng(seed)
    ref = oracle.project(A.astype(np.float64), cam, deg, blur=blur, eps_g=EPS_G, tight=True)
    d = rng.standard_normal((n, 12)).astype(np.float32)
    d[:, [3, 7, 11]] = 0.0
    d[:, 4:7] *= 0.01
    r.d_splats.copy_(up(d))
    dA = torch.zeros_like(attrs)
    r.project_bwd(attrs, c, blur, dA)
    torch.cuda.synchronize()
    got = dA.cpu().numpy()[:, :n]
    want = oracle.project_bwd(A.astype(np.float64), cam, deg, d[:, 0:2].T, d[:, 4:7].T, d[:, 2], d[:, 8:11].T,
                              blur=blur)
    ok = ref["fragile"] == 0
    for name, sl in (("position", slice(0, 3)), ("quaternion", slice(3, 7)), ("log-scale", slice(7, 10)),
                     ("opacity", slice(10, 11)), ("sh", slice(11, None))):
        close(got[sl][:, ok], want[sl][:, ok], floor_frac=GRAD_FLOOR, what=name)


@pytest.mark.parametrize("blur", [0.3, 0.0])
def test_project_bwd_of_needles_matches_oracle(blur):
    """Needle-like Gaussians only (one axis 17x the other two), whose projected
    covariances reach condition numbers kappa ~ 300, the largest the
    benchmark scenes hold.  The kernel forms Sigma' from V = T R S (sums of
    squares, a Cauchy-Binet determinant) and dL/dSigma' in its eigenbasis, so
    nothing cancels by kappa^2: positions, scales and opacity within 1e-4.
    The rotation gradient keeps an FP32 error that grows with kappa and the
    anisotropy (the small eigenvalue of Sigma' is carried by sums over the
    long axis): it is held to RTOL_NEEDLE_ROT."""
    n, W, H, deg, seed = 1500, 256, 256, 1, 11
    A, cam = _scene(n, W, H, deg, seed)
    A[7] = -1.0
    A[8:10] = -3.8
    r, c, attrs = gpu_raster(A, cam, deg, blur)
    rng = np.random.default_rng(seed)
    ref = oracle.project(A.astype(np.float64), cam, deg, blur=blur, eps_g=EPS_G, tight=True)
    a_, b_, c_ = ref["conic"]
    tr, dt = a_ + c_, a_ * c_ - b_ * b_
    disc = np.sqrt(np.maximum(tr * tr / 4 - dt, 0.0))
    kappa = np.where(dt > 0, (tr / 2 + disc) / np.maximum(tr / 2 - disc, 1e-30), 1.0)
    ok = (ref["fragile"] == 0) & (ref["radius"] > 0)
    assert (kappa[ok] > 200).sum() >= 300, np.sort(kappa[ok])[-5:]
    d = rng.standard_normal((n, 12)).astype(np.float32)
    d[:, [3, 7, 11]] = 0.0
    d[:, 4:7] *= 0.01
    r.d_splats.copy_(up(d))
    dA = torch.zeros_like(attrs)
    r.project_bwd(attrs, c, blur, dA)
    torch.cuda.synchronize()
    got = dA.cpu().numpy()[:, :n]
    want = oracle.project_bwd(A.astype(np.float64), cam, deg, d[:, 0:2].T, d[:, 4:7].T, d[:, 2], d[:, 8:11].T,
                              blur=blur)
    for k in range(11):                 # each plane against its own 1% floor
        close(got[k, ok], want[k, ok], rtol=RTOL_NEEDLE_ROT if 3 <= k <= 6 else 1e-4, floor_frac=GRAD_FLOOR,
              what=f"plane {k}")
    # and the forward records of the same needles
    sp = r.splats.cpu().numpy()[:n]
    close(sp[ok, 4:7].T, ref["conic"][:, ok], what="conic")
    close(sp[ok, 0:2].T, ref["mean2d"][:, ok], what="mean2d")


# ---------------------------------------------------------------- binning
BIN_CASES = [  # n, tiles_x, tiles_y, seed, max_extent
    (0, 3, 2, 0, 4), (1, 1, 1, 1, 1), (7, 4, 3, 2, 3), (257, 9, 7, 3, 5), (2049, 17, 5, 6, 3),
    (5000, 85, 64, 4, 12), (3000, 120, 68, 5, 40), (20000, 256, 3, 7, 200), (60000, 85, 64, 8, 9),
]


def _gpu_bin(depth, rect, tx, ty, capacity=None, with_keys=True, vals_offset=0):
    n = depth.size
    buf = np.zeros((max(n, 1), 12), np.float32)
    buf[:n, 3] = depth
    sp = up(buf)
    rc = up(np.ascontiguousarray(rect.T) if n else np.zeros((1, 4), np.int32), torch.int32)
    ws = torch.zeros(max(B().qn_bin_sort_workspace_size(n, tx, ty), 256), device="cuda", dtype=torch.uint8)
    P_ref = int(np.maximum(rect[2] - rect[0], 0).dot(np.maximum(rect[3] - rect[1], 0))) if n else 0
    cap = P_ref if capacity is None else capacity
    vals = torch.zeros(max(cap, 1) + vals_offset, device="cuda", dtype=torch.int32)[vals_offset:]
    keys = torch.zeros(max(cap, 1), device="cuda", dtype=torch.int64) if with_keys else None
    ranges = torch.full((tx * ty, 2), 7, device="cuda", dtype=torch.int32)
    npairs = torch.zeros(1, device="cuda", dtype=torch.int64)
    P = B().qn_bin_sort(n, sp.data_ptr() + 12, 12, rc, tx, ty, ws, cap, vals, keys, ranges, npairs, sync=True)
    return P, (keys.cpu().numpy().view(np.uint64)[:P] if with_keys else None), \
        vals.cpu().numpy().view(np.uint32)[:P], ranges.cpu().numpy().view(np.uint32), int(npairs.item())


@pytest.mark.parametrize("n,tx,ty,seed,ext", BIN_CASES)
def test_bin_sort_bit_exact(n, tx, ty, seed, ext):
    depth, rect = S.make_bin_inputs(n, tx, ty, seed, max_extent=ext)
    k_ref, v_ref, r_ref = oracle.bin_sort(depth, rect, tx, ty)
    P, k, v, r, p_dev = _gpu_bin(depth, rect, tx, ty)
    assert P == k_ref.size == p_dev
    assert np.array_equal(k, k_ref)
    assert np.array_equal(v, v_ref)
    assert np.array_equal(r, r_ref)


@pytest.mark.parametrize("n,tx,ty,seed,ext", [BIN_CASES[i] for i in (2, 4, 5, 6, 8)])
@pytest.mark.parametrize("offset", [0, 1])
def test_bin_sort_without_keys(n, tx, ty, seed, ext, offset):
    """Without keys the scatter writes four members per 16-byte store where
    the slots allow (a 16-byte aligned vals, offset 0) and single stores
    otherwise (offset 1): the same values either way."""
    depth, rect = S.make_bin_inputs(n, tx, ty, seed, max_extent=ext)
    _, v_ref, r_ref = oracle.bin_sort(depth, rect, tx, ty)
    P, _, v, r, _ = _gpu_bin(depth, rect, tx, ty, with_keys=False, vals_offset=offset)
    assert np.array_equal(v, v_ref) and np.array_equal(r, r_ref)


def test_bin_sort_capacity_overflow():
    depth, rect = S.make_bin_inputs(500, 9, 7, 11, max_extent=4)
    k_ref, _, _ = oracle.bin_sort(depth, rect, 9, 7)
    from paper_2412_04469_gb300.binding import QueenError, QN_ERR_CAPACITY
    with pytest.raises(QueenError) as e:
        _gpu_bin(depth, rect, 9, 7, capacity=k_ref.size - 1)
    assert e.value.code == QN_ERR_CAPACITY


def test_pair_buffer_sizing_and_overflow_report():
    """Rasterizer.size_for_views sizes the pair buffer from every view's
    pair count; check_capacity reports the count, and raises after a binning
    that overflowed a buffer made too small (which wrote empty ranges)."""
    from paper_2412_04469_gb300.pipeline import QueenFrame, Rasterizer, training_iteration
    n, deg, W, H = 3000, 1, 200, 150
    lay = DecoderLayout.default(sh_degree=deg, latent=8)
    prev = S.make_scene(n, deg, 9)
    res = S.make_residuals(n, lay, 9)
    frame = QueenFrame(prev, deg, lay, res.lat, res.dec, res.lp, res.log_alpha)
    rast = Rasterizer(n, frame.S, deg, W, H, 1)
    cams = [B().make_camera(c) for c in S.make_arc_cameras(3, W, H)]
    frame.decode()
    counts = []
    for c in cams:
        rast.project(frame.attrs, c, frame.hp.blur)
        rast.bin_sort(sync=False)
        torch.cuda.synchronize()
        counts.append(int(rast.n_pairs.item()))
    P = rast.size_for_views(frame.attrs, cams, frame.hp.blur, margin=1.25)
    assert P == max(counts) > 0 and rast.capacity == int(P * 1.25) + 4096
    targets = [up(S.make_image(W, H, v)) for v in range(3)]
    for it in range(3):
        training_iteration(frame, rast, cams[it], targets[it])
    assert 0 < rast.check_capacity() <= rast.capacity
    rast.set_capacity(min(counts) // 2)
    rast.project(frame.attrs, cams[0], frame.hp.blur)
    rast.bin_sort(sync=False)
    with pytest.raises(RuntimeError, match="overflow"):
        rast.check_capacity()
    assert not rast.ranges.cpu().numpy().any()          # every range (0, 0): nothing to composite


@pytest.mark.parametrize("low_zero", [False, True])
@pytest.mark.parametrize("empty_frac", [0.0, 0.1])
def test_bin_sort_with_constant_digits(low_zero, empty_frac):
    """Depths in [2, 4) share their top byte, and with low_zero their low byte
    too: a radix pass on a digit every key shares is a copy on the GPU.  With
    culled Gaussians (empty rects, keys all ones) no digit is shared."""
    n, tx, ty = 20000, 85, 64
    depth, rect = S.make_bin_inputs(n, tx, ty, 21, max_extent=9, empty_frac=empty_frac)
    depth = (2.0 + (depth - 0.2) / 9.8 * 1.999).astype(np.float32)
    if low_zero:
        depth = (depth.view(np.uint32) & np.uint32(0xFFFFFF00)).view(np.float32)
    k_ref, v_ref, r_ref = oracle.bin_sort(depth, rect, tx, ty)
    P, k, v, r, _ = _gpu_bin(depth, rect, tx, ty)
    assert np.array_equal(k, k_ref) and np.array_equal(v, v_ref) and np.array_equal(r, r_ref)


def test_bin_sort_all_culled_and_tie_heavy():
    depth, rect = S.make_bin_inputs(1000, 8, 8, 12, max_extent=8, tie_frac=0.9, empty_frac=0.0)
    depth[:] = depth[0]                                  # every key's depth bits equal
    k_ref, v_ref, r_ref = oracle.bin_sort(depth, rect, 8, 8)
    P, k, v, r, _ = _gpu_bin(depth, rect, 8, 8)
    assert np.array_equal(k, k_ref) and np.array_equal(v, v_ref) and np.array_equal(r, r_ref)
    rect[:] = 0
    P, _, _, r, _ = _gpu_bin(depth, rect, 8, 8)
    assert P == 0 and np.all(r == 0)


# ---------------------------------------------------------------- compositing
@pytest.mark.parametrize("n,W,H,deg,blur,seed", SCENES)
def test_render_forward_matches_oracle(n, W, H, deg, blur, seed):
    A, cam = _scene(n, W, H, deg, seed)
    bg = (0.1, 0.3, 0.2)
    r, _, _ = gpu_raster(A, cam, deg, blur, bg)
    proj = oracle.project(A.astype(np.float64), cam, deg, blur=blur, eps_g=EPS_G, tight=True)
    img, T, last, frag = oracle.render_fwd(proj, bg, eps=EPS_A, eps_d=EPS_D)
    ok = frag == 0
    assert (~ok).mean() <= MAX_FRAGILE
    gi = r.img.cpu().numpy()
    close(gi[:, ok], img[:, ok], what="image")
    close(r.T_final.cpu().numpy()[ok], T[ok], what="T_final")
    ids_g = gpu_last_ids(r, W, H)
    ids_o = oracle_last_ids(proj, last, W, H)
    assert np.array_equal(ids_g[ok], ids_o[ok])      # last contributor: bit-exact identity


@pytest.mark.parametrize("n,W,H,deg,blur,seed", SCENES)
def test_render_backward_matches_oracle(n, W, H, deg, blur, seed):
    A, cam = _scene(n, W, H, deg, seed)
    bg = (0.2, 0.1, 0.05)
    r, c, _ = gpu_raster(A, cam, deg, blur, bg)
    proj = oracle.project(A.astype(np.float64), cam, deg, blur=blur, eps_g=EPS_G, tight=True)
    _, _, _, frag = oracle.render_fwd(proj, bg, eps=EPS_A, eps_d=EPS_D)
    d_img = (S.make_image(W, H, seed) - 0.5) * (frag == 0)[None]
    r.d_img.copy_(up(d_img))
    r.render_bwd(c, bg)
    torch.cuda.synchronize()
    g = r.d_splats.cpu().numpy()[:n]
    ref = oracle.render_bwd(proj, d_img, bg, magnitudes=True)
    close_grads(g, ref, rtol=RTOL_GRAD_PROJ64)


def _fed(r, n, W, H):
    return proj_from_gpu(r.splats.cpu().numpy(), r.rects.cpu().numpy(), n, W, H)


@pytest.mark.parametrize("n,W,H,deg,blur,seed", SCENES)
def test_render_matches_oracle_fed_the_gpu_projection(n, W, H, deg, blur, seed):
    """Compositing and its adjoint against the oracle composited from the
    GPU's own FP32 records and rects: the same tile lists, so only the alpha
    and termination decisions can flip (< 0.1% of the pixels excluded)."""
    A, cam = _scene(n, W, H, deg, seed)
    bg = (0.1, 0.3, 0.2)
    r, c, _ = gpu_raster(A, cam, deg, blur, bg)
    proj = _fed(r, n, W, H)
    img, T, last, frag = oracle.render_fwd(proj, bg, eps=EPS_A_FED, eps_t=EPS_T_FED,
                                           eps_d=-1.0)   # equal depths sort alike on both sides
    ok = frag == 0
    assert (~ok).mean() <= MAX_FRAGILE_FED, (~ok).mean()
    close(r.img.cpu().numpy()[:, ok], img[:, ok], what="image")
    close(r.T_final.cpu().numpy()[ok], T[ok], what="T_final")
    assert np.array_equal(r.last.cpu().numpy()[ok], last[ok])      # same lists: positions compare directly
    d_img = (S.make_image(W, H, seed) - 0.5) * ok[None]
    r.d_img.copy_(up(d_img))
    r.render_bwd(c, bg)
    torch.cuda.synchronize()
    g = r.d_splats.cpu().numpy()[:n]
    ref = oracle.render_bwd(proj, d_img, bg, magnitudes=True)
    close_grads(g, ref)


def test_render_bwd_call_alone_gives_per_gaussian_gradients():
    """qn_render_bwd called directly through the C ABI on raw buffers (the
    binning's workspace, a pair scratch, per-Gaussian output): against the
    oracle fed the same FP32 projection; the forward's composited marks,
    which let the walk drop the Gaussians no pixel composites, and the call
    split into its two passes give the same records bit for bit; a skip mask
    zeroes exactly the skipped Gaussians and leaves the others' gradients.
    The scene holds faint Gaussians and opaque ones whose alpha is capped, so
    both of the adjoint's branches (records that can reach the cap and those
    that cannot) are compared."""
    from paper_2412_04469_gb300 import binding as Bd
    n, W, H, deg, blur, seed = 1500, 150, 110, 2, 0.3, 9
    A, cam = _scene(n, W, H, deg, seed)
    A[10, ::10] = np.log(0.004 / 0.996)    # faint: in the tile lists, below 1/255 at most pixels
    A[10, 5::40] = 6.0                      # opaque (o = 0.9975): alpha capped at 0.99 near their centres
    bg = (0.05, 0.1, 0.2)
    r, c, _ = gpu_raster(A, cam, deg, blur, bg)
    comp = torch.zeros(n, device="cuda", dtype=torch.uint8)
    Bd.qn_render_fwd(c, r.ranges, r.vals, r.splats, bg, r.img, r.T_final, r.last, composited=comp)
    proj = _fed(r, n, W, H)
    _, _, _, frag = oracle.render_fwd(proj, bg, eps=EPS_A_FED, eps_t=EPS_T_FED, eps_d=-1.0)
    d_img = up((S.make_image(W, H, seed) - 0.5) * (frag == 0)[None])
    scratch = torch.zeros((r.capacity, 12), device="cuda")
    outs = {}
    for name, marks in (("plain", None), ("marks", comp)):
        d = torch.full((n, 12), 7.0, device="cuda")
        Bd.qn_render_bwd(c, n, r.rects, r.ranges, r.vals, r.splats, bg, r.T_final, r.last, d_img, None, marks,
                         r.workspace, scratch, d)
        outs[name] = d
    d2 = torch.full((n, 12), 7.0, device="cuda")
    Bd.qn_render_bwd_pairs(c, n, r.ranges, r.vals, r.splats, bg, r.T_final, r.last, d_img, None, comp, r.workspace,
                           scratch)
    Bd.qn_render_bwd_gather(c, n, r.rects, None, r.workspace, scratch, d2)
    torch.cuda.synchronize()
    assert torch.equal(outs["plain"], outs["marks"]) and torch.equal(outs["plain"], d2)
    assert 0 < int(comp.sum()) < n
    assert not outs["plain"][~comp.bool()].any()          # uncomposited: zero gradient
    g = outs["plain"].cpu().numpy()
    ref = oracle.render_bwd(proj, d_img.cpu().numpy(), bg, magnitudes=True)
    close_grads(g, ref)
    assert not g[:, [3, 7, 11]].any()                     # the records' padding lanes are zero
    # skip half of the composited Gaussians: they get zero, the others the same
    skip = torch.zeros(n, device="cuda", dtype=torch.uint8)
    skip[torch.nonzero(comp)[::2, 0]] = 1
    ds = torch.full((n, 12), 7.0, device="cuda")
    Bd.qn_render_bwd(c, n, r.rects, r.ranges, r.vals, r.splats, bg, r.T_final, r.last, d_img, skip, comp,
                     r.workspace, scratch, ds)
    torch.cuda.synchronize()
    sk = skip.bool()
    assert not ds[sk].any() and torch.equal(ds[~sk], outs["plain"][~sk])


def test_render_backward_large_footprints():
    """A fifth of the Gaussians scaled up (log-scale + 2) on a ragged 33 x 26
    tile grid: rects above 384 tiles, up to the whole grid, are listed by the
    binning and summed by a whole block each, the rest by one warp each, in
    the same launch."""
    n, W, H, deg, blur = 400, 520, 410, 1, 0.3
    A, cam = _scene(n, W, H, deg, 4)
    big = np.random.default_rng(4).choice(n, n // 5, replace=False)
    A[7:10, big] += 2.0
    bg = (0.2, 0.1, 0.05)
    r, c, _ = gpu_raster(A, cam, deg, blur, bg)
    proj = oracle.project(A.astype(np.float64), cam, deg, blur=blur, eps_g=EPS_G, tight=True)
    _, _, _, frag = oracle.render_fwd(proj, bg, eps=EPS_A, eps_d=EPS_D)
    assert (frag != 0).mean() < MAX_FRAGILE
    d_img = (S.make_image(W, H, 4) - 0.5) * (frag == 0)[None]
    r.d_img.copy_(up(d_img))
    r.render_bwd(c, bg)
    torch.cuda.synchronize()
    g = r.d_splats.cpu().numpy()[:n]
    ref = oracle.render_bwd(proj, d_img, bg, magnitudes=True)
    rect = proj["rect"]
    area = (rect[2] - rect[0]) * (rect[3] - rect[1])
    touched = np.abs(ref["d_rgb"]).max(axis=0) > 0
    assert (touched & (area > 384)).sum() >= 5 and (touched & (area <= 384)).sum() >= 100
    close_grads(g, ref, rtol=RTOL_GRAD_PROJ64)


@pytest.mark.parametrize("n,W,H,deg,blur,seed", SCENES[:2])
def test_tight_rects_leave_rendering_unchanged(n, W, H, deg, blur, seed):
    """The tile lists built from tight rects are a subset of the 3-sigma ones
    and give the same image, transmittance, last contributor and adjoint."""
    A, cam = _scene(n, W, H, deg, seed)
    A[10] += np.linspace(-6, 3, n).astype(np.float32)
    bg = (0.3, 0.2, 0.1)
    out = []
    for tight in (False, True):
        r, c, _ = gpu_raster(A, cam, deg, blur, bg, tight=tight)
        r.d_img.copy_(up(S.make_image(W, H, seed) - 0.5))
        r.render_bwd(c, bg)
        torch.cuda.synchronize()
        out.append((r.img.cpu().numpy(), r.T_final.cpu().numpy(), gpu_last_ids(r, W, H),
                    r.d_splats.cpu().numpy(), int(r.n_pairs.item())))
    (i0, t0, l0, g0, p0), (i1, t1, l1, g1, p1) = out
    assert p1 < p0
    assert np.array_equal(i0, i1) and np.array_equal(t0, t1) and np.array_equal(l0, l1)
    # the lists differ by pairs that no pixel composites, whose records are zero
    close(g1, g0, rtol=1e-5, floor_frac=GRAD_FLOOR, what="adjoint")


def test_render_skip_mask_zeroes_skipped():
    """Skipped Gaussians get zero gradient, the others exactly their
    unskipped one (a composited skipped Gaussian still enters the others'
    T and colour behind); the forward's composited marks cover skipped and
    unskipped Gaussians alike, and qn_clear_marked un-skips exactly the
    composited ones."""
    A, cam = _scene(800, 64, 64, 0, 3)
    r, c, _ = gpu_raster(A, cam, 0, 0.3)
    r.render_fwd(c, (0, 0, 0), mark=True)
    r.d_img.copy_(up(S.make_image(64, 64, 4) - 0.5))
    r.render_bwd(c, (0, 0, 0))
    full = r.d_splats.cpu().numpy().copy()
    hit_full = r.composited.cpu().numpy().copy()[:800]
    skip = (np.arange(800) % 3 == 0).astype(np.uint8)
    r.render_bwd(c, (0, 0, 0), skip=up(skip, torch.uint8))
    part = r.d_splats.cpu().numpy()
    assert np.all(part[skip == 1] == 0)
    assert np.array_equal(part[skip == 0], full[skip == 0])
    assert np.all(full[hit_full == 0] == 0) and hit_full.any() and (hit_full[skip == 1] != 0).any()
    flags = up(skip, torch.uint8)
    B().qn_clear_marked(800, r.composited, flags)
    assert np.array_equal(flags.cpu().numpy(), skip * (hit_full == 0))


def test_empty_and_culled_scenes_render_background():
    cam = S.make_camera(40, 24, 60.0)
    bg = (0.25, 0.5, 0.75)
    for A in (S.make_scene(0, 0, 0), S.make_scene(50, 0, 1) + np.array([[0], [0], [10.0]] + [[0]] * 11, np.float32)):
        r, _, _ = gpu_raster(A, cam, 0, 0.3, bg)
        img = r.img.cpu().numpy()
        assert np.array_equal(img, np.broadcast_to(np.array(bg, np.float32)[:, None, None], img.shape))
        assert np.all(r.T_final.cpu().numpy() == 1.0) and np.all(r.last.cpu().numpy() == 0)


# ---------------------------------------------------------------- decode and gate
def _decode_problem(n, deg, seed, latent=8):
    lay = DecoderLayout.default(sh_degree=deg, latent=latent)
    prev = S.make_scene(n, deg, seed)
    res = S.make_residuals(n, lay, seed)
    ties = np.array([0.5, 1.5, -2.5, 130.2, -200.0], np.float32)[:n]      # rounding ties and saturation
    res.lat[:, :ties.size] = ties[None, :]
    return lay, prev, res


@pytest.mark.parametrize("n,deg,seed,latent", [(1000, 3, 0, 8), (37, 1, 1, 8), (1, 0, 2, 8), (1000, 2, 5, 4)])
def test_decode_matches_oracle(n, deg, seed, latent):
    from paper_2412_04469_gb300.pipeline import QueenFrame
    lay, prev, res = _decode_problem(n, deg, seed, latent)
    f = QueenFrame(prev, deg, lay, res.lat, res.dec, res.lp, res.log_alpha)
    f.decode()
    torch.cuda.synchronize()
    out, gate, lreg = oracle.decode(prev.astype(np.float64), res.lat, res.dec, res.lp, res.log_alpha, lay, TAU, G0, G1)
    got = f.attrs.cpu().numpy()[:, :n]
    close(got[:3], out[:3], what="position")
    close(got[3:] - prev[3:], out[3:] - prev[3:].astype(np.float64), rtol=RTOL_BF16, what="decoded residual")
    close(f.gate.cpu().numpy()[:n], gate, what="gate")
    assert float(f.lreg.item()) == pytest.approx(lreg, rel=1e-5)


@pytest.mark.parametrize("n,deg,seed,latent", [(1000, 3, 0, 8), (37, 1, 1, 8), (1000, 3, 0, 4), (40_000, 3, 3, 8),
                                               (40_000, 1, 4, 4)])
def test_decode_bwd_matches_oracle(n, deg, seed, latent):
    """Latent width 8 takes the specialised adjoint, width 4 the general one;
    the 40k cases span many tiles per block, with a contiguous skipped run."""
    from paper_2412_04469_gb300.pipeline import QueenFrame
    lay, prev, res = _decode_problem(n, deg, seed, latent)
    res.log_alpha[: n // 2] = np.linspace(-1, 1, n // 2)      # inside the open gate interval
    from paper_2412_04469_gb300.pipeline import HParams
    f = QueenFrame(prev, deg, lay, res.lat, res.dec, res.lp, res.log_alpha, HParams(lreg_mean=False))
    rng = np.random.default_rng(seed)
    d_out = rng.standard_normal((prev.shape[0], n)).astype(np.float32)
    f.d_attrs[:, :n] = up(d_out)
    skip = (rng.uniform(size=n) < 0.2).astype(np.uint8)
    if n > 10_000:
        skip[n // 3: 2 * n // 3] = 1                            # whole tiles of skipped Gaussians
    f.decode_bwd(skip=up(skip, torch.uint8))
    torch.cuda.synchronize()
    want = oracle.decode_bwd(res.lat, res.dec, res.lp, res.log_alpha, lay, TAU, G0, G1, d_out, f.d_lreg,
                             skip=skip)
    close(f.d_lat.cpu().numpy()[:, :n], want[0], floor_frac=GRAD_FLOOR, what="d_lat")
    close(f.d_dec.cpu().numpy(), want[1], floor_frac=GRAD_FLOOR, what="d_dec")
    close(f.d_lp.cpu().numpy()[:, :n], want[2], floor_frac=GRAD_FLOOR, what="d_lp")
    close(f.d_log_alpha.cpu().numpy()[:n], want[3], floor_frac=GRAD_FLOOR, what="d_log_alpha")


# ---------------------------------------------------------------- loss and Adam
def test_image_loss_matches_oracle():
    img = S.make_image(37, 29, 1)
    tgt = S.make_image(37, 29, 2)
    loss = torch.zeros(1, device="cuda")
    d = torch.zeros((3, 29, 37), device="cuda")
    for mse in (False, True):
        B().qn_image_loss(img.size, up(img), up(tgt), 1.0, mse, loss, d)
        torch.cuda.synchronize()
        if mse:
            ref_g = oracle.mse_grad(img, tgt)
            ref_l = float(((img.astype(np.float64) - tgt) ** 2).mean())
        else:
            ref_l, ref_g = oracle.l1_loss(img, tgt)
        assert float(loss.item()) == pytest.approx(ref_l, rel=1e-5)
        close(d.cpu().numpy(), ref_g, floor_frac=GRAD_FLOOR, what="d_img")


def test_adam_matches_oracle():
    rng = np.random.default_rng(0)
    rows, n, stride = 3, 1000, 1024
    p = rng.standard_normal((rows, n)).astype(np.float32)
    skip = (rng.uniform(size=n) < 0.3).astype(np.uint8)
    P, M, V = planes(p, stride), torch.zeros((rows, stride), device="cuda"), torch.zeros((rows, stride), device="cuda")
    pb = torch.zeros((rows, stride), device="cuda", dtype=torch.bfloat16)
    rp, rm, rv = p.astype(np.float64), np.zeros((rows, n)), np.zeros((rows, n))
    for step in (1, 2, 3):
        g = rng.standard_normal((rows, n)).astype(np.float32)
        B().qn_adam(rows, n, stride, P, planes(g, stride), M, V, step, 0.01, 0.9, 0.999, 1e-8, up(skip, torch.uint8), pb)
        rp, rm, rv = oracle.adam_step(rp, g, rm, rv, step, 0.01, mask=np.broadcast_to(skip, (rows, n)))
    torch.cuda.synchronize()
    close(P.cpu().numpy()[:, :n], rp, rtol=1e-5, what="param")
    close(M.cpu().numpy()[:, :n], rm, rtol=1e-5, what="m")
    got_b = pb.float().cpu().numpy()[:, :n]
    assert np.array_equal(got_b[:, skip == 0], S.to_bf16_values(P.cpu().numpy()[:, :n][:, skip == 0]))


def test_decode_skip_freezes_columns():
    """Skipped Gaussians keep their out columns and gate entries; the others
    match the oracle; L_reg sums the others only."""
    from paper_2412_04469_gb300.pipeline import QueenFrame
    n, deg = 3000, 1
    lay = DecoderLayout.default(sh_degree=deg, latent=8)
    prev = S.make_scene(n, deg, 21)
    res = S.make_residuals(n, lay, 21)
    skip = (np.random.default_rng(4).uniform(size=n) < 0.6).astype(np.uint8)
    f = QueenFrame(prev, deg, lay, res.lat, res.dec, res.lp, res.log_alpha)
    f.attrs.fill_(7.0)
    f.gate.fill_(3.0)
    f.decode(skip=up(skip, torch.uint8))
    torch.cuda.synchronize()
    A_ref, g_ref, _ = oracle.decode(prev.astype(np.float64), res.lat, res.dec, res.lp, res.log_alpha, lay, TAU, G0, G1)
    got = f.attrs.cpu().numpy()[:, :n]
    gg = f.gate.cpu().numpy()[:n]
    assert np.all(got[:, skip == 1] == 7.0) and np.all(gg[skip == 1] == 3.0)
    close(got[:, skip == 0], A_ref[:, skip == 0], rtol=2e-3, floor_frac=0.01, what="A_t")
    close(gg[skip == 0], g_ref[skip == 0], rtol=1e-5, floor_frac=0.01, what="gate")
    keep = skip == 0
    shift = TAU * np.log(-G0 / G1)
    lreg_ref = float((1 / (1 + np.exp(-(res.log_alpha.astype(np.float64)[keep] - shift)))).sum())
    assert float(f.lreg.item()) == pytest.approx(lreg_ref, rel=1e-4)


B1_F32, B2_F32 = float(np.float32(0.9)), float(np.float32(0.999))


def test_adam_groups_match_oracle():
    """Three groups in one launch, the step count on the device: two planes
    with the skip mask, one without (and with a bf16 copy)."""
    rng = np.random.default_rng(1)
    n, stride = 700, 704
    specs = [(2, n, stride, 0.01, True, False), (1, 96, 96, 0.001, False, True), (3, n, stride, 0.05, True, False)]
    skip = (rng.uniform(size=n) < 0.4).astype(np.uint8)
    dev, ref, groups = [], [], []
    for rows, nn, st, lr, use_skip, bf in specs:
        p = rng.standard_normal((rows, nn)).astype(np.float32)
        P, G = planes(p, st), torch.zeros((rows, st), device="cuda")
        M, V = torch.zeros((rows, st), device="cuda"), torch.zeros((rows, st), device="cuda")
        PB = torch.zeros((rows, st), device="cuda", dtype=torch.bfloat16) if bf else None
        dev.append((P, G, M, V, PB))
        ref.append([p.astype(np.float64), np.zeros((rows, nn)), np.zeros((rows, nn))])
        groups.append(B().adam_group(P, G, M, V, lr, rows, nn, st, param_bf16=PB, use_skip=use_skip))
    step = torch.zeros(1, device="cuda", dtype=torch.int32)
    for t in (1, 2, 3, 4):
        gs = []
        for (rows, nn, st, lr, use_skip, bf), d in zip(specs, dev):
            g = rng.standard_normal((rows, nn)).astype(np.float32)
            d[1][:, :nn] = up(g)
            gs.append(g)
        B().qn_adam_groups(groups, step, 0.9, 0.999, 1e-8, up(skip, torch.uint8))
        for (rows, nn, st, lr, use_skip, bf), r, g in zip(specs, ref, gs):
            mask = np.broadcast_to(skip, (rows, nn)) if use_skip else None
            # the betas reach the kernel as f32 values: the reference uses those
            r[0], r[1], r[2] = oracle.adam_step(r[0], g, r[1], r[2], t, float(np.float32(lr)), beta1=B1_F32,
                                                beta2=B2_F32, mask=mask)
    torch.cuda.synchronize()
    assert int(step.item()) == 4
    for (rows, nn, st, lr, use_skip, bf), d, r in zip(specs, dev, ref):
        close(d[0].cpu().numpy()[:, :nn], r[0], rtol=1e-5, what="param")
        close(d[3].cpu().numpy()[:, :nn], r[2], rtol=1e-5, what="v")
        if bf:
            assert np.array_equal(d[4].float().cpu().numpy()[:, :nn], S.to_bf16_values(d[0].cpu().numpy()[:, :nn]))


def test_graph_replay_equals_eager():
    """IterationGraph replays give the eager iterations' results bit for bit,
    the device step count included, across two views and a skip mask."""
    from paper_2412_04469_gb300.pipeline import IterationGraph, QueenFrame, Rasterizer, training_iteration
    n, deg, W, H = 3000, 1, 96, 80
    lay = DecoderLayout.default(sh_degree=deg, latent=8)
    prev = S.make_scene(n, deg, 11)
    res = S.make_residuals(n, lay, 11)
    cams = [B().make_camera(c) for c in S.make_arc_cameras(2, W, H, arc_deg=30)]
    tg = [up(S.make_image(W, H, 30 + v)) for v in range(2)]
    skip = up((np.random.default_rng(2).uniform(size=n) < 0.3).astype(np.uint8), torch.uint8)
    outs = []
    for use_graph in (False, True):
        f = QueenFrame(prev, deg, lay, res.lat, res.dec, res.lp, res.log_alpha)
        r = Rasterizer(n, f.S, deg, W, H, 1 << 20)
        ig = IterationGraph(f, r)
        for it in range(7):
            v, sk = it % 2, (skip if it >= 4 else None)
            if use_graph:
                ig.run((v, sk is not None), cams[v], tg[v], sk)
            else:
                training_iteration(f, r, cams[v], tg[v], sk)
        torch.cuda.synchronize()
        if use_graph:
            assert len(ig.graphs) >= 3
        outs.append([t.clone() for t in (f.lat, f.dec, f.dec_bf16.view(torch.int16), f.lp, f.log_alpha, f.step,
                                          r.d_splats, r.img, r.loss)])
    for a, b in zip(*outs):
        assert torch.equal(a, b)


@pytest.mark.parametrize("n,frac", [(1, 0.5), (1000, 0.0), (1000, 1.0), (2500, 0.8), (70_001, 0.3)])
def test_partition_is_a_stable_partition(n, frac):
    rng = np.random.default_rng(n)
    flags = (rng.uniform(size=n) < frac).astype(np.uint8)
    perm = torch.zeros(n, device="cuda", dtype=torch.int32)
    nf = torch.zeros(1, device="cuda", dtype=torch.int32)
    ws = torch.zeros(B().qn_partition_workspace_size(n), device="cuda", dtype=torch.uint8)
    B().qn_partition(n, up(flags, torch.uint8), perm, nf, ws)
    torch.cuda.synchronize()
    ref = np.argsort(flags, kind="stable")
    assert np.array_equal(perm.cpu().numpy(), ref)
    assert int(nf.item()) == int((flags == 0).sum())


@pytest.mark.parametrize("dtype", [torch.uint8, torch.int16, torch.float32, torch.float64])
def test_gather_columns(dtype):
    rng = np.random.default_rng(3)
    rows, n, ss, ds = 3, 1500, 1504, 1600
    src = torch.from_numpy(rng.integers(0, 100, size=(rows, ss))).to("cuda", dtype)
    perm = rng.permutation(n).astype(np.int32)
    dst = torch.zeros((rows, ds), device="cuda", dtype=dtype)
    B().qn_gather_columns(rows, n, src, ss, up(perm, torch.int32), dst, ds)
    torch.cuda.synchronize()
    assert torch.equal(dst[:, :n].cpu(), src.cpu()[:, perm])
    assert torch.count_nonzero(dst[:, n:]) == 0


# ---------------------------------------------------------------- whole iteration
@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_end_to_end_gradients_match_oracle_chain(lam):
    """decode -> project -> bin -> composite -> Eq. 3's loss ((1 - lam) L1 +
    lam D-SSIM) -> every adjoint, against the oracle's chain on the same inputs
    (the small config's camera, SH degree 1)."""
    from paper_2412_04469_gb300.pipeline import QueenFrame, Rasterizer
    n, deg, W, H = 1500, 1, 96, 80
    lay = DecoderLayout.default(sh_degree=deg, latent=4)
    prev = S.make_scene(n, deg, 5)
    res = S.make_residuals(n, lay, 5)
    res.log_alpha[:] = np.random.default_rng(5).uniform(-0.8, 0.8, n).astype(np.float32)
    cam = S.make_camera(W, H, 60.0, eye=(0.5, 0.2, 4.0))
    target = S.make_image(W, H, 9)
    bg = (0.0, 0.0, 0.0)
    f = QueenFrame(prev, deg, lay, res.lat, res.dec, res.lp, res.log_alpha)
    f.decode()
    A_ref, _, _ = oracle.decode(prev.astype(np.float64), res.lat, res.dec, res.lp, res.log_alpha, lay, TAU, G0, G1)
    proj = oracle.project(A_ref, cam, deg, blur=0.3, eps_g=EPS_G, tight=True)
    img_ref, _, _, frag = oracle.render_fwd(proj, bg, eps=EPS_A, eps_d=EPS_D)
    _, g_ref = oracle.l1_loss(img_ref, target)
    g_ref = (1 - lam) * g_ref
    near = np.abs(img_ref - target).min(axis=0) < 1e-4          # sign of the L1 term could flip
    mask = (frag == 0) & ~near
    if lam > 0:
        g_ref = g_ref + lam * oracle.dssim_loss(img_ref, target)[1]
        mask &= ~oracle.dilate(frag != 0, 22)                   # D-SSIM's gradient reads 10 pixels around
        assert mask.mean() > 0.5
    g_ref = g_ref * mask[None]
    r = Rasterizer(n, f.S, deg, W, H, 1)
    c = B().make_camera(cam)
    r.project(f.attrs, c, 0.3)
    r.bin_sort()
    torch.cuda.synchronize()
    r.set_capacity(int(r.n_pairs.item()) + 16)
    r.bin_sort(sync=True)
    r.render_fwd(c, bg)
    r.photometric_loss(up(target), lam)
    r.d_img.mul_(up(mask.astype(np.float32))[None])
    r.render_bwd(c, bg)
    r.project_bwd(f.attrs, c, 0.3, f.d_attrs)
    f.decode_bwd()
    torch.cuda.synchronize()
    close(r.d_img.cpu().numpy(), g_ref, rtol=RTOL_GRAD_PROJ64, floor_frac=GRAD_FLOOR, what="d_img")
    g2 = oracle.render_bwd(proj, g_ref, bg)
    dA = oracle.project_bwd(A_ref, cam, deg, g2["d_mean2d"], g2["d_conic"], g2["d_opac"], g2["d_rgb"], blur=0.3)
    want = oracle.decode_bwd(res.lat, res.dec, res.lp, res.log_alpha, lay, TAU, G0, G1, dA, f.d_lreg)
    close(f.d_attrs.cpu().numpy()[:, :n], dA, rtol=RTOL_GRAD_PROJ64, floor_frac=GRAD_FLOOR, what="d_attrs")
    close(f.d_lat.cpu().numpy()[:, :n], want[0], rtol=RTOL_GRAD_PROJ64, floor_frac=GRAD_FLOOR, what="d_lat")
    close(f.d_dec.cpu().numpy(), want[1], rtol=RTOL_GRAD_PROJ64, floor_frac=GRAD_FLOOR, what="d_dec")
    close(f.d_lp.cpu().numpy()[:, :n], want[2], rtol=RTOL_GRAD_PROJ64, floor_frac=GRAD_FLOOR, what="d_lp")
    close(f.d_log_alpha.cpu().numpy()[:n], want[3], rtol=RTOL_GRAD_PROJ64, floor_frac=GRAD_FLOOR, what="d_log_alpha")
