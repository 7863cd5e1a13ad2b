"""Tile lists formed inside the compositing forward (qn_bin_sort_partial,
which writes only the lists of at most list_max pairs, then
qn_render_fwd_binned) against fully written lists (qn_bin_sort,
qn_render_fwd): every output of the forward bit for bit, every written
position equal to the full list's, the short lists written whole, every
position below a tile's largest `last` written, and the adjoint bit for bit --
on scenes of one chunk to ~80 chunks (several 32-chunk windows per tile), for
list_max from none to all, with contributor counts, composited marks and tile
orders, on masked ranges and on an overflowing pair buffer."""
import numpy as np
import pytest
import torch

from paper_2412_04469_gb300 import synthetic as S

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


def _raster(n, W, H, deg, seed, capacity=None):
    from paper_2412_04469_gb300.pipeline import Rasterizer
    A = S.make_scene(n, deg, seed)
    A[10] += np.linspace(-4, 4, n).astype(np.float32)          # opacities from faint to saturating
    cam = S.make_camera(W, H, 60.0, eye=(0.4, 0.3, 4.0))
    Sd = max(4, (n + 31) // 32 * 32)
    attrs = torch.zeros((A.shape[0], Sd), device="cuda")
    attrs[:, :n] = up(A)
    r = Rasterizer(n, Sd, deg, W, H, 1)
    c = B().make_camera(cam)
    r.project(attrs, c, 0.3)
    r.bin_sort(sync=False)
    torch.cuda.synchronize()
    P = int(r.n_pairs.item())
    r.set_capacity(P + 16 if capacity is None else capacity)
    return r, c, P


FWD_OUT = ("img", "T_final", "last", "composited", "tile_cost")


ALL = 0xffffffff


def _forward(r, c, bg, lazy, count, mark, order, ranges=None, list_max=0):
    r.vals.fill_(-1)                                             # what nothing writes stays -1
    r.tile_order.copy_(torch.arange(r.TX * r.TY, device="cuda", dtype=torch.int32).flip(0))
    r.tile_cost.zero_()
    r.bin_sort(sync=True, lazy=lazy, list_max=list_max)
    ncon = torch.zeros((r.H, r.W), device="cuda", dtype=torch.int32) if count else None
    r.render_fwd(c, bg, n_contrib=ncon, ranges=ranges, mark=mark, order=order)
    torch.cuda.synchronize()
    out = {k: getattr(r, k).clone() for k in FWD_OUT}
    out["ncon"] = ncon
    out["vals"] = r.vals.clone()
    return out


def _tile_max_last(r):
    pad = torch.zeros((r.TY * 16, r.TX * 16), dtype=torch.long, device="cuda")
    pad[:r.H, :r.W] = r.last.long()
    return pad.view(r.TY, 16, r.TX, 16).amax(dim=(1, 3)).reshape(-1).cpu().numpy()


SCENES = [  # n, W, H, sh degree, seed
    (200, 64, 48, 0, 0),         # one chunk
    (3000, 160, 120, 3, 1),      # 12 chunks, ragged tiles
    (20000, 256, 192, 1, 2),     # 79 chunks: three 32-chunk windows per tile
]


@pytest.mark.parametrize("n,W,H,deg,seed", SCENES)
@pytest.mark.parametrize("count,mark,order,list_max", [(False, False, False, 0), (True, True, True, 0),
                                                       (False, True, False, 300), (True, False, True, 2048),
                                                       (False, False, True, ALL)])
def test_lazy_forward_equals_written_lists(n, W, H, deg, seed, count, mark, order, list_max):
    r, c, P = _raster(n, W, H, deg, seed)
    bg = (0.3, 0.2, 0.1)
    full = _forward(r, c, bg, False, count, mark, order)
    vm = _tile_max_last(r)
    lazy = _forward(r, c, bg, True, count, mark, order, list_max=list_max)
    for k in FWD_OUT:
        assert torch.equal(lazy[k], full[k]), k
    if count:
        assert torch.equal(lazy["ncon"], full["ncon"])
    assert np.array_equal(_tile_max_last(r), vm)
    vf, vl = full["vals"].cpu().numpy()[:P], lazy["vals"].cpu().numpy()[:P]
    written = vl != -1
    assert np.array_equal(vl[written], vf[written])              # what is written is the list
    rg = r.ranges.cpu().numpy().astype(np.int64)
    need = np.zeros(P, bool)
    for t in np.nonzero(vm)[0]:
        need[rg[t, 0]:rg[t, 0] + vm[t]] = True                  # all the adjoint reads
    for t in np.nonzero(rg[:, 1] - rg[:, 0] <= list_max)[0]:
        need[rg[t, 0]:rg[t, 1]] = True                          # the short lists, whole
    assert written[need].all()


@pytest.mark.parametrize("n,W,H,deg,seed", SCENES[1:])
def test_lazy_adjoint_equals_written_lists(n, W, H, deg, seed):
    r, c, _ = _raster(n, W, H, deg, seed)
    bg = (0.3, 0.2, 0.1)
    d_img = up(S.make_image(W, H, seed) - 0.5)
    out = []
    for lazy, lm in ((False, 0), (True, 0), (True, 300)):
        _forward(r, c, bg, lazy, False, True, True, list_max=lm)
        r.d_img.copy_(d_img)
        r.d_splats.zero_()
        r.render_bwd(c, bg, marks=True, order=True)
        torch.cuda.synchronize()
        out.append(r.d_splats.clone())
    assert torch.equal(out[0], out[1]) and torch.equal(out[0], out[2])


def test_lazy_forward_on_masked_ranges():
    n, W, H = 3000, 160, 120
    r, c, P = _raster(n, W, H, 2, 3)
    rng = np.random.default_rng(3)
    tiles = up((rng.uniform(size=r.TX * r.TY) < 0.4).astype(np.uint8), torch.uint8)
    outs = []
    for lazy in (False, True):
        r.vals.fill_(-1)
        r.bin_sort(sync=True, lazy=lazy, list_max=0)
        B().qn_mask_ranges(r.TX * r.TY, r.ranges, tiles, r.ranges_masked)
        r.render_fwd(c, (0.0, 0.0, 0.0), ranges=r.ranges_masked)
        torch.cuda.synchronize()
        outs.append((r.img.clone(), r.T_final.clone(), r.last.clone(), r.vals.clone()))
    for k in range(3):
        assert torch.equal(outs[0][k], outs[1][k])
    # masked-out tiles walk nothing: none of their list positions is written
    rm = r.ranges.cpu().numpy().astype(np.int64)
    vl = outs[1][3].cpu().numpy()
    for t in np.nonzero(tiles.cpu().numpy() == 0)[0]:
        assert (vl[rm[t, 0]:rm[t, 1]] == -1).all()


def test_lazy_forward_with_an_overflowing_pair_buffer():
    r, c, P = _raster(3000, 160, 120, 0, 4, capacity=100)
    assert P > 100
    r.vals.fill_(-1)
    r.bin_sort(sync=False, lazy=True, list_max=2048)
    r.render_fwd(c, (0.25, 0.5, 0.75))
    torch.cuda.synchronize()
    assert (r.vals == -1).all()                                   # nothing walked, nothing written
    img = r.img.cpu().numpy()
    for k, v in enumerate((0.25, 0.5, 0.75)):
        assert np.all(img[k] == v)
    assert (r.last == 0).all() and (r.T_final == 1).all()
