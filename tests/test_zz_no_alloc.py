"""qn_bin_sort_noalloc: binning for callers that may not allocate device
memory (allocator hooks, plugins inside another application's memory pool,
real-time loops), using the library's fixed device workspace.

Checked through the C ABI, bit for bit like the rest of the integer binning
tests, against the oracle's stable sort and against qn_bin_sort with a caller
workspace, on two calls in a row (a large problem, then a small one, so
stale contents of the shared array would show).  The file is named to be
collected last.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2412_04469_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_04469_gb300 import build
    build.build()


def _inputs(n, tx, ty, seed, ext):
    depth, rect = S.make_bin_inputs(n, tx, ty, seed, max_extent=ext)
    buf = np.zeros((max(n, 1), 12), np.float32)
    buf[:n, 3] = depth
    sp = torch.from_numpy(buf).cuda()
    rc = torch.from_numpy(np.ascontiguousarray(rect.T)).cuda()
    P = int(np.maximum(rect[2] - rect[0], 0).dot(np.maximum(rect[3] - rect[1], 0)))
    return sp, rc, P


def _outs(P, tiles):
    return (torch.zeros(max(P, 1), device="cuda", dtype=torch.int32),
            torch.zeros(max(P, 1), device="cuda", dtype=torch.int64),
            torch.full((tiles, 2), 3, device="cuda", dtype=torch.int32),
            torch.zeros(1, device="cuda", dtype=torch.int64))


def _compare(n, tx, ty, seed, ext):
    from paper_2412_04469_gb300 import binding as B
    sp, rc, P = _inputs(n, tx, ty, seed, ext)
    ws = torch.zeros(B.qn_bin_sort_workspace_size(n, tx, ty), device="cuda", dtype=torch.uint8)
    v1, k1, r1, p1 = _outs(P, tx * ty)
    got1 = B.qn_bin_sort(n, sp.data_ptr() + 12, 12, rc, tx, ty, ws, P, v1, k1, r1, p1, sync=True)
    v2, k2, r2, p2 = _outs(P, tx * ty)
    got2 = B.qn_bin_sort_noalloc(n, sp.data_ptr() + 12, 12, rc, tx, ty, P, v2, k2, r2, p2, sync=True)
    torch.cuda.synchronize()
    assert got1 == got2 == P
    assert torch.equal(v1[:P], v2[:P]) and torch.equal(k1[:P], k2[:P])
    assert torch.equal(r1, r2) and torch.equal(p1, p2)
    keys, vals, ranges = oracle.bin_sort(sp[:n, 3].cpu().numpy(), rc[:n].cpu().numpy().T, tx, ty)
    assert keys.size == P
    assert np.array_equal(v2[:P].cpu().numpy().view(np.uint32), vals)
    assert np.array_equal(k2[:P].cpu().numpy().view(np.uint64), keys)
    assert np.array_equal(r2.cpu().numpy().view(np.uint32), ranges)


def test_noalloc_matches_workspace_version_twice():
    # first the largest problem the static array was sized for (300,000
    # Gaussians on the 85 x 64 tile grid of a 1352 x 1014 image), then a small
    # one whose ranges would expose anything left over from the first call
    _compare(300_000, 85, 64, 21, 9)
    _compare(2_049, 17, 5, 22, 3)


def test_noalloc_rejects_oversized_problems():
    from paper_2412_04469_gb300 import binding as B
    n, tx, ty = 4_000_000, 256, 256
    assert B.qn_bin_sort_workspace_size(n, tx, ty) > (40 << 20)
    v, k, r, p = _outs(1, tx * ty)
    with pytest.raises(B.QueenError) as e:
        B.qn_bin_sort_noalloc(n, 0, 12, 0, tx, ty, 1, v, k, r, p)
    assert e.value.code == B.QN_ERR_INVALID_ARG
    assert "static" in str(e.value)
