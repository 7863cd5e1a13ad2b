"""The learned static-skip MLP over a short synthetic sequence: trained on
the first frames' gates by the library's own kernels, it must pick out the
static Gaussians (high precision and recall against the ground-truth motion)
and skip most Gaussians without the held-out PSNR falling more than 0.05 dB
below plain gated training (the fallback guarantees the bound)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_04469_gb300 import build
    build.build()


def test_learned_skip_on_short_sequence():
    from paper_2412_04469_gb300.sequence import SequenceConfig, compare
    cfg = SequenceConfig(n=20_000, sh_degree=1, width=160, height=120, views=6, frames=15, iters=80,
                         train_frames=10, seed=3)
    out = compare(cfg)
    plain, learned = out["plain"], out["learned"]
    assert all(np.isfinite(r.psnr) for r in plain + learned)
    skip = [r for r in learned if r.t > cfg.train_frames]
    assert len(skip) == 4
    for r, p in zip(skip, plain[-4:]):
        assert r.psnr >= p.psnr - cfg.max_dpsnr - 1e-9
    assert out["mean_skipped"] > 0.5
    assert min(r.static_precision for r in skip) > 0.95
    assert min(r.static_recall for r in skip) > 0.6
