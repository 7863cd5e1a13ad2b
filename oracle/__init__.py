"""CPU FP64 oracle of QUEEN's per-frame residual-training path (arXiv 2412.04469).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import or call this package.  It shares no
code with the CUDA path (paper_2412_04469_gb300) and never imports it.

Two halves:
  raster  -- ctypes front-end to queen_oracle.c (decode, gate, projection,
             binning, compositing and their analytic adjoints), Sec. 3.1-3.2.
  learn   -- numpy FP64 code for the loss, the viewspace gradient difference
             and gate initialisation (Sec. 3.3, Eq. 9-10), the adaptive
             training mask (Sec. 3.3), Adam, and the static-skip MLP.
  ssim    -- numpy FP64 D-SSIM term of Eq. 3 and its gradient.
  rng     -- Philox4x32-10 gate noise for the stochastic hard-concrete gate.
  packet  -- the compressed per-frame packet (entropy-coded latents, decoders,
             COO position residuals; App. B storage) and its rANS coder.

Parity status per function is recorded in each function's docstring; every
function listed here is pinned by tests/test_oracle_*.py (closed forms,
brute force, finite differences or a library routine) except where a
docstring says "parity unpinned".
"""
from .raster import (build, OracleCamera, sh_basis, decode, decode_bwd, project, project_bwd,
                     bin_sort, render_fwd, render_bwd, num_threads)
from .learn import (l1_loss, mse_grad, viewspace_score, gate_init, adam_step, mlp_forward,
                    mlp_backward, bce_loss, skip_features, dynamic_flags, dynamic_pixels, dilate, tile_mask,
                    masked_l1_loss, MASK_T_D, MASK_KERNEL)
from . import packet, rng
from .ssim import (ssim_window, window_filter, window_filter_adjoint, ssim_map, dssim_loss, SSIM_WINDOW,
                   SSIM_SIGMA, SSIM_C1, SSIM_C2)

__all__ = [
    "build", "OracleCamera", "sh_basis", "decode", "decode_bwd", "project", "project_bwd",
    "bin_sort", "render_fwd", "render_bwd", "num_threads", "l1_loss", "mse_grad",
    "viewspace_score", "gate_init", "adam_step", "mlp_forward", "mlp_backward", "bce_loss",
    "skip_features", "dynamic_flags", "dynamic_pixels", "dilate", "tile_mask", "masked_l1_loss",
    "MASK_T_D", "MASK_KERNEL", "ssim_window", "window_filter", "window_filter_adjoint", "ssim_map", "dssim_loss",
    "SSIM_WINDOW", "SSIM_SIGMA", "SSIM_C1", "SSIM_C2", "packet", "rng",
]
