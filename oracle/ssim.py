"""FP64 numpy oracle of the D-SSIM term of Eq. 3 (Sec. 3.1) and its gradient.
Test infrastructure only; shares no code with the CUDA path.

Eq. 3 combines L1 with D-SSIM, the structural dissimilarity built on the SSIM
index of the work it cites: for every channel and pixel, local means,
variances and the covariance of the two images under a normalised Gaussian
window give

    SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),

and D-SSIM = 1 - the mean of SSIM over channels and pixels.  The paper does
not restate the window or constants; this oracle takes those of the 3D-GS
training code it builds on: an 11 x 11 Gaussian window with sigma 1.5,
C1 = 0.01^2, C2 = 0.03^2 (data range 1), outputs of the image's own size with
the window's taps outside the image reading zero.
"""
from __future__ import annotations

import numpy as np

SSIM_WINDOW = 11
SSIM_SIGMA = 1.5
SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2


def ssim_window(size: int = SSIM_WINDOW, sigma: float = SSIM_SIGMA) -> np.ndarray:
    """[size][size] window: the outer product of the normalised 1-D Gaussian
    exp(-r^2 / (2 sigma^2)), r = -(size-1)/2 ... (size-1)/2."""
    r = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-r * r / (2.0 * sigma * sigma))
    g /= g.sum()
    return np.outer(g, g)


def window_filter(a, w) -> np.ndarray:
    """out[y][x] = sum_{i,j} w[i][j] a[y + i - k][x + j - k], k = size // 2,
    with a read as zero outside its [H][W] extent."""
    a = np.asarray(a, np.float64)
    k = w.shape[0] // 2
    H, W = a.shape
    p = np.zeros((H + 2 * k, W + 2 * k))
    p[k:k + H, k:k + W] = a
    out = np.zeros((H, W))
    for i in range(w.shape[0]):
        for j in range(w.shape[1]):
            out += w[i, j] * p[i:i + H, j:j + W]
    return out


def window_filter_adjoint(g, w) -> np.ndarray:
    """The transpose of window_filter: every out[y][x] spreads w[i][j] g[y][x]
    back onto input pixel (y + i - k, x + j - k); contributions that fall
    outside the image are dropped (they met zeros in the forward)."""
    g = np.asarray(g, np.float64)
    k = w.shape[0] // 2
    H, W = g.shape
    p = np.zeros((H + 2 * k, W + 2 * k))
    for i in range(w.shape[0]):
        for j in range(w.shape[1]):
            p[i:i + H, j:j + W] += w[i, j] * g
    return p[k:k + H, k:k + W].copy()


def _stats(x, y, w):
    mx, my = window_filter(x, w), window_filter(y, w)
    vx = window_filter(x * x, w) - mx * mx
    vy = window_filter(y * y, w) - my * my
    cxy = window_filter(x * y, w) - mx * my
    return mx, my, vx, vy, cxy


def ssim_map(img, target) -> np.ndarray:
    """SSIM of every channel and pixel of two [C][H][W] images."""
    x, y = np.asarray(img, np.float64), np.asarray(target, np.float64)
    w = ssim_window()
    out = np.zeros(x.shape)
    for c in range(x.shape[0]):
        mx, my, vx, vy, cxy = _stats(x[c], y[c], w)
        out[c] = ((2 * mx * my + SSIM_C1) * (2 * cxy + SSIM_C2)
                  / ((mx * mx + my * my + SSIM_C1) * (vx + vy + SSIM_C2)))
    return out


def dssim_loss(img, target, mask=None):
    """D-SSIM = 1 - mean SSIM of img against target ([C][H][W]); returns
    (loss, dD/dimg).  The gradient is the chain rule through the three window
    statistics that depend on img -- mu_x, E[x^2] and E[xy] under the window --
    followed by the transpose of the window filter:
      dD/dx = F^T(a) + 2 x F^T(b) + y F^T(c),
    a, b, c = -1/(C H W) times dSSIM/dmu_x, dSSIM/dE[x^2], dSSIM/dE[xy].
    With mask ([H][W] bool, Sec. 3.3's masked training) the mean runs over the
    C x (masked pixels) values only, the windows still reading every pixel;
    (0, 0) for an empty mask."""
    x, y = np.asarray(img, np.float64), np.asarray(target, np.float64)
    w = ssim_window()
    sel = np.ones(x.shape[1:], bool) if mask is None else np.asarray(mask, bool)
    count = x.shape[0] * int(sel.sum())
    if count == 0:
        return 0.0, np.zeros(x.shape)
    scale = np.where(sel, -1.0 / count, 0.0)
    total = 0.0
    grad = np.zeros(x.shape)
    for c in range(x.shape[0]):
        mx, my, vx, vy, cxy = _stats(x[c], y[c], w)
        A1 = 2 * mx * my + SSIM_C1
        A2 = 2 * cxy + SSIM_C2
        B1 = mx * mx + my * my + SSIM_C1
        B2 = vx + vy + SSIM_C2
        S = A1 * A2 / (B1 * B2)
        total += S[sel].sum()
        # E[x^2] and E[xy] enter through the variance and covariance only;
        # mu_x also enters both of those (s_x^2 = E[x^2] - mu_x^2, s_xy = E[xy] - mu_x mu_y)
        dS_dmx = (2 * my * A2 - 2 * my * A1) / (B1 * B2) - S * (2 * mx / B1 - 2 * mx / B2)
        dS_dexx = -S / B2
        dS_dexy = 2 * A1 / (B1 * B2)
        grad[c] = (window_filter_adjoint(scale * dS_dmx, w)
                   + 2 * x[c] * window_filter_adjoint(scale * dS_dexx, w)
                   + y[c] * window_filter_adjoint(scale * dS_dexy, w))
    return 1.0 - total / count, grad
