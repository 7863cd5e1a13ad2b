"""FP64 numpy half of the oracle: loss, viewspace gradient difference and gate
initialisation (Sec. 3.3), Adam, and the static-skip MLP.  Test
infrastructure only; shares no code with the CUDA path.
"""
from __future__ import annotations

import numpy as np

from . import raster


def l1_loss(img, target):
    """L1 term of Eq. 3 as a mean over the 3 H W values; returns (loss, dL/dimg)
    with sign(0) = 0.  Pinned by a closed-form test."""
    d = np.asarray(img, np.float64) - np.asarray(target, np.float64)
    return float(np.abs(d).mean()), np.sign(d) / d.size


def mse_grad(img, target):
    """dL/dimg of the mean squared error used by Eq. 9."""
    d = np.asarray(img, np.float64) - np.asarray(target, np.float64)
    return 2.0 * d / d.size


def viewspace_score(projs, gt_t, gt_prev, bg=(0.0, 0.0, 0.0)):
    """Eq. 9 as written: for every view v the renderer's gradient w.r.t. the 2D
    means of the MSE to the new frame minus that of the MSE to the previous
    frame, both at the previous frame's rendering, averaged over views.
    projs[v] is the oracle projection of A_{t-1} in view v.  Returns d[2][n]."""
    d = None
    for proj, It, Ip in zip(projs, gt_t, gt_prev):
        img, _, _, _ = raster.render_fwd(proj, bg)
        g_t = raster.render_bwd(proj, mse_grad(img, It), bg)["d_mean2d"]
        g_p = raster.render_bwd(proj, mse_grad(img, Ip), bg)["d_mean2d"]
        d = (g_t - g_p) if d is None else d + (g_t - g_p)
    return d / len(projs)


def gate_init(d, tau, gamma0, gamma1, nonzero_median=True):
    """Eq. 10 and Eq. 8 solved for log alpha:
         d_i = |d_i| / (|d_i| + median |d|),  sigmoid(log a_i - tau log(-g0/g1)) = d_i.
    Median of an even count is the lower median; with nonzero_median it is
    taken over the non-zero |d_i| only (0 if there are none); with a zero
    median d_i is 1 for |d_i| > 0 and 0 otherwise; d_i is clamped to
    [1e-6, 1 - 1e-6]."""
    nrm = np.sqrt((np.asarray(d, np.float64) ** 2).sum(axis=0))
    pool = nrm[nrm > 0] if nonzero_median else nrm
    med = np.sort(pool)[(pool.size - 1) // 2] if pool.size else 0.0
    if med > 0:
        p = nrm / (nrm + med)
    else:
        p = (nrm > 0).astype(np.float64)
    p = np.clip(p, 1e-6, 1.0 - 1e-6)
    return np.log(p / (1.0 - p)) + tau * np.log(-gamma0 / gamma1), nrm, med


def adam_step(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, mask=None):
    """One Adam update (Kingma & Ba, Algorithm 1) in FP64; `step` counts from 1.
    Elements with mask != 0 keep their parameter and moments.  Returns new
    (param, m, v)."""
    p = np.asarray(param, np.float64).copy()
    g = np.asarray(grad, np.float64)
    m1 = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v1 = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mh = m1 / (1.0 - beta1 ** step)
    vh = v1 / (1.0 - beta2 ** step)
    p1 = p - lr * mh / (np.sqrt(vh) + eps)
    if mask is not None:
        keep = np.asarray(mask) != 0
        p1 = np.where(keep, p, p1)
        m1 = np.where(keep, m, m1)
        v1 = np.where(keep, v, v1)
    return p1, m1, v1


# --------------------------------------------------------------------------
# Static-skip features (16 per Gaussian), written from their definition:
#   0 p_i of Eq. 10 (|d| / (|d| + median); 1 or 0 for a zero median; the
#     median as in gate_init)
#   1 clip(log(|d| / median + 1e-6), -8, 8) / 4  (0 for a zero median)
#   2, 3 direction of d_t (d / (|d| + 1e-20))
#   4, 5, 6 position of A_{t-1}
#   7 previous frame's gate g_{t-1}
#   8 previous frame's p of Eq. 8: sigmoid(log a_{t-1} - tau log(-g0/g1))
#   9 opacity sigmoid(logit o)
#   10, 11, 12 (log-scale + 3) / 2
#   13 clip(100 |g_{t-1} lp_{t-1}|, 0, 8)  (previous position residual)
#   14 the previous frame's zero-residual label (prev_static), or
#      [g_{t-1} == 0] without one
#   15 1
# --------------------------------------------------------------------------
def skip_features(score, prev, prev_gate, prev_log_alpha, prev_lp, tau, gamma0, gamma1, nonzero_median=True,
                  prev_static=None):
    """Returns X[16][n] (float64).  score [2][n], prev [n_attr][n] (A_{t-1}),
    prev_gate [n], prev_log_alpha [n], prev_lp [3][n].  The paper does not
    define these features (the MLP is not part of it); a hand example with
    every feature worked out pins them."""
    d = np.asarray(score, np.float64)
    A = np.asarray(prev, np.float64)
    n = d.shape[1]
    nrm = np.sqrt((d ** 2).sum(axis=0))
    pool = nrm[nrm > 0] if nonzero_median else nrm
    med = np.sort(pool)[(pool.size - 1) // 2] if pool.size else 0.0
    X = np.zeros((16, n))
    if med > 0:
        X[0] = nrm / (nrm + med)
        X[1] = np.clip(np.log(nrm / med + 1e-6), -8, 8) / 4
    else:
        X[0] = (nrm > 0).astype(np.float64)
    X[2] = d[0] / (nrm + 1e-20)
    X[3] = d[1] / (nrm + 1e-20)
    X[4:7] = A[0:3]
    g = np.asarray(prev_gate, np.float64)
    X[7] = g
    X[8] = 1 / (1 + np.exp(-(np.asarray(prev_log_alpha, np.float64) - tau * np.log(-gamma0 / gamma1))))
    X[9] = 1 / (1 + np.exp(-A[10]))
    X[10:13] = (A[7:10] + 3) / 2
    X[13] = np.clip(100 * np.abs(g) * np.sqrt((np.asarray(prev_lp, np.float64) ** 2).sum(axis=0)), 0, 8)
    X[14] = (g == 0).astype(np.float64) if prev_static is None else (np.asarray(prev_static) != 0).astype(np.float64)
    X[15] = 1.0
    return X


# --------------------------------------------------------------------------
# Static-skip MLP 16 -> 64 -> 64 -> 1 (ReLU, ReLU, logit).  params is a dict
# W1[64][16], b1[64], W2[64][64], b2[64], W3[1][64], b3[1].
# --------------------------------------------------------------------------
def mlp_forward(X, params):
    """Returns (logit[n], cache).  X is [n][16]."""
    X = np.asarray(X, np.float64)
    z1 = X @ params["W1"].T + params["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ params["W3"].T + params["b3"]
    return z3[:, 0], (X, z1, h1, z2, h2)


def bce_loss(logit, label):
    """Mean binary cross-entropy on logits; returns (loss, dL/dlogit)."""
    z = np.asarray(logit, np.float64)
    y = np.asarray(label, np.float64)
    loss = np.mean(np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z))))
    return float(loss), (1.0 / (1.0 + np.exp(-z)) - y) / z.size


def mlp_backward(d_logit, params, cache):
    """Gradients of the MLP parameters for an upstream d_logit[n]."""
    X, z1, h1, z2, h2 = cache
    d3 = np.asarray(d_logit, np.float64)[:, None]
    g = {"W3": d3.T @ h2, "b3": d3.sum(axis=0)}
    d2 = (d3 @ params["W3"]) * (z2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ params["W2"]) * (z1 > 0)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    return g


# --------------------------------------------------------------------------
# Adaptive masked training (Sec. 3.3; App. B: t_d = 0.001, a 48 x 48
# dilation, masked iterations for a fraction of the frame's iterations).
MASK_T_D = 0.001
MASK_KERNEL = 48


def dynamic_flags(d, width, height, t_d=MASK_T_D):
    """Dynamic Gaussians: |d_t| above the threshold t_d, with d_t (Eq. 9,
    [2][n], pixel units) taken in normalised device coordinates -- the units
    of the 3D-GS rasterizer's viewspace gradients that t_d refers to: a
    position in NDC moves W/2 (H/2) pixels per unit, so the gradient w.r.t.
    it is the pixel-unit gradient times W/2 (H/2)."""
    d = np.asarray(d, np.float64)
    return np.hypot(d[0] * (width / 2.0), d[1] * (height / 2.0)) > t_d


def dynamic_pixels(proj, flags, bg=(0.0, 0.0, 0.0)):
    """Pixels where the dynamic Gaussians rendered alone produce a contributor:
    the oracle rendering with every other Gaussian's tile rect emptied, and
    last > 0 (the first Gaussian that passes the alpha test at a pixel always
    contributes, so this is the union of the dynamic Gaussians' alpha >= 1/255
    footprints).  Returns bool [H][W]."""
    p = dict(proj)
    rect = np.array(proj["rect"], copy=True)
    rect[:, ~np.asarray(flags, bool)] = 0
    p["rect"] = rect
    _, _, last, _ = raster.render_fwd(p, bg)
    return last > 0


def dilate(mask, k=MASK_KERNEL):
    """Box dilation with a k x k kernel: out[y][x] is set when some input
    pixel (x', y') has x in [x' - k/2, x' + k/2 - 1] and y likewise, i.e. the
    input window of out[y][x] is [x - k/2 + 1, x + k/2] (k even)."""
    m = np.asarray(mask, bool)
    H, W = m.shape
    lo, hi = k // 2 - 1, k // 2
    cs = np.zeros((H + 1, W + 1), np.int64)
    cs[1:, 1:] = np.cumsum(np.cumsum(m, axis=0), axis=1)
    y0 = np.clip(np.arange(H) - lo, 0, H)
    y1 = np.clip(np.arange(H) + hi + 1, 0, H)
    x0 = np.clip(np.arange(W) - lo, 0, W)
    x1 = np.clip(np.arange(W) + hi + 1, 0, W)
    s = cs[y1][:, x1] - cs[y0][:, x1] - cs[y1][:, x0] + cs[y0][:, x0]
    return s > 0


def tile_mask(pixel_mask, tile=16):
    """Tiles (row-major over the tile grid) holding at least one masked pixel."""
    m = np.asarray(pixel_mask, bool)
    H, W = m.shape
    TX, TY = (W + tile - 1) // tile, (H + tile - 1) // tile
    pad = np.zeros((TY * tile, TX * tile), bool)
    pad[:H, :W] = m
    return pad.reshape(TY, tile, TX, tile).any(axis=(1, 3)).reshape(-1)


def masked_l1_loss(img, target, pixel_mask):
    """L1 term of Eq. 3 restricted to the masked pixels: the mean of |img -
    target| over the C x (masked pixels) values; dL/dimg = sign / that count on
    masked pixels and 0 elsewhere (both 0 for an empty mask)."""
    d = np.asarray(img, np.float64) - np.asarray(target, np.float64)
    m = np.broadcast_to(np.asarray(pixel_mask, bool)[None], d.shape)
    cnt = int(m.sum())
    if cnt == 0:
        return 0.0, np.zeros_like(d)
    return float(np.abs(d[m]).sum() / cnt), np.where(m, np.sign(d), 0.0) / cnt
