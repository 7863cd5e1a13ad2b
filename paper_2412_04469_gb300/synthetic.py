"""Seeded synthetic inputs shaped like QUEEN's multi-view captures.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic, and both the CUDA path and the CPU oracle consume it.

Scene recipe (per Gaussian, numpy PCG64, seed given):
  position   ~ U[-1, 1]^3
  log-scale  ~ N(-3, 0.5^2) per axis
  quaternion ~ normalised N(0, I_4)   (uniform on S^3; stored in (w, x, y, z))
  logit(o)   ~ N(0, 1)
  SH DC      ~ U[-1.7725, 1.7725] per channel, which makes the DC colour
               uniform in [0, 1]; higher-order coefficients ~ N(0, 0.1^2).
Residual parameters (Sec. 3.2): continuous latents ~ N(0, 1), decoders
  ~ N(0, 0.01^2) rounded to bfloat16, log-alpha ~ N(-2, 1),
  pre-gated position residuals ~ N(0, 0.01^2).
Cameras: pinhole, square pixels, horizontal field of view `fov_deg`,
  principal point at the image centre, looking at the origin with world +y
  up (camera x right, y down, z forward).

Attribute planes ([n_attr][n], float32): 0-2 position, 3-6 quaternion,
7-9 log-scale, 10 logit-opacity, 11 + 3 k + ch SH coefficient k of channel ch.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SH_DC_HALF_RANGE = 1.7724538509055159  # 0.5 / (SH degree-0 basis value)


def n_sh(degree: int) -> int:
    return (degree + 1) * (degree + 1)


def n_attr(degree: int) -> int:
    return 11 + 3 * n_sh(degree)


@dataclass
class DecoderLayout:
    """Residual categories of Sec. 3.4: which attribute planes each decoder
    writes and its latent width.  Default: rotation (4), scale (3),
    opacity (1), SH (3 K) with latent width 8 each."""

    attr_begin: list = field(default_factory=list)
    attr_count: list = field(default_factory=list)
    lat_dim: list = field(default_factory=list)

    @staticmethod
    def default(sh_degree: int = 3, latent: int = 8) -> "DecoderLayout":
        return DecoderLayout([3, 7, 10, 11], [4, 3, 1, 3 * n_sh(sh_degree)], [latent] * 4)

    @staticmethod
    def paper_n3dv(sh_degree: int = 2) -> "DecoderLayout":
        """The N3DV decoders of the paper's quantisation table (App. B):
        rotation (latent width 6), scale (8), opacity (3), colour base = the
        SH DC coefficients (8) and colour frequency = the higher SH
        coefficients (4); N3DV trains SH degree 2."""
        K = n_sh(sh_degree)
        if K < 2:
            raise ValueError("the colour-frequency decoder needs SH degree >= 1")
        return DecoderLayout([3, 7, 10, 11, 14], [4, 3, 1, 3, 3 * (K - 1)], [6, 8, 3, 8, 4])

    @property
    def n_cat(self) -> int:
        return len(self.attr_begin)

    @property
    def n_latent(self) -> int:
        return int(sum(self.lat_dim))

    @property
    def n_dec(self) -> int:
        return int(sum(m * l for m, l in zip(self.attr_count, self.lat_dim)))


def to_bf16_values(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even); returns
    float32 holding exactly representable bfloat16 values."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """Upper 16 bits of float32 values that are exact bfloat16 values."""
    return (np.ascontiguousarray(x, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)


def make_scene(n: int, sh_degree: int, seed: int = 0) -> np.ndarray:
    """Raw attributes A_{t-1} as float32 planes [n_attr][n]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    K = n_sh(sh_degree)
    A = np.zeros((n_attr(sh_degree), n), np.float32)
    A[0:3] = rng.uniform(-1.0, 1.0, (3, n))
    q = rng.standard_normal((4, n))
    A[3:7] = q / np.linalg.norm(q, axis=0, keepdims=True)
    A[7:10] = rng.normal(-3.0, 0.5, (3, n))
    A[10] = rng.standard_normal(n)
    A[11:14] = rng.uniform(-SH_DC_HALF_RANGE, SH_DC_HALF_RANGE, (3, n))
    if K > 1:
        A[14:] = rng.normal(0.0, 0.1, (3 * (K - 1), n))
    return A


@dataclass
class Residuals:
    lat: np.ndarray        # [n_latent][n] float32 continuous latents
    dec: np.ndarray        # [n_dec] float32, exact bfloat16 values
    lp: np.ndarray         # [3][n] float32 pre-gated position residuals
    log_alpha: np.ndarray  # [n] float32


def make_residuals(n: int, layout: DecoderLayout, seed: int = 0) -> Residuals:
    rng = np.random.Generator(np.random.PCG64(seed + 1000003))
    lat = rng.standard_normal((layout.n_latent, n)).astype(np.float32)
    dec = to_bf16_values(rng.normal(0.0, 0.01, layout.n_dec).astype(np.float32))
    lp = rng.normal(0.0, 0.01, (3, n)).astype(np.float32)
    la = rng.normal(-2.0, 1.0, n).astype(np.float32)
    return Residuals(lat, dec, lp, la)


@dataclass
class Camera:
    R: np.ndarray          # [3][3] world -> camera rotation (rows: right, down, forward)
    t: np.ndarray          # [3]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float
    campos: np.ndarray     # [3] camera centre in world coordinates


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)):
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    return R, -R @ eye


def make_camera(width: int, height: int, fov_deg: float = 60.0, eye=(0.0, 0.0, 4.0),
                target=(0.0, 0.0, 0.0), near: float = 0.2) -> Camera:
    R, t = look_at(eye, target)
    f = 0.5 * width / math.tan(math.radians(fov_deg) / 2.0)
    return Camera(R.astype(np.float32).astype(np.float64), t.astype(np.float32).astype(np.float64),
                  float(np.float32(f)), float(np.float32(f)), 0.5 * width, 0.5 * height,
                  width, height, near, np.asarray(eye, np.float32).astype(np.float64))


def make_arc_cameras(views: int, width: int, height: int, radius: float = 4.0,
                     arc_deg: float = 120.0, fov_deg: float = 60.0) -> list:
    """`views` cameras on an arc of `arc_deg` degrees in the y = 0 plane."""
    cams = []
    for v in range(views):
        th = math.radians(-0.5 * arc_deg + arc_deg * (v / max(1, views - 1)))
        eye = (radius * math.sin(th), 0.0, radius * math.cos(th))
        cams.append(make_camera(width, height, fov_deg, eye))
    return cams


def make_image(width: int, height: int, seed: int) -> np.ndarray:
    """Uniform [0, 1] image [3][H][W] (an upstream-gradient or target stand-in)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    return rng.uniform(0.0, 1.0, (3, height, width)).astype(np.float32)


def make_bin_inputs(n: int, tiles_x: int, tiles_y: int, seed: int, max_extent: int = 6,
                    tie_frac: float = 0.25, empty_frac: float = 0.1):
    """Random float32 depths (with deliberate exact ties) and tile rects
    (x0, y0, x1, y1) [4][n] for the binning path; some rects are empty."""
    rng = np.random.Generator(np.random.PCG64(seed + 31337))
    depth = rng.uniform(0.2, 10.0, n).astype(np.float32)
    tie = rng.uniform(size=n) < tie_frac
    if n > 1 and tie.any():
        depth[tie] = depth[rng.integers(0, n, int(tie.sum()))]
    x0 = rng.integers(0, tiles_x, n)
    y0 = rng.integers(0, tiles_y, n)
    w = rng.integers(1, max_extent + 1, n)
    h = rng.integers(1, max_extent + 1, n)
    x1 = np.minimum(x0 + w, tiles_x)
    y1 = np.minimum(y0 + h, tiles_y)
    empty = rng.uniform(size=n) < empty_frac
    x0[empty] = x1[empty] = y0[empty] = y1[empty] = 0
    rect = np.stack([x0, y0, x1, y1]).astype(np.int32)
    return depth, rect


@dataclass
class Motion:
    """Ground-truth motion of a synthetic streaming sequence: a random
    `frac` of the Gaussians rotate rigidly about the world y axis through the
    origin by `deg_per_frame` per frame and jitter by
    amp sin(2 pi t / period + phi_i) u_i (u_i uniform on the sphere)."""
    dynamic: np.ndarray    # [n] bool
    phase: np.ndarray      # [n]
    direction: np.ndarray  # [3][n]
    deg_per_frame: float = 0.5
    amp: float = 0.01
    period: float = 30.0


def make_motion(n: int, frac: float = 0.1, seed: int = 0, deg_per_frame: float = 0.5, amp: float = 0.01,
                period: float = 30.0, positions: np.ndarray | None = None,
                centre=(0.0, 0.0, 1.0)) -> Motion:
    """With `positions` ([3][n]) the dynamic set is a rigid object: the
    frac * n Gaussians nearest `centre` (by default the middle of the cube face
    the cameras look at, so the object is visible); without, a uniformly random
    subset."""
    rng = np.random.Generator(np.random.PCG64(seed + 4242))
    dyn = np.zeros(n, bool)
    k = int(round(frac * n))
    if positions is not None:
        d2 = ((np.asarray(positions, np.float64) - np.asarray(centre, np.float64)[:, None]) ** 2).sum(axis=0)
        dyn[np.argsort(d2, kind="stable")[:k]] = True
    else:
        dyn[rng.choice(n, size=k, replace=False)] = True
    u = rng.standard_normal((3, n))
    u /= np.linalg.norm(u, axis=0, keepdims=True)
    return Motion(dyn, rng.uniform(0, 2 * math.pi, n), u, deg_per_frame, amp, period)


def frame_attrs(A0: np.ndarray, motion: Motion, t: int) -> np.ndarray:
    """Raw attributes of frame t (frame 0 is A0): positions and orientations of
    the dynamic Gaussians follow the motion, everything else is unchanged."""
    A = A0.copy()
    d = motion.dynamic
    th = math.radians(motion.deg_per_frame * t)
    c, s = math.cos(th), math.sin(th)
    x, y, z = A0[0, d].astype(np.float64), A0[1, d].astype(np.float64), A0[2, d].astype(np.float64)
    jit = motion.amp * (np.sin(2 * math.pi * t / motion.period + motion.phase[d])
                        - np.sin(motion.phase[d]))[None, :] * motion.direction[:, d]
    A[0, d] = c * x + s * z + jit[0]
    A[1, d] = y + jit[1]
    A[2, d] = -s * x + c * z + jit[2]
    # orientation: q_t = q_y(th) * q_0 with q_y(th) = (cos th/2, 0, sin th/2, 0)
    hw, hy = math.cos(th / 2), math.sin(th / 2)
    w0, x0, y0, z0 = (A0[3 + k, d].astype(np.float64) for k in range(4))
    A[3, d] = hw * w0 - hy * y0
    A[4, d] = hw * x0 + hy * z0
    A[5, d] = hw * y0 + hy * w0
    A[6, d] = hw * z0 - hy * x0
    return A
