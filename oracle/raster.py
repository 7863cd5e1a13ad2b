"""ctypes front-end of the C oracle (queen_oracle.c).  Test infrastructure only.

All arrays go in and come out as float64 planes ([.][n]); integer outputs are
int32.  The C code is compiled with gcc on first use (or by build()).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "queen_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_F = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_I = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_U8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_U32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_U64 = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, OpenMP, -O2)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                                   "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB_PATH)
    lib.or_sh_basis.argtypes = [C.c_int, _D, C.c_int, _D, C.c_void_p]
    lib.or_decode.argtypes = [C.c_int, C.c_int, _D, C.c_int, _I, _I, _I, _D, _D, C.c_int, _D, _D,
                              C.c_double, C.c_double, C.c_double, _D, _D, _D]
    lib.or_decode_bwd.argtypes = [C.c_int, C.c_int, C.c_int, _I, _I, _I, _D, _D, C.c_int, _D, _D,
                                  C.c_double, C.c_double, C.c_double, _D, C.c_double, C.c_void_p,
                                  _D, _D, _D, _D]
    lib.or_project.argtypes = [C.c_int, C.c_int, C.c_int, _D, _D, C.c_int, C.c_int, C.c_double, C.c_int,
                               C.c_double, _D, _D, _D, _D, _D, _I, _I, _I, _I]
    lib.or_project_bwd.argtypes = [C.c_int, C.c_int, C.c_int, _D, _D, C.c_int, C.c_int, C.c_double,
                                   _D, _D, _D, _D, _D]
    lib.or_bin_count.argtypes = [C.c_int, _I]
    lib.or_bin_count.restype = C.c_int64
    lib.or_bin_sort.argtypes = [C.c_int, _F, _I, C.c_int, C.c_int, _U64, _U32, _U32]
    lib.or_bin_sort.restype = C.c_int64
    lib.or_render_fwd.argtypes = [C.c_int, _D, _D, _D, _D, _D, _I, _I, _I, C.c_int, C.c_int, _D,
                                  C.c_double, C.c_double, C.c_double, C.c_void_p, C.c_int, _D, _D, _I, _I]
    lib.or_render_bwd.argtypes = [C.c_int, _D, _D, _D, _D, _D, _I, C.c_int, C.c_int, _D, _D,
                                  C.c_void_p, C.c_int, _D, _D, _D, _D, C.c_void_p]
    lib.or_num_threads.restype = C.c_int
    _lib = lib
    return lib


def num_threads() -> int:
    return int(_load().or_num_threads())


def _d(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _i(x):
    return np.ascontiguousarray(x, dtype=np.int32)


@dataclass
class OracleCamera:
    R: np.ndarray
    t: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float
    campos: np.ndarray

    @staticmethod
    def of(cam) -> "OracleCamera":
        return OracleCamera(np.asarray(cam.R, np.float64), np.asarray(cam.t, np.float64), float(cam.fx),
                            float(cam.fy), float(cam.cx), float(cam.cy), int(cam.width), int(cam.height),
                            float(cam.near), np.asarray(cam.campos, np.float64))

    def packed(self) -> np.ndarray:
        return _d(np.concatenate([self.R.reshape(9), self.t.reshape(3),
                                  [self.fx, self.fy, self.cx, self.cy, self.near],
                                  self.campos.reshape(3)]))


def sh_basis(degree: int, dirs: np.ndarray, grad: bool = False):
    """Real SH basis Y[n][K] (and polynomial gradient dY[n][K][3]) at unit
    directions dirs[n][3].  Pinned: orthonormality, scipy sph_harm_y, FD."""
    lib = _load()
    dirs = _d(dirs).reshape(-1, 3)
    n = dirs.shape[0]
    K = (degree + 1) ** 2
    Y = np.zeros((n, K))
    dY = np.zeros((n, K, 3)) if grad else None
    lib.or_sh_basis(degree, dirs, n, Y, dY.ctypes.data if grad else None)
    return (Y, dY) if grad else Y


def _layout_arrays(layout):
    return (_i(layout.attr_begin), _i(layout.attr_count), _i(layout.lat_dim))


def _noise_shift(log_alpha, noise):
    """log alpha + logit(u): the stochastic hard-concrete sample is Eq. 6 with
    log alpha shifted by the logistic noise log u - log(1 - u)."""
    u = np.asarray(noise, np.float64)
    return _d(log_alpha) + (np.log(u) - np.log1p(-u))


def _lreg(log_alpha, tau, gamma0, gamma1):
    """Eq. 8 (independent of the noise)."""
    z = _d(log_alpha) - tau * np.log(-gamma0 / gamma1)
    return 1.0 / (1.0 + np.exp(-z))


def decode(prev, lat, dec, lp, log_alpha, layout, tau, gamma0, gamma1, round_latents=True, noise=None):
    """Eq. 4-8: A_t = A_{t-1} + R_t with r = D float(round(l_hat)) and
    dp = g l_p; returns (A_t, gate, L_reg).  With noise (u [n] in (0, 1)) the
    gate is the stochastic hard-concrete sample sigmoid((log alpha + log u -
    log(1 - u)) / tau), stretched and clipped as in Eq. 7; L_reg (Eq. 8) stays
    on log alpha.  Pinned: hand example, closed-form gate values,
    rounding/saturation cases; the noisy gate against its closed form."""
    if noise is not None:
        out, gate, _ = decode(prev, lat, dec, lp, _noise_shift(log_alpha, noise), layout, tau, gamma0, gamma1,
                              round_latents)
        return out, gate, float(_lreg(log_alpha, tau, gamma0, gamma1).sum())
    lib = _load()
    prev = _d(prev)
    na, n = prev.shape
    out = np.zeros_like(prev)
    gate = np.zeros(n)
    lreg = np.zeros(1)
    ab, ac, ld = _layout_arrays(layout)
    lib.or_decode(n, na, prev, layout.n_cat, ab, ac, ld, _d(lat), _d(dec), int(round_latents), _d(lp),
                  _d(log_alpha), tau, gamma0, gamma1, out, gate, lreg)
    return out, gate, float(lreg[0])


def decode_bwd(lat, dec, lp, log_alpha, layout, tau, gamma0, gamma1, d_out, d_lreg=0.0, skip=None,
               round_latents=True, noise=None):
    """Adjoint of decode (STE for the latents).  Returns (d_lat, d_dec, d_lp,
    d_log_alpha).  With noise, the gate's path takes the shifted log alpha
    and the L_reg path the plain one.  Pinned: finite differences with
    rounding switched off (also with noise)."""
    if noise is not None:
        d_lat, d_dec, d_lp, d_la = decode_bwd(lat, dec, lp, _noise_shift(log_alpha, noise), layout, tau, gamma0,
                                              gamma1, d_out, 0.0, skip, round_latents)
        p = _lreg(log_alpha, tau, gamma0, gamma1)
        d_la = d_la + float(d_lreg) * p * (1.0 - p)
        if skip is not None:
            d_la = np.where(np.asarray(skip) != 0, 0.0, d_la)
        return d_lat, d_dec, d_lp, d_la
    lib = _load()
    d_out = _d(d_out)
    na, n = d_out.shape
    ab, ac, ld = _layout_arrays(layout)
    d_lat = np.zeros((layout.n_latent, n))
    d_dec = np.zeros(layout.n_dec)
    d_lp = np.zeros((3, n))
    d_la = np.zeros(n)
    sk = None if skip is None else np.ascontiguousarray(skip, dtype=np.uint8)
    lib.or_decode_bwd(n, na, layout.n_cat, ab, ac, ld, _d(lat), _d(dec), int(round_latents), _d(lp),
                      _d(log_alpha), tau, gamma0, gamma1, d_out, float(d_lreg),
                      None if sk is None else sk.ctypes.data, d_lat, d_dec, d_lp, d_la)
    return d_lat, d_dec, d_lp, d_la


def project(attrs, cam, sh_degree, blur=0.3, eps_g=0.0, tight=False):
    """Eq. 1 + SH colour.  Returns a dict of planes (see queen_oracle.c).
    With tight=True the tile rects are limited to the tiles the
    alpha >= 1/255 ellipse can reach (same rendering, shorter tile lists)."""
    lib = _load()
    oc = cam if isinstance(cam, OracleCamera) else OracleCamera.of(cam)
    A = _d(attrs)
    na, n = A.shape
    r = dict(mean2d=np.zeros((2, n)), conic=np.zeros((3, n)), opac=np.zeros(n), rgb=np.zeros((3, n)),
             depth=np.zeros(n), radius=np.zeros(n, np.int32), rect=np.zeros((4, n), np.int32),
             fragile=np.zeros(n, np.int32), frag_rect=np.zeros((4, n), np.int32))
    lib.or_project(n, na, sh_degree, A, oc.packed(), oc.width, oc.height, blur, int(tight), eps_g, r["mean2d"],
                   r["conic"], r["opac"], r["rgb"], r["depth"], r["radius"], r["rect"], r["fragile"],
                   r["frag_rect"])
    r["width"], r["height"] = oc.width, oc.height
    return r


def project_bwd(attrs, cam, sh_degree, d_mean2d, d_conic, d_opac, d_rgb, blur=0.3):
    """Adjoint of project.  Pinned by central finite differences."""
    lib = _load()
    oc = cam if isinstance(cam, OracleCamera) else OracleCamera.of(cam)
    A = _d(attrs)
    na, n = A.shape
    dA = np.zeros_like(A)
    lib.or_project_bwd(n, na, sh_degree, A, oc.packed(), oc.width, oc.height, blur, _d(d_mean2d),
                       _d(d_conic), _d(d_opac), _d(d_rgb), dA)
    return dA


def bin_sort(depth_f32, rect, tiles_x, tiles_y):
    """Integer binning: keys (tile << 32 | float bits of depth), values, and
    per-tile ranges [n_tiles][2] of the stable sort.  Pinned by a pure-Python
    brute force and partition invariants."""
    lib = _load()
    depth = np.ascontiguousarray(depth_f32, dtype=np.float32)
    rect = _i(rect)
    n = depth.shape[0]
    P = int(lib.or_bin_count(n, rect))
    keys = np.zeros(max(P, 1), np.uint64)
    vals = np.zeros(max(P, 1), np.uint32)
    ranges = np.zeros((tiles_x * tiles_y, 2), np.uint32)
    got = lib.or_bin_sort(n, depth, rect, tiles_x, tiles_y, keys, vals, ranges)
    if got != P:
        raise RuntimeError("oracle bin_sort failed")
    return keys[:P], vals[:P], ranges


def _tiles(tiles):
    if tiles is None:
        return None, 0, None
    t = np.ascontiguousarray(tiles, dtype=np.int32)
    return t.ctypes.data, int(t.size), t


def render_fwd(proj, bg=(0.0, 0.0, 0.0), eps=0.0, eps_d=0.0, tiles=None, eps_t=None):
    """Eq. 2 per pixel.  Returns (img[3][H][W], T_final, last, fragile).
    Pinned: single-Gaussian footprint closed form, two-Gaussian hand blend,
    transmittance invariants, pure-Python brute force.  `tiles` (optional)
    restricts the work to those tile indices.  Fragility flags (pinned by
    tests/test_oracle_fragility.py): eps is the relative margin of the alpha
    decisions (threshold and cap), eps_t that of the termination product
    (default eps); consecutive contributors whose depths lie within eps_d
    relative are flagged (eps_d < 0 flags none, for depths that are the GPU's
    own FP32 values, which both sides order alike)."""
    lib = _load()
    tp, tn, _keep = _tiles(tiles)
    W, H = proj["width"], proj["height"]
    n = proj["opac"].shape[0]
    img = np.zeros((3, H, W))
    T = np.zeros((H, W))
    last = np.zeros((H, W), np.int32)
    frag = np.zeros((H, W), np.int32)
    lib.or_render_fwd(n, _d(proj["mean2d"]), _d(proj["conic"]), _d(proj["opac"]), _d(proj["rgb"]),
                      _d(proj["depth"]), _i(proj["rect"]), _i(proj["fragile"]), _i(proj["frag_rect"]),
                      W, H, _d(bg), eps, eps if eps_t is None else eps_t, eps_d, tp, tn, img, T, last, frag)
    return img, T, last, frag


def render_bwd(proj, d_img, bg=(0.0, 0.0, 0.0), tiles=None, magnitudes=False):
    """Adjoint of render_fwd.  Returns dict d_mean2d[2][n], d_conic[3][n],
    d_opac[n], d_rgb[3][n].  Pinned by central finite differences.
    magnitudes: also "mag", the same keys holding each entry's sum of term
    magnitudes (dL/dalpha's signed parts taken as T sum |dC| (|c| + |B|)),
    which bounds what floating-point summation of the entry can keep.
    Pinned: never below the entry's magnitude, and equal to it where no term
    and no factor changes sign."""
    lib = _load()
    tp, tn, _keep = _tiles(tiles)
    W, H = proj["width"], proj["height"]
    n = proj["opac"].shape[0]
    g = dict(d_mean2d=np.zeros((2, n)), d_conic=np.zeros((3, n)), d_opac=np.zeros(n),
             d_rgb=np.zeros((3, n)))
    m = np.zeros((9, n)) if magnitudes else None
    lib.or_render_bwd(n, _d(proj["mean2d"]), _d(proj["conic"]), _d(proj["opac"]), _d(proj["rgb"]),
                      _d(proj["depth"]), _i(proj["rect"]), W, H, _d(bg), _d(d_img), tp, tn, g["d_mean2d"],
                      g["d_conic"], g["d_opac"], g["d_rgb"], m.ctypes.data if m is not None else None)
    if m is not None:
        g["mag"] = dict(d_mean2d=m[0:2], d_conic=m[2:5], d_opac=m[5], d_rgb=m[6:9])
    return g
