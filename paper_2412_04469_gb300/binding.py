"""Thin ctypes binding of libqueen_gb300.so (include/queen.h).

Each function has the name of its C entry point, takes torch tensors (device
memory) or plain numbers, marshals them to pointers and raises QueenError on
a non-zero status.  No computation happens here.  Loading fails loudly when
the library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqueen_gb300.so")

QN_OK, QN_ERR_INVALID_ARG, QN_ERR_CUDA, QN_ERR_CAPACITY, QN_ERR_TIMEOUT, QN_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5
QN_TILE = 16
QN_MAX_CATEGORIES = 8


class QueenError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"queen status {code}: {msg}")
        self.code = code


class qn_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("near_plane", C.c_float), ("campos", C.c_float * 3),
                ("width", C.c_int32), ("height", C.c_int32)]


class qn_decoder_layout(C.Structure):
    _fields_ = [("n_cat", C.c_int32), ("attr_begin", C.c_int32 * QN_MAX_CATEGORIES),
                ("attr_count", C.c_int32 * QN_MAX_CATEGORIES), ("lat_dim", C.c_int32 * QN_MAX_CATEGORIES)]


class qn_gate_params(C.Structure):
    _fields_ = [("tau", C.c_float), ("gamma0", C.c_float), ("gamma1", C.c_float), ("noise", C.c_void_p)]


QN_ADAM_MAX_GROUPS = 16


class qn_adam_group(C.Structure):
    _fields_ = [("param", C.c_void_p), ("grad", C.c_void_p), ("m", C.c_void_p), ("v", C.c_void_p),
                ("param_bf16", C.c_void_p), ("rows", C.c_int32), ("n", C.c_int32), ("stride", C.c_int32),
                ("lr", C.c_float), ("use_skip", C.c_int32)]


_lib = None
_P = C.c_void_p
_I32, _I64, _F32, _SZ, _U32 = C.c_int32, C.c_int64, C.c_float, C.c_size_t, C.c_uint32

_SIGS = {
    "qn_last_error": ([], C.c_char_p),
    "qn_version": ([], C.c_char_p),
    "qn_decode_residuals": ([_I32, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "qn_decode_project": ([_I32, _I32, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _F32, _I32, _P, _P, _P, _P,
                           _P, _P], C.c_int),
    "qn_decode_residuals_bwd": ([_I32, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _F32, _P, _P, _P, _P, _P, _P,
                                 _P], C.c_int),
    "qn_decode_project_bwd": ([_I32, _I32, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _F32, _P, _F32, _P, _P,
                               _P, _P, _P, _P], C.c_int),
    "qn_project": ([_I32, _I32, _I32, _P, _P, _F32, _I32, _P, _P, _P], C.c_int),
    "qn_project_bwd": ([_I32, _I32, _I32, _P, _P, _F32, _P, _P, _P, _P], C.c_int),
    "qn_bin_sort_workspace_size": ([_I32, _I32, _I32], _SZ),
    "qn_bin_sort": ([_I32, _P, _I32, _P, _I32, _I32, _P, _SZ, _I64, _P, _P, _P, _P, _P, _P], C.c_int),
    "qn_bin_sort_noalloc": ([_I32, _P, _I32, _P, _I32, _I32, _I64, _P, _P, _P, _P, _P, _P], C.c_int),
    "qn_render_fwd": ([_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "qn_render_fwd_binned": ([_P, _I32, _P, _SZ, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "qn_bin_sort_partial": ([_I32, _P, _I32, _P, _I32, _I32, _P, _SZ, _I64, _U32, _P, _P, _P, _P, _P], C.c_int),
    "qn_tile_order": ([_I32, _P, _P, _P], C.c_int),
    "qn_render_bwd": ([_P, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P, _P, _P], C.c_int),
    "qn_render_bwd_pairs": ([_P, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P, _P], C.c_int),
    "qn_render_bwd_gather": ([_P, _I32, _P, _P, _P, _SZ, _P, _P, _P], C.c_int),
    "qn_image_loss": ([_I64, _P, _P, _F32, _I32, _P, _P, _P, _P], C.c_int),
    "qn_viewspace_accum": ([_I32, _I32, _P, _F32, _P, _P], C.c_int),
    "qn_gate_init": ([_I32, _I32, _P, _P, _I32, _P, _P, _P, _P], C.c_int),
    "qn_skip_features": ([_I32, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "qn_skip_mlp_fwd": ([_I32, _I32, _P, _P, _F32, _P, _P, _P], C.c_int),
    "qn_skip_mlp_bwd": ([_I32, _I32, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "qn_skip_labels": ([_I32, _I32, _I32, _P, _P, _P, _P, _P], C.c_int),
    "qn_or_marks": ([_I32, _P, _P, _P], C.c_int),
    "qn_clear_marked": ([_I32, _P, _P, _P], C.c_int),
    "qn_adam": ([_I32, _I32, _I32, _P, _P, _P, _P, _I32, _F32, _F32, _F32, _F32, _P, _P, _P], C.c_int),
    "qn_adam_groups": ([_I32, _P, _P, _F32, _F32, _F32, _P, _P], C.c_int),
    "qn_partition_workspace_size": ([_I32], C.c_size_t),
    "qn_select_rects": ([_I32, _I32, _P, _P, _F32, _F32, _F32, _P, _P], C.c_int),
    "qn_dilate_mask": ([_I32, _I32, _P, _I32, _P, _P, _P, _P, _P], C.c_int),
    "qn_mask_ranges": ([_I32, _P, _P, _P, _P], C.c_int),
    "qn_masked_image_loss": ([_I64, _I32, _P, _P, _P, _P, _F32, _I32, _P, _P, _P, _P], C.c_int),
    "qn_dssim_workspace_size": ([_I32, _I32, _I32], _SZ),
    "qn_dssim_loss": ([_I32, _I32, _I32, _P, _P, _P, _P, _F32, _P, _P, _P, _SZ, _P], C.c_int),
    "qn_pack_workspace_size": ([_I32, _P], _SZ),
    "qn_packet_max_bytes": ([_I32, _P], _SZ),
    "qn_pack_frame": ([_I32, _I32, _P, _P, _P, _P, _P, _P, _SZ, _P, _SZ, _P, _P], C.c_int),
    "qn_unpack_workspace_size": ([_I32, _I32, _P, _SZ], _SZ),
    "qn_unpack_frame": ([_P, _SZ, _I32, _I32, _I32, _P, _P, _P, _P, _SZ, _P], C.c_int),
    "qn_gate_uniform": ([_I32, C.c_uint64, _P, _P, _P], C.c_int),
    "qn_partition": ([_I32, _P, _P, _P, _P, C.c_size_t, _P], C.c_int),
    "qn_gather_columns": ([_I32, _I32, _I32, _P, C.c_int64, _P, _P, C.c_int64, _P], C.c_int),
}


def lib():
    """Loads the library (built by paper_2412_04469_gb300.build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise QueenError(QN_ERR_UNSUPPORTED, f"{LIB_PATH} is missing: run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise QueenError(QN_ERR_INVALID_ARG, "expected a CUDA tensor")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _check(code):
    if code != QN_OK:
        raise QueenError(code, lib().qn_last_error().decode())


def make_camera(cam) -> qn_camera:
    """qn_camera from any object with R, t, fx, fy, cx, cy, near, campos, width, height."""
    c = qn_camera()
    R = [float(v) for row in cam.R for v in row]
    for k in range(9):
        c.R[k] = R[k]
    for k in range(3):
        c.t[k] = float(cam.t[k])
        c.campos[k] = float(cam.campos[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.near_plane = float(cam.near)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def make_layout(layout) -> qn_decoder_layout:
    L = qn_decoder_layout()
    L.n_cat = layout.n_cat
    for c in range(layout.n_cat):
        L.attr_begin[c] = layout.attr_begin[c]
        L.attr_count[c] = layout.attr_count[c]
        L.lat_dim[c] = layout.lat_dim[c]
    return L


def make_gate(tau, gamma0, gamma1, noise=None) -> qn_gate_params:
    """Gate parameters; noise (device float tensor [n], u in (0, 1)) selects
    the stochastic hard-concrete sample, None the gate of Eq. 6."""
    return qn_gate_params(tau, gamma0, gamma1, _ptr(noise))


def qn_decode_residuals(n, n_stride, n_attr, prev, lat, dec, layout, lp, log_alpha, gate_params, out, gate=None,
                        lreg=None, stream=None, skip=None):
    _check(lib().qn_decode_residuals(n, n_stride, n_attr, _ptr(prev), _ptr(lat), _ptr(dec), C.byref(layout),
                                     _ptr(lp), _ptr(log_alpha), C.byref(gate_params), _ptr(skip), _ptr(out),
                                     _ptr(gate), _ptr(lreg), _stream(stream)))


QN_DECODE_BWD_BLOCKS = 1216
QN_MLP_BWD_BLOCKS = 256


def qn_decode_project(n, n_stride, n_attr, sh_degree, prev, lat, dec, layout, lp, log_alpha, gate_params, skip, cam,
                      blur, tight_rects, gate, lreg, out, splats, rects, stream=None):
    _check(lib().qn_decode_project(n, n_stride, n_attr, sh_degree, _ptr(prev), _ptr(lat), _ptr(dec),
                                   C.byref(layout), _ptr(lp), _ptr(log_alpha), C.byref(gate_params), _ptr(skip),
                                   C.byref(cam), float(blur), int(bool(tight_rects)), _ptr(gate), _ptr(lreg),
                                   _ptr(out), _ptr(splats), _ptr(rects), _stream(stream)))


def qn_decode_project_bwd(n, n_stride, n_attr, sh_degree, prev, lat, dec, layout, lp, log_alpha, gate_params, skip,
                          cam, blur, d_splats, d_lreg, d_lat, d_dec, d_lp, d_log_alpha, partials, stream=None):
    """partials: QN_DECODE_BWD_BLOCKS * d_dec.numel() floats of scratch."""
    _check(lib().qn_decode_project_bwd(n, n_stride, n_attr, sh_degree, _ptr(prev), _ptr(lat), _ptr(dec),
                                       C.byref(layout), _ptr(lp), _ptr(log_alpha), C.byref(gate_params), _ptr(skip),
                                       C.byref(cam), float(blur), _ptr(d_splats), float(d_lreg), _ptr(d_lat),
                                       _ptr(d_dec), _ptr(d_lp), _ptr(d_log_alpha), _ptr(partials), _stream(stream)))


def qn_decode_residuals_bwd(n, n_stride, n_attr, lat, dec, layout, lp, log_alpha, gate_params, d_out, d_lreg,
                            skip, d_lat, d_dec, d_lp, d_log_alpha, partials, stream=None):
    """partials: QN_DECODE_BWD_BLOCKS * d_dec.numel() floats of scratch."""
    _check(lib().qn_decode_residuals_bwd(n, n_stride, n_attr, _ptr(lat), _ptr(dec), C.byref(layout), _ptr(lp),
                                         _ptr(log_alpha), C.byref(gate_params), _ptr(d_out), float(d_lreg),
                                         _ptr(skip), _ptr(d_lat), _ptr(d_dec), _ptr(d_lp), _ptr(d_log_alpha),
                                         _ptr(partials), _stream(stream)))


def qn_project(n, n_stride, sh_degree, attrs, cam, blur, splats, rects, tight_rects=True, stream=None):
    _check(lib().qn_project(n, n_stride, sh_degree, _ptr(attrs), C.byref(cam), float(blur), int(tight_rects),
                            _ptr(splats), _ptr(rects), _stream(stream)))


def qn_project_bwd(n, n_stride, sh_degree, attrs, cam, blur, d_splats, skip, d_attrs, stream=None):
    _check(lib().qn_project_bwd(n, n_stride, sh_degree, _ptr(attrs), C.byref(cam), float(blur), _ptr(d_splats),
                                _ptr(skip), _ptr(d_attrs), _stream(stream)))


def qn_bin_sort_workspace_size(n, tiles_x, tiles_y):
    return int(lib().qn_bin_sort_workspace_size(n, tiles_x, tiles_y))


def qn_bin_sort(n, depth, depth_stride, rects, tiles_x, tiles_y, workspace, pair_capacity, vals, keys, ranges,
                n_pairs, sync=True, stream=None):
    """Returns P (int) when sync is True (the call synchronises), else None."""
    host = C.c_int64(0)
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().qn_bin_sort(n, _ptr(depth), depth_stride, _ptr(rects), tiles_x, tiles_y, _ptr(workspace),
                             ws_bytes, int(pair_capacity), _ptr(vals), _ptr(keys), _ptr(ranges), _ptr(n_pairs),
                             C.addressof(host) if sync else None, _stream(stream)))
    return int(host.value) if sync else None


def qn_bin_sort_partial(n, depth, depth_stride, rects, tiles_x, tiles_y, workspace, pair_capacity, list_max, vals,
                        ranges, n_pairs, sync=True, stream=None):
    """qn_bin_sort writing only the lists of at most list_max pairs; returns P
    (int) when sync is True (the call synchronises), else None."""
    host = C.c_int64(0)
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().qn_bin_sort_partial(n, _ptr(depth), depth_stride, _ptr(rects), tiles_x, tiles_y, _ptr(workspace),
                                     ws_bytes, int(pair_capacity), int(list_max), _ptr(vals), _ptr(ranges),
                                     _ptr(n_pairs), C.addressof(host) if sync else None, _stream(stream)))
    return int(host.value) if sync else None


def qn_bin_sort_noalloc(n, depth, depth_stride, rects, tiles_x, tiles_y, pair_capacity, vals, keys, ranges,
                        n_pairs, sync=True, stream=None):
    """qn_bin_sort on the library's fixed device workspace, for callers that
    may not allocate device memory (allocator hooks, plugins in another
    application's memory pool, real-time loops); returns P when sync is True."""
    host = C.c_int64(0)
    _check(lib().qn_bin_sort_noalloc(n, _ptr(depth), depth_stride, _ptr(rects), tiles_x, tiles_y,
                                     int(pair_capacity), _ptr(vals), _ptr(keys), _ptr(ranges), _ptr(n_pairs),
                                     C.addressof(host) if sync else None, _stream(stream)))
    return int(host.value) if sync else None


def _bg(bg):
    return (C.c_float * 3)(*[float(v) for v in bg])


def qn_render_fwd(cam, ranges, vals, splats, bg, img, T_final, last, n_contrib=None, stream=None, composited=None,
                  tile_order=None, tile_cost=None):
    _check(lib().qn_render_fwd(C.byref(cam), _ptr(ranges), _ptr(vals), _ptr(splats), _bg(bg), _ptr(img),
                               _ptr(T_final), _ptr(last), _ptr(n_contrib), _ptr(composited), _ptr(tile_order),
                               _ptr(tile_cost), _stream(stream)))


def qn_render_fwd_binned(cam, n, workspace, ranges, vals, splats, bg, img, T_final, last, n_contrib=None,
                         stream=None, composited=None, tile_order=None, tile_cost=None):
    """qn_render_fwd after qn_bin_sort_partial: the lists it left unwritten are
    formed from the binning workspace; their walked positions are written to vals."""
    _check(lib().qn_render_fwd_binned(C.byref(cam), n, _ptr(workspace), _nbytes(workspace), _ptr(ranges),
                                      _ptr(vals), _ptr(splats), _bg(bg), _ptr(img), _ptr(T_final), _ptr(last),
                                      _ptr(n_contrib), _ptr(composited), _ptr(tile_order), _ptr(tile_cost),
                                      _stream(stream)))


def qn_tile_order(n_tiles, tile_cost, tile_order, stream=None):
    _check(lib().qn_tile_order(n_tiles, _ptr(tile_cost), _ptr(tile_order), _stream(stream)))


def _nbytes(t):
    return t.numel() * t.element_size()


def qn_render_bwd(cam, n, rects, ranges, vals, splats, bg, T_final, last, d_img, skip, composited, workspace,
                  pair_scratch, d_splats, stream=None, tile_order=None):
    _check(lib().qn_render_bwd(C.byref(cam), n, _ptr(rects), _ptr(ranges), _ptr(vals), _ptr(splats), _bg(bg),
                               _ptr(T_final), _ptr(last), _ptr(d_img), _ptr(skip), _ptr(composited),
                               _ptr(tile_order), _ptr(workspace), _nbytes(workspace), _ptr(pair_scratch),
                               _ptr(d_splats), _stream(stream)))


def qn_render_bwd_pairs(cam, n, ranges, vals, splats, bg, T_final, last, d_img, skip, composited, workspace,
                        pair_scratch, stream=None, tile_order=None):
    _check(lib().qn_render_bwd_pairs(C.byref(cam), n, _ptr(ranges), _ptr(vals), _ptr(splats), _bg(bg),
                                     _ptr(T_final), _ptr(last), _ptr(d_img), _ptr(skip), _ptr(composited),
                                     _ptr(tile_order), _ptr(workspace), _nbytes(workspace), _ptr(pair_scratch),
                                     _stream(stream)))


def qn_render_bwd_gather(cam, n, rects, skip, workspace, pair_scratch, d_splats, stream=None):
    _check(lib().qn_render_bwd_gather(C.byref(cam), n, _ptr(rects), _ptr(skip), _ptr(workspace),
                                      _nbytes(workspace), _ptr(pair_scratch), _ptr(d_splats), _stream(stream)))


QN_LOSS_BLOCKS = 2048
_loss_scratch = {}


def _loss_partials(dev):
    if dev not in _loss_scratch:
        _loss_scratch[dev] = torch.zeros(QN_LOSS_BLOCKS, device=dev)
    return _loss_scratch[dev]


def qn_image_loss(count, img, target, w, mse, loss, d_img, partials=None, stream=None):
    """partials: QN_LOSS_BLOCKS floats of scratch (one per device is kept here
    when not given)."""
    if partials is None:
        partials = _loss_partials(loss.device)
    _check(lib().qn_image_loss(count, _ptr(img), _ptr(target), float(w), int(mse), _ptr(loss), _ptr(d_img),
                               _ptr(partials), _stream(stream)))


def qn_adam(rows, n, stride, param, grad, m, v, step, lr, beta1, beta2, eps, skip=None, param_bf16=None,
            stream=None):
    _check(lib().qn_adam(rows, n, stride, _ptr(param), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr),
                         float(beta1), float(beta2), float(eps), _ptr(skip), _ptr(param_bf16), _stream(stream)))


def adam_group(param, grad, m, v, lr, rows, n, stride, param_bf16=None, use_skip=True):
    """One qn_adam_group over device tensors (views are fine: their data
    pointers are taken)."""
    return qn_adam_group(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), _ptr(param_bf16), int(rows), int(n), int(stride),
                         float(lr), int(bool(use_skip)))


def qn_adam_groups(groups, step, beta1, beta2, eps, skip=None, stream=None):
    """groups: a sequence of qn_adam_group, or a ctypes array of them."""
    if not isinstance(groups, C.Array):
        groups = (qn_adam_group * len(groups))(*groups)
    _check(lib().qn_adam_groups(len(groups), groups, _ptr(step), float(beta1), float(beta2), float(eps), _ptr(skip),
                                _stream(stream)))


def qn_viewspace_accum(n, n_stride, d_splats, scale, score, stream=None):
    _check(lib().qn_viewspace_accum(n, n_stride, _ptr(d_splats), float(scale), _ptr(score), _stream(stream)))


def qn_gate_init(n, n_stride, score, gate_params, norms, median, log_alpha, nonzero_median=True, stream=None):
    _check(lib().qn_gate_init(n, n_stride, _ptr(score), C.byref(gate_params), int(nonzero_median), _ptr(norms),
                              _ptr(median), _ptr(log_alpha), _stream(stream)))


QN_MLP_FEATURES = 16
QN_MLP_PARAMS = 5313


def qn_skip_features(n, n_stride, n_attr, score, median, prev, prev_gate, prev_log_alpha, prev_lp, gate_params,
                     X, prev_static=None, stream=None):
    _check(lib().qn_skip_features(n, n_stride, n_attr, _ptr(score), _ptr(median), _ptr(prev), _ptr(prev_gate),
                                  _ptr(prev_log_alpha), _ptr(prev_lp), _ptr(prev_static), C.byref(gate_params),
                                  _ptr(X), _stream(stream)))


def qn_skip_mlp_fwd(n, n_stride, X, params_bf16, threshold, logits=None, skip=None, stream=None):
    _check(lib().qn_skip_mlp_fwd(n, n_stride, _ptr(X), _ptr(params_bf16), float(threshold), _ptr(logits),
                                 _ptr(skip), _stream(stream)))


def qn_skip_mlp_bwd(n, n_stride, X, labels, params_bf16, d_params, loss, partials, stream=None):
    """partials: QN_MLP_BWD_BLOCKS * (QN_MLP_PARAMS + 1) floats of scratch."""
    _check(lib().qn_skip_mlp_bwd(n, n_stride, _ptr(X), _ptr(labels), _ptr(params_bf16), _ptr(d_params),
                                 _ptr(loss), _ptr(partials), _stream(stream)))


def qn_skip_labels(n, n_stride, n_latent, gate, lat, labels, stream=None, hit=None):
    _check(lib().qn_skip_labels(n, n_stride, n_latent, _ptr(gate), _ptr(lat), _ptr(hit), _ptr(labels),
                                _stream(stream)))


def qn_or_marks(n, src, dst, stream=None):
    _check(lib().qn_or_marks(n, _ptr(src), _ptr(dst), _stream(stream)))


def qn_partition_workspace_size(n):
    return int(lib().qn_partition_workspace_size(n))


def qn_partition(n, flags, perm, n_first, workspace, stream=None):
    ws_bytes = workspace.numel() * workspace.element_size()
    _check(lib().qn_partition(n, _ptr(flags), _ptr(perm), _ptr(n_first), _ptr(workspace), ws_bytes,
                              _stream(stream)))


def qn_gather_columns(rows, n, src, src_stride, perm, dst, dst_stride, stream=None):
    """dst[r][i] = src[r][perm[i]]; element size from src's dtype."""
    _check(lib().qn_gather_columns(rows, n, src.element_size(), _ptr(src), int(src_stride), _ptr(perm), _ptr(dst),
                                   int(dst_stride), _stream(stream)))


def qn_select_rects(n, n_stride, rects, score, ndc_x, ndc_y, t_d, rects_out, stream=None):
    _check(lib().qn_select_rects(n, n_stride, _ptr(rects), _ptr(score), float(ndc_x), float(ndc_y), float(t_d),
                                 _ptr(rects_out), _stream(stream)))


def qn_dilate_mask(width, height, last, k, tmp, pixel_mask, tile_mask, n_masked, stream=None):
    _check(lib().qn_dilate_mask(width, height, _ptr(last), int(k), _ptr(tmp), _ptr(pixel_mask), _ptr(tile_mask),
                                _ptr(n_masked), _stream(stream)))


def qn_mask_ranges(n_tiles, ranges, tile_mask, ranges_out, stream=None):
    _check(lib().qn_mask_ranges(n_tiles, _ptr(ranges), _ptr(tile_mask), _ptr(ranges_out), _stream(stream)))


def qn_masked_image_loss(hw, channels, img, target, pixel_mask, n_masked, w, mse, loss, d_img, stream=None):
    part = _loss_partials(img.device)
    _check(lib().qn_masked_image_loss(int(hw), int(channels), _ptr(img), _ptr(target), _ptr(pixel_mask),
                                      _ptr(n_masked), float(w), int(bool(mse)), _ptr(loss), _ptr(d_img), _ptr(part),
                                      _stream(stream)))


def qn_dssim_workspace_size(width, height, channels):
    return int(lib().qn_dssim_workspace_size(width, height, channels))


def qn_dssim_loss(width, height, channels, img, target, w, loss, d_img, workspace, pixel_mask=None, n_masked=None,
                  stream=None):
    """loss += w (1 - mean SSIM), d_img += w dD/dimg (Eq. 3's D-SSIM term)."""
    ws_bytes = workspace.numel() * workspace.element_size()
    _check(lib().qn_dssim_loss(width, height, channels, _ptr(img), _ptr(target), _ptr(pixel_mask), _ptr(n_masked),
                               float(w), _ptr(loss), _ptr(d_img), _ptr(workspace), ws_bytes, _stream(stream)))


def qn_pack_workspace_size(n, layout):
    return int(lib().qn_pack_workspace_size(n, C.byref(layout)))


def qn_packet_max_bytes(n, layout):
    return int(lib().qn_packet_max_bytes(n, C.byref(layout)))


def qn_pack_frame(n, n_stride, layout, lat, dec_bf16, lp, gate, workspace, packet, stream=None):
    """Writes the frame's packet into packet (device uint8); returns its size."""
    size = C.c_size_t(0)
    _check(lib().qn_pack_frame(n, n_stride, C.byref(layout), _ptr(lat), _ptr(dec_bf16), _ptr(lp), _ptr(gate),
                               _ptr(workspace), workspace.numel() * workspace.element_size(), _ptr(packet),
                               packet.numel(), C.byref(size), _stream(stream)))
    return int(size.value)


def qn_unpack_workspace_size(n, n_stride, layout, packet_bytes):
    return int(lib().qn_unpack_workspace_size(n, n_stride, C.byref(layout), packet_bytes))


def qn_unpack_frame(packet: bytes, n, n_stride, n_attr, layout, prev, out, workspace, stream=None):
    """A_t = prev + R_t from a packet held in host memory (bytes)."""
    buf = C.create_string_buffer(bytes(packet), len(packet))
    _check(lib().qn_unpack_frame(C.cast(buf, C.c_void_p), len(packet), n, n_stride, n_attr, C.byref(layout),
                                 _ptr(prev), _ptr(out), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                 _stream(stream)))


def qn_gate_uniform(n, seed, step, u, stream=None):
    """u[i] = Philox4x32-10 uniform of counter (i, *step) under seed."""
    _check(lib().qn_gate_uniform(n, int(seed) & ((1 << 64) - 1), _ptr(step), _ptr(u), _stream(stream)))


def qn_clear_marked(n, marks, flags, stream=None):
    _check(lib().qn_clear_marked(n, _ptr(marks), _ptr(flags), _stream(stream)))
