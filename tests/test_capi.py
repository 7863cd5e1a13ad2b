"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point declared in include/queen.h, and host-side argument validation
returns the documented status codes before any device work."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "queen.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qn_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2412_04469_gb300 import build
    path = build.build()
    from paper_2412_04469_gb300 import binding
    return binding.lib(), C.CDLL(path)


def test_exports_every_declared_symbol(lib):
    _, raw = lib
    names = _declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(raw, name), name


def test_binding_covers_header(lib):
    from paper_2412_04469_gb300 import binding
    assert set(_declared()) <= set(binding.exported_symbols())


def test_version_and_error_string(lib):
    L, _ = lib
    assert b"sm_103a" in L.qn_version()


def test_invalid_arguments_fail_before_any_launch(lib):
    from paper_2412_04469_gb300 import binding as B
    cam = B.qn_camera()
    cam.width, cam.height, cam.fx, cam.fy, cam.near_plane = 64, 64, 50.0, 50.0, 0.2
    assert B.lib().qn_project(-1, 4, 0, None, C.byref(cam), 0.3, 1, None, None, None) == B.QN_ERR_INVALID_ARG
    assert b"n_stride" in B.lib().qn_last_error() or b"n" in B.lib().qn_last_error()
    assert B.lib().qn_project(8, 8, 4, None, C.byref(cam), 0.3, 1, None, None, None) == B.QN_ERR_INVALID_ARG
    assert b"sh_degree" in B.lib().qn_last_error()
    bad = B.qn_camera()
    bad.width, bad.height = 0, 64
    assert B.lib().qn_project(8, 8, 0, None, C.byref(bad), 0.3, 1, None, None, None) == B.QN_ERR_INVALID_ARG
    assert B.lib().qn_bin_sort(4, None, 1, None, 300, 2, None, 0, 0, None, None, None, None, None, None) == \
        B.QN_ERR_INVALID_ARG
    lay = B.qn_decoder_layout()
    lay.n_cat = 1
    lay.attr_begin[0], lay.attr_count[0], lay.lat_dim[0] = 1, 2, 4      # overlaps the position planes
    gp = B.make_gate(0.3, -0.5, 1.01)
    assert B.lib().qn_decode_residuals(4, 4, 14, None, None, None, C.byref(lay), None, None, C.byref(gp),
                                       None, None, None, None, None) == B.QN_ERR_INVALID_ARG
    assert b"category" in B.lib().qn_last_error()
    assert B.lib().qn_render_bwd(None, 0, None, None, None, None, None, None, None, None, None, None, None, None, 0,
                                 None, None, None) == B.QN_ERR_INVALID_ARG
    assert B.lib().qn_render_bwd(C.byref(cam), 4, 16, 16, 16, 32, None, 64, 128, 256, None, None, None, 512, 0,
                                 1024, 2048, None) == B.QN_ERR_INVALID_ARG
    assert b"workspace too small" in B.lib().qn_last_error()
    assert B.lib().qn_render_bwd_gather(C.byref(cam), 4, 16, None, 256, 1 << 20, 1024, 40, None) == \
        B.QN_ERR_INVALID_ARG
    assert b"misaligned" in B.lib().qn_last_error()
    assert B.lib().qn_tile_order(-1, None, None, None) == B.QN_ERR_INVALID_ARG
    assert B.lib().qn_tile_order(4, None, 16, None) == B.QN_ERR_INVALID_ARG
    bg = (C.c_float * 3)()
    assert B.lib().qn_render_fwd(C.byref(cam), 16, None, 32, bg, 64, 128, 256, None, None, None, None, None) == \
        B.QN_ERR_INVALID_ARG
    assert b"vals" in B.lib().qn_last_error()                                        # sorted pair values missing
    assert B.lib().qn_render_fwd(C.byref(cam), 16, 16, 40, bg, 64, 128, 256, None, None, None, None, None) == \
        B.QN_ERR_INVALID_ARG
    assert b"aligned" in B.lib().qn_last_error()                                     # splats misaligned
    assert B.lib().qn_bin_sort(4, 16, 1, 32, 4, 4, 256, 16, 1 << 40, 64, None, 128, 256, None, None) == \
        B.QN_ERR_INVALID_ARG                                                          # workspace too small
    assert b"workspace too small" in B.lib().qn_last_error()
    assert B.lib().qn_bin_sort_partial(4, 16, 1, 32, 4, 4, 256, 1 << 20, 64, 2048, None, 128, 256, None, None) == \
        B.QN_ERR_INVALID_ARG                                                          # vals is the output
    assert b"vals is required" in B.lib().qn_last_error()
    assert B.lib().qn_bin_sort_partial(4, 16, 1, 32, 4, 4, 256, 16, 64, 0, 64, 128, 256, None, None) == \
        B.QN_ERR_INVALID_ARG                                                          # workspace too small
    assert b"workspace too small" in B.lib().qn_last_error()
    for ws, nb, what in ((None, 0, b"workspace is required"), (264, 1 << 20, b"256-byte aligned"),
                         (256, 16, b"too small")):
        assert B.lib().qn_render_fwd_binned(C.byref(cam), 4, ws, nb, 16, 16, 32, bg, 64, 128, 256, None, None,
                                            None, None, None) == B.QN_ERR_INVALID_ARG
        assert what in B.lib().qn_last_error()
    gp_bad = B.make_gate(0.3, 0.5, 1.01)
    lay.attr_begin[0] = 3
    assert B.lib().qn_decode_residuals(4, 4, 14, None, None, None, C.byref(lay), None, None, C.byref(gp_bad),
                                       None, None, None, None, None) == B.QN_ERR_INVALID_ARG
    gp = B.make_gate(0.3, -0.5, 1.01)
    assert B.lib().qn_decode_project(4, 4, 14, 1, 16, 16, 16, C.byref(lay), 16, 16, C.byref(gp), None,
                                     C.byref(cam), 0.3, 1, None, None, 64, 48, 96, None) == B.QN_ERR_INVALID_ARG
    assert b"sh_degree" in B.lib().qn_last_error()                                   # 14 planes are degree 0
    assert B.lib().qn_decode_project(4, 4, 14, 0, 16, 16, 16, C.byref(lay), 16, 16, C.byref(gp), None,
                                     C.byref(cam), 0.3, 1, None, None, 64, 40, 96, None) == B.QN_ERR_INVALID_ARG
    assert b"aligned" in B.lib().qn_last_error()                                     # splats misaligned
    assert B.lib().qn_decode_project(4, 4, 14, 0, 16, 16, 16, C.byref(lay), 16, 16, C.byref(gp), None,
                                     C.byref(cam), 0.3, 1, None, None, 16, 48, 96, None) == B.QN_ERR_INVALID_ARG
    assert b"alias" in B.lib().qn_last_error()                                       # out aliases prev
    assert B.lib().qn_adam(1, 4, 4, None, None, None, None, 0, 0.1, 0.9, 0.999, 1e-8, None, None, None) == \
        B.QN_ERR_INVALID_ARG
    assert B.lib().qn_bin_sort_workspace_size(-1, 4, 4) == 0
    groups = (B.qn_adam_group * 1)()
    assert B.lib().qn_adam_groups(0, groups, None, 0.9, 0.999, 1e-8, None, None) == B.QN_ERR_INVALID_ARG
    assert B.lib().qn_adam_groups(B.QN_ADAM_MAX_GROUPS + 1, groups, None, 0.9, 0.999, 1e-8, None, None) == \
        B.QN_ERR_INVALID_ARG
    groups[0].rows, groups[0].n, groups[0].stride = 1, 8, 4                  # stride < n
    assert B.lib().qn_adam_groups(1, groups, 16, 0.9, 0.999, 1e-8, None, None) == B.QN_ERR_INVALID_ARG
    assert b"stride" in B.lib().qn_last_error()
    assert B.lib().qn_partition_workspace_size(-1) == 0
    assert B.lib().qn_partition_workspace_size(2049) == 4 * 4
    assert B.lib().qn_partition(-1, None, None, None, None, 0, None) == B.QN_ERR_INVALID_ARG
    assert B.lib().qn_partition(10, 16, 16, 16, 16, 4, None) == B.QN_ERR_INVALID_ARG      # workspace too small
    assert b"workspace" in B.lib().qn_last_error()
    assert B.lib().qn_gather_columns(1, 4, 3, 16, 4, 16, 32, 4, None) == B.QN_ERR_INVALID_ARG   # elem_bytes
    assert B.lib().qn_gather_columns(1, 4, 4, 16, 4, 16, 16, 4, None) == B.QN_ERR_INVALID_ARG   # aliasing
    assert B.lib().qn_dilate_mask(64, 64, 16, 47, 16, 16, 16, 16, None) == B.QN_ERR_INVALID_ARG     # odd k
    assert b"k must be even" in B.lib().qn_last_error()
    assert B.lib().qn_dilate_mask(0, 64, 16, 48, 16, 16, 16, 16, None) == B.QN_ERR_INVALID_ARG
    assert B.lib().qn_mask_ranges(4, 16, 32, 16, None) == B.QN_ERR_INVALID_ARG                      # aliasing
    assert B.lib().qn_select_rects(4, 4, 8, 32, 1.0, 1.0, 0.001, 48, None) == B.QN_ERR_INVALID_ARG  # misaligned
    assert B.lib().qn_select_rects(4, 2, 16, 32, 1.0, 1.0, 0.001, 48, None) == B.QN_ERR_INVALID_ARG  # stride < n
    assert B.lib().qn_select_rects(4, 4, 16, 32, 1.0, 1.0, -1.0, 48, None) == B.QN_ERR_INVALID_ARG   # t_d < 0
    assert B.lib().qn_masked_image_loss(16, 0, None, None, None, None, 1.0, 0, None, None, None, None) == \
        B.QN_ERR_INVALID_ARG
    assert B.lib().qn_pack_workspace_size(10, None) == 0 and B.lib().qn_packet_max_bytes(-1, None) == 0
    assert B.lib().qn_pack_frame(10, 12, None, 16, 16, 16, 16, 256, 1 << 20, 16, 64, 16, None) == \
        B.QN_ERR_INVALID_ARG                                                                          # no layout
    assert B.lib().qn_unpack_frame(None, 0, 10, 12, 59, None, 16, 16, 256, 1 << 20, None) == B.QN_ERR_INVALID_ARG
    assert B.lib().qn_dssim_workspace_size(0, 8, 3) == 0
    ws = B.lib().qn_dssim_workspace_size(40, 20, 3)
    assert ws >= 3 * 3 * 40 * 20 * 4
    assert B.lib().qn_dssim_loss(40, 20, 0, 16, 32, None, None, 0.2, 48, 64, 128, ws, None) == B.QN_ERR_INVALID_ARG
    assert B.lib().qn_dssim_loss(40, 20, 3, 16, 32, None, None, 0.2, 48, 64, 128, ws - 4, None) == \
        B.QN_ERR_INVALID_ARG                                                                          # workspace
    assert b"workspace too small" in B.lib().qn_last_error()
    assert B.lib().qn_dssim_loss(40, 20, 3, 16, 32, 80, None, 0.2, 48, 64, 128, ws, None) == \
        B.QN_ERR_INVALID_ARG                                                                          # mask, no count
    assert B.lib().qn_dssim_loss(40, 20, 3, 16, 32, None, None, 0.2, 48, 16, 128, ws, None) == \
        B.QN_ERR_INVALID_ARG                                                                          # aliasing
    assert B.lib().qn_dssim_loss(40, 20, 3, 16, 32, None, None, 0.2, 48, 64, 136, ws, None) == \
        B.QN_ERR_INVALID_ARG                                                                          # misaligned
