"""torch.autograd.Functions over the C ABI: decode + gate, projection, and
rasterisation (binning + compositing).  Forward and backward both run the
library's kernels; these classes only save tensors and marshal arguments.

    A_t, L_reg = DecodeGate.apply(prev, lat, dec_f32, lp, log_alpha, ctx_args)
    splat      = Project.apply(A_t, ctx_args)
    image      = Rasterize.apply(splat, ctx_args)

ctx_args are small holder objects (DecodeArgs, ProjectArgs, RasterArgs)
carrying the non-tensor arguments and preallocated buffers.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import binding as B
from .pipeline import Rasterizer


@dataclass
class DecodeArgs:
    n: int
    n_stride: int
    n_attr: int
    layout: object          # binding.qn_decoder_layout
    gate: object            # binding.qn_gate_params


class DecodeGate(torch.autograd.Function):
    """Eq. 4-8 forward; straight-through estimator and gate adjoint backward."""

    @staticmethod
    def forward(ctx, prev, lat, dec, lp, log_alpha, args: DecodeArgs):
        dec_bf16 = dec.detach().to(torch.bfloat16).contiguous()
        out = torch.empty_like(prev)
        lreg = torch.zeros(1, device=prev.device)
        B.qn_decode_residuals(args.n, args.n_stride, args.n_attr, prev, lat, dec_bf16, args.layout, lp, log_alpha,
                              args.gate, out, None, lreg)
        ctx.save_for_backward(lat, dec_bf16, lp, log_alpha)
        ctx.args = args
        ctx.dec_shape = dec.shape
        return out, lreg

    @staticmethod
    def backward(ctx, d_out, d_lreg):
        lat, dec_bf16, lp, log_alpha = ctx.saved_tensors
        a = ctx.args
        d_out = d_out.contiguous()
        dl = float(d_lreg.reshape(-1)[0]) if d_lreg is not None else 0.0
        d_lat = torch.zeros_like(lat)
        d_dec = torch.zeros(ctx.dec_shape, device=lat.device)
        d_lp = torch.zeros_like(lp)
        d_la = torch.zeros_like(log_alpha)
        partials = torch.zeros(B.QN_DECODE_BWD_BLOCKS * d_dec.numel(), device=lat.device)
        B.qn_decode_residuals_bwd(a.n, a.n_stride, a.n_attr, lat, dec_bf16, a.layout, lp, log_alpha, a.gate, d_out,
                                  dl, None, d_lat, d_dec, d_lp, d_la, partials)
        return None, d_lat, d_dec, d_lp, d_la, None


@dataclass
class RasterArgs:
    rast: Rasterizer
    cam: object             # binding.qn_camera
    blur: float = 0.3
    bg: tuple = (0.0, 0.0, 0.0)


class Project(torch.autograd.Function):
    """Eq. 1 + SH colour; returns the projected records [n][12]."""

    @staticmethod
    def forward(ctx, attrs, args: RasterArgs):
        r = args.rast
        r.project(attrs, args.cam, args.blur)
        ctx.save_for_backward(attrs)
        ctx.args = args
        return r.splats.clone()

    @staticmethod
    def backward(ctx, d_splat):
        (attrs,) = ctx.saved_tensors
        a = ctx.args
        r = a.rast
        d_attrs = torch.zeros_like(attrs)
        B.qn_project_bwd(r.n, r.S, r.sh_degree, attrs, a.cam, a.blur, d_splat.contiguous(), None, d_attrs)
        return d_attrs, None


class Rasterize(torch.autograd.Function):
    """Binning + Eq. 2; saves only the final transmittance and the last
    contributor per pixel, and the adjoint recomputes alpha."""

    @staticmethod
    def forward(ctx, splat, args: RasterArgs):
        r = args.rast
        if splat.data_ptr() != r.splats.data_ptr():
            r.splats.copy_(splat)
        try:
            r.bin_sort(sync=True)
        except B.QueenError as e:
            if e.code != B.QN_ERR_CAPACITY:
                raise
            r.set_capacity(int(int(r.n_pairs.item()) * 1.25) + 1024)
            r.bin_sort(sync=True)
        r.render_fwd(args.cam, args.bg)
        ctx.args = args
        ctx.save_for_backward(splat)
        return r.img.clone()

    @staticmethod
    def backward(ctx, d_img):
        a = ctx.args
        r = a.rast
        r.d_img.copy_(d_img)
        r.render_bwd(a.cam, a.bg)
        return r.d_splats.clone(), None
