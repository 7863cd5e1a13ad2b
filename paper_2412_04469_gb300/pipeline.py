"""Device-resident buffers and the per-view training iteration of QUEEN's
residual training (Sec. 3.2-3.4), every step a C-ABI call:

  decode+gate -> project -> bin/sort -> composite -> loss -> composite adjoint
  -> projection adjoint -> decode/gate adjoint -> Adam

PyTorch only allocates device memory and provides the stream.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import binding as B
from .synthetic import DecoderLayout, n_attr as n_attr_of, bf16_bits

TILE = B.QN_TILE
MASK_T_D = 0.001          # Sec. 3.3 threshold on |d_t| (App. B)
MASK_KERNEL = 48          # dilation of the mask (App. B)


def _stride(n: int) -> int:
    return max(4, (n + 31) // 32 * 32)


@dataclass
class HParams:
    """Hyper-parameters, N3DV rows of the paper's tables (App. B)."""
    tau: float = 0.3
    gamma0: float = -0.5
    gamma1: float = 1.01
    lambda_reg: float = 0.01
    # weight of the D-SSIM term of Eq. 3 (L = (1 - lambda) L1 + lambda D-SSIM);
    # the paper does not give it: 0.2, the value of the 3D-GS training it builds on
    lambda_dssim: float = 0.2
    # the stochastic hard-concrete sample (noise on log alpha) during training
    # iterations instead of Eq. 6's deterministic gate; decodes outside
    # training (A_t, the packet) keep Eq. 6
    gate_noise: bool = False
    gate_seed: int = 0
    # Eq. 11 weights Eq. 8's sum by lambda_reg / n (the penalty averaged over
    # Gaussians): with the L1 term a per-pixel mean, the plain sum closes every
    # gate within a frame, unlike the few percent of open gates the paper reports.
    lreg_mean: bool = True
    lr_gate: float = 0.1
    lr_pos: float = 0.00016
    # per decoder category (rotation, scale, opacity, colour)
    lr_latent: tuple = (0.025, 0.01, 0.05, 0.0125)
    lr_decoder: tuple = (1e-3, 1e-4, 1e-4, 1e-3)
    blur: float = 0.3
    bg: tuple = (0.0, 0.0, 0.0)
    # the forward marks the Gaussians some pixel composites and the adjoint
    # drops the others from its per-tile walk (the same result; the marks
    # cost the forward about what they save the adjoint, so plain training
    # leaves them off and the learned skip, which needs them, turns them on)
    mark_composited: bool = False
    # the compositing kernels start their tiles heaviest first (by the
    # per-tile visited prefixes of the last forward; the same result)
    order_tiles: bool = True
    # the training iteration decodes and projects in one pass (a skipped
    # Gaussian is then rendered with the current decoders)
    fused: bool = True
    # with fused, the projection and decode adjoints can also run in one
    # pass that rebuilds A_t in shared memory, so A_t is never written (d_dec
    # is then summed in another order).  Off: at 300k Gaussians it measured
    # 0.129 ms against 0.105 ms for the two kernels (its ~800 bytes of shared
    # memory per Gaussian leave ~8 warps per SM for a long serial chain)
    fused_bwd: bool = False
    # the binning writes only the tile lists of at most list_max pairs; the
    # compositing forward forms each longer list from the binning's chunk
    # masks as it goes, writing only the prefix it walks (~1 M of the 21.8 M
    # pairs of a 300k-Gaussian view); the same result.  Writing the short
    # lists in the binning measured slower (list_max 1024 / 2048 / 4096:
    # 0.949 / 0.957 / 0.966 ms a step against 0.929 for none)
    lazy_lists: bool = True
    list_max: int = 0
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15


def n3dv_hparams() -> HParams:
    """HParams for DecoderLayout.paper_n3dv: the latent learning rates of the
    paper's quantisation table for N3DV (rotation, scale, opacity, colour
    base, colour frequency) and App. B's decoder rates (1e-3 for colour and
    rotation, 1e-4 for opacity and scale)."""
    return HParams(lr_latent=(0.025, 0.01, 0.05, 0.0125, 0.000625), lr_decoder=(1e-3, 1e-4, 1e-4, 1e-3, 1e-3))


class _Adam:
    def __init__(self, shape, dev):
        self.m = torch.zeros(shape, device=dev, dtype=torch.float32)
        self.v = torch.zeros(shape, device=dev, dtype=torch.float32)


class QueenFrame:
    """One time-step's trainable residuals on top of the fixed A_{t-1}."""

    def __init__(self, prev: np.ndarray, sh_degree: int, layout: DecoderLayout, lat: np.ndarray, dec: np.ndarray,
                 lp: np.ndarray, log_alpha: np.ndarray, hp: HParams | None = None, device="cuda"):
        self.dev = torch.device(device)
        self.hp = hp or HParams()
        self.sh_degree = sh_degree
        self.layout = layout
        self.n = n = prev.shape[1]
        self.n_attr = n_attr_of(sh_degree)
        assert prev.shape[0] == self.n_attr
        self.S = S = _stride(n)
        dev = self.dev

        def planes(a, rows):
            t = torch.zeros((rows, S), device=dev, dtype=torch.float32)
            if n:
                t[:, :n] = torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev)
            return t

        self.prev = planes(prev, self.n_attr)
        self.lat = planes(lat, layout.n_latent)
        self.lp = planes(lp, 3)
        self.log_alpha = torch.zeros(S, device=dev, dtype=torch.float32)
        self.log_alpha[:n] = torch.from_numpy(np.ascontiguousarray(log_alpha, np.float32)).to(dev)
        self.dec = torch.from_numpy(np.ascontiguousarray(dec, np.float32)).to(dev)
        self.dec_bf16 = torch.from_numpy(bf16_bits(dec).view(np.int16)).to(dev).view(torch.bfloat16)
        self.c_layout = B.make_layout(layout)
        self.c_gate = B.make_gate(self.hp.tau, self.hp.gamma0, self.hp.gamma1)
        self.noise = torch.zeros(S, device=dev) if self.hp.gate_noise else None
        self.c_gate_train = (B.make_gate(self.hp.tau, self.hp.gamma0, self.hp.gamma1, self.noise)
                             if self.hp.gate_noise else self.c_gate)
        # outputs and gradients
        self.attrs = torch.zeros((self.n_attr, S), device=dev)
        self.gate = torch.zeros(S, device=dev)
        self.lreg = torch.zeros(1, device=dev)
        self.d_attrs = torch.zeros((self.n_attr, S), device=dev)
        self.d_lat = torch.zeros_like(self.lat)
        self.d_dec = torch.zeros_like(self.dec)
        self.d_lp = torch.zeros_like(self.lp)
        self.d_log_alpha = torch.zeros_like(self.log_alpha)
        self.dec_partials = torch.zeros(B.QN_DECODE_BWD_BLOCKS * max(1, layout.n_dec), device=dev)
        self.opt = {k: _Adam(getattr(self, k).shape, dev) for k in ("lat", "dec", "lp", "log_alpha")}
        self.step = torch.zeros(1, device=dev, dtype=torch.int32)     # Adam step count, on the device
        self._adam_groups = self._make_adam_groups()

    def _make_adam_groups(self):
        """Every trainable tensor as qn_adam groups: latents and decoders per
        category (each its own learning rate), position residuals and gate
        parameters; the decoders also refresh their bf16 copy."""
        hp, n, S, lay = self.hp, self.n, self.S, self.layout
        groups = []
        lo, dofs = 0, 0
        o = self.opt["lat"]
        for c in range(lay.n_cat):
            L = lay.lat_dim[c]
            groups.append(B.adam_group(self.lat[lo:lo + L], self.d_lat[lo:lo + L], o.m[lo:lo + L], o.v[lo:lo + L],
                                       hp.lr_latent[min(c, len(hp.lr_latent) - 1)], L, n, S))
            lo += L
        o = self.opt["dec"]
        for c in range(lay.n_cat):
            k = lay.attr_count[c] * lay.lat_dim[c]
            groups.append(B.adam_group(self.dec[dofs:dofs + k], self.d_dec[dofs:dofs + k], o.m[dofs:dofs + k],
                                       o.v[dofs:dofs + k], hp.lr_decoder[min(c, len(hp.lr_decoder) - 1)], 1, k, k,
                                       param_bf16=self.dec_bf16[dofs:dofs + k], use_skip=False))
            dofs += k
        o = self.opt["lp"]
        groups.append(B.adam_group(self.lp, self.d_lp, o.m, o.v, hp.lr_pos, 3, n, S))
        o = self.opt["log_alpha"]
        groups.append(B.adam_group(self.log_alpha, self.d_log_alpha, o.m, o.v, hp.lr_gate, 1, n, S))
        return (B.qn_adam_group * len(groups))(*groups)

    def reset_optimizer(self):
        """Clears Adam's moments and step count (device work, no sync)."""
        for o in self.opt.values():
            o.m.zero_()
            o.v.zero_()
        self.step.zero_()

    # ---------------------------------------------------------------- steps
    def decode(self, stream=None, skip=None, train=False):
        """A_t from A_{t-1} and the residuals; Gaussians with skip set are
        frozen and keep their columns of attrs and gate.  train: the
        iteration's gate (with HParams.gate_noise, fresh noise drawn for the
        current Adam step first)."""
        gate = self.c_gate
        if train and self.noise is not None:
            B.qn_gate_uniform(self.n, self.hp.gate_seed, self.step, self.noise, stream)
            gate = self.c_gate_train
        B.qn_decode_residuals(self.n, self.S, self.n_attr, self.prev, self.lat, self.dec_bf16, self.c_layout,
                              self.lp, self.log_alpha, gate, self.attrs, self.gate, self.lreg, stream, skip)

    def pack(self, stream=None) -> bytes:
        """The frame's compressed packet (App. B storage; layout in the C
        header): entropy-coded integer latents, bf16 decoders, COO position
        residuals of the Gaussians whose gate is on.  Reads the gate of the
        last decode."""
        if getattr(self, "_pack_ws", None) is None:
            self._pack_ws = torch.zeros(max(B.qn_pack_workspace_size(self.n, self.c_layout), 256), device=self.dev,
                                        dtype=torch.uint8)
            self._packet = torch.zeros(B.qn_packet_max_bytes(self.n, self.c_layout), device=self.dev,
                                       dtype=torch.uint8)
        size = B.qn_pack_frame(self.n, self.S, self.c_layout, self.lat, self.dec_bf16, self.lp, self.gate,
                               self._pack_ws, self._packet, stream)
        return bytes(self._packet[:size].cpu().numpy().tobytes())

    def unpack(self, packet: bytes, out, stream=None):
        """out = A_{t-1} + R_t decoded from a packet (what a receiver holding
        A_{t-1} reconstructs)."""
        need = B.qn_unpack_workspace_size(self.n, self.S, self.c_layout, len(packet))
        ws = getattr(self, "_unpack_ws", None)
        if ws is None or ws.numel() < need:
            ws = self._unpack_ws = torch.zeros(need, device=self.dev, dtype=torch.uint8)
        B.qn_unpack_frame(packet, self.n, self.S, self.n_attr, self.c_layout, self.prev, out, ws, stream)

    @property
    def d_lreg(self) -> float:
        """dL_total / dL_reg of Eq. 11."""
        return self.hp.lambda_reg / max(1, self.n) if self.hp.lreg_mean else self.hp.lambda_reg

    def _train_gate(self, stream=None):
        """The gate parameters of a training iteration (with HParams.gate_noise,
        fresh noise drawn for the current Adam step first)."""
        if self.noise is not None:
            B.qn_gate_uniform(self.n, self.hp.gate_seed, self.step, self.noise, stream)
            return self.c_gate_train
        return self.c_gate

    def decode_project(self, rast: "Rasterizer", cam, stream=None, skip=None, keep_attrs: bool = True):
        """A training iteration's decode (Eq. 4-8) and projection (Eq. 1) in
        one pass into rast's records and rects, A_t into attrs (for the
        projection adjoint) unless keep_attrs is False.  Gaussians with skip
        set keep their gate entries and add nothing to lreg; their A_t is
        rebuilt from the current decoders like every other."""
        B.qn_decode_project(self.n, self.S, self.n_attr, self.sh_degree, self.prev, self.lat, self.dec_bf16,
                            self.c_layout, self.lp, self.log_alpha, self._train_gate(stream), skip, cam,
                            self.hp.blur, rast.tight_rects, self.gate, self.lreg,
                            self.attrs if keep_attrs else None, rast.splats, rast.rects, stream)

    def decode_project_bwd(self, rast: "Rasterizer", cam, skip=None, stream=None):
        """The projection adjoint (from rast.d_splats) and the decode adjoint
        in one pass, A_t rebuilt from prev and the residuals as
        decode_project forms it (the iteration's gate noise included)."""
        B.qn_decode_project_bwd(self.n, self.S, self.n_attr, self.sh_degree, self.prev, self.lat, self.dec_bf16,
                                self.c_layout, self.lp, self.log_alpha, self.c_gate_train, skip, cam, self.hp.blur,
                                rast.d_splats, self.d_lreg, self.d_lat, self.d_dec, self.d_lp, self.d_log_alpha,
                                self.dec_partials, stream)

    def decode_bwd(self, skip=None, stream=None):
        B.qn_decode_residuals_bwd(self.n, self.S, self.n_attr, self.lat, self.dec_bf16, self.c_layout, self.lp,
                                  self.log_alpha, self.c_gate_train, self.d_attrs, self.d_lreg, skip, self.d_lat,
                                  self.d_dec, self.d_lp, self.d_log_alpha, self.dec_partials, stream)

    def adam(self, skip=None, stream=None):
        """One Adam step on every trainable tensor: a single launch (after
        the device step counter's increment)."""
        hp = self.hp
        B.qn_adam_groups(self._adam_groups, self.step, hp.beta1, hp.beta2, hp.eps, skip, stream)


class Rasterizer:
    """Projection, binning and compositing buffers for n Gaussians on one
    image size."""

    def __init__(self, n: int, n_stride: int, sh_degree: int, width: int, height: int, pair_capacity: int,
                 device="cuda", keep_keys: bool = False, tight_rects: bool = True):
        dev = torch.device(device)
        self.tight_rects = tight_rects
        self.n, self.S, self.sh_degree = n, n_stride, sh_degree
        self.W, self.H = width, height
        self.TX, self.TY = (width + TILE - 1) // TILE, (height + TILE - 1) // TILE
        nn = max(n, 1)
        self.splats = torch.zeros((nn, 12), device=dev)
        self.rects = torch.zeros((nn, 4), device=dev, dtype=torch.int32)
        self.d_splats = torch.zeros((nn, 12), device=dev)
        ws = B.qn_bin_sort_workspace_size(n, self.TX, self.TY)
        self.workspace = torch.zeros(max(ws, 256), device=dev, dtype=torch.uint8)
        self.ranges = torch.zeros((self.TX * self.TY, 2), device=dev, dtype=torch.int32)
        self.n_pairs = torch.zeros(1, device=dev, dtype=torch.int64)
        self.ranges_masked = torch.zeros_like(self.ranges)         # masked iterations: inactive tiles emptied
        self.rects_sel = torch.zeros_like(self.rects)              # mask building: dynamic Gaussians' rects
        self.mask_tmp = torch.zeros((height, width), device=dev, dtype=torch.uint8)
        self.composited = torch.zeros(nn, device=dev, dtype=torch.uint8)     # Gaussians some pixel composited
        # tiles by descending work: written after each forward from its
        # per-tile visited prefix (tile_cost), read by the adjoint of the same
        # iteration and the forward of the next (neighbouring views cost alike)
        self.tile_cost = torch.zeros(self.TX * self.TY, device=dev, dtype=torch.int32)
        self.tile_order = torch.arange(self.TX * self.TY, device=dev, dtype=torch.int32)
        self.keep_keys = keep_keys
        self.lazy = False                                          # the last bin_sort left the lists unwritten
        # tile_order is refreshed on a side stream while the loss runs; the
        # next reader of tile_order waits for it
        self._order_stream = None
        self._order_pending = False
        self.set_capacity(pair_capacity)
        self.img = torch.zeros((3, height, width), device=dev)
        self.T_final = torch.zeros((height, width), device=dev)
        self.last = torch.zeros((height, width), device=dev, dtype=torch.int32)
        self.d_img = torch.zeros((3, height, width), device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.dssim_ws = torch.zeros(B.qn_dssim_workspace_size(width, height, 3), device=dev, dtype=torch.uint8)

    def set_capacity(self, cap: int):
        dev = self.splats.device
        self.capacity = int(cap)
        self.vals = torch.zeros(max(self.capacity, 1), device=dev, dtype=torch.int32)
        self.pair_grads = torch.zeros((max(self.capacity, 1), 12), device=dev)
        self.keys = torch.zeros(max(self.capacity, 1), device=dev, dtype=torch.int64) if self.keep_keys else None

    def project(self, attrs, cam, blur, stream=None):
        B.qn_project(self.n, self.S, self.sh_degree, attrs, cam, blur, self.splats, self.rects, self.tight_rects,
                     stream)

    def bin_sort(self, sync=False, stream=None, rects=None, lazy=False, list_max=0):
        """With lazy, only the tile lists of at most list_max pairs are
        written: the next render_fwd forms the others from the binning
        workspace and writes the part of each it walks (all the adjoint
        reads); the keys are then not written either."""
        depth_ptr = self.splats.data_ptr() + 3 * 4
        rc = self.rects if rects is None else rects
        self.lazy = bool(lazy)
        if lazy:
            return B.qn_bin_sort_partial(self.n, depth_ptr, 12, rc, self.TX, self.TY, self.workspace, self.capacity,
                                         list_max, self.vals, self.ranges, self.n_pairs, sync, stream)
        return B.qn_bin_sort(self.n, depth_ptr, 12, rc, self.TX, self.TY, self.workspace, self.capacity,
                             self.vals, self.keys, self.ranges, self.n_pairs, sync, stream)

    @staticmethod
    def _torch_stream(stream):
        if stream is None:
            return torch.cuda.current_stream()
        return torch.cuda.ExternalStream(stream) if isinstance(stream, int) else stream

    def _join_order(self, stream):
        """The stream waits for the last tile_order refresh (on the side stream)."""
        if self._order_pending:
            self._torch_stream(stream).wait_event(self._order_done)
            self._order_pending = False

    def render_fwd(self, cam, bg, n_contrib=None, stream=None, ranges=None, mark=False, order=False):
        """Compositing; with mark, `composited` holds afterwards the Gaussians
        some pixel composited; with order, the tiles start heaviest first (by
        the previous ordered forward's costs) and tile_order is refreshed from
        this forward's costs -- on a side stream, forked from `stream` here and
        joined by the next call that reads tile_order (render_fwd,
        render_bwd, render_bwd_pairs), so that it overlaps the loss."""
        self._join_order(stream)
        if mark:
            self.composited.zero_()
        rg = self.ranges if ranges is None else ranges
        if self.lazy:
            B.qn_render_fwd_binned(cam, self.n, self.workspace, rg, self.vals, self.splats, bg, self.img,
                                   self.T_final, self.last, n_contrib, stream,
                                   composited=self.composited if mark else None,
                                   tile_order=self.tile_order if order else None,
                                   tile_cost=self.tile_cost if order else None)
        else:
            B.qn_render_fwd(cam, rg, self.vals, self.splats, bg, self.img, self.T_final, self.last, n_contrib,
                            stream, composited=self.composited if mark else None,
                            tile_order=self.tile_order if order else None,
                            tile_cost=self.tile_cost if order else None)
        if order:
            main = self._torch_stream(stream)
            if self._order_stream is None:
                self._order_stream = torch.cuda.Stream(device=self.splats.device)
                self._order_fork, self._order_done = torch.cuda.Event(), torch.cuda.Event()
            self._order_fork.record(main)
            self._order_stream.wait_event(self._order_fork)
            B.qn_tile_order(self.TX * self.TY, self.tile_cost, self.tile_order, self._order_stream)
            self._order_done.record(self._order_stream)
            self._order_pending = True

    def loss_grad(self, target, w=1.0, mse=False, stream=None):
        B.qn_image_loss(self.img.numel(), self.img, target, w, mse, self.loss, self.d_img, stream)

    def dssim_grad(self, target, w, mask: "ViewMask | None" = None, stream=None):
        """Adds w D-SSIM (Eq. 3) to the loss and its gradient to d_img; with a
        mask, over the masked pixels."""
        B.qn_dssim_loss(self.W, self.H, 3, self.img, target, w, self.loss, self.d_img, self.dssim_ws,
                        None if mask is None else mask.pixel, None if mask is None else mask.count, stream)

    def photometric_loss(self, target, lambda_dssim, mask: "ViewMask | None" = None, stream=None):
        """Eq. 3: (1 - lambda) L1 + lambda D-SSIM, into loss and d_img (both
        over the masked pixels when a mask is given)."""
        if mask is None:
            self.loss_grad(target, 1.0 - lambda_dssim, False, stream)
        else:
            self.masked_loss_grad(target, mask, 1.0 - lambda_dssim, False, stream)
        if lambda_dssim > 0:
            self.dssim_grad(target, lambda_dssim, mask, stream)

    def render_bwd(self, cam, bg, skip=None, stream=None, ranges=None, marks=False, order=False):
        """Compositing adjoint into d_splats; with marks, the adjoint drops the
        Gaussians the last marked forward did not composite; with order, the
        tiles start in tile_order."""
        self._join_order(stream)
        B.qn_render_bwd(cam, self.n, self.rects, self.ranges if ranges is None else ranges, self.vals, self.splats,
                        bg, self.T_final, self.last, self.d_img, skip, self.composited if marks else None,
                        self.workspace, self.pair_grads, self.d_splats, stream,
                        tile_order=self.tile_order if order else None)

    def render_bwd_pairs(self, cam, bg, skip=None, stream=None, ranges=None, marks=False, order=False):
        """First pass of render_bwd (per-pair records)."""
        self._join_order(stream)
        B.qn_render_bwd_pairs(cam, self.n, self.ranges if ranges is None else ranges, self.vals, self.splats, bg,
                              self.T_final, self.last, self.d_img, skip, self.composited if marks else None,
                              self.workspace, self.pair_grads, stream, tile_order=self.tile_order if order else None)

    def gather(self, cam, skip=None, stream=None):
        """Second pass of render_bwd (per-Gaussian sums)."""
        B.qn_render_bwd_gather(cam, self.n, self.rects, skip, self.workspace, self.pair_grads, self.d_splats, stream)

    def project_bwd(self, attrs, cam, blur, d_attrs, skip=None, stream=None):
        B.qn_project_bwd(self.n, self.S, self.sh_degree, attrs, cam, blur, self.d_splats, skip, d_attrs, stream)

    # ------------------------------------------------------------ masked training
    def build_mask(self, attrs, cam, blur, score, vm: "ViewMask", t_d=MASK_T_D, k=MASK_KERNEL, bg=(0.0, 0.0, 0.0),
                   stream=None):
        """Sec. 3.3's mask of one view: the dynamic Gaussians (|d_t| > t_d,
        d_t = score [2][S] in pixel units, compared in normalised device
        coordinates) rendered alone, their pixels dilated with a k x k box,
        the tiles holding a masked pixel marked.  Overwrites the rasterizer's
        projection, binning and image buffers."""
        self.project(attrs, cam, blur, stream)
        B.qn_select_rects(self.n, self.S, self.rects, score, self.W / 2.0, self.H / 2.0, t_d, self.rects_sel, stream)
        self.bin_sort(False, stream, rects=self.rects_sel)
        self.render_fwd(cam, bg, stream=stream)
        B.qn_dilate_mask(self.W, self.H, self.last, k, self.mask_tmp, vm.pixel, vm.tiles, vm.count, stream)

    def mask_ranges(self, vm: "ViewMask", stream=None):
        B.qn_mask_ranges(self.TX * self.TY, self.ranges, vm.tiles, self.ranges_masked, stream)

    def masked_loss_grad(self, target, vm: "ViewMask", w=1.0, mse=False, stream=None):
        B.qn_masked_image_loss(self.W * self.H, 3, self.img, target, vm.pixel, vm.count, w, mse, self.loss,
                               self.d_img, stream)

    def ensure_capacity(self, margin: float = 1.25):
        """Synchronising: re-runs the binning with a larger buffer if it overflowed."""
        P = int(self.n_pairs.item())
        if P > self.capacity:
            self.set_capacity(int(P * margin) + 1024)
            self.bin_sort(sync=True)
        return P

    def size_for_views(self, attrs, cams, blur, margin: float = 1.25, stream=None) -> int:
        """Synchronising: bins attrs for every camera and sets the pair buffer
        to margin x the largest pair count (+ 4096); returns that count.  The
        training iteration never synchronises, so the buffer is sized before
        training; a binning that overflows it writes empty ranges (nothing is
        composited in that iteration), which check_capacity() reports."""
        P = 0
        for c in cams:
            self.project(attrs, c, blur, stream)
            self.bin_sort(False, stream)
            torch.cuda.synchronize()
            P = max(P, int(self.n_pairs.item()))
        self.set_capacity(int(P * margin) + 4096)
        return P

    def check_capacity(self) -> int:
        """Synchronising: the last binning's pair count; raises if it
        overflowed the pair buffer."""
        P = int(self.n_pairs.item())
        if P > self.capacity:
            raise RuntimeError(f"pair buffer overflow ({P} > {self.capacity})")
        return P


@dataclass
class ViewMask:
    """The adaptive training mask of one view (Sec. 3.3): pixel mask [H][W]
    u8, tile mask [tiles] u8, number of masked pixels [1] i32 (device)."""
    pixel: torch.Tensor
    tiles: torch.Tensor
    count: torch.Tensor

    @classmethod
    def empty(cls, width, height, device="cuda"):
        tx, ty = (width + TILE - 1) // TILE, (height + TILE - 1) // TILE
        return cls(torch.zeros((height, width), device=device, dtype=torch.uint8),
                   torch.zeros(tx * ty, device=device, dtype=torch.uint8),
                   torch.zeros(1, device=device, dtype=torch.int32))


def training_iteration(frame: QueenFrame, rast: Rasterizer, cam, target, skip=None, stream=None,
                       mask: ViewMask | None = None, unskip: bool = False, mark: bool = False):
    """One view of Eq. 11's optimisation: forward, Eq. 3's loss ((1 - lambda)
    L1 + lambda D-SSIM) + lambda_reg L_reg (the L_reg gradient is folded into
    the gate adjoint), full adjoint and the Adam step.  No host
    synchronisation.  Gaussians with skip set are frozen: no gradient and no
    update of their residual parameters (with HParams.fused they are rendered
    with the current decoders; otherwise their decoded columns are reused, and
    frame.attrs must hold their A_t, e.g. from a decode without skip).  With
    unskip, a skipped Gaussian
    that some pixel composites in this iteration is un-skipped before the
    adjoint (the forward marks the composited Gaussians), so it takes this
    iteration's update as plain training does and trains like the others from
    then on; the adjoint drops the Gaussians left skipped, which no pixel
    composites.  With HParams.mark_composited (or mark) the forward marks the
    composited Gaussians in rast.composited and the adjoint drops the others.
    With a mask (Sec. 3.3's masked training) only the masked tiles are
    composited and the loss is the mean over the masked pixels."""
    hp = frame.hp
    unskip = unskip and skip is not None
    mark = mark or unskip or hp.mark_composited
    fused_bwd = hp.fused and hp.fused_bwd
    if hp.fused:
        frame.decode_project(rast, cam, stream, skip, keep_attrs=not fused_bwd)
    else:
        frame.decode(stream, skip, train=True)
        rast.project(frame.attrs, cam, hp.blur, stream)
    rast.bin_sort(False, stream, lazy=hp.lazy_lists, list_max=hp.list_max)
    ranges = None
    if mask is not None:
        rast.mask_ranges(mask, stream)
        ranges = rast.ranges_masked
    rast.render_fwd(cam, hp.bg, stream=stream, ranges=ranges, mark=mark, order=hp.order_tiles)
    rast.photometric_loss(target, hp.lambda_dssim, mask, stream)
    if unskip:
        B.qn_clear_marked(rast.n, rast.composited, skip, stream)
    rast.render_bwd(cam, hp.bg, skip, stream, ranges=ranges, marks=mark, order=hp.order_tiles)
    if fused_bwd:
        frame.decode_project_bwd(rast, cam, skip, stream)
    else:
        rast.project_bwd(frame.attrs, cam, hp.blur, frame.d_attrs, skip, stream)
        frame.decode_bwd(skip, stream)
    frame.adam(skip, stream)


class IterationGraph:
    """training_iteration captured as CUDA graphs and replayed: one graph per
    key (normally the view index and whether a skip mask is used), captured
    on first use.  A replay issues the whole iteration with one host call, so
    the loop's speed is the GPU's.  Everything an iteration reads is bound at
    capture: the camera, and the addresses of the target, the skip mask and
    the frame's and rasterizer's buffers; a graph is captured again when one
    of those addresses changes (e.g. after Rasterizer.set_capacity).  The
    Adam step count lives on the device, so replays keep counting."""

    def __init__(self, frame: QueenFrame, rast: Rasterizer):
        self.frame, self.rast = frame, rast
        self.graphs = {}
        self.pool = None
        self.warm = False

    def _signature(self, target, skip, mask, unskip, mark, loss_out):
        r = self.rast
        return (target.data_ptr(), None if skip is None else skip.data_ptr(), r.vals.data_ptr(),
                r.pair_grads.data_ptr(), r.workspace.data_ptr(), None if mask is None else mask.pixel.data_ptr(),
                bool(unskip), bool(mark), None if loss_out is None else loss_out.data_ptr())

    def run(self, key, cam, target, skip=None, mask=None, unskip=False, mark=False, loss_out=None):
        """loss_out (optional, a one-element device tensor): the iteration's
        loss is copied there at its end, inside the graph, so a caller can
        read it back while the next iteration overwrites rast.loss."""
        sig = self._signature(target, skip, mask, unskip, mark, loss_out)
        ent = self.graphs.get(key)
        if ent is None or ent[1] != sig:
            if not self.warm:
                # one eager iteration first: lazily allocated scratch must
                # exist before capture; it is a real training step
                training_iteration(self.frame, self.rast, cam, target, skip, mask=mask, unskip=unskip, mark=mark)
                if loss_out is not None:
                    loss_out.copy_(self.rast.loss)
                self.warm = True
                return
            if self.pool is None:
                self.pool = torch.cuda.graph_pool_handle()
            g = torch.cuda.CUDAGraph()
            torch.cuda.synchronize()
            with torch.cuda.graph(g, pool=self.pool):
                training_iteration(self.frame, self.rast, cam, target, skip, mask=mask, unskip=unskip, mark=mark)
                if loss_out is not None:
                    loss_out.copy_(self.rast.loss)
            ent = (g, sig, cam, target, skip, mask, loss_out)   # keep what the graph points at alive
            self.graphs[key] = ent
        ent[0].replay()

    def clear(self):
        self.graphs.clear()
