"""Benchmark of QUEEN's per-frame residual-training iteration on one GB300.

One step = one training view through every stage of the hot path:
decode + gate -> projection -> binning -> compositing -> L1 loss ->
compositing adjoint -> projection adjoint -> decode/gate adjoint -> Adam.
Workload: 300,000 Gaussians, SH degree 3, 20 cameras at 1352 x 1014 on a
120-degree arc, int8 latents of width 8 per attribute category, synthetic
inputs (seeded), views cycled.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on a bounded tile sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: n, sh degree, width, height, views, latent width
    "full": (300_000, 3, 1352, 1014, 20, 8),
    "small": (2_000, 0, 128, 128, 1, 8),
    "large": (1_000_000, 3, 1920, 1080, 15, 8),
}
METRIC = "fwd+bwd rasterize it/s @300k Gaussians 1352x1014; s/frame learned vs plain @dPSNR<=.05"
L2_FLUSH_BYTES = 256 << 20
# the reference arm times whole oracle iterations when its K + W steps fit in this
REF_WHOLE_BUDGET_S = 300.0
# kernels each stage launches (memsets are not counted); the step decodes and
# projects in one kernel
KERNELS_PER_STAGE = {"decode_project": 1, "bin_sort": 14, "render_fwd": 2, "loss": 4, "render_bwd": 1,
                     "gather": 1, "project_bwd": 1, "decode_bwd": 2, "adam": 2}
STAGES = list(KERNELS_PER_STAGE)
# DRAM bytes per launch of a kernel on one workload, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum); valid for that workload while
# the sources it was built from are unchanged (their SHA-256 is checked), else
# reported null
NCU_TRAFFIC = {
    "render_bwd": {"workload": "full", "bytes": 38.054912e6 + 12.604672e6,
                   "sources": ("paper_2412_04469_gb300/csrc/render.cu", "paper_2412_04469_gb300/csrc/common.cuh",
                               "paper_2412_04469_gb300/csrc/bins.cuh", "paper_2412_04469_gb300/csrc/packed.cuh"),
                   "sha256": "86ed94babe90132465e0fa313a113cab0b0b8a260a715ef6f2c85050740fd9a5"},
}


def ncu_traffic(stage, workload):
    import hashlib
    rec = NCU_TRAFFIC.get(stage)
    if rec is None or rec["workload"] != workload:
        return None
    h = hashlib.sha256()
    for f in rec["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return rec["bytes"] if h.hexdigest() == rec["sha256"] else None


def workload_name(name):
    n, deg, W, H, V, L = WORKLOADS[name]
    return f"queen_residual_step_n{n}_sh{deg}_{W}x{H}_v{V}"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")

        sm = [num(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        loaded = [s for s in sm if not math.isnan(s)]
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": num(rows[0][2]),
                "samples": len(rows), "power_w_max": max(num(r[3]) for r in rows), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ GPU arm
def setup(name, seed=0, quick=False):
    import torch

    from paper_2412_04469_gb300 import binding as B
    from paper_2412_04469_gb300 import synthetic as S
    from paper_2412_04469_gb300.pipeline import QueenFrame, Rasterizer

    n, deg, W, H, V, L = WORKLOADS[name]
    lay = S.DecoderLayout.default(sh_degree=deg, latent=L)
    prev = S.make_scene(n, deg, seed)
    res = S.make_residuals(n, lay, seed)
    cams = S.make_arc_cameras(V, W, H) if V > 1 else [S.make_camera(W, H, 60.0)]
    if quick:
        V, cams = 1, cams[:1]
    frame = QueenFrame(prev, deg, lay, res.lat, res.dec, res.lp, res.log_alpha)
    rast = Rasterizer(n, frame.S, deg, W, H, 1)
    ccams = [B.make_camera(c) for c in cams]
    targets_host = [torch.from_numpy(S.make_image(W, H, 100 + v)).pin_memory() for v in range(V)]
    targets = [t.cuda() for t in targets_host]
    # size the pair buffer from every view (synchronising, outside any timing)
    frame.decode()
    rast.size_for_views(frame.attrs, ccams, frame.hp.blur, margin=1.25)
    return frame, rast, ccams, targets, targets_host, lay, prev, res, cams


def reduce_max(x, world, device):
    """The maximum of x over the ranks of the process group (x itself for one
    rank): every rank's timed region is bracketed by barriers, so the slowest
    rank's time is the job's."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, steps, max_ms):
    """Whole-job throughput: the iterations all ranks ran (each rank a replica
    running `steps` of them) over the slowest rank's time."""
    return world * steps / (max_ms * 1e-3)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2412_04469_gb300 import build as pbuild
    from paper_2412_04469_gb300.pipeline import IterationGraph, training_iteration

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pbuild.build()
    name = args.workload
    frame, rast, cams, targets, targets_host, lay, prev, res, cams_py = setup(name, quick=args.quick)
    n, deg, W, H, V, L = WORKLOADS[name]
    V = len(cams)
    hp = frame.hp
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return reduce_max(x, world, "cuda")

    def staged_step(v, ev):
        """One iteration issued stage by stage with an event between stages."""
        c = cams[v]
        mk, od = hp.mark_composited, hp.order_tiles
        calls = (lambda: frame.decode_project(rast, c), lambda: rast.bin_sort(False, lazy=hp.lazy_lists, list_max=hp.list_max),
                 lambda: rast.render_fwd(c, hp.bg, mark=mk, order=od),
                 lambda: rast.photometric_loss(targets[v], hp.lambda_dssim),
                 lambda: rast.render_bwd_pairs(c, hp.bg, marks=mk, order=od), lambda: rast.gather(c),
                 lambda: rast.project_bwd(frame.attrs, c, hp.blur, frame.d_attrs), lambda: frame.decode_bwd(),
                 lambda: frame.adam())
        for i, f in enumerate(calls):
            ev[i].record(stream)
            f()
        ev[len(calls)].record(stream)

    for w in range(args.warmup):
        training_iteration(frame, rast, cams[w % V], targets[w % V])
    torch.cuda.synchronize()
    assert int(rast.n_pairs.item()) <= rast.capacity, "pair buffer overflow during warm-up"

    # ---- per-stage breakdown: eager launches, CUDA events between stages
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(STAGES) + 1)] for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.zero_()                       # L2 flush between timed steps (outside the step events)
        staged_step((args.warmup + k) % V, evs[k])
    barrier()
    stage_ms = {s: [e[i].elapsed_time(e[i + 1]) for e in evs] for i, s in enumerate(STAGES)}
    staged_ms = max_over_ranks(float(sum(e[0].elapsed_time(e[-1]) for e in evs)))

    # ---- headline: the iteration replayed as one CUDA graph per view
    graphs = IterationGraph(frame, rast)
    for w in range(V + 1):                  # warm-up: the eager step, then one capture per view
        graphs.run(w % V, cams[w % V], targets[w % V])
    for w in range(args.warmup):
        graphs.run(w % V, cams[w % V], targets[w % V])
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        v = (args.warmup + k) % V
        flush.zero_()
        gev[k][0].record(stream)
        graphs.run(v, cams[v], targets[v])
        gev[k][1].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    overflow = int(rast.n_pairs.item()) > rast.capacity
    step_ms = [a.elapsed_time(b) for a, b in gev]
    max_ms = max_over_ranks(float(sum(step_ms)))
    median_ms = max_over_ranks(float(statistics.median(step_ms)))
    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "ms_per_step": max_ms / args.steps,
                              "staged_ms_per_step": staged_ms / args.steps,
                              "stage_ms": {s: float(np.mean(stage_ms[s])) for s in STAGES}}), flush=True)
        return

    # ---- end to end through the public API with host buffers: every step
    # copies its view's target from pinned host memory to the device and reads
    # the loss back.  The copies run on their own stream into two target
    # buffers, so step k + 1's copy overlaps step k's compute; each step waits
    # for its copy, and a buffer is refilled only after the step that read it.
    # The loss goes, inside the step's graph, to one of two device slots, and
    # is read back from there on the copy stream while the next step runs; a
    # slot is rewritten only after its read-back, and the timed region ends
    # after the last one.
    loss_host = torch.zeros(2).pin_memory()
    loss_slots = [torch.zeros(1, device="cuda") for _ in range(2)]
    tgt_bufs = [torch.empty_like(targets[0]) for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    for b in range(2):
        for v in range(V):
            tgt_bufs[b].copy_(targets_host[v], non_blocking=True)
            graphs.run(("e2e", v, b), cams[v], tgt_bufs[b], loss_out=loss_slots[b])
    barrier()
    ready = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    read = [torch.cuda.Event() for _ in range(2)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def upload(k):
        b, v = k % 2, (args.warmup + k) % V
        with torch.cuda.stream(copy_stream):
            tgt_bufs[b].copy_(targets_host[v], non_blocking=True)
            ready[b].record(copy_stream)

    e0.record(stream)
    copy_stream.wait_event(e0)                 # no copy before the timed region starts
    upload(0)
    for k in range(args.steps):
        b, v = k % 2, (args.warmup + k) % V
        if k + 1 < args.steps:
            if k >= 1:
                copy_stream.wait_event(done[1 - b])   # step k - 1 has read that buffer
            upload(k + 1)
        stream.wait_event(ready[b])
        if k >= 2:
            stream.wait_event(read[b])                # step k - 2's loss has been read from slot b
        graphs.run(("e2e", v, b), cams[v], tgt_bufs[b], loss_out=loss_slots[b])
        done[b].record(stream)
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(done[b])
            loss_host[b:b + 1].copy_(loss_slots[b], non_blocking=True)
            read[b].record(copy_stream)
    stream.wait_event(read[(args.steps - 1) % 2])     # the last read-back is inside the timed region
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1))

    # ---- work counts for the roofline (after timing; one forward per view)
    P_list, Pvis_list, last_sum, contrib_sum = [], [], [], []
    ncon = torch.zeros((H, W), device="cuda", dtype=torch.int32)
    frame.decode()
    for v in range(V):
        c = cams[v]
        rast.project(frame.attrs, c, hp.blur)
        rast.bin_sort(False)
        rast.render_fwd(c, hp.bg, n_contrib=ncon)
        torch.cuda.synchronize()
        P_list.append(int(rast.n_pairs.item()))
        TY, TX = rast.TY, rast.TX
        last = rast.last.long()
        pad = torch.zeros((TY * 16, TX * 16), dtype=torch.long, device="cuda")
        pad[:H, :W] = last
        tile_max = pad.view(TY, 16, TX, 16).amax(dim=(1, 3))
        Pvis_list.append(int(tile_max.sum().item()))
        last_sum.append(int(last.sum().item()))
        contrib_sum.append(int(ncon.long().sum().item()))
    P = float(np.mean(P_list))
    Pvis = float(np.mean(Pvis_list))
    n_vis = int((rast.rects[:, 2] > rast.rects[:, 0]).sum().item())
    px = W * H
    chunks, tiles = (n_vis + 255) // 256, rast.TX * rast.TY
    # algorithmic bytes per launch: what each stage must read and write once
    # (a projected record or a pair's gradient record is 48 bytes)
    algo_bytes = {
        # read A_{t-1} 236 + latents 128 + lp 12 + log alpha 4, write the 2D record 48
        # (and A_t 236 for the projection adjoint)
        "decode_project": (428.0 + 236.0) * n,
        # depth sort: key and index in, out, and the rect read (20 per Gaussian); then with the lists
        # written, the lower bound of a (key, value) sort over the P pairs (36 per pair), else the
        # (chunk, tile) counts (written, read twice, written back) and the chunk masks (written)
        "bin_sort": 20.0 * n + (16.0 * chunks * tiles + 32.0 * chunks * (rast.TX + rast.TY) if hp.lazy_lists
                                else 36.0 * P),
        # (with lists formed in the forward, it also writes the walked prefix: 4 per visited pair)
        "render_fwd": 20.0 * px + (8.0 if hp.lazy_lists else 4.0) * Pvis + 48.0 * n_vis,
        # L1: img, target, d_img; D-SSIM: img, target, 3 maps out, 3 maps in, img, target, d_img += (3 channels)
        "loss": 36.0 * px + (144.0 * px if hp.lambda_dssim > 0 else 0.0),
        "render_bwd": 20.0 * px + 52.0 * Pvis + 48.0 * n_vis, "gather": 48.0 * Pvis + 48.0 * n_vis,
        "project_bwd": 508.0 * n, "decode_bwd": 524.0 * n,
        "adam": 28.0 * ((lay.n_latent + 4) * n + lay.n_dec),
    }
    avg = {s: float(np.mean(stage_ms[s])) for s in STAGES}
    # the dominant kernel: the longest stage that is one kernel (the binning
    # stage is 14 kernels, none of them as long as the compositing adjoint)
    dom = max((s for s in STAGES if KERNELS_PER_STAGE[s] == 1), key=lambda s: avg[s])
    hbm_peak, peak_kind = peaks()
    achieved = algo_bytes[dom] / (avg[dom] * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(achieved / hbm_peak, 4), "peak_source": f"{peak_kind} hbm_gbs",
            "traffic": ncu_traffic(dom, args.workload), "algorithmic_bytes": algo_bytes[dom]}
    # FP32 arithmetic of the compositing adjoint as the method defines it:
    # 12 flop per alpha evaluation (every pixel up to its last contributor),
    # 41 more per contributing evaluation, and a 45-flop reduction of the
    # nine per-Gaussian sums per 32 contributions
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
    flops_bwd = 12.0 * np.mean(last_sum) + 41.0 * np.mean(contrib_sum) + 45.0 * np.mean(contrib_sum) / 32.0
    alu = {"kernel": "render_bwd", "achieved": round(flops_bwd / (avg["render_bwd"] * 1e-3) / 1e12, 3),
           "peak": round(fp32_peak, 2), "unit": "TFLOP/s"}
    alu["frac"] = round(alu["achieved"] / alu["peak"], 4)
    # special-function unit: one ex2 per alpha evaluation, one reciprocal per
    # contributing evaluation (T rebuilt in front of the Gaussian), against 32
    # MUFU results per SM and clock (an independent-chain ex2.approx loop
    # measures 30.4 on this part)
    sfu_ops = float(np.mean(last_sum) + np.mean(contrib_sum))
    sfu = {"kernel": "render_bwd", "achieved": round(sfu_ops / (avg["render_bwd"] * 1e-3) / 1e12, 3),
           "peak": round(n_sm * 32 * sm_mhz * 1e6 / 1e12, 3), "unit": "Tops/s",
           "peak_source": f"{n_sm} SM x 32 MUFU results x median SM clock"}
    sfu["frac"] = round(sfu["achieved"] / sfu["peak"], 4)
    if dom == "render_bwd" and alu["frac"] > roof["frac"]:
        roof_alu = dict(roof)
        roof = {"bound": "alu", "kernel": dom, "achieved": alu["achieved"], "peak": alu["peak"],
                "unit": "TFLOP/s", "frac": alu["frac"], "peak_source": f"{n_sm} SM x 128 FP32 lanes x 2 x median SM clock",
                "traffic": ncu_traffic(dom, args.workload), "algorithmic_bytes": algo_bytes[dom],
                "hbm": {k: roof_alu[k] for k in ("achieved", "peak", "unit", "frac")}, "sfu": sfu}
    else:
        roof["alu_render_bwd"] = alu
        roof["sfu_render_bwd"] = sfu

    value = job_rate(world, args.steps, max_ms)
    launches = args.steps * (sum(KERNELS_PER_STAGE.values()) - (2 if hp.lambda_dssim == 0 else 0)
                             + (1 if hp.gate_noise else 0))
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "it/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(max_ms / args.steps, 4),
        "median_ms_per_step": round(median_ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (bf16 decoder weights)",
        "data": "synthetic (seeded scene, residuals and target images; no dataset)",
        "config": {"workload": workload_name(name), "n_gaussians": n, "sh_degree": deg, "width": W, "height": H,
                   "views": V, "latent_dim": L, "pairs_per_view": round(P), "visited_pairs_per_view": round(Pvis),
                   "loss": f"{1 - hp.lambda_dssim:g} L1 + {hp.lambda_dssim:g} D-SSIM (Eq. 3) + lambda_reg L_reg",
                   "visible_gaussians": n_vis, "l2": "flushed between timed steps (256 MB write outside step events)",
                   "launch": "one CUDA graph replay per step (iteration captured once per view)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "stage_ms": {s: round(avg[s], 4) for s in STAGES},
        # algorithmic bytes of each stage over its warm time (HBM-side work rate)
        "stage_gbs": {s: round(algo_bytes[s] / (avg[s] * 1e-3) / 1e9, 1) for s in STAGES},
        "staged_ms_per_step": round(staged_ms / args.steps, 4),
        "roofline": roof,
        "clocks": clocks,
        "e2e": {"value": round(job_rate(world, args.steps, e2e_ms), 3), "unit": "it/s",
                "h2d_bytes_per_step": int(targets[0].numel() * 4), "d2h_bytes_per_step": 4,
                "l2": "not flushed: steps back to back, as a training loop runs them"},
        "gpu_launches": launches,
        "pair_overflow": overflow,
        "wall_s": round(t_wall, 3),
    }
    if not args.no_seq and (name == "full" or args.seq_config == "large"):
        del graphs, frame, rast, targets, flush
        torch.cuda.empty_cache()
        out["sequence"] = run_sequence(args)
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(name)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_sequence(args):
    """The learned static-skip comparison on the full workload's scene and
    cameras: plain gated training and learned skip over the same streamed
    frames (the MLP trains on the first 10, skips from frame 11 on), at the
    configured skip threshold and at each --seq-extra-threshold; then plain
    gated training with Sec. 3.3's masked training on each --seq-masked
    fraction of the iterations, against the plain arm."""
    from paper_2412_04469_gb300.sequence import SequenceConfig, compare

    if args.seq_config == "large":
        # 1M Gaussians, 15 views at 1920x1080, 5% dynamic content, 30 frames
        n, deg, W, H, V, L = WORKLOADS["large"]
        cfg = SequenceConfig(n=n, sh_degree=deg, width=W, height=H, views=V, frames=30, iters=args.seq_iters,
                             frac_dynamic=0.05)
    else:
        cfg = SequenceConfig(frames=args.seq_frames, iters=args.seq_iters, frac_dynamic=args.seq_dynamic)
    t0 = time.perf_counter()
    out = compare(cfg, extra_thresholds=args.seq_extra_threshold, masked_fractions=args.seq_masked,
                  learned=not args.seq_masked_only, no_unskip=not args.seq_masked_only)

    def arm(summary, learned, thr):
        skip = [r for r in learned if r.t > cfg.train_frames]
        kept = [r.seconds for r in skip if not r.fallback]
        return {"threshold": thr,
                "s_per_frame_plain": round(summary["s_per_frame_plain_skip_frames"], 4),
                "s_per_frame_learned": round(summary["s_per_frame_learned_skip_frames"], 4),
                "speedup": round(summary["s_per_frame_plain_skip_frames"]
                                 / summary["s_per_frame_learned_skip_frames"], 4),
                "skip_frames": len(skip), "fallbacks": summary["fallbacks"],
                "mean_skipped_fraction": round(summary["mean_skipped"], 4),
                # against the Gaussians static by construction (the 90% that do not move)
                "static_recall": round(summary["static_recall"], 4),
                "static_precision": round(summary["static_precision"], 4),
                "plain_gate0_static_recall": round(summary["plain_gate0_recall"], 4),
                "plain_gate0_static_precision": round(summary["plain_gate0_precision"], 4),
                "dpsnr_train_views_min": round(summary["min_dpsnr_train_skip_frames"], 4),
                "dpsnr_train_views_mean": round(summary["mean_dpsnr_train_skip_frames"], 4),
                "dpsnr_heldout_min": round(summary["min_dpsnr_skip_frames"], 4),
                "dpsnr_heldout_mean": round(summary["mean_dpsnr_skip_frames"], 4),
                "frame_s_learned": [round(r.seconds, 4) for r in skip],
                "s_per_frame_learned_kept": round(float(np.mean(kept)), 4) if kept else None,
                "fallback_dpsnr_train_before": [round(r.psnr_skip_train - r.psnr_plain_train, 4)
                                                for r in skip if r.fallback],
                # the compositing adjoint of one view at each skip frame's end, with and without the skip
                "render_bwd_ms_skip": round(summary["render_bwd_ms_skip"], 4),
                "render_bwd_ms_plain": round(summary["render_bwd_ms_plain"], 4)}

    res = {"config": {"n_gaussians": cfg.n, "sh_degree": cfg.sh_degree, "width": cfg.width, "height": cfg.height,
                      "views": cfg.views, "frames": cfg.frames, "iters_per_frame": cfg.iters,
                      "frac_dynamic": cfg.frac_dynamic, "mlp_train_frames": cfg.train_frames,
                      "max_dpsnr": cfg.max_dpsnr, "fallback_psnr": cfg.fallback_psnr,
                      "dpsnr_reference": "plain gated training of the same frame from the same state",
                      "timed": "training work only (PSNR evaluation and the reference run excluded)",
                      "launch": "CUDA graph replays" if cfg.graphs else "eager"}}
    if "learned" in out:
        res["configured"] = arm(out, out["learned"], cfg.threshold)
    for thr, v in out["by_threshold"].items():
        res[f"threshold_{thr:g}"] = arm(v, v["learned"], thr)
    if "rule" in out:
        # the non-learned skip: what the previous frame's label called static
        res["rule_previous_label"] = arm(out["rule"], out["rule"]["learned"], None)
    if "no_unskip" in out:
        # the learned skip with composited skipped Gaussians kept skipped: the
        # compositing adjoint drops their gradients, the frame may fall back
        res["learned_no_unskip"] = arm(out["no_unskip"], out["no_unskip"]["learned"], cfg.threshold)
    plain = out["plain"]
    if cfg.packet:
        res["packet"] = {
            "mb_per_frame": round(float(np.mean([r.packet_bytes for r in plain])) / 1e6, 4),
            "mb_per_frame_each": [round(r.packet_bytes / 1e6, 4) for r in plain],
            "pack_unpack_s": round(float(np.mean([r.packet_s for r in plain])), 4),
            "dpsnr_gate_binarised_mean": round(float(np.mean([r.psnr_packet - r.psnr for r in plain])), 4),
            "contents": "rANS-coded integer latents, bf16 decoders, COO position residuals (gate binarised)"}
    for mf, recs in out["masked"].items():
        res[f"masked_{mf:g}"] = {
            "masked_fraction": mf, "t_d_ndc": cfg.mask_t_d, "dilation": 48,
            "s_per_frame_plain": round(float(np.mean([r.seconds for r in plain])), 4),
            "s_per_frame_masked": round(float(np.mean([r.seconds for r in recs])), 4),
            "speedup": round(float(np.mean([r.seconds for r in plain]) / np.mean([r.seconds for r in recs])), 4),
            "dpsnr_heldout_mean": round(float(np.mean([m.psnr - p.psnr for m, p in zip(recs, plain)])), 4),
            "dpsnr_heldout_min": round(float(np.min([m.psnr - p.psnr for m, p in zip(recs, plain)])), 4),
            "mask_tile_fraction_mean": round(float(np.mean([r.mask_tiles for r in recs])), 4)}
    res["wall_s"] = round(time.perf_counter() - t0, 1)
    return res


# ------------------------------------------------------------------ CPU oracle
_ORACLE = {}


def _oracle_state(name, seed, m):
    """The workload's seeded inputs for the oracle, built once per process
    outside every timed region, and the column sample of m Gaussians that the
    per-Gaussian stages are timed on."""
    from paper_2412_04469_gb300 import synthetic as S

    st = _ORACLE.get((name, seed))
    if st is None:
        n, deg, W, H, V, L = WORKLOADS[name]
        lay = S.DecoderLayout.default(sh_degree=deg, latent=L)
        st = {"lay": lay, "prev": S.make_scene(n, deg, seed).astype(np.float64),
              "res": S.make_residuals(n, lay, seed),
              "cams": S.make_arc_cameras(V, W, H) if V > 1 else [S.make_camera(W, H, 60.0)],
              "views": {}, "cols": {}, "dssim_s": None}
        _ORACLE[(name, seed)] = st
    if m not in st["cols"]:
        n = WORKLOADS[name][0]
        idx = (np.sort(np.random.default_rng(seed + 29).choice(n, size=m, replace=False)) if m < n
               else np.arange(n))
        r = st["res"]
        st["cols"][m] = (idx, np.ascontiguousarray(st["prev"][:, idx]), np.ascontiguousarray(r.lat[:, idx]),
                         np.ascontiguousarray(r.lp[:, idx]), np.ascontiguousarray(r.log_alpha[idx]))
    return st


def oracle_step(name, n_tiles_sample, seed=0, view=0, m=None, tile_seed=None, calib=1.0):
    """One oracle training iteration of the workload, timed on a bounded
    sample and scaled to the whole of it:
      - decode, projection and their adjoints (linear in the Gaussians) on a
        seeded sample of m of the n Gaussians, scaled by n / m;
      - compositing and its adjoint on a seeded sample of tiles (tile_seed,
        else one per view), against the view's full projection (computed
        once per view, untimed); their per-call set-up (a pass over every
        rect) does not grow with the tiles, so it is timed apart on the
        corner tile, once per view, and added once; the per-tile time is
        multiplied by calib
        (small samples overstate it: the few deep tiles keep some threads busy
        while the others wait, so the caller calibrates against a composite
        of every tile);
      - the L1 term on the whole image;
      - D-SSIM, timed once per process on the whole image (on crops its
        numpy filters cost up to half as much again per pixel).
    Returns a dict: seconds of the sampled work, the whole-iteration
    estimate, the tiles and Gaussians sampled, and the parts."""
    import oracle

    n, deg, W, H, V, L = WORKLOADS[name]
    m = n if m is None else max(1, min(n, int(m)))
    st = _oracle_state(name, seed, m)
    lay, res = st["lay"], st["res"]
    tau, g0, g1, lam = 0.3, -0.5, 1.01, 0.2            # Eq. 3 weights, as the GPU step uses them
    cam = st["cams"][view % V]
    vw = st["views"].get(view % V)
    if vw is None:
        A, _, _ = oracle.decode(st["prev"], res.lat, res.dec, res.lp, res.log_alpha, lay, tau, g0, g1)
        from paper_2412_04469_gb300 import synthetic as S
        vw = {"proj": oracle.project(A, cam, deg, blur=0.3), "target": S.make_image(W, H, 100 + view % V)}
        st["views"][view % V] = vw
    if st["dssim_s"] is None:
        t = time.perf_counter()
        oracle.dssim_loss(0.5 * vw["target"], vw["target"])
        st["dssim_s"] = time.perf_counter() - t
    TX, TY = (W + 15) // 16, (H + 15) // 16
    rng = np.random.default_rng(seed + 17 + view if tile_seed is None else tile_seed)
    tiles = np.sort(rng.choice(TX * TY, size=min(n_tiles_sample, TX * TY), replace=False))
    idx, prev_m, lat_m, lp_m, la_m = st["cols"][m]
    proj = vw["proj"]
    if "setup" not in vw:                                # the same pass over every rect in every call
        corner = np.array([0])
        ts = time.perf_counter()
        oracle.render_fwd(proj, tiles=corner)
        oracle.render_bwd(proj, np.zeros((3, H, W)), tiles=corner)
        vw["setup"] = time.perf_counter() - ts
    setup = vw["setup"]
    t0 = time.perf_counter()
    A_m, _, _ = oracle.decode(prev_m, lat_m, res.dec, lp_m, la_m, lay, tau, g0, g1)
    proj_m = oracle.project(A_m, cam, deg, blur=0.3)
    t1 = time.perf_counter()
    img, _, _, _ = oracle.render_fwd(proj, tiles=tiles)
    t2 = time.perf_counter()
    _, g = oracle.l1_loss(img, vw["target"])
    g *= 1 - lam
    t3 = time.perf_counter()
    gr = oracle.render_bwd(proj, g, tiles=tiles)
    t4 = time.perf_counter()
    dA = oracle.project_bwd(A_m, cam, deg, gr["d_mean2d"][:, idx], gr["d_conic"][:, idx], gr["d_opac"][idx],
                            gr["d_rgb"][:, idx], blur=0.3)
    oracle.decode_bwd(lat_m, res.dec, lp_m, la_m, lay, tau, g0, g1, dA, 0.01)
    t5 = time.perf_counter()
    del proj_m
    per_gauss = ((t1 - t0) + (t5 - t4)) * n / m
    per_tile = max(0.0, (t2 - t1) + (t4 - t3) - setup) / len(tiles)
    full = per_gauss + setup + calib * per_tile * TX * TY + (t3 - t2) + st["dssim_s"]
    return {"sampled": t5 - t0, "full": full, "tiles": len(tiles), "n_tiles": TX * TY, "m": m, "n": n,
            "per_gauss": per_gauss, "per_tile": per_tile, "setup": setup, "l1": t3 - t2, "dssim": st["dssim_s"]}


def oracle_iteration(name, n_tiles_sample, seed=0, view=0):
    """oracle_step with every Gaussian: (sampled seconds, whole-iteration
    estimate, tiles sampled)."""
    r = oracle_step(name, n_tiles_sample, seed, view)
    return r["sampled"], r["full"], r["tiles"]


def oracle_whole_step(name, view, seed=0):
    """One oracle training iteration of the workload, all of it measured:
    decode and projection of every Gaussian, compositing of every tile, the
    L1 and D-SSIM terms of Eq. 3 on the whole image, the compositing
    adjoint of every tile, the projection and decode adjoints of every
    Gaussian.  Returns its wall seconds."""
    import oracle

    n, deg, W, H, V, L = WORKLOADS[name]
    st = _oracle_state(name, seed, n)
    lay, res = st["lay"], st["res"]
    tau, g0, g1, lam = 0.3, -0.5, 1.01, 0.2
    cam = st["cams"][view % V]
    tgt = st.setdefault("targets", {})
    if view % V not in tgt:
        from paper_2412_04469_gb300 import synthetic as S
        tgt[view % V] = S.make_image(W, H, 100 + view % V)
    target = tgt[view % V]
    t0 = time.perf_counter()
    A, _, _ = oracle.decode(st["prev"], res.lat, res.dec, res.lp, res.log_alpha, lay, tau, g0, g1)
    proj = oracle.project(A, cam, deg, blur=0.3, tight=True)
    img, _, _, _ = oracle.render_fwd(proj)
    _, g = oracle.l1_loss(img, target)
    g *= 1 - lam
    _, gs = oracle.dssim_loss(img, target)
    g += lam * gs
    gr = oracle.render_bwd(proj, g)
    dA = oracle.project_bwd(A, cam, deg, gr["d_mean2d"], gr["d_conic"], gr["d_opac"], gr["d_rgb"], blur=0.3)
    oracle.decode_bwd(res.lat, res.dec, res.lp, res.log_alpha, lay, tau, g0, g1, dA, 0.01)
    return time.perf_counter() - t0


ORACLE_SAMPLE = ("one iteration: decode, projection and their adjoints on {m} of {n} Gaussians{gauss_note}, "
                 "compositing and its adjoint on {k} of {nt} tiles{tiles_note}, the L1 term on the whole image, "
                 "D-SSIM timed once on the whole image ({dssim:.1f} s)")


def cpu_single_thread(name, tiles=48):
    """The same oracle iteration on one core (OMP_NUM_THREADS=1, in a child
    process so the parent's thread pool is untouched), on a smaller tile
    sample; None if the child fails."""
    import subprocess
    code = ("import json, sys; sys.path.insert(0, %r); import bench, oracle; oracle.build(); "
            "s, f, k = bench.oracle_iteration(%r, %d); print(json.dumps([s, f, k, oracle.num_threads()]))"
            % (ROOT, name, tiles))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, env=env)
        s, f, k, cores = json.loads(out.stdout.strip().splitlines()[-1])
    except Exception:
        return None
    return {"value": round(1.0 / f, 6), "unit": "it/s", "cores": cores,
            "sample": f"as above on {k} random tiles; sampled run {s:.1f} s"}


def cpu_baseline(name):
    """The oracle's iteration on the machine's host cores, every Gaussian and
    every tile (10-30 s of CPU work at the benchmark's sizes)."""
    import oracle
    oracle.build()
    nt = ((WORKLOADS[name][2] + 15) // 16) * ((WORKLOADS[name][3] + 15) // 16)
    r = oracle_step(name, nt)
    single = cpu_single_thread(name)
    return {"value": round(1.0 / r["full"], 6), "unit": "it/s", "cores": oracle.num_threads(), "kind": "oracle",
            "single_thread": single,
            "sample": ORACLE_SAMPLE.format(m=r["m"], n=r["n"], k=r["tiles"], nt=r["n_tiles"], dssim=r["dssim"],
                                           tiles_note="", gauss_note="")
            + f"; sampled run {r['sampled']:.1f} s"}


def run_reference(args):
    """The oracle's line (the paper ships no code; the reference arm is the
    FP64 CPU oracle on the machine's host cores): whole iterations, nothing
    extrapolated.  One untimed whole iteration sizes the run and counts as
    the first warm-up step.  When the requested K + W steps would not fit in
    --ref-budget seconds, it times fewer whole iterations (3 warm-up steps, as
    many timed steps as fit, at least 3) and the line says so: `steps` is the
    count timed, `steps_requested` the count asked for."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    name = args.workload
    n, deg, W, H, V, L = WORKLOADS[name]
    ntiles = ((W + 15) // 16) * ((H + 15) // 16)
    t_one = oracle_whole_step(name, 0)
    budget = args.ref_budget
    if (args.steps + args.warmup) * t_one <= budget:
        steps, warmup = args.steps, args.warmup
    else:
        warmup = 3
        steps = min(args.steps, max(3, int((budget - warmup * t_one) // max(t_one, 1e-9))))
    for w in range(1, warmup):
        oracle_whole_step(name, w)
    secs = [oracle_whole_step(name, warmup + s) for s in range(steps)]
    value = steps / sum(secs)
    sample = (f"whole iterations, nothing extrapolated: per step decode, projection and their adjoints on all "
              f"{n} Gaussians, compositing and its adjoint on all {ntiles} tiles, L1 and D-SSIM (Eq. 3) on the "
              f"whole image; {sum(secs):.1f} s over the {steps} timed steps")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "it/s", "n_gpus": world,
           "steps": steps, "warmup": warmup, "ms_per_step": round(1e3 * sum(secs) / steps, 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_name(name), "n_gaussians": n, "width": W, "height": H, "views": V,
                      "sh_degree": deg}}
    if (steps, warmup) != (args.steps, args.warmup):
        out["steps_requested"], out["warmup_requested"] = args.steps, args.warmup
        out["note"] = (f"{args.steps + args.warmup} whole iterations (~{t_one:.1f} s each) would not fit in "
                       f"{budget:g} s, so {steps} timed after {warmup} warm-up steps")
    out["cpu_baseline"] = {"value": out["value"], "unit": "it/s", "cores": oracle.num_threads(), "kind": "oracle",
                           "sample": sample}
    out["e2e"] = {"value": out["value"], "unit": "it/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--ref-budget", type=float, default=REF_WHOLE_BUDGET_S,
                    help="reference arm: seconds of whole oracle iterations to fit the K + W steps in")
    ap.add_argument("--workload", default="full", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-seq", action="store_true", help="skip the learned-skip sequence comparison")
    ap.add_argument("--seq-frames", type=int, default=60, help="frames of the learned-skip sequence comparison")
    ap.add_argument("--seq-iters", type=int, default=250, help="training iterations per frame in that comparison")
    ap.add_argument("--seq-config", default="full", choices=["full", "large"],
                    help="sequence of the learned-skip comparison: the 300k one (60 frames by default) or the "
                         "1M-Gaussian 1920x1080 one (30 frames, 5%% dynamic)")
    ap.add_argument("--seq-dynamic", type=float, default=0.10,
                    help="fraction of the Gaussians that move in the 300k sequence (the ones nearest the middle "
                         "of the face the cameras see)")
    ap.add_argument("--seq-masked-only", action="store_true",
                    help="sequence: the plain and masked-training arms only (no skip arms)")
    ap.add_argument("--seq-masked", type=float, nargs="*", default=[],
                    help="fractions of iterations trained on Sec. 3.3's adaptive masks (plain gating otherwise)")
    ap.add_argument("--seq-extra-threshold", type=float, nargs="*", default=[],
                    help="further skip thresholds to run in that comparison (same plain arm)")
    ap.add_argument("--quick", action="store_true",
                    help="one view, timed steps only (for profiler captures); prints stage times")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
