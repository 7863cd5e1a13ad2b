"""Variants of the path.  The paper's own N3DV configuration: five decoders
(rotation, scale, opacity, colour base, colour frequency with latent widths
6, 8, 3, 8, 4 from the quantisation table) on SH degree 2 -- the decode and
its adjoint against the oracle, a training iteration (eager and
graph-replayed, bit-identical) with the table's learning rates, and the packet
against the oracle's bytes.  The stochastic hard-concrete gate: the Philox
noise bit-identical to the oracle's, the noisy decode and its adjoint against
the oracle, and training iterations that draw fresh noise per step and still
replay bit-identically."""
import numpy as np
import pytest
import torch

import oracle
from oracle import packet as OP
from paper_2412_04469_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

TAU, G0, G1 = 0.3, -0.5, 1.01


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_04469_gb300 import build
    build.build()


def up(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def close(got, ref, rtol, floor_frac, what):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    err = np.abs(got - ref) / np.maximum(np.abs(ref), floor_frac * np.abs(ref).max())
    assert err.max() <= rtol, f"{what}: {err.max():.3e}"


@pytest.mark.parametrize("n", [1000, 40_000])
def test_paper_layout_decode_and_adjoint(n):
    from paper_2412_04469_gb300.pipeline import HParams, QueenFrame
    deg = 2
    lay = S.DecoderLayout.paper_n3dv(deg)
    assert lay.n_cat == 5 and lay.lat_dim == [6, 8, 3, 8, 4] and lay.attr_count[4] == 24
    prev = S.make_scene(n, deg, 3)
    res = S.make_residuals(n, lay, 3)
    res.lat[:, :5] = np.array([0.5, 1.5, -2.5, 130.2, -200.0], np.float32)[None, :]
    res.log_alpha[: n // 2] = np.linspace(-1, 1, n // 2)
    f = QueenFrame(prev, deg, lay, res.lat, res.dec, res.lp, res.log_alpha, HParams(lreg_mean=False))
    f.decode()
    torch.cuda.synchronize()
    out, gate, lreg = oracle.decode(prev.astype(np.float64), res.lat, res.dec, res.lp, res.log_alpha, lay, TAU, G0,
                                    G1)
    got = f.attrs.cpu().numpy()[:, :n]
    close(got[:3], out[:3], 1e-4, 1e-2, "position")
    close(got[3:] - prev[3:], out[3:] - prev[3:].astype(np.float64), 2e-3, 1e-2, "decoded residual")
    rng = np.random.default_rng(4)
    d_out = rng.standard_normal((prev.shape[0], n)).astype(np.float32)
    f.d_attrs[:, :n] = up(d_out)
    f.decode_bwd()
    torch.cuda.synchronize()
    want = oracle.decode_bwd(res.lat, res.dec, res.lp, res.log_alpha, lay, TAU, G0, G1, d_out, f.d_lreg)
    for got_t, ref, what in ((f.d_lat.cpu().numpy()[:, :n], want[0], "d_lat"), (f.d_dec.cpu().numpy(), want[1], "d_dec"),
                             (f.d_lp.cpu().numpy()[:, :n], want[2], "d_lp"),
                             (f.d_log_alpha.cpu().numpy()[:n], want[3], "d_log_alpha")):
        close(got_t, ref, 1e-4, 0.05, what)


def test_paper_layout_training_iteration_and_graph():
    from paper_2412_04469_gb300 import binding as B
    from paper_2412_04469_gb300.pipeline import IterationGraph, QueenFrame, Rasterizer, n3dv_hparams, training_iteration
    n, deg, W, H = 6000, 2, 120, 90
    lay = S.DecoderLayout.paper_n3dv(deg)
    prev = S.make_scene(n, deg, 5)
    res = S.make_residuals(n, lay, 5)
    cams = [B.make_camera(c) for c in S.make_arc_cameras(3, W, H)]
    tg = [up(S.make_image(W, H, 40 + v)) for v in range(3)]
    outs = []
    for graphs in (False, True):
        f = QueenFrame(prev, deg, lay, res.lat, res.dec, res.lp, res.log_alpha, n3dv_hparams())
        r = Rasterizer(n, f.S, deg, W, H, 1 << 20)
        g = IterationGraph(f, r) if graphs else None
        for it in range(7):
            if g is None:
                training_iteration(f, r, cams[it % 3], tg[it % 3])
            else:
                g.run(it % 3, cams[it % 3], tg[it % 3])
        torch.cuda.synchronize()
        assert torch.isfinite(f.lat).all() and torch.isfinite(f.dec).all() and torch.isfinite(r.loss).all()
        outs.append([t.clone() for t in (f.lat, f.dec, f.lp, f.log_alpha, r.loss)])
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def test_paper_layout_packet():
    from paper_2412_04469_gb300 import binding as B
    n, deg = 12_000, 2
    lay = S.DecoderLayout.paper_n3dv(deg)
    rng = np.random.default_rng(8)
    Sd = (n + 3) // 4 * 4
    lat = np.where(rng.uniform(size=(lay.n_latent, Sd)) < 0.85, 0.0, rng.normal(0, 3, (lay.n_latent, Sd))).astype(
        np.float32)
    dec = S.bf16_bits(rng.normal(0, 0.01, lay.n_dec).astype(np.float32))
    lp = rng.normal(0, 0.01, (3, Sd)).astype(np.float32)
    gate = np.where(rng.uniform(size=n) < 0.05, 1.0, 0.0).astype(np.float32)
    L = B.make_layout(lay)
    ws = torch.zeros(B.qn_pack_workspace_size(n, L), device="cuda", dtype=torch.uint8)
    pkt = torch.zeros(B.qn_packet_max_bytes(n, L), device="cuda", dtype=torch.uint8)
    size = B.qn_pack_frame(n, Sd, L, up(lat), up(dec.view(np.int16), torch.int16), up(lp), up(gate), ws, pkt)
    got = bytes(pkt[:size].cpu().numpy().tobytes())
    assert got == OP.pack_frame(n, lat, lay.lat_dim, lay.attr_count, dec, lp, gate)


@pytest.mark.parametrize("n,seed,step", [(1, 0, 0), (1000, 7, 5), (300_001, (3 << 40) + 11, 123_456)])
def test_gate_noise_matches_oracle_philox(n, seed, step):
    from oracle import rng
    from paper_2412_04469_gb300 import binding as B
    u = torch.zeros(n, device="cuda")
    st = torch.tensor([step], device="cuda", dtype=torch.int32)
    B.qn_gate_uniform(n, seed, st, u)
    torch.cuda.synchronize()
    assert np.array_equal(u.cpu().numpy(), rng.gate_uniform(n, seed, step))


@pytest.mark.parametrize("n,latent", [(1000, 8), (40_000, 8), (3000, 4)])
def test_noisy_gate_decode_and_adjoint(n, latent):
    from oracle import rng
    from paper_2412_04469_gb300 import binding as B
    from paper_2412_04469_gb300.pipeline import HParams, QueenFrame
    deg = 1
    lay = S.DecoderLayout.default(sh_degree=deg, latent=latent)
    prev = S.make_scene(n, deg, 13)
    res = S.make_residuals(n, lay, 13)
    res.log_alpha[:] = np.random.default_rng(13).uniform(-1.5, 1.5, n).astype(np.float32)
    f = QueenFrame(prev, deg, lay, res.lat, res.dec, res.lp, res.log_alpha, HParams(lreg_mean=False))
    u = rng.gate_uniform(n, 99, 3)
    noise = torch.zeros(f.S, device="cuda")
    noise[:n] = up(u)
    f.c_gate = f.c_gate_train = B.make_gate(TAU, G0, G1, noise)
    f.decode()
    torch.cuda.synchronize()
    out, gate, lreg = oracle.decode(prev.astype(np.float64), res.lat, res.dec, res.lp, res.log_alpha, lay, TAU, G0,
                                    G1, noise=u)
    got = f.attrs.cpu().numpy()[:, :n]
    close(got[:3], out[:3], 1e-4, 1e-2, "position")
    close(f.gate.cpu().numpy()[:n], gate, 1e-4, 1e-2, "gate")
    assert float(f.lreg.item()) == pytest.approx(lreg, rel=1e-5)
    d_out = np.random.default_rng(14).standard_normal((prev.shape[0], n)).astype(np.float32)
    f.d_attrs[:, :n] = up(d_out)
    f.decode_bwd()
    torch.cuda.synchronize()
    want = oracle.decode_bwd(res.lat, res.dec, res.lp, res.log_alpha, lay, TAU, G0, G1, d_out, f.d_lreg, noise=u)
    close(f.d_lp.cpu().numpy()[:, :n], want[2], 1e-4, 0.05, "d_lp")
    close(f.d_log_alpha.cpu().numpy()[:n], want[3], 1e-4, 0.05, "d_log_alpha")


def test_noisy_gate_training_draws_per_step_and_replays():
    from paper_2412_04469_gb300 import binding as B
    from paper_2412_04469_gb300.pipeline import HParams, IterationGraph, QueenFrame, Rasterizer, training_iteration
    n, deg, W, H = 5000, 1, 96, 80
    lay = S.DecoderLayout.default(sh_degree=deg, latent=8)
    prev = S.make_scene(n, deg, 6)
    res = S.make_residuals(n, lay, 6)
    cams = [B.make_camera(c) for c in S.make_arc_cameras(2, W, H)]
    tg = [up(S.make_image(W, H, 60 + v)) for v in range(2)]
    outs, noises = [], []
    for graphs in (False, True):
        f = QueenFrame(prev, deg, lay, res.lat, res.dec, res.lp, res.log_alpha, HParams(gate_noise=True, gate_seed=5))
        r = Rasterizer(n, f.S, deg, W, H, 1 << 20)
        g = IterationGraph(f, r) if graphs else None
        seen = []
        for it in range(6):
            if g is None:
                training_iteration(f, r, cams[it % 2], tg[it % 2])
            else:
                g.run(it % 2, cams[it % 2], tg[it % 2])
            seen.append(f.noise[:n].clone())
        torch.cuda.synchronize()
        outs.append([t.clone() for t in (f.lat, f.dec, f.lp, f.log_alpha, r.loss)])
        noises.append(seen)
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    for a, b in zip(*noises):
        assert torch.equal(a, b)
    assert not torch.equal(noises[0][0], noises[0][1])          # fresh noise every step
