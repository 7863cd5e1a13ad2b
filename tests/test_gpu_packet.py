"""The compressed per-frame packet on the GPU (qn_pack_frame, qn_unpack_frame)
against the oracle: packets bit-identical to the oracle's on seeded inputs
(rounding ties, saturation, ragged last streams, no Gaussian at all); at the
full 300k-Gaussian size the frequency tables, the COO section and sampled
streams identical, every stream within its information content; the
unpacked A_t equal to the oracle's decode of the integer latents with the gate
binarised; corrupt packets rejected without a fault."""
import struct

import numpy as np
import pytest
import torch

import oracle
from oracle import packet as OP
from paper_2412_04469_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_04469_gb300 import build
    build.build()


def B():
    from paper_2412_04469_gb300 import binding
    return binding


def up(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _inputs(n, deg, latent, seed, stride_pad=5):
    """Seeded residual parameters shaped like a trained frame's: most latents
    round to 0, a tenth of the gates open."""
    lay = S.DecoderLayout.default(sh_degree=deg, latent=latent)
    rng = np.random.default_rng(seed)
    Sd = (n + stride_pad + 3) // 4 * 4
    lat = np.where(rng.uniform(size=(lay.n_latent, Sd)) < 0.8, rng.uniform(-0.49, 0.49, (lay.n_latent, Sd)),
                   rng.normal(0, 4, (lay.n_latent, Sd))).astype(np.float32)
    ties = np.array([0.5, 1.5, -2.5, 130.2, -200.0, 2.5], np.float32)
    k = min(n, ties.size)
    lat[0, :k] = ties[:k]
    dec = S.bf16_bits(rng.normal(0, 0.01, lay.n_dec).astype(np.float32))
    lp = rng.normal(0, 0.01, (3, Sd)).astype(np.float32)
    gate = np.where(rng.uniform(size=max(n, 1)) < 0.1, rng.uniform(0.0, 1.0, max(n, 1)), 0.0).astype(np.float32)
    return lay, Sd, lat, dec, lp, gate


def _gpu_pack(n, Sd, lay, lat, dec, lp, gate):
    L = B().make_layout(lay)
    ws = torch.zeros(max(B().qn_pack_workspace_size(n, L), 256), device="cuda", dtype=torch.uint8)
    pkt = torch.zeros(B().qn_packet_max_bytes(n, L), device="cuda", dtype=torch.uint8)
    size = B().qn_pack_frame(n, Sd, L, up(lat), up(dec.view(np.int16), torch.int16), up(lp), up(gate), ws, pkt)
    return bytes(pkt[:size].cpu().numpy().tobytes())


@pytest.mark.parametrize("n,deg,latent", [(0, 1, 8), (1, 0, 8), (100, 1, 8), (1025, 3, 8), (20_000, 3, 8),
                                          (3001, 2, 4)])
def test_packet_matches_oracle_bytes(n, deg, latent):
    lay, Sd, lat, dec, lp, gate = _inputs(n, deg, latent, n + deg)
    got = _gpu_pack(n, Sd, lay, lat, dec, lp, gate)
    want = OP.pack_frame(n, lat, lay.lat_dim, lay.attr_count, dec, lp, gate[:n])
    assert len(got) == len(want) and got == want


def _sections(data):
    magic, version, n, n_cat, ss, sb = struct.unpack_from("<6I", data, 0)
    pos = 24
    meta = [struct.unpack_from("<4I", data, pos + 16 * c) for c in range(n_cat)]
    pos += 16 * n_cat
    freqs = [np.frombuffer(data, "<u2", 256, pos + 512 * c) for c in range(n_cat)]
    pos += 512 * n_cat
    sizes = []
    for (L, A, ns, pb) in meta:
        sizes.append(np.frombuffer(data, "<u4", ns, pos).astype(np.int64))
        pos += 4 * ns
    starts = []
    for (L, A, ns, pb), sz in zip(meta, sizes):
        starts.append(pos + np.concatenate([[0], np.cumsum(sz)[:-1]]))
        pos += pb + (-pb % 4)
    for (L, A, ns, pb) in meta:
        pos += 2 * L * A + (-(2 * L * A) % 4)
    return meta, freqs, sizes, starts, pos


def test_packet_full_size():
    n, deg = 300_000, 3
    lay, Sd, lat, dec, lp, gate = _inputs(n, deg, 8, 11)
    got = _gpu_pack(n, Sd, lay, lat, dec, lp, gate)
    meta, freqs, sizes, starts, coo = _sections(got)
    syms = OP.latent_symbols(lat, lay.lat_dim, n)
    rng = np.random.default_rng(0)
    for c, s in enumerate(syms):
        f = OP.normalize_freqs(np.bincount(s, minlength=256))
        assert np.array_equal(freqs[c], f)
        ns = meta[c][2]
        assert ns == -(-s.size // OP.STREAM_SYMBOLS) and sizes[c].sum() == meta[c][3]
        for k in sorted(set(rng.choice(ns, 4, replace=False).tolist()) | {ns - 1}):
            chunk = s[k * OP.STREAM_SYMBOLS:(k + 1) * OP.STREAM_SYMBOLS]
            want = OP.rans_encode(chunk, f)
            assert got[starts[c][k]:starts[c][k] + sizes[c][k]] == want, (c, k)
        # every stream is within the 4-byte state of its information content
        for k in range(ns):
            chunk = s[k * OP.STREAM_SYMBOLS:(k + 1) * OP.STREAM_SYMBOLS]
            ideal = OP.entropy_bits(chunk, f) / 8
            assert ideal - 1 <= sizes[c][k] <= ideal + 5
    idx = np.nonzero(gate[:n])[0]
    (n_coo,) = struct.unpack_from("<I", got, coo)
    assert n_coo == idx.size and len(got) == coo + 4 + 16 * n_coo
    assert np.array_equal(np.frombuffer(got, "<u4", n_coo, coo + 4), idx)
    assert np.array_equal(np.frombuffer(got, "<f4", 3 * n_coo, coo + 4 + 4 * n_coo).reshape(3, n_coo), lp[:, idx])
    # mostly-zero latents: about a bit per latent, far below the 8 of raw int8
    assert sum(m[3] for m in meta) < 0.25 * sum(s.size for s in syms)


@pytest.mark.parametrize("n,deg", [(5000, 1), (300_000, 3)])
def test_unpack_matches_oracle_decode(n, deg):
    lay, Sd, lat, dec, lp, gate = _inputs(n, deg, 8, 21)
    prev = S.make_scene(n, deg, 22)
    data = _gpu_pack(n, Sd, lay, lat, dec, lp, gate)
    L = B().make_layout(lay)
    n_attr = prev.shape[0]
    prev_d = torch.zeros((n_attr, Sd), device="cuda")
    prev_d[:, :n] = up(prev)
    out = torch.zeros_like(prev_d)
    ws = torch.zeros(B().qn_unpack_workspace_size(n, Sd, L, len(data)), device="cuda", dtype=torch.uint8)
    B().qn_unpack_frame(data, n, Sd, n_attr, L, prev_d, out, ws)
    torch.cuda.synchronize()
    # the oracle: integer latents, the decoders, and the gate binarised
    lat_int = np.clip(np.rint(lat[:, :n]), -128, 127).astype(np.float32)
    dec_f = (dec.astype(np.uint32) << 16).view(np.float32)
    on = gate[:n] != 0
    la = np.where(on, 1e30, -1e30).astype(np.float32)
    want, g, _ = oracle.decode(prev.astype(np.float64), lat_int, dec_f, lp[:, :n], la, lay, 1.0, -0.5, 1.5)
    assert np.array_equal(g, on.astype(np.float64))
    got = out.cpu().numpy()[:, :n].astype(np.float64)
    pos_err = np.abs(got[:3] - want[:3]) / np.maximum(np.abs(want[:3]), 1e-2)
    assert pos_err.max() <= 1e-6
    res = got[3:] - prev[3:]
    ref = want[3:] - prev[3:].astype(np.float64)
    err = np.abs(res - ref) / np.maximum(np.abs(ref), 1e-2 * np.abs(ref).max())
    assert err.max() <= 2e-3


def test_corrupt_packets_are_rejected():
    n, deg = 20_000, 1
    lay, Sd, lat, dec, lp, gate = _inputs(n, deg, 8, 31)
    data = bytearray(_gpu_pack(n, Sd, lay, lat, dec, lp, gate))
    L = B().make_layout(lay)
    n_attr = S.n_attr(deg)
    prev = torch.zeros((n_attr, Sd), device="cuda")
    out = torch.zeros_like(prev)
    ws = torch.zeros(B().qn_unpack_workspace_size(n, Sd, L, len(data)) + 4096, device="cuda", dtype=torch.uint8)

    def rejected(buf, what):
        with pytest.raises(B().QueenError) as e:
            B().qn_unpack_frame(bytes(buf), n, Sd, n_attr, L, prev, out, ws)
        assert e.value.code == B().QN_ERR_INVALID_ARG, what

    rejected(data[:-1], "truncated")
    bad = bytearray(data)
    bad[0] ^= 1
    rejected(bad, "magic")
    meta, freqs, sizes, starts, coo = _sections(bytes(data))
    # move bytes from stream 0 of category 0 to stream 1: the sums still add
    # up, stream 0 now ends inside its own data and its decode runs out
    tab = 24 + 16 * len(meta) + 512 * len(meta)
    s0, s1 = int(sizes[0][0]), int(sizes[0][1])
    bad = bytearray(data)
    struct.pack_into("<2I", bad, tab, 4, s0 + s1 - 4)
    rejected(bad, "stream size")
    # a COO index past n
    bad = bytearray(data)
    (n_coo,) = struct.unpack_from("<I", bad, coo)
    assert n_coo > 1
    struct.pack_into("<I", bad, coo + 4 + 4 * (n_coo - 1), n + 5)
    rejected(bad, "COO index")
    # the context still works
    B().qn_unpack_frame(bytes(data), n, Sd, n_attr, L, prev, out, ws)
    torch.cuda.synchronize()
