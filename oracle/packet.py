"""Oracle of the compressed per-frame packet (Sec. 3.2.1 and App. B, storage):
the integer latents of every category flattened and entropy coded, the
decoders stored as they are, and the position residuals of the Gaussians
whose gate is on stored in coordinate (COO) form.  Test infrastructure only;
shares no code with the CUDA path.

Entropy coder: range asymmetric numeral systems (rANS, Duda 2013), an
arithmetic-coding variant, with a static model per category and frame:
  - frequencies f_s quantised to M = 2^12 (normalize_freqs), cumulative c_s;
  - 32-bit state x kept in [L, 256 L), L = 2^23, renormalised a byte at a time;
  - encoding runs over the symbols in reverse: before coding s, while
    x >= (L >> 12 << 8) f_s, emit x & 255 and shift x right by 8; then
    x = (x // f_s) << 12 + x % f_s + c_s;
  - a stream is the final state as 4 little-endian bytes followed by the
    emitted bytes in reverse order of emission, so decoding reads forward:
    s = the symbol whose [c_s, c_s + f_s) holds x & (M - 1),
    x = f_s (x >> 12) + (x & (M - 1)) - c_s, then while x < L, x = x << 8 | next byte.
The flattened vector of a category (latent-major: latent dimension k, then
Gaussian i; symbol = integer latent + 128) is cut into streams of 8192
symbols coded independently (the last one ragged).

Packet layout (little-endian):
  u32 magic 0x4650_4e51 ('QNPF'), u32 version 1, u32 n, u32 n_cat,
  u32 stream_symbols, u32 scale_bits;
  per category: u32 lat_dim, u32 attr_count, u32 n_streams, u32 payload_bytes;
  per category: u16 freq[256];
  per category: u32 stream_bytes[n_streams];
  per category: the streams' bytes, concatenated, zero-padded to 4 bytes;
  per category: the decoder's bf16 bits, attr_count x lat_dim, row-major,
                zero-padded to 4 bytes;
  u32 n_coo, u32 index[n_coo] (increasing), f32 l_p[3][n_coo].
The gate is binarised for storage: Gaussian i is listed when g_i != 0 and its
position residual is l_p_i (the gate taken as 1), as App. B describes.
"""
from __future__ import annotations

import struct

import numpy as np

MAGIC = 0x46504E51
VERSION = 1
SCALE_BITS = 12
M = 1 << SCALE_BITS
RANS_L = 1 << 23
STREAM_SYMBOLS = 8192


def latent_symbols(lat, lat_dims, n):
    """Integer latents (Eq. 5 forward: round half to even, saturate to int8)
    of the FP32 continuous latents lat [sum lat_dims][>= n], + 128, as one
    uint8 vector per category, latent-major."""
    q = np.clip(np.rint(np.asarray(lat, np.float32)[:, :n]), -128, 127).astype(np.int64) + 128
    out, row = [], 0
    for L in lat_dims:
        out.append(q[row:row + L].reshape(-1).astype(np.uint8))
        row += L
    return out


def normalize_freqs(counts, scale_bits=SCALE_BITS):
    """Quantised frequencies summing to 2^scale_bits from symbol counts:
    f_s = max(1, floor(c_s 2^b / T)) for c_s > 0 (else 0), T = sum c.  A
    shortfall d > 0 goes to the most frequent symbol (the smallest such s);
    an excess is taken back in one pass over the symbols in order of
    decreasing f_s (then increasing s), each giving up to f_s - 1.  An empty
    histogram gives all zeros."""
    c = np.asarray(counts, np.int64)
    total = int(c.sum())
    Mb = 1 << scale_bits
    f = np.zeros(256, np.int64)
    if total == 0:
        return f
    for s in range(256):
        if c[s] > 0:
            f[s] = max(1, (int(c[s]) * Mb) // total)
    d = Mb - int(f.sum())
    if d > 0:
        best = max(range(256), key=lambda s: (int(c[s]), -s))
        f[best] += d
    elif d < 0:
        order = sorted(range(256), key=lambda s: (-int(f[s]), s))
        for s in order:
            if d == 0:
                break
            t = min(-d, int(f[s]) - 1)
            if t > 0:
                f[s] -= t
                d += t
    assert int(f.sum()) == Mb
    return f


def _cum(freqs):
    f = np.asarray(freqs, np.int64)
    return np.concatenate([[0], np.cumsum(f)[:-1]])


def rans_encode(symbols, freqs):
    """One rANS stream of the symbols (uint8 values) under freqs (sum M)."""
    f = [int(v) for v in freqs]
    c = [int(v) for v in _cum(freqs)]
    x = RANS_L
    emitted = bytearray()
    for s in reversed([int(v) for v in symbols]):
        fs = f[s]
        assert fs > 0, "symbol with zero frequency"
        x_max = ((RANS_L >> SCALE_BITS) << 8) * fs
        while x >= x_max:
            emitted.append(x & 0xFF)
            x >>= 8
        x = ((x // fs) << SCALE_BITS) + (x % fs) + c[s]
    return struct.pack("<I", x) + bytes(reversed(emitted))


def rans_decode(data, count, freqs):
    """count symbols from one rANS stream."""
    f = [int(v) for v in freqs]
    c = [int(v) for v in _cum(freqs)]
    slot2sym = np.repeat(np.arange(256), np.asarray(freqs, np.int64))
    x = struct.unpack_from("<I", data, 0)[0]
    pos = 4
    out = np.zeros(count, np.uint8)
    for k in range(count):
        slot = x & (M - 1)
        s = int(slot2sym[slot])
        out[k] = s
        x = f[s] * (x >> SCALE_BITS) + slot - c[s]
        while x < RANS_L:
            x = (x << 8) | data[pos]
            pos += 1
    return out


def encode_category(symbols, stream_symbols=STREAM_SYMBOLS):
    """(freqs, [stream bytes]) of one category's symbol vector."""
    counts = np.bincount(np.asarray(symbols, np.int64), minlength=256)
    freqs = normalize_freqs(counts)
    streams = [rans_encode(symbols[k:k + stream_symbols], freqs) for k in range(0, len(symbols), stream_symbols)]
    return freqs, streams


def _pad4(b: bytes) -> bytes:
    return b + b"\0" * (-len(b) % 4)


def pack_frame(n, lat, lat_dims, attr_counts, dec_bf16, lp, gate):
    """The packet of one frame.  lat [sum lat_dims][>= n] f32, dec_bf16 the
    concatenated row-major decoder blocks as uint16 bf16 bits, lp [3][>= n]
    f32, gate [n] (g_i; listed where != 0)."""
    syms = latent_symbols(lat, lat_dims, n)
    cats = [encode_category(s) for s in syms]
    head = struct.pack("<6I", MAGIC, VERSION, n, len(lat_dims), STREAM_SYMBOLS, SCALE_BITS)
    for L, A, (fr, st) in zip(lat_dims, attr_counts, cats):
        head += struct.pack("<4I", L, A, len(st), sum(len(b) for b in st))
    for fr, _ in cats:
        head += np.asarray(fr, "<u2").tobytes()
    for _, st in cats:
        head += np.asarray([len(b) for b in st], "<u4").tobytes()
    body = b"".join(_pad4(b"".join(st)) for _, st in cats)
    dec = np.asarray(dec_bf16, np.uint16)
    off = 0
    for L, A in zip(lat_dims, attr_counts):
        body += _pad4(dec[off:off + L * A].astype("<u2").tobytes())
        off += L * A
    idx = np.nonzero(np.asarray(gate)[:n] != 0)[0].astype(np.uint32)
    body += struct.pack("<I", len(idx)) + idx.astype("<u4").tobytes()
    body += np.asarray(lp, np.float32)[:, idx].astype("<f4").tobytes()
    return head + body


def unpack_frame(data):
    """Inverse of pack_frame: dict with n, lat_dims, attr_counts, symbols (per
    category), dec_bf16 (concatenated), coo_index, coo_lp [3][n_coo]."""
    magic, version, n, n_cat, stream_symbols, scale_bits = struct.unpack_from("<6I", data, 0)
    assert magic == MAGIC and version == VERSION and scale_bits == SCALE_BITS
    pos = 24
    meta = []
    for _ in range(n_cat):
        meta.append(struct.unpack_from("<4I", data, pos))
        pos += 16
    freqs = []
    for _ in range(n_cat):
        freqs.append(np.frombuffer(data, "<u2", 256, pos).astype(np.int64))
        pos += 512
    sizes = []
    for (L, A, ns, pb) in meta:
        sizes.append(np.frombuffer(data, "<u4", ns, pos).astype(np.int64))
        pos += 4 * ns
    symbols = []
    for (L, A, ns, pb), fr, sz in zip(meta, freqs, sizes):
        total = L * n
        out, p = [], pos
        for k in range(ns):
            cnt = min(stream_symbols, total - k * stream_symbols)
            out.append(rans_decode(data[p:p + int(sz[k])], cnt, fr))
            p += int(sz[k])
        symbols.append(np.concatenate(out) if out else np.zeros(0, np.uint8))
        pos += pb + (-pb % 4)
    dec = []
    for (L, A, ns, pb) in meta:
        dec.append(np.frombuffer(data, "<u2", L * A, pos))
        pos += 2 * L * A + (-(2 * L * A) % 4)
    (n_coo,) = struct.unpack_from("<I", data, pos)
    pos += 4
    idx = np.frombuffer(data, "<u4", n_coo, pos).astype(np.int64)
    pos += 4 * n_coo
    lp = np.frombuffer(data, "<f4", 3 * n_coo, pos).reshape(3, n_coo)
    pos += 12 * n_coo
    assert pos == len(data)
    return {"n": n, "lat_dims": [m[0] for m in meta], "attr_counts": [m[1] for m in meta], "freqs": freqs,
            "symbols": symbols, "dec_bf16": np.concatenate(dec) if dec else np.zeros(0, np.uint16),
            "coo_index": idx, "coo_lp": lp.astype(np.float64)}


def entropy_bits(symbols, freqs):
    """Information content of the symbols under the quantised model, in bits
    (the length arithmetic coding approaches)."""
    f = np.asarray(freqs, np.float64)
    s = np.asarray(symbols, np.int64)
    return float(-np.log2(f[s] / M).sum())
