"""Pins of the packet oracle (App. B storage): the rANS coder against closed
forms worked out by hand (a one-symbol alphabet codes to its 4-byte state; a
uniform 256-symbol alphabet emits one byte per symbol whose values follow
from the update rule), invertibility on random and ragged inputs, code
lengths within a few bytes of the information content, the frequency
normalisation's invariants and edge cases, and the packet's round trip."""
import struct

import numpy as np
import pytest

from oracle import packet as P


def test_single_symbol_alphabet_codes_to_the_initial_state():
    f = np.zeros(256, np.int64)
    f[7] = P.M
    data = P.rans_encode(np.full(1000, 7, np.uint8), f)
    # f = M: x_max = 2^31, the update keeps x = L, nothing is emitted
    assert data == struct.pack("<I", 1 << 23)
    assert np.array_equal(P.rans_decode(data, 1000, f), np.full(1000, 7))


def test_uniform_alphabet_closed_form():
    # f_s = 16 = M / 256, c_s = 16 s.  From x = 2^23 the first step emits 0x00
    # and leaves 2^23 + 16 s; from x = 2^23 + 16 s + q (q < 16) a step emits
    # (16 s + q) & 255 = 16 (s mod 16) + q and leaves 2^23 + 16 s' + s // 16.
    # Coding runs backwards, so with s_n = 0: final state 2^23 + 16 s_0 +
    # s_1 // 16, emitted bytes e_0 = 0 and e_k = 16 (s_{n-k} mod 16) +
    # s_{n-k+1} // 16; the stream holds them in reverse after the state.
    rng = np.random.default_rng(0)
    s = rng.integers(0, 256, 300)
    n = len(s)
    f = np.full(256, 16, np.int64)
    data = P.rans_encode(s.astype(np.uint8), f)
    ext = list(s) + [0]
    e = [0] + [16 * (ext[n - k] % 16) + ext[n - k + 1] // 16 for k in range(1, n)]
    state = (1 << 23) + 16 * s[0] + s[1] // 16
    assert data == struct.pack("<I", state) + bytes(reversed(e))
    assert len(data) == n + 4


@pytest.mark.parametrize("n", [0, 1, 2, 100, 8191, 8192, 8193])
@pytest.mark.parametrize("kind", ["peaked", "uniform", "two"])
def test_round_trip_and_code_length(n, kind):
    rng = np.random.default_rng(n + len(kind))
    if kind == "peaked":
        sym = np.clip(np.rint(rng.laplace(128, 0.6, n)), 0, 255).astype(np.uint8)
    elif kind == "uniform":
        sym = rng.integers(0, 256, n).astype(np.uint8)
    else:
        sym = np.where(rng.uniform(size=n) < 0.97, 128, 129).astype(np.uint8)
    counts = np.bincount(sym, minlength=256)
    f = P.normalize_freqs(counts)
    data = P.rans_encode(sym, f)
    assert np.array_equal(P.rans_decode(data, n, f), sym)
    ideal = P.entropy_bits(sym, f) / 8
    # within the 4-byte state flush (and one byte of rounding) of the information content
    assert ideal - 1 <= len(data) <= ideal + 5


def test_normalize_freqs_invariants_and_edges():
    rng = np.random.default_rng(3)
    for _ in range(200):
        k = rng.integers(1, 257)
        counts = np.zeros(256, np.int64)
        idx = rng.choice(256, k, replace=False)
        counts[idx] = rng.integers(1, 10 ** rng.integers(1, 7), k)
        f = P.normalize_freqs(counts)
        assert f.sum() == P.M and np.array_equal(f > 0, counts > 0)
    one = np.zeros(256, np.int64)
    one[200] = 5
    assert P.normalize_freqs(one)[200] == P.M
    assert np.array_equal(P.normalize_freqs(np.full(256, 9)), np.full(256, 16))
    assert not P.normalize_freqs(np.zeros(256)).any()
    # proportional counts are kept exactly
    c = np.zeros(256, np.int64)
    c[[3, 4, 5]] = [1, 1, 2]
    f = P.normalize_freqs(c)
    assert (f[3], f[4], f[5]) == (1024, 1024, 2048)
    # 200 rare symbols bumped to 1 push the sum over M: the excess comes back
    # from the largest frequencies first
    c = np.zeros(256, np.int64)
    c[:200] = 1
    c[200:] = 10 ** 6
    f = P.normalize_freqs(c)
    assert f.sum() == P.M and (f[:200] == 1).all() and (f[200:] >= 1).all()
    # shortfall goes to the most frequent symbol (smallest index on ties)
    c = np.zeros(256, np.int64)
    c[[10, 11, 12]] = [3, 3, 1]
    f = P.normalize_freqs(c)
    assert f.sum() == P.M and f[10] == 4096 * 3 // 7 + (4096 - (2 * (4096 * 3 // 7) + 4096 // 7))


def test_packet_round_trip():
    rng = np.random.default_rng(5)
    n = 9000
    lat_dims, attr_counts = [8, 8, 8, 8], [4, 3, 1, 48]
    lat = np.where(rng.uniform(size=(32, n + 7)) < 0.8, 0.0, rng.normal(0, 3, (32, n + 7))).astype(np.float32)
    lat[0, :4] = [0.5, 1.5, -0.5, 200.0]                   # half to even, saturation
    dec = rng.integers(0, 1 << 16, sum(a * l for a, l in zip(attr_counts, lat_dims))).astype(np.uint16)
    lp = rng.normal(0, 0.01, (3, n + 7)).astype(np.float32)
    gate = np.where(rng.uniform(size=n) < 0.1, rng.uniform(0.01, 1, n), 0.0).astype(np.float32)
    data = P.pack_frame(n, lat, lat_dims, attr_counts, dec, lp, gate)
    out = P.unpack_frame(data)
    assert out["n"] == n and out["lat_dims"] == lat_dims and out["attr_counts"] == attr_counts
    want = np.clip(np.rint(lat[:, :n]), -128, 127) + 128
    assert want[0, :4].tolist() == [128, 130, 128, 255]
    got = np.concatenate([s.reshape(8, n) for s in out["symbols"]])
    assert np.array_equal(got, want)
    assert np.array_equal(out["dec_bf16"], dec)
    idx = np.nonzero(gate)[0]
    assert np.array_equal(out["coo_index"], idx)
    assert np.array_equal(out["coo_lp"], lp[:, idx].astype(np.float64))
    # mostly-zero latents code far below 8 bits per symbol
    assert len(data) < 0.3 * 32 * n
