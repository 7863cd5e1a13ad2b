"""Pins of the stochastic hard-concrete gate's oracle: Philox4x32-10 against
the known-answer vectors published with the generator (Salmon et al., SC
2011; the Random123 known-answer tests), the uniform mapping's range and
exactness, and the noisy decode: u = 1/2 reduces it to the deterministic
Eq. 6 exactly, L_reg (Eq. 8) does not see the noise, and the adjoint matches
central differences of the noisy forward."""
import numpy as np
import pytest

import oracle
from oracle import rng
from paper_2412_04469_gb300 import synthetic as S

KAT = [  # counter (4 words), key (2 words), output (4 words)
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,want", KAT)
def test_philox_known_answers(ctr, key, want):
    got = rng.philox4x32_10([np.uint64(v) for v in ctr], [np.uint64(v) for v in key])
    assert [int(v) for v in got] == list(want)


def test_gate_uniform_range_and_streams():
    u = rng.gate_uniform(100_000, seed=12345, step=7)
    assert u.dtype == np.float32 and (u > 0).all() and (u < 1).all()
    k = u.astype(np.float64) * (1 << 23) - 0.5
    assert np.array_equal(k, np.round(k))                      # ((x >> 9) + 1/2) / 2^23 exactly
    assert abs(u.mean() - 0.5) < 0.005 and abs(np.var(u) - 1 / 12) < 0.002
    assert np.array_equal(u, rng.gate_uniform(100_000, seed=12345, step=7))
    assert (u != rng.gate_uniform(100_000, seed=12345, step=8)).mean() > 0.99
    assert (u != rng.gate_uniform(100_000, seed=12346, step=7)).mean() > 0.99


def _problem(n, seed):
    lay = S.DecoderLayout.default(sh_degree=0, latent=4)
    prev = S.make_scene(n, 0, seed).astype(np.float64)
    res = S.make_residuals(n, lay, seed)
    res.log_alpha[:] = np.random.default_rng(seed).uniform(-1.5, 1.5, n).astype(np.float32)
    return lay, prev, res


def test_noisy_decode_reduces_to_eq6_and_keeps_lreg():
    lay, prev, res = _problem(200, 1)
    args = (prev, res.lat, res.dec, res.lp, res.log_alpha, lay, 0.3, -0.5, 1.01)
    det = oracle.decode(*args)
    half = oracle.decode(*args, noise=np.full(200, 0.5, np.float32))
    assert np.array_equal(half[0], det[0]) and np.array_equal(half[1], det[1])
    assert half[2] == pytest.approx(det[2], rel=1e-14)
    u = rng.gate_uniform(200, 3, 1)
    noisy = oracle.decode(*args, noise=u)
    assert noisy[2] == pytest.approx(det[2], rel=1e-15) and not np.array_equal(noisy[1], det[1])


def test_noisy_decode_adjoint_matches_central_differences():
    n = 40
    lay, prev, res = _problem(n, 2)
    u = rng.gate_uniform(n, 9, 4)
    rng_ = np.random.default_rng(5)
    d_out = rng_.standard_normal((prev.shape[0], n))
    d_lreg = 0.3
    _, _, d_lp, d_la = oracle.decode_bwd(res.lat, res.dec, res.lp, res.log_alpha, lay, 0.3, -0.5, 1.01, d_out,
                                         d_lreg, round_latents=False, noise=u)

    def f(la):
        out, _, lr = oracle.decode(prev, res.lat, res.dec, res.lp, la, lay, 0.3, -0.5, 1.01, round_latents=False,
                                   noise=u)
        return float((out * d_out).sum() + d_lreg * lr)

    la0 = res.log_alpha.astype(np.float64)
    checked = 0
    for i in range(n):
        g = oracle.decode(prev, res.lat, res.dec, res.lp, la0, lay, 0.3, -0.5, 1.01, noise=u)[1][i]
        if not 0.01 < g < 0.99:
            continue                                     # clipped: derivative 0 on one side only near the edge
        h = 1e-6
        lp_, lm_ = la0.copy(), la0.copy()
        lp_[i] += h
        lm_[i] -= h
        fd = (f(lp_) - f(lm_)) / (2 * h)
        assert d_la[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)
        checked += 1
    assert checked >= 5
