"""Pins of the oracle's random numbers (Philox4x32-10 + Box-Muller).

Philox (Salmon et al., SC'11) is pinned against an independent library:
numpy.random.Philox implements the 4x64-10 instance of the same round
structure, and the oracle's 4x64 routine must reproduce it bit for bit (numpy
advances the counter by one before each block).  The 4x32 instance used by the
method shares that structure with the published 32-bit multipliers and Weyl
constants; it is additionally pinned on the GPU against cuRAND's
Philox4_32_10 generator.  Gaussian statistics are checked against the
standard normal distribution.
"""
import math

import numpy as np
import pytest

from paper_2302_11719_gb300.inputs import DEFAULT_PARAMS


@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((7, 9), (0, 0, 0, 0)),
                                     ((2**64 - 1, 12345), (5, 2**63, 77, 1)),
                                     ((0xDEADBEEF, 1 << 40), (2**64 - 3, 0, 0, 9))])
def test_philox4x64_matches_numpy(orc, key, ctr):
    g = np.random.Philox(key=np.array(key, dtype=np.uint64),
                         counter=np.array(ctr, dtype=np.uint64))
    raw = [int(x) for x in g.random_raw(12)]
    c = list(ctr)
    for blk in range(3):
        # numpy increments the 256-bit counter (little-endian words) first
        carry = 1
        for i in range(4):
            s = c[i] + carry
            c[i] = s & (2**64 - 1)
            carry = s >> 64
        assert orc.philox4x64(c, key) == raw[4 * blk:4 * blk + 4]


def test_philox4x32_bits_balanced(orc):
    # 2^14 blocks of 4 words: every bit position is set about half the time
    n = 1 << 14
    words = np.array([orc.philox4x32((i, 3, 1, 0), (0, 0)) for i in range(n)], dtype=np.uint64)
    bits = np.array([(words >> b) & 1 for b in range(32)]).reshape(32, -1).mean(axis=1)
    sd = math.sqrt(0.25 / (4 * n))
    assert np.all(np.abs(bits - 0.5) < 6 * sd)
    # distinct counters -> distinct blocks (a keyed bijection)
    assert len({tuple(w) for w in words.tolist()}) == n


def test_philox4x32_key_and_counter_sensitivity(orc):
    base = orc.philox4x32((1, 2, 3, 4), (5, 6))
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        other = orc.philox4x32(c, (5, 6))
        flips = sum(bin(a ^ b).count("1") for a, b in zip(base, other))
        assert 30 < flips < 98          # avalanche: about half of 128 bits
    other = orc.philox4x32((1, 2, 3, 4), (5, 7))
    assert sum(bin(a ^ b).count("1") for a, b in zip(base, other)) > 30


def test_uniform_exact_and_open(orc):
    assert orc.uniform(0) == 0.5 * 2.0 ** -23
    assert orc.uniform(0xFFFFFFFF) == 1.0 - 0.5 * 2.0 ** -23
    for x in (0, 1 << 9, 0x12345678, 0xFFFFFFFF):
        u = orc.uniform(x)
        assert float(np.float32(u)) == u        # representable in float32
        assert 0.0 < u < 1.0


def test_box_muller_radius_and_angle(orc):
    # u1 = uniform(a): radius^2 = -2 ln u1; u2 = uniform(b): angle = 2 pi u2
    for a, b in [(0, 0), (123456789, 987654321), (0xFFFFFFFF, 1 << 31)]:
        z = orc.box_muller(a, b)
        u1, u2 = orc.uniform(a), orc.uniform(b)
        assert math.isclose(z[0] ** 2 + z[1] ** 2, -2 * math.log(u1), rel_tol=1e-12)
        ang = math.atan2(z[1], z[0]) % (2 * math.pi)
        assert math.isclose(ang, (2 * math.pi * u2) % (2 * math.pi), rel_tol=1e-9, abs_tol=1e-9)
    # u2 = 1/2 - 2^-24 (b = 2^31 - 2^9... ) gives an angle just below pi: z1 ~ 0+, z0 < 0
    z = orc.box_muller(1 << 31, (1 << 31) - 512)
    assert z[0] < 0 and 0 < z[1] < 1e-5


def test_gaussian_moments(orc):
    n = 200000
    m = orc.Model(dict(DEFAULT_PARAMS), np.zeros((4, 2), np.float32))
    z = np.array([orc.normal_pair(0, 0, 0, 0, k, t) for k in range(n // 20) for t in range(20)])
    assert z.shape == (n, 2)
    se = 1 / math.sqrt(n)
    assert np.all(np.abs(z.mean(axis=0)) < 5 * se)
    assert np.all(np.abs(z.var(axis=0) - 1) < 5 * math.sqrt(2) * se)
    assert abs(np.mean(z[:, 0] * z[:, 1])) < 5 * se
    kurt = np.mean(z ** 4, axis=0)
    assert np.all(np.abs(kurt - 3) < 5 * math.sqrt(96) * se)
    # control noise eps = (sigma_delta z0, sigma_a z1)
    e = orc.noise(m, 0, 0, 3, 7)
    zz = orc.normal_pair(0, 0, 0, 0, 3, 7)
    assert np.allclose(e, [np.float32(0.15) * zz[0], np.float32(0.3) * zz[1]], rtol=1e-15)


def test_noise_counter_layout(orc):
    # even and odd steps of a pair come from one Philox block: words (0,1) and (2,3)
    blk = orc.philox4x32((11, 4, 2, 0 | (5 << 8)), (0x2A, 0))
    z_even = orc.normal_pair(0x2A, 2, 5, 0, 11, 8)
    z_odd = orc.normal_pair(0x2A, 2, 5, 0, 11, 9)
    assert np.array_equal(z_even, orc.box_muller(blk[0], blk[1]))
    assert np.array_equal(z_odd, orc.box_muller(blk[2], blk[3]))
    # streams, instances and iterations are independent draws
    assert not np.array_equal(z_even, orc.normal_pair(0x2A, 2, 5, 1, 11, 8))
    assert not np.array_equal(z_even, orc.normal_pair(0x2A, 2, 6, 0, 11, 8))
    assert not np.array_equal(z_even, orc.normal_pair(0x2A, 3, 5, 0, 11, 8))
