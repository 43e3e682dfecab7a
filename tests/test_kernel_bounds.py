"""Integer bounds that the CUDA NTT butterflies rely on, checked with exact Python integers on
a model of their arithmetic (no GPU).

mul_shoup_lazy (he_common.cuh) estimates Shoup's quotient floor(a w' / 2^64) from three of the
four 32x32 partial products and forms a w - h q mod 2^64 as a w + h (2^64 - q).  The forward
butterflies keep values in [0, 8q) and the inverse ones in [0, 4q); both need q < 2^61, the
largest modulus the library accepts."""
import random

import pytest

M64 = (1 << 64) - 1


def lazy_shoup(a, w, wp, q):
    a0, a1, p0, p1 = a & 0xFFFFFFFF, a >> 32, wp & 0xFFFFFFFF, wp >> 32
    h = (a1 * p1 + ((a0 * p1) >> 32) + ((a1 * p0) >> 32)) & M64
    return (a * w + h * ((1 << 64) - q)) & M64, h


def _cases(rng, q):
    edge = [0, 1, q - 1, q, 2 * q - 1, 4 * q - 1, 8 * q - 1, M64, 1 << 63, (1 << 32) - 1, 1 << 32]
    return edge + [rng.getrandbits(64) for _ in range(300)]


@pytest.mark.parametrize("bits", [20, 42, 50, 58, 60, 61])
def test_lazy_shoup_product_is_congruent_and_below_4q(bits):
    rng = random.Random(bits)
    for _ in range(20):
        q = rng.randrange(1 << (bits - 1), 1 << bits) | 1
        for w in (0, 1, q - 1, rng.randrange(q)):
            wp = (w << 64) // q
            for a in _cases(rng, q):
                r, h = lazy_shoup(a, w, wp, q)
                exact = (a * wp) >> 64
                assert exact - 2 <= h <= exact
                assert r < 4 * q and r % q == (a * w) % q


def test_butterfly_ranges_fit_64_bits():
    """Forward: u < 8q reduced by 4q, x < 4q, outputs u + x and u - x + 4q in [0, 8q).
    Inverse: u, x < 4q, s = u + x reduced by 4q, d = u - x + 4q in (0, 8q), Shoup(d) < 4q.
    The largest value formed is below 8q, so every sum is exact for q < 2^61."""
    q = (1 << 61) - 1
    assert 8 * q <= M64
    u, x = 4 * q - 1, 4 * q - 1
    assert u + x < 8 * q and u - 0 + 4 * q < 8 * q and 0 - x + 4 * q > 0
    rng = random.Random(5)
    for _ in range(2000):
        qq = rng.randrange(1 << 40, 1 << 61) | 1
        w = rng.randrange(qq)
        wp = (w << 64) // qq
        u, v = rng.randrange(8 * qq), rng.randrange(8 * qq)
        if u >= 4 * qq:
            u -= 4 * qq
        x, _ = lazy_shoup(v, w, wp, qq)
        hi, lo = u + x, u - x + 4 * qq
        assert 0 <= hi < 8 * qq and 0 < lo < 8 * qq
        assert (hi - u - v * w) % qq == 0 and (lo - u + v * w) % qq == 0
