"""Integer bounds that the CUDA NTT butterflies rely on, checked with exact Python integers on
a model of their arithmetic (no GPU).

mul_shoup_lazy (he_common.cuh) estimates Shoup's quotient floor(a w' / 2^64) from three of the
four 32x32 partial products and forms a w - h q mod 2^64 as a w + h (2^64 - q).  The forward
butterflies of a 16-coefficient register block reduce u by 8q only in every other stage, so
values alternate between [0, 12q) and [0, 16q); the inverse ones stay in [0, 4q).  Both need
q < 2^60, the largest modulus the library accepts."""
import random

import pytest

M64 = (1 << 64) - 1


def lazy_shoup(a, w, wp, q):
    a0, a1, p0, p1 = a & 0xFFFFFFFF, a >> 32, wp & 0xFFFFFFFF, wp >> 32
    h = (a1 * p1 + ((a0 * p1) >> 32) + ((a1 * p0) >> 32)) & M64
    return (a * w + h * ((1 << 64) - q)) & M64, h


def lazy_shoup_words(a, w, wp, q):
    """The same product as the kernel forms it, from 32-bit multiply-adds only: h = H + t2 with
    H = a1 w'1 + hi(a0 w'1) and t2 = hi(a1 w'0), and h nq = H nq + t2 nq."""
    m, nq = 0xFFFFFFFF, (1 << 64) - q
    a0, a1, p0, p1, w0, w1, n0, n1 = a & m, a >> 32, wp & m, wp >> 32, w & m, w >> 32, nq & m, nq >> 32
    t2 = (a1 * p0) >> 32
    H = a1 * p1 + ((a0 * p1) >> 32)
    assert H <= M64
    h0, h1 = H & m, H >> 32
    acc = (a0 * w0 + h0 * n0 + t2 * n0) & M64
    hi = ((acc >> 32) + a0 * w1 + a1 * w0 + h0 * n1 + h1 * n0 + t2 * n1) & m
    return (hi << 32) | (acc & m)


def _cases(rng, q):
    edge = [0, 1, q - 1, q, 2 * q - 1, 4 * q - 1, 8 * q - 1, M64, 1 << 63, (1 << 32) - 1, 1 << 32]
    return edge + [rng.getrandbits(64) for _ in range(300)]


@pytest.mark.parametrize("bits", [20, 42, 50, 58, 60])
def test_lazy_shoup_product_is_congruent_and_below_4q(bits):
    rng = random.Random(bits)
    for _ in range(20):
        q = rng.randrange(1 << (bits - 1), 1 << bits) | 1
        for w in (0, 1, q - 1, rng.randrange(q)):
            wp = (w << 64) // q
            for a in _cases(rng, q):
                r, h = lazy_shoup(a, w, wp, q)
                assert lazy_shoup_words(a, w, wp, q) == r
                exact = (a * wp) >> 64
                assert exact - 2 <= h <= exact
                assert r < 4 * q and r % q == (a * w) % q


def _forward_block(v, ws, q, reduce_every_stage):
    """Radix-2 stages of one 16-coefficient register block as the forward kernel runs them:
    stage p pairs (j, j + t), t = 8 >> p; returns the values after each stage."""
    out = []
    for p in range(4):
        t = 8 >> p
        red = 4 * q if reduce_every_stage else 8 * q
        for b in range(8):
            grp, jj = b // t, 2 * (b // t) * t + b % t
            w = ws[p][grp]
            u = v[jj]
            if (reduce_every_stage or p & 1) and u >= red:
                u -= red
            x, _ = lazy_shoup(v[jj + t], w, (w << 64) // q, q)
            v[jj], v[jj + t] = u + x, u - x + 4 * q
        out.append(list(v))
    return out


def test_forward_butterfly_ranges_fit_64_bits():
    """Inputs below 12q (canonical on entry, below 12q after each block): stages 0 and 2 leave
    values below 16q, stages 1 and 3 below 12q, and every value is congruent to the textbook
    radix-2 result; the largest q allowed (2^60 - 1) keeps 16q < 2^64."""
    assert 16 * ((1 << 60) - 1) <= M64
    rng = random.Random(5)
    for trial in range(300):
        q = ((1 << 60) - 1 - 2 * trial) if trial < 5 else (rng.randrange(1 << 40, 1 << 60) | 1)
        ws = [[rng.randrange(q) for _ in range(8)] for _ in range(4)]
        v = [rng.randrange(12 * q) if trial % 2 else 12 * q - 1 - rng.randrange(4) for _ in range(16)]
        ref = [x % q for x in v]
        for p, lazy in enumerate(_forward_block(list(v), ws, q, False)):
            t = 8 >> p
            for b in range(8):
                grp, jj = b // t, 2 * (b // t) * t + b % t
                w = ws[p][grp]
                u, x = ref[jj], ref[jj + t] * w % q
                ref[jj], ref[jj + t] = (u + x) % q, (u - x) % q
            bound = 16 * q if p % 2 == 0 else 12 * q
            assert all(0 <= y < bound for y in lazy), (p, q)
            assert [y % q for y in lazy] == ref


def test_inverse_butterfly_ranges_fit_64_bits():
    """Inverse: u, x < 4q, s = u + x reduced by 4q, d = u - x + 4q in (0, 8q), Shoup(d) < 4q."""
    rng = random.Random(6)
    for _ in range(2000):
        qq = rng.randrange(1 << 40, 1 << 60) | 1
        w = rng.randrange(qq)
        u, x = rng.randrange(4 * qq), rng.randrange(4 * qq)
        s = u + x
        if s >= 4 * qq:
            s -= 4 * qq
        d = u - x + 4 * qq
        y, _ = lazy_shoup(d, w, (w << 64) // qq, qq)
        assert 0 <= s < 4 * qq and 0 < d < 8 * qq and 0 <= y < 4 * qq
        assert (s - u - x) % qq == 0 and (y - (u - x) * w) % qq == 0


def test_final_reduction_small_quotient_barrett():
    """The forward row pass reduces r < 16q to [0, q) with k = floor(floor(r / 2^(s-6)) mu6 / 2^12),
    mu6 = floor(mu / 2^57) where mu = floor(2^(s+63) / q) is the stored Barrett constant; k is
    floor(r / q) or one less, so one conditional subtraction finishes."""
    rng = random.Random(7)
    for _ in range(20000):
        s = rng.randrange(20, 61)
        q = rng.randrange(1 << (s - 1), 1 << s) | 1
        mu6 = ((1 << (s + 63)) // q) >> 57
        assert mu6 == (1 << (s + 6)) // q
        for r in (0, q - 1, q, 12 * q - 1, 16 * q - 1, rng.randrange(16 * q)):
            t = r >> (s - 6)
            assert t < 1 << 10
            k = (t * mu6) >> 12
            x = (r + k * ((1 << 64) - q)) & M64
            assert k * q <= r and x == r - k * q < 2 * q
            assert (x - q if x >= q else x) == r % q
