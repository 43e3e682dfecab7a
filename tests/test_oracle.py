"""Pins for the CPU oracle against definitions, published values and invariants."""
import math

import numpy as np
import pytest

import oracle as O


def small_oracle(params, log_n=8, nq=6, keyseed=5):
    ch = dict(params[0]["toy"])
    ch["log_n"] = log_n
    ch["q"] = ch["q"][:nq]
    ch["h"] = min(ch["h"], (1 << log_n) // 2)
    o = O.Oracle(ch)
    o.keygen(keyseed)
    return o


def crt(residues, mods):
    X, M = 0, 1
    for r, m in zip(residues, mods):
        # solve X' = X mod M, X' = r mod m
        t = ((int(r) - X) * pow(M, -1, m)) % m
        X += M * t
        M *= m
    return X, M


def centred(x, m):
    x %= m
    return x - m if x > m // 2 else x


# ------------------------------------------------------------------ randomness
def test_splitmix_published_outputs(golden):
    g = 0x9e3779b97f4a7c15
    outs = [int(h, 16) for h in golden["splitmix64_outputs_state0"]]
    assert O.lib().orc_mix(g) == outs[0]
    assert O.lib().orc_mix((2 * g) & (2 ** 64 - 1)) == outs[1]


def test_samplers(toy_oracle):
    o = toy_oracle
    L = O.lib()
    e = np.array([L.orc_rng_gauss(o.ptr, 9, 77, i) for i in range(60000)])
    assert abs(e.mean()) < 0.05 and abs(e.std() - 3.2) < 0.05 and np.abs(e).max() <= 20
    q = o.q[1]
    u = np.array([L.orc_rng_uniform(9, 78, i, q) for i in range(20000)], dtype=np.float64)
    assert u.max() < q and abs(u.mean() / q - 0.5) < 0.01
    s = np.zeros(4096, dtype=np.int8)
    L.orc_hwt(4096, 64, 123, s.ctypes.data)
    assert (s != 0).sum() == 64 and set(np.unique(s)) <= {-1, 0, 1}


# ------------------------------------------------------------------ transforms
def test_ntt_product_equals_schoolbook(params):
    o = small_oracle(params)
    rng = np.random.default_rng(0)
    for t in range(3):
        q = o.q[t]
        a = rng.integers(0, q, o.n, dtype=np.uint64)
        b = rng.integers(0, q, o.n, dtype=np.uint64)
        sb = np.zeros(o.n, dtype=np.uint64)
        O.lib().orc_polymul_schoolbook(o.n, q, O.P(a), O.P(b), O.P(sb))
        assert np.array_equal(o.polymul(t, a, b), sb)
        assert np.array_equal(o.ntt(t, o.ntt(t, a), inverse=True), a)


def test_ntt_is_evaluation_at_odd_powers(params):
    o = small_oracle(params, log_n=5)
    q = o.q[1]
    psi = O.lib().orc_psi(o.ptr, 1)
    assert pow(psi, o.n, q) == q - 1
    a = np.random.default_rng(1).integers(0, q, o.n, dtype=np.uint64)
    ah = o.ntt(1, a)
    for k in range(o.n):
        r = pow(psi, 2 * k + 1, q)
        v = sum(int(a[i]) * pow(r, i, q) for i in range(o.n)) % q
        assert int(ah[k]) == v


def test_special_fft_is_canonical_embedding(params):
    o = small_oracle(params, log_n=8)
    rng = np.random.default_rng(2)
    w = rng.normal(size=o.n0) + 1j * rng.normal(size=o.n0)
    zeta = np.exp(1j * np.pi / o.n)
    g = np.array([pow(5, j, 2 * o.n) for j in range(o.n0)])
    V = zeta ** (np.outer(g, np.arange(o.n0)) % (2 * o.n))
    assert np.abs(o.special_fft(w) - V @ w).max() < 1e-11
    assert np.abs(o.special_fft(o.special_fft(w), inverse=True) - w).max() < 1e-13


def test_encode_definition(params):
    o = small_oracle(params, log_n=8)
    rng = np.random.default_rng(3)
    z = rng.uniform(-1, 1, o.n0) + 1j * rng.uniform(-1, 1, o.n0)
    scale = 2.0 ** 30
    pt = o.encode(z, scale, 2)
    t = o.decode_coeffs(pt, 2)
    # slots of the integer polynomial: t(zeta^{5^j})
    zeta = np.exp(1j * np.pi / o.n)
    g = np.array([pow(5, j, 2 * o.n) for j in range(o.n0)])
    Vf = zeta ** (np.outer(g, np.arange(o.n)) % (2 * o.n))
    assert np.abs(Vf @ t / scale - z).max() < o.n / scale
    # a real constant encodes to a constant polynomial
    pc = o.decode_coeffs(o.encode(np.full(o.n0, 0.75), scale, 2), 2)
    assert pc[0] == round(0.75 * scale) and np.all(pc[1:] == 0)


# ------------------------------------------------------------------ keys and ciphertexts
def test_public_and_switching_keys(params):
    o = small_oracle(params, log_n=6, nq=6)
    s = o.secret().astype(np.int64)
    assert (s != 0).sum() == o.chain["h"]
    mods = o.q + o.p
    nl = len(mods)

    def limb(v, m):
        return np.array([x % m for x in v.tolist()], dtype=np.uint64)

    alpha = o.chain["alpha"]
    pmod = [math.prod(o.p) % m for m in mods]
    for g in (0, o.galois(1), 2 * o.n - 1):
        # integer target secret s'
        if g == 0:
            sp = np.zeros(o.n, dtype=object)
            for i in range(o.n):
                for j in range(o.n):
                    k = i + j
                    v = int(s[i]) * int(s[j])
                    if k < o.n:
                        sp[k] += v
                    else:
                        sp[k - o.n] -= v
        else:
            sp = np.zeros(o.n, dtype=object)
            for i in range(o.n):
                k = (i * g) % (2 * o.n)
                if k < o.n:
                    sp[k] += int(s[i])
                else:
                    sp[k - o.n] -= int(s[i])
        nd = (len(o.q) + alpha - 1) // alpha
        for j in range(nd):
            b, a = o.key_digit(g, j)
            for t in range(nl):
                m = mods[t]
                as_ = o.polymul(t, a[t], limb(s, m)) if t < nl else None
                e = [(int(b[t][i]) + int(as_[i])) % m for i in range(o.n)]
                if t < len(o.q) and t // alpha == j:
                    e = [(e[i] - pmod[t] * (int(sp[i]) % m)) % m for i in range(o.n)]
                e = [centred(x, m) for x in e]
                assert max(abs(x) for x in e) <= 20, (g, j, t)


def test_tensor_is_exact_product(params):
    o = small_oracle(params, log_n=6)
    rng = np.random.default_rng(4)
    s = o.secret().astype(np.int64)
    a = O.Ct(np.stack([rng.integers(0, 1, (4, o.n), dtype=np.uint64)] * 2), 3, 1.0)
    for p in range(2):
        for t in range(4):
            a.data[p, t] = rng.integers(0, o.q[t], o.n, dtype=np.uint64)
    b = O.Ct(a.data[:, :, ::-1].copy(), 3, 1.0)
    d = o.tensor(a, b)
    for t in range(4):
        q = o.q[t]
        st = np.array([x % q for x in s.tolist()], dtype=np.uint64)
        s2 = o.polymul(t, st, st)
        lhs = (d[0, t].astype(object) + o.polymul(t, d[1, t], st).astype(object)
               + o.polymul(t, d[2, t], s2).astype(object)) % q
        da = (a.data[0, t].astype(object) + o.polymul(t, a.data[1, t], st).astype(object)) % q
        db = (b.data[0, t].astype(object) + o.polymul(t, b.data[1, t], st).astype(object)) % q
        rhs = o.polymul(t, np.array(da, dtype=np.uint64), np.array(db, dtype=np.uint64))
        assert np.array_equal(np.array(lhs, dtype=np.uint64), rhs)


def test_rescale_is_rounded_division(params):
    o = small_oracle(params, log_n=5)
    rng = np.random.default_rng(5)
    lv = 3
    data = np.zeros((2, lv + 1, o.n), dtype=np.uint64)
    for t in range(lv + 1):
        data[:, t] = rng.integers(0, o.q[t], (2, o.n), dtype=np.uint64)
    r = o.rescale(O.Ct(data, lv, 2.0 ** 40))
    mods = o.q[:lv + 1]
    for p in range(2):
        for k in range(o.n):
            X, _ = crt(data[p, :, k], mods)
            rt = centred(X % mods[-1], mods[-1])
            Y = (X - rt) // mods[-1]
            assert (X - rt) % mods[-1] == 0
            for t in range(lv):
                assert int(r.data[p, t, k]) == Y % mods[t]
    assert r.scale == 2.0 ** 40 / o.q[lv]


def test_modup_is_crt_lift_plus_small_multiple(params):
    """ModUp of hybrid key switching (Sec. 2.2): for every digit D (alpha consecutive primes),
    limbs inside D are copied, and every other limb t (Q or P) holds Y mod m_t for ONE integer
    Y = X + u Q_D, X the centred CRT value of the digit's residues (|X| <= Q_D / 2) and u small:
    the fast basis conversion with centred representatives has |Y| <= |D| Q_D / 2.  Centring
    also makes u average about 0 (representatives in [0, q_i) would put Y in [0, |D| Q_D) and
    give u a mean near |D| / 2)."""
    o = small_oracle(params, log_n=8, nq=8)
    rng = np.random.default_rng(9)
    lv, alpha = 6, o.chain["alpha"]
    d = np.stack([rng.integers(0, o.q[t], o.n, dtype=np.uint64) for t in range(lv + 1)])
    out = o.modup(d, lv)
    mods = list(o.q[:lv + 1]) + [int(v) for v in o.chain["p"]]
    assert out.shape == (-(-(lv + 1) // alpha), len(mods), o.n)
    us = []
    for j in range(out.shape[0]):
        D = list(range(j * alpha, min((j + 1) * alpha, lv + 1)))
        for k in range(o.n):
            X, QD = crt([int(d[i, k]) for i in D], [o.q[i] for i in D])
            X = centred(X, QD)
            bound = len(D) // 2 + 1
            u_seen = set()
            for t, mt in enumerate(mods):
                v = int(out[j, t, k])
                if t in D:
                    assert v == int(d[t, k])
                    continue
                cand = [u for u in range(-bound, bound + 1) if (X + u * QD - v) % mt == 0]
                assert len(cand) == 1, (j, k, t)
                u_seen.add(cand[0])
            assert len(u_seen) == 1, (j, k, u_seen)   # one integer Y on every limb
            us.append(u_seen.pop())
    assert abs(np.mean(us)) < 0.2


def test_relinearisation_noise_is_small(params):
    o = small_oracle(params, log_n=6)
    rng = np.random.default_rng(6)
    s = o.secret().astype(np.int64)
    lv = 4
    d = np.zeros((3, lv + 1, o.n), dtype=np.uint64)
    for t in range(lv + 1):
        d[:, t] = rng.integers(0, o.q[t], (3, o.n), dtype=np.uint64)
    k = o.relin(d, lv)
    mods = o.q[:lv + 1]
    Q = math.prod(mods)
    diffs = []
    for t in range(lv + 1):
        q = mods[t]
        st = np.array([x % q for x in s.tolist()], dtype=np.uint64)
        s2 = o.polymul(t, st, st)
        want = (d[0, t].astype(object) + o.polymul(t, d[1, t], st).astype(object)
                + o.polymul(t, d[2, t], s2).astype(object)) % q
        got = (k[0, t].astype(object) + o.polymul(t, k[1, t], st).astype(object)) % q
        diffs.append([(int(g) - int(w)) % q for g, w in zip(got, want)])
    worst = max(abs(centred(crt([diffs[t][i] for t in range(lv + 1)], mods)[0], Q)) for i in range(o.n))
    assert worst < 2 ** 20  # key-switching error, far below Q ~ 2^220


def test_relin_rescale_is_rounded_division(params):
    """The merged relinearisation + rescale: (M0 + M1 s) equals (d0 + d1 s + d2 s^2) / q_l over
    Q_{l-1} up to the key-switching and conversion error, checked with exact integers."""
    o = small_oracle(params, log_n=6)
    rng = np.random.default_rng(16)
    s = o.secret().astype(np.int64)
    lv = 4
    d = np.zeros((3, lv + 1, o.n), dtype=np.uint64)
    for t in range(lv + 1):
        d[:, t] = rng.integers(0, o.q[t], (3, o.n), dtype=np.uint64)
    got_ct = o.relin_rescale(d, lv)
    mods, mods_out = o.q[:lv + 1], o.q[:lv]
    Q, Qo = math.prod(mods), math.prod(mods_out)

    def dec(parts, ms):
        # coefficients of parts[0] + parts[1] s (+ parts[2] s^2) per limb, CRT-combined, centred
        limbs = []
        for t, q in enumerate(ms):
            st = np.array([x % q for x in s.tolist()], dtype=np.uint64)
            acc = parts[0][t].astype(object) + o.polymul(t, parts[1][t], st).astype(object)
            if len(parts) > 2:
                acc = acc + o.polymul(t, parts[2][t], o.polymul(t, st, st)).astype(object)
            limbs.append([int(v) % q for v in acc])
        M = math.prod(ms)
        return [centred(crt([limbs[t][i] for t in range(len(ms))], ms)[0], M) for i in range(o.n)]

    want = dec(d, mods)
    got = dec(got_ct, mods_out)
    ql = o.q[lv]
    worst = max(abs(g - w / ql) for g, w in zip(got, want))
    assert worst < 2 ** 12  # key-switch error / P plus the conversion error, far below Q_{l-1}
    assert Qo > 2 ** 100


def test_ciphertext_semantics(toy_oracle):
    o = toy_oracle
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, o.n0)
    y = rng.uniform(-1, 1, o.n0)
    a = o.encrypt(x, 20, 2.0 ** 40, 1, 0)
    b = o.encrypt(y, 20, 2.0 ** 40, 1, 1)
    assert np.abs(o.decrypt(a).real - x).max() < 2 ** -20
    pr = o.hmult(a, b)
    assert pr.level == 19 and np.abs(o.decrypt(pr).real - x * y).max() < 2 ** -20
    for r in (1, 5, o.n0 - 3):
        assert np.abs(o.decrypt(o.rotate(a, r)).real - np.roll(x, -r)).max() < 2 ** -20
    c = o.encrypt(x + 1j * y, 20, 2.0 ** 40, 2)
    assert np.abs(o.decrypt(o.conjugate(c)) - (x - 1j * y)).max() < 2 ** -20
    assert np.abs(o.decrypt(o.add(a, b)).real - (x + y)).max() < 2 ** -20


@pytest.mark.parametrize("deg", [7, 15, 63])
def test_poly_eval_depth_and_value(toy_oracle, deg):
    o = toy_oracle
    rng = np.random.default_rng(deg)
    u = rng.uniform(-1, 1, o.n0)
    c = rng.normal(size=deg + 1) / (1 + np.arange(deg + 1)) ** 1.5
    top = 20
    ct = o.encrypt(u, top, float(o.q[top]), 3)
    d = math.ceil(math.log2(deg + 1))
    r = o.poly_eval(ct, c, top - d, 2.0 ** 40)
    assert r.level == top - d
    assert np.abs(o.decrypt(r).real - O.cheb_eval(c, u)).max() < 2 ** -18


# ------------------------------------------------------------------ bootstrapping
def test_stc_places_slots_in_coefficients(toybts_oracle):
    o = toybts_oracle
    rng = np.random.default_rng(8)
    x = rng.uniform(-1, 1, o.n0)
    y = o.encrypt(x, 3, 2.0 ** 42, 5)
    for g in range(3):
        y = o.lintrans(y, 3, False, g, 1.0, float(o.q[y.level]))
    s = o.secret().astype(np.int64)
    q0 = o.q[0]
    st = np.array([v % q0 for v in s.tolist()], dtype=np.uint64)
    m = (y.data[0, 0].astype(object) + o.polymul(0, y.data[1, 0], st).astype(object)) % q0
    m = np.array([centred(int(v), q0) for v in m], dtype=np.float64) / y.scale
    bits = int(math.log2(o.n0))
    perm = np.array([int(format(i, "0%db" % bits)[::-1], 2) for i in range(o.n0)])
    assert np.abs(m[:o.n0] - x[perm]).max() < 2 ** -24
    assert np.abs(m[o.n0:]).max() < 2 ** -24


@pytest.mark.parametrize("inverse,which,level", [(False, 0, 3), (True, 1, 23)])
def test_shared_giant_step_moddown(toybts_oracle, inverse, which, level):
    """A linear-transform level whose giant-step rotations share one ModDown (their key-switch
    inner products summed over Q_l u P and divided by P once) against the textbook evaluation of
    the same level (every giant step a complete rotation with its own ModDown), both before the
    level's rescale.  Under exact decryption (c0 + c1 s per limb) the two differ only by the
    ModDowns' rounding: the same small integer on every limb, at most
    (giant steps) (1 + h)(alpha + 1)/2 in size.  A dropped key-switch term, a wrong sign or a
    wrong Galois element would put a residue of size ~q in the difference."""
    o = toybts_oracle
    rng = np.random.default_rng(12 + level)
    a = o.encrypt(rng.uniform(-1, 1, o.n0) + 1j * rng.uniform(-1, 1, o.n0), level, 2.0 ** 42, 13)
    pt_scale = float(o.q[level])
    shared = o.lintrans_unrescaled(a, 3, inverse, which, 1.0, pt_scale)
    text = o.lintrans_unrescaled(a, 3, inverse, which, 1.0, pt_scale, textbook=True)
    assert shared.scale == text.scale
    s = o.secret().astype(np.int64)
    deltas = []
    for t in range(level + 1):
        q = o.q[t]
        st = np.mod(s, q).astype(np.uint64)
        dec = []
        for ct in (shared, text):
            c0, c1 = ct.data[0, t].astype(object), o.polymul(t, ct.data[1, t], st).astype(object)
            dec.append((c0 + c1) % q)
        d = (dec[0] - dec[1]) % q
        deltas.append(np.where(d > q // 2, d - q, d).astype(np.int64))
    for t in range(1, level + 1):
        assert np.array_equal(deltas[t], deltas[0]), t    # one small integer polynomial
    # the 11 stages at N = 2^12 form levels of 4, 4, 3 stages (SlotToCoeff) and 3, 4, 4
    # (CoeffToSlot); both levels tested have r = 4 stages and several non-zero giant steps
    r = 4
    E, g = (1 << r) - 1, 1 << ((r + 2) // 2)
    giants = E // g + (E + g - 1) // g + 1
    bound = giants * (1 + o.chain["h"]) * (o.chain["alpha"] + 1) / 2
    assert 0 < np.abs(deltas[0]).max() <= bound, (np.abs(deltas[0]).max(), bound)
    # the shared form and the rescaling entry point agree after the rescale
    assert np.array_equal(o.rescale(shared).data, o.lintrans(a, 3, inverse, which, 1.0, pt_scale).data)


def test_bootstrap_precision(toybts_oracle, params):
    o = toybts_oracle
    em = params[2]["toybts"]
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, o.n0)
    ct = o.encrypt(x, 3, 2.0 ** 42, 5)
    b = o.bootstrap(ct, em, gain=16.0)
    assert b.level == o.chain["user_top_level"]
    err = np.abs(o.decrypt(b).real / 16.0 - x).max()
    assert err < 2 ** -22


# ------------------------------------------------------------------ FP64 references
def test_softmax_fp64_definition_and_lemma():
    rng = np.random.default_rng(10)
    x = rng.uniform(-20, 0, (5, 7))
    y = O.softmax_fp64(x)
    for r in range(5):
        den = sum(math.exp(v) for v in x[r])
        for i in range(7):
            assert abs(y[r, i] - math.exp(x[r, i]) / den) < 1e-15
    assert np.allclose(O.softmax_fp64(x - 3.7), y, atol=1e-15)          # Lemma 3.2a
    y2 = O.softmax_fp64(2 * x)                                         # Eq. doubling identity
    assert np.allclose(y2, y * y / np.sum(y * y, axis=1, keepdims=True), atol=1e-15)
    s = np.sum(y * y, axis=1)                                          # Lemma 3.4
    assert np.all(s >= 1 / 7 - 1e-15) and np.all(s <= 1 + 1e-15)


def test_alg2_with_exact_functions_is_softmax():
    rng = np.random.default_rng(11)
    n, M, k = 32, 64.0, 4
    x = rng.uniform(-M, 0, (9, n))
    y = np.exp(x / 2 ** k)
    for _ in range(k):
        lam = np.sum(y * y, axis=1, keepdims=True) ** -0.5
        z = lam * y
        y = z * z
    assert np.abs(y - O.softmax_fp64(x)).max() < 1e-14


def test_simulation_precision_and_invariants(params):
    rng = np.random.default_rng(12)
    for name in ("cfg1_n16_M8", "n256_M128", "toybts_n16_M32"):
        pl = params[1][name]
        x = rng.uniform(-pl["M"], 0, (64, pl["n"]))
        y, sums = O.simulate(x, pl)
        ref = O.softmax_fp64(x)
        assert np.abs(y - ref).max() < 2 ** -17, name
        assert np.abs(y.sum(axis=1) - 1).max() < 2 ** -16
        for j, S in enumerate(sums[1:], start=1):
            a = pl["iters"][j - 1]["alpha"]
            assert np.all(S >= (1 - a) ** 2 / pl["n"]) and np.all(S <= (1 + a) ** 2)


def test_pack_unpack_roundtrip():
    rng = np.random.default_rng(13)
    x = rng.normal(size=(64, 8))
    assert np.array_equal(O.unpack(O.pack(x, 2, 256), 8), x)
    x = rng.normal(size=(128, 16))
    p = O.pack(x, 1, 2048)
    assert p[0, 3 * 128 + 5] == x[5, 3]


# ------------------------------------------------------------------ end to end
def test_softmax_circuit_toy(toy_oracle, params):
    o = toy_oracle
    pl = params[1]["cfg1_n16_M8"]
    rng = np.random.default_rng(14)
    n = pl["n"]
    L = o.n0 // n
    x = rng.uniform(-pl["M"], 0, (L, n))
    top = o.chain["user_top_level"]
    ct = o.encrypt(O.pack(x, 1, o.n0)[0], top, (2 / pl["M"]) * o.q[top], 21)
    out = o.softmax([ct], pl)
    y = O.unpack(o.decrypt(out[0]).real[None, :], n)
    ref = O.softmax_fp64(x)
    assert np.abs(y - ref).max() < 2 ** -15
    assert np.abs(y.sum(axis=1) - 1).max() < 2 ** -14
    assert y.min() > -2 ** -15 and y.max() < 1 + 2 ** -15


def test_softmax_circuit_bootstrapped(toybts_oracle, params):
    o = toybts_oracle
    pl = params[1]["toybts_n16_M32"]
    rng = np.random.default_rng(15)
    n, m = pl["n"], 2
    L = m * o.n0 // n
    x = rng.uniform(-pl["M"], 0, (L, n))
    top = o.chain["user_top_level"]
    slots = O.pack(x, m, o.n0)
    cts = [o.encrypt(slots[i], top, (2 / pl["M"]) * o.q[top], 22, i) for i in range(m)]
    o.reset_counters()
    out = o.softmax(cts, pl, params[2]["toybts"])
    y = O.unpack(np.stack([o.decrypt(c).real for c in out]), n)
    assert np.abs(y - O.softmax_fp64(x)).max() < 2 ** -15
    # 3 sums, 1 lambda, and the main thread once (z, per ciphertext) on this schedule
    assert o.counters()["bts"] == 4 + m
