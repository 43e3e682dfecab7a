"""GPU path (C ABI through the thin binding) against the CPU oracle.

Ciphertexts are compared limb by limb in coefficient form, bit for bit: the two sides use
different NTT orderings and roots, so equality in coefficient form is independent of them.
Decrypted values are compared with the FP64 references within the stated tolerances."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2410_11184_gb300 import he  # noqa: E402

SEED = 7


def _rand_ct(o, level, rng, nct=1):
    d = np.zeros((nct, 2, level + 1, o.n), dtype=np.uint64)
    for t in range(level + 1):
        d[:, :, t] = rng.integers(0, o.q[t], (nct, 2, o.n), dtype=np.uint64)
    return d


@pytest.fixture(scope="module")
def toy(params):
    ch = params[0]["toy"]
    g = he.Context(ch)
    g.keygen(SEED, rot_steps=[1, 3, 5, 64])
    o = O.Oracle(ch)
    o.keygen(SEED)
    return g, o


@pytest.fixture(scope="module")
def toybts(params):
    ch = params[0]["toybts"]
    em = params[2]["toybts"]
    g = he.Context(ch, em)
    g.keygen(SEED, rot_steps=[1])
    o = O.Oracle(ch)
    o.keygen(SEED)
    return g, o, em


def test_library_exports_and_bounded_wait(toy):
    g, _ = toy
    assert he.lib().he_ring_degree(g.h) == 4096
    assert g.selftest_bounded_wait(1000) == -6  # HE_ETIMEOUT, context still usable
    assert g.counters()["ks"] >= 0


def test_ntt_product_matches_oracle(toy):
    g, o = toy
    rng = np.random.default_rng(1)
    lv = 4
    a = _rand_ct(o, lv, rng)
    a[:, 1] = 0
    b = np.stack([rng.integers(0, o.q[t], o.n, dtype=np.uint64) for t in range(lv + 1)])
    ga = g.from_coeff(a, lv, 1.0)
    pt = torch.from_numpy(b.view(np.int64).reshape(-1).copy()).to(g.device)
    g.ntt(pt, 1, lv + 1)
    g.mul_plain(ga, pt)
    out = g.to_coeff(ga)
    for t in range(lv + 1):
        assert np.array_equal(out[0, 0, t], o.polymul(t, a[0, 0, t], b[t]))
    # inverse . forward = identity
    assert np.array_equal(g.to_coeff(g.from_coeff(a, lv, 1.0)), a)


def test_encode_bit_exact(toy):
    g, o = toy
    rng = np.random.default_rng(2)
    z = rng.uniform(-1, 1, o.n0) + 1j * rng.uniform(-1, 1, o.n0)
    for scale in (2.0 ** 40, float(o.q[7]) * 3.5, 2.0 ** 70):
        pt = g.encode(z, scale, 7)
        g.ntt(pt, 1, 8, inverse=True)
        got = pt.cpu().numpy().view(np.uint64).reshape(8, o.n)
        assert np.array_equal(got, o.encode(z, scale, 7))


def test_encrypt_bit_exact_and_decrypt(toy):
    g, o = toy
    rng = np.random.default_rng(3)
    z = rng.uniform(-1, 1, o.n0)
    for idx in (0, 5):
        gc = g.encrypt_slots(z, 20, 2.0 ** 40, 99, ct_index=idx)
        oc = o.encrypt(z, 20, 2.0 ** 40, 99, idx)
        assert np.array_equal(g.to_coeff(gc)[0], oc.data)
        assert np.abs(g.decrypt_slots(gc).real - z).max() < 2 ** -20


def test_rescale_hmult_relin_bit_exact(toy):
    g, o = toy
    rng = np.random.default_rng(4)
    x, y = rng.uniform(-1, 1, o.n0), rng.uniform(-1, 1, o.n0)
    a, b = o.encrypt(x, 12, 2.0 ** 40, 5, 0), o.encrypt(y, 11, 2.0 ** 40, 5, 1)
    ga, gb = g.from_coeff(a.data, 12, a.scale), g.from_coeff(b.data, 11, b.scale)
    r = o.rescale(a)
    gr = g.rescale(ga)
    assert np.array_equal(g.to_coeff(gr)[0], r.data) and gr.scale == r.scale
    p = o.hmult(a, b)
    gp = g.hmult(ga, gb)
    assert gp.level == p.level and gp.scale == p.scale
    assert np.array_equal(g.to_coeff(gp)[0], p.data)
    d = np.stack([rng.integers(0, o.q[t], (3, o.n), dtype=np.uint64) for t in range(6)], axis=1)
    dt = torch.from_numpy(d.view(np.int64).reshape(-1).copy()).to(g.device)
    g.ntt(dt, 3, 6)
    gk = g.relinearize(dt, 5, 1)
    assert np.array_equal(g.to_coeff(gk)[0], o.relin(d, 5))


def test_rotations_bit_exact(toy):
    g, o = toy
    rng = np.random.default_rng(5)
    a = o.encrypt(rng.uniform(-1, 1, o.n0) + 1j * rng.uniform(-1, 1, o.n0), 9, 2.0 ** 40, 6)
    ga = g.from_coeff(a.data, 9, a.scale)
    for r in (1, 3, 64):
        assert np.array_equal(g.to_coeff(g.rotate(ga, r))[0], o.rotate(a, r).data)
    assert np.array_equal(g.to_coeff(g.conjugate(ga))[0], o.conjugate(a).data)


@pytest.mark.parametrize("deg", [7, 15, 63])
def test_poly_eval_bit_exact(toy, deg):
    g, o = toy
    rng = np.random.default_rng(deg)
    c = rng.normal(size=deg + 1) / (1 + np.arange(deg + 1)) ** 1.5
    a = o.encrypt(rng.uniform(-1, 1, o.n0), 20, float(o.q[20]), 8)
    d = math.ceil(math.log2(deg + 1))
    r = o.poly_eval(a, c, 20 - d, 2.0 ** 40)
    gr = g.poly_eval(g.from_coeff(a.data, 20, a.scale), c, 20 - d, 2.0 ** 40)
    assert gr.scale == r.scale
    assert np.array_equal(g.to_coeff(gr)[0], r.data)


def test_lintrans_and_modraise_bit_exact(toybts):
    g, o, em = toybts
    rng = np.random.default_rng(6)
    a = o.encrypt(rng.uniform(-1, 1, o.n0), 3, 2.0 ** 42, 9)
    ga = g.from_coeff(a.data, 3, a.scale)
    for which in range(3):
        r = o.lintrans(a, 3, False, which, 16.0 if which == 0 else 1.0, float(o.q[a.level]))
        gr = g.lintrans(ga, 3, False, which, 16.0 if which == 0 else 1.0, float(o.q[a.level]))
        assert np.array_equal(g.to_coeff(gr)[0], r.data), which
        a, ga = r, gr
    top = len(o.q) - 1
    mr = o.mod_raise(a, top)
    assert np.array_equal(g.to_coeff(g.mod_raise(ga, top))[0], mr.data)
    r = o.lintrans(mr, 3, True, 0, 1.0, float(o.q[top]))
    gr = g.lintrans(g.from_coeff(mr.data, top, mr.scale), 3, True, 0, 1.0, float(o.q[top]))
    assert np.array_equal(g.to_coeff(gr)[0], r.data)


def test_bootstrap_bit_exact(toybts):
    g, o, em = toybts
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, o.n0)
    a = o.encrypt(x, 3, 2.0 ** 42, 10)
    r = o.bootstrap(a, em, gain=16.0)
    gr = g.bootstrap(g.from_coeff(a.data, 3, a.scale), 16.0, 2.0 ** 42)
    assert gr.level == r.level and gr.scale == r.scale
    assert np.array_equal(g.to_coeff(gr)[0], r.data)
    assert np.abs(g.decrypt_slots(gr).real / 16.0 - x).max() < 2 ** -22


def test_softmax_toy_bit_exact(toy, params):
    g, o = toy
    pl = params[1]["cfg1_n16_M8"]
    n = pl["n"]
    g.keygen_softmax(n, 1)
    rng = np.random.default_rng(8)
    L = o.n0 // n
    x = rng.uniform(-pl["M"], 0, (L, n))
    gc = g.encrypt(x, n, 1, pl["M"], 31)
    top = o.chain["user_top_level"]
    oc = o.encrypt(O.pack(x, 1, o.n0)[0], top, (2 / pl["M"]) * o.q[top], 31, 0)
    assert np.array_equal(g.to_coeff(gc)[0], oc.data)
    g.softmax(gc, pl)
    out = o.softmax([oc], pl)[0]
    assert gc.level == out.level and gc.scale == out.scale
    assert np.array_equal(g.to_coeff(gc)[0], out.data)
    y = g.decrypt(gc, n)
    assert np.abs(y - O.softmax_fp64(x)).max() < 2 ** -15


@pytest.mark.parametrize("batched", [True, False])
def test_softmax_bootstrapped_bit_exact(toybts, params, batched):
    g, o, em = toybts
    pl = params[1]["toybts_n16_M32"]
    n, m = pl["n"], 2
    g.keygen_softmax(n, m)
    rng = np.random.default_rng(9)
    L = m * o.n0 // n
    x = rng.uniform(-pl["M"], 0, (L, n))
    gc = g.encrypt(x, n, m, pl["M"], 32)
    top = o.chain["user_top_level"]
    slots = O.pack(x, m, o.n0)
    ocs = [o.encrypt(slots[i], top, (2 / pl["M"]) * o.q[top], 32, i) for i in range(m)]
    g.softmax(gc, pl, batched=batched)
    outs = o.softmax(ocs, pl, em)
    assert gc.level == outs[0].level and gc.scale == outs[0].scale
    got = g.to_coeff(gc)
    for i in range(m):
        assert np.array_equal(got[i], outs[i].data), i
    assert np.abs(g.decrypt(gc, n) - O.softmax_fp64(x)).max() < 2 ** -15


def test_softmax_graph_replay_bit_exact(toybts, params):
    """he_softmax_graph: captured on the first call, replayed on the next ones; every result
    equals the oracle's Softmax limb for limb, and the replay counts the captured launches."""
    g, o, em = toybts
    pl = params[1]["toybts_n16_M32"]
    n, m = pl["n"], 2
    g.keygen_softmax(n, m)
    rng = np.random.default_rng(19)
    L = m * o.n0 // n
    x = rng.uniform(-pl["M"], 0, (L, n))
    src = g.encrypt(x, n, m, pl["M"], 33)
    top = o.chain["user_top_level"]
    slots = O.pack(x, m, o.n0)
    outs = o.softmax([o.encrypt(slots[i], top, (2 / pl["M"]) * o.q[top], 33, i) for i in range(m)], pl, em)
    work = g.like(src)
    per_call = []
    for call in range(3):
        work.tensor.copy_(src.tensor)
        work.level, work.scale, work.n_ct = src.level, src.scale, src.n_ct
        l0 = g.launch_count()
        g.softmax(work, pl, graph=True)
        per_call.append(g.launch_count() - l0)
        assert work.level == outs[0].level and work.scale == outs[0].scale, call
        got = g.to_coeff(work)
        for i in range(m):
            assert np.array_equal(got[i], outs[i].data), (call, i)
    # the first call also ran the circuit once eagerly to fill the caches
    assert per_call[1] == per_call[2] > 0 and per_call[0] >= 2 * per_call[1]


def test_large_batch_paths_bit_exact(toybts):
    """Batches of more than 4 ciphertexts take the per-digit ModUp, per-rotation key switches and
    separate giant-step ModUps (smaller batches take the merged launches): 6 ciphertexts through
    multiplication, rotation, a CoeffToSlot level and bootstrapping, each against the oracle."""
    g, o, em = toybts
    rng = np.random.default_rng(17)
    m = 6
    lv = 5
    cts = [o.encrypt(rng.uniform(-1, 1, o.n0), lv, 2.0 ** 42, 40 + i) for i in range(m)]
    ga = g.from_coeff(np.stack([c.data for c in cts]), lv, cts[0].scale)
    assert ga.n_ct == m
    gp = g.hmult(ga, ga)
    got = g.to_coeff(gp)
    for i in range(m):
        assert np.array_equal(got[i], o.hmult(cts[i], cts[i]).data), ("hmult", i)
    got = g.to_coeff(g.rotate(ga, 1))
    for i in range(m):
        assert np.array_equal(got[i], o.rotate(cts[i], 1).data), ("rotate", i)
    b3 = [o.encrypt(rng.uniform(-1, 1, o.n0), 3, 2.0 ** 42, 60 + i) for i in range(m)]
    gb = g.from_coeff(np.stack([c.data for c in b3]), 3, b3[0].scale)
    got = g.to_coeff(g.lintrans(gb, 3, False, 0, 16.0, float(o.q[3])))
    for i in range(m):
        assert np.array_equal(got[i], o.lintrans(b3[i], 3, False, 0, 16.0, float(o.q[3])).data), ("lintrans", i)
    gr = g.bootstrap(gb, 16.0, 2.0 ** 42)
    got = g.to_coeff(gr)
    for i in range(m):
        r = o.bootstrap(b3[i], em, gain=16.0)
        assert gr.level == r.level and gr.scale == r.scale
        assert np.array_equal(got[i], r.data), ("bootstrap", i)


def test_second_keygen_replaces_every_key(params):
    """A second he_keygen with another seed replaces the secret and every evaluation key: a
    multiplication and a rotation afterwards equal the oracle's under the second seed, limb for
    limb, and the Softmax rotation keys must be generated again."""
    ch = params[0]["toy"]
    g = he.Context(ch)
    g.keygen(SEED, rot_steps=[1])
    g.keygen_softmax(16, 1)
    g.keygen(SEED + 1, rot_steps=[1])
    o = O.Oracle(ch)
    o.keygen(SEED + 1)
    rng = np.random.default_rng(21)
    a = o.encrypt(rng.uniform(-1, 1, o.n0), 8, 2.0 ** 40, 3, 0)
    b = o.encrypt(rng.uniform(-1, 1, o.n0), 8, 2.0 ** 40, 3, 1)
    ga, gb = g.from_coeff(a.data, 8, a.scale), g.from_coeff(b.data, 8, b.scale)
    assert np.array_equal(g.to_coeff(g.hmult(ga, gb))[0], o.hmult(a, b).data)
    assert np.array_equal(g.to_coeff(g.rotate(ga, 1))[0], o.rotate(a, 1).data)
    # the stride-128 rotation key of the first secret's he_keygen_softmax(16, 1) is gone
    with pytest.raises(RuntimeError, match="-5"):
        g.rotate(ga, 128)


@pytest.mark.parametrize("mode", ["batched", "plain", "graph"])
def test_softmax_alg4_bit_exact(toybts, params, mode):
    """Alg. 4 (version B, Sec. 4.3) with the auxiliary thread of Alg. 3, two ciphertexts of the
    many-ciphertext packing: every output limb equals the oracle's, in the batched form, the
    per-ciphertext form and by graph replay; only the auxiliary ciphertext is bootstrapped."""
    g, o, em = toybts
    pl = he.load_plans_b()["toybts_n16_M32_B"]
    n, m = pl["n"], 2
    g.keygen_softmax(n, m)
    rng = np.random.default_rng(23)
    L = m * o.n0 // n
    x = rng.uniform(-pl["M"], 0, (L, n))
    gc = g.encrypt(x, n, m, pl["M"], 34)
    top = o.chain["user_top_level"]
    slots = O.pack(x, m, o.n0)
    outs = o.softmax_b([o.encrypt(slots[i], top, (2 / pl["M"]) * o.q[top], 34, i) for i in range(m)], pl, em)
    c0 = g.counters()
    if mode == "graph":
        work = g.like(gc)
        for _ in range(2):
            work.tensor.copy_(gc.tensor)
            work.level, work.scale, work.n_ct = gc.level, gc.scale, gc.n_ct
            g.softmax(work, pl, graph=True)
        gc = work
    else:
        g.softmax(gc, pl, batched=mode == "batched")
        # bootstrapping calls: S_j and lambda_j in each of the k rounds, nothing of the main thread
        assert g.counters()["bts"] - c0["bts"] == 2 * pl["k"]
    assert gc.level == outs[0].level and gc.scale == outs[0].scale
    got = g.to_coeff(gc)
    for i in range(m):
        assert np.array_equal(got[i], outs[i].data), i
    assert np.abs(g.decrypt(gc, n) - O.softmax_fp64(x)).max() < 2 ** -15


@pytest.mark.parametrize("split", [(2, 2), (1, 3)])
def test_softmax_alg4_split_shares_equal_unsplit(toybts, split):
    """Alg. 4 split over shares of the main-thread ciphertexts (the multi-device form: one share
    per device, the shares' sums of squares added as integers, the auxiliary thread on every
    device): two shares in one process, sums added on the host side of the boundary; every
    share's output equals the unsplit batched he_softmax's, bit for bit."""
    g, o, em = toybts
    pl = he.load_plans_b()["toybts_n16_M32_B"]
    n, m = pl["n"], sum(split)
    g.keygen_softmax(n, m)
    L = m * o.n0 // n
    x = np.random.default_rng(29).uniform(-pl["M"], 0, (L, n))
    whole = g.encrypt(x, n, m, pl["M"], 35)
    ref = g.like(whole)
    ref.tensor.copy_(whole.tensor)
    g.softmax(ref, pl, batched=True)
    cw = 2 * (whole.level + 1) * g.n
    shares, lo = [], 0
    for cnt in split:
        t = whole.tensor[lo * cw:(lo + cnt) * cw].clone()
        shares.append(he.Ciphertexts(g, t, whole.level, whole.scale, cnt))
        lo += cnt
    y0 = [g.softmax_share_exp(s_, pl) for s_ in shares]
    ys = [g.like(s_) for s_ in shares]
    lam, lr = g.alloc(o.chain["user_top_level"], 1), g.alloc(o.chain["user_top_level"], 1)
    for j in range(1, pl["k"] + 1):
        src = y0 if j == 1 else ys
        d = [g.softmax_share_square_sum(s_) for s_ in src]
        dsum = d[0] + d[1]   # integer sum of residues (< 2^61): exact
        g.softmax_aux_round(pl, j, m, dsum, src[0].level, src[0].scale, y0[0], lam, lr)
        ys = [g.softmax_share_update(pl, j, lr, y0[i], g.like(y0[i])) for i in range(2)]
    assert all(y.level == ref.level and y.scale == ref.scale for y in ys)
    got = torch.cat([y.tensor[:y.n_ct * 2 * (y.level + 1) * g.n] for y in ys])
    assert torch.equal(got, ref.tensor[:m * 2 * (ref.level + 1) * g.n])


def test_autotune_variants_bit_identical(toybts):
    """Every launch strategy the autotuner chooses between gives the same words: each variant of
    each operation forced in turn (branches on side streams or one stream, transform CTA size,
    basis conversions fused into the transforms or separate) on
    multiplications, hoisted rotations, SlotToCoeff / CoeffToSlot levels and a degree-31
    polynomial at batch sizes 1, 2 and 6; then he_autotune fills its table (one entry per timed
    operation, level and batch size) and results stay the same."""
    g, o, em = toybts
    rng = np.random.default_rng(31)
    top = len(o.q) - 1

    def run():
        out = []
        for nct in (1, 2, 6):
            a = g.from_coeff(_rand_ct(o, 3, rng_fixed(nct), nct), 3, 2.0 ** 42)
            b = g.from_coeff(_rand_ct(o, top, rng_fixed(nct + 10), nct), top, float(o.q[0]))
            out.append(g.to_coeff(g.hmult(a, a)))
            out.append(g.to_coeff(g.lintrans(a, 3, False, 0, 16.0, float(o.q[3]))))
            out.append(g.to_coeff(g.lintrans(b, 3, True, 1, 1.0, float(o.q[top]))))
            u = g.from_coeff(_rand_ct(o, 20, rng_fixed(nct + 20), nct), 20, float(o.q[20]))
            out.append(g.to_coeff(g.poly_eval(u, np.linspace(0.3, -0.2, 32), 15, 2.0 ** 42)))
        return out

    def rng_fixed(k):
        return np.random.default_rng(1000 + k)

    ref = run()
    for op in ("modup", "rot", "lt_small", "lt_rows", "branches", "ntt_small", "fuse_conv", "ntt_1pass"):
        for choice in (0, 1):
            g.tune_force(op, choice)
            got = run()
            g.tune_force(op, -1)
            for i, (x, y) in enumerate(zip(ref, got)):
                assert np.array_equal(x, y), (op, choice, i)
    g.autotune([3, top - 1, top], [1, 6], reps=1)
    table = g.tune_table()
    ops = {e["op"] for e in table}
    assert ops == {"modup", "rot", "lt_small", "lt_rows", "ntt_small", "fuse_conv"}, ops
    assert all(e["choice"] in (0, 1) and min(e["ms"]) > 0 for e in table)
    assert {(e["limbs"], e["n_ct"]) for e in table if e["op"] == "modup"} == {(4, 1), (4, 6), (top, 1), (top, 6),
                                                                                 (top + 1, 1), (top + 1, 6)}
    assert ({(e["limbs"], e["n_ct"]) for e in table if e["op"] == "fuse_conv"}
            == {(e["limbs"], e["n_ct"]) for e in table if e["op"] == "modup"})
    # transform CTA size: both directions (n_ct holds the direction) over the limb-count ladder
    assert {e["n_ct"] for e in table if e["op"] == "ntt_small"} == {0, 1}
    got = run()
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)
    del rng


@pytest.mark.parametrize("mode", ["batched", "graph"])
def test_softmax_alg4_split_first_polynomial_bit_exact(toybts, mode):
    """A first polynomial one level deeper than the room above the bootstrapping input (degree
    1023, Chebyshev interpolant of v^(-1/2) on the plan's interval) is evaluated as A + T_512 B:
    T_256 and B bootstrapped on two side streams beside A.  Every output limb equals the oracle's
    (which evaluates the three parts one after the other), eagerly and by graph replay."""
    import copy

    from paper_2410_11184_gb300 import design as D

    g, o, em = toybts
    pl = copy.deepcopy(he.load_plans_b()["toybts_n16_M32_B"])
    it = pl["iters"][0]
    a, b = it["a"], it["b"]
    c, _ = D.cheb_interp(lambda u: (0.5 * (b - a) * u + 0.5 * (a + b)) ** -0.5, 1023)
    it["coeffs"] = D.hexlist(c)
    it["deg"] = 1023
    D.bts_gains_b(pl, o.chain)
    assert it["b_max"] > 0
    n, m = pl["n"], 2
    g.keygen_softmax(n, m)
    L = m * o.n0 // n
    x = np.random.default_rng(37).uniform(-pl["M"], 0, (L, n))
    gc = g.encrypt(x, n, m, pl["M"], 38)
    top = o.chain["user_top_level"]
    slots = O.pack(x, m, o.n0)
    outs = o.softmax_b([o.encrypt(slots[i], top, (2 / pl["M"]) * o.q[top], 38, i) for i in range(m)], pl, em)
    c0 = g.counters()
    if mode == "graph":
        work = g.like(gc)
        for _ in range(2):
            work.tensor.copy_(gc.tensor)
            work.level, work.scale, work.n_ct = gc.level, gc.scale, gc.n_ct
            g.softmax(work, pl, graph=True)
        gc = work
    else:
        g.softmax(gc, pl, batched=True)
        assert g.counters()["bts"] - c0["bts"] == 2 * pl["k"] + 2
    assert gc.level == outs[0].level and gc.scale == outs[0].scale
    got = g.to_coeff(gc)
    for i in range(m):
        assert np.array_equal(got[i], outs[i].data), i
