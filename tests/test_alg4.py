"""Alg. 4 (version B) in FP64: the reading of its lambda_j, the designed polynomials, and the
level budget that lets the many-ciphertext main thread run without bootstrapping.

Alg. 4 prints lambda_j = (sum (y^(j-1))^2)^(-2^-(j-1)).  With that exponent iteration 1 gives
sum y^(1) = 1 / S_1, not 1.  The reading lambda_j = S_j^(-1/2^j) normalises every round:
lambda^(2^j) sum (y^(0))^(2^j) = 1, and y^(k) = Softmax(x) (Sec. 4.3)."""
import math
import time
import os

import numpy as np
import pytest

import oracle as O
from paper_2410_11184_gb300 import workloads as W


def _alg4_exact(x, k, exponent):
    """Alg. 4 with exact exp and exact powers; exponent(j) is the power applied to S_j."""
    y0 = np.exp(x / 2.0 ** k)
    lam = np.ones((x.shape[0], 1))
    y, sums = y0, []
    for j in range(1, k + 1):
        S = np.sum(y * y, axis=1, keepdims=True)
        lam = lam * S ** exponent(j)
        y = (lam * y0) ** (2 ** j)
        sums.append(np.sum(y, axis=1))
    return y, sums


def test_reading_normalises_every_round_and_gives_softmax():
    x = W.uniform_inputs(200, 64, seed=2, M=32.0)
    y, sums = _alg4_exact(x, 4, lambda j: -(2.0 ** -j))
    for s in sums:
        assert np.allclose(s, 1.0, atol=1e-12)
    assert np.abs(y - O.softmax_fp64(x)).max() < 1e-12
    # the printed exponent -2^-(j-1): the first round already misses the normalisation
    _, printed = _alg4_exact(x, 4, lambda j: -(2.0 ** -(j - 1)))
    assert np.abs(printed[0] - 1.0).min() > 1e-3


def test_simulation_with_exact_polynomials_is_softmax(params):
    """simulate_b with near-exact polynomials (degree-120 interpolants of v^(-1/2^j) on wide
    intervals, exp of degree 40) reproduces Softmax: pins the simulation's bookkeeping (gains,
    the accumulated lambda, the squarings) independently of the designed minimax."""
    from paper_2410_11184_gb300 import design as D

    n, M, k = 16, 8.0, 3
    A = M / 2.0 ** k
    ce, _ = D.cheb_interp(lambda u: np.exp(A * (u - 1.0) / 2.0), 40)
    iters = []
    for j in range(1, k + 1):
        e = 2.0 ** -j
        a, b = (math.exp(-2 * A) * 0.9, 1.1) if j == 1 else (0.5 / n, 1.5)
        c, _ = D.cheb_interp(lambda u, a=a, b=b, e=e: (0.5 * (b - a) * u + 0.5 * (a + b)) ** -e, 120)
        iters.append({"a": a, "b": b, "coeffs": D.hexlist(c), "exponent": e, "gain_s": 1.0 / n if j == 1 else 1.0})
    plan = {"n": n, "M": M, "k": k, "exp": {"coeffs": D.hexlist(ce)}, "iters": iters}
    x = W.uniform_inputs(300, n, seed=3, M=M)
    y, _ = O.simulate_b(x, plan)
    assert np.abs(y - O.softmax_fp64(x)).max() < 1e-9


plans_b = O.load_plans_b()


FULL_SIZE = sorted(k for k, p in plans_b.items() if p["chain"] == "fgb16")


@pytest.mark.skipif(not FULL_SIZE, reason="params/plans_b.json not generated")
@pytest.mark.parametrize("name", FULL_SIZE)
def test_designed_plan_precision(name):
    """Each stored N = 2^16 plan (k = 4) against FP64 Softmax on the three input models: at
    least 20 bits (the circuit then loses a few more to encryption noise).  The last round's
    relative error of sum y is below 2^-20, or 2^-17 for n = 32768, whose rounds 2-4 are
    degree-1023 Chebyshev interpolants on intervals spanning a ratio of 2^15."""
    plan = plans_b[name]
    for it in plan["iters"]:
        assert it["delta"] < 1.0 and it["a"] < it["b"]
    assert plan["iters"][-1]["delta"] < 2.0 ** (-17 if plan["n"] >= 32768 else -20)
    n, M = plan["n"], plan["M"]
    for x in (W.attention_logits(300, n, seed=5, M=M), W.paper_normal_inputs(300, n, 6, M),
              W.uniform_inputs(300, n, 7, M)):
        y, sums = O.simulate_b(x, plan)
        assert -math.log2(np.abs(y - O.softmax_fp64(x)).max()) >= 20.0
        # every S_j lies in the interval its polynomial was designed for
        for it, S in zip(plan["iters"], sums):
            v = it["gain_s"] * S
            assert v.min() >= it["a"] and v.max() <= it["b"]


@pytest.mark.skipif(not FULL_SIZE, reason="params/plans_b.json not generated")
@pytest.mark.parametrize("name", FULL_SIZE)
def test_main_thread_fits_the_chain_without_bootstrapping(params, name):
    """Main thread: exp (ceil(log2(deg + 1)) levels), z = lambda y0 (1), y^(j) = z^(2^j) (j).
    The output y^(k) needs a level >= 0; the last auxiliary input (y^(k-1))^2 is summed and
    bootstrapped, so it must stay at or above the level the bootstrapping starts from."""
    plan = plans_b[name]
    ch = params[0][plan["chain"]]
    top, bts = ch["user_top_level"], ch["bts_min_level"]
    z_level = top - math.ceil(math.log2(plan["exp"]["deg"] + 1)) - 1
    k = plan["k"]
    assert z_level - k >= 0                   # y^(k), the output
    assert z_level - (k - 1) - 1 >= bts       # (y^(k-1))^2, summed into S_k and bootstrapped
    assert z_level - (5 - 1) - 1 < bts        # k = 5 (Thm 3.3's k for M = 128, n = 256) would not fit
    # polynomials deeper than the room above the bootstrapping input are evaluated split
    # (one level deeper at most)
    for it in plan["iters"]:
        assert math.ceil(math.log2(it["deg"] + 1)) <= (top - bts) + 1


@pytest.mark.skipif("toybts_n16_M32_B" not in plans_b, reason="params/plans_b.json not generated")
def test_ciphertext_circuit_toy(params):
    """Alg. 4 as a ciphertext circuit in the oracle (N = 2^12, m = 2 ciphertexts of 256 Softmax
    of dimension 16 on [-32, 0], k = 4): within 2^-15 of FP64 Softmax, the outputs at the
    bootstrapping input level (9 main-thread levels below the top), and only the auxiliary
    thread bootstraps: two bootstrappings per iteration whatever m is."""
    chains, _, evalmod = params
    chain, em = chains["toybts"], evalmod["toybts"]
    plan = plans_b["toybts_n16_M32_B"]
    o = O.Oracle(chain)
    o.keygen(11)
    m, n, M = 2, plan["n"], plan["M"]
    x = W.uniform_inputs(m * o.n0 // n, n, seed=5, M=M)
    top = chain["user_top_level"]
    slots = O.pack(x, m, o.n0)
    cts = [o.encrypt(slots[i], top, (2 / M) * o.q[top], 21, i) for i in range(m)]
    o.reset_counters()
    outs = o.softmax_b(cts, plan, em)
    assert [c.level for c in outs] == [chain["bts_min_level"]] * m
    assert o.counters()["bts"] == 2 * plan["k"]
    y = O.unpack(np.stack([o.decrypt(c).real for c in outs]), n)
    assert np.abs(y - O.softmax_fp64(x)).max() < 2 ** -15


@pytest.mark.skipif("toybts_n16_M32_B" not in plans_b, reason="params/plans_b.json not generated")
def test_ciphertext_circuit_split_first_polynomial(params):
    """A first polynomial one level deeper than the room above the bootstrapping input (degree
    1023: a Chebyshev interpolant of the same v^(-1/2) on the same interval) is evaluated as
    A + T_512 B with T_256 and B bootstrapped: same precision, two more bootstrappings."""
    import copy

    from paper_2410_11184_gb300 import design as D

    chains, _, evalmod = params
    chain, em = chains["toybts"], evalmod["toybts"]
    plan = copy.deepcopy(plans_b["toybts_n16_M32_B"])
    it = plan["iters"][0]
    a, b = it["a"], it["b"]
    c, _ = D.cheb_interp(lambda u: (0.5 * (b - a) * u + 0.5 * (a + b)) ** -0.5, 1023)
    it["coeffs"] = D.hexlist(c)
    D.bts_gains_b(plan, chain)   # the split's B now needs a bootstrapping gain
    assert it["b_max"] > 0
    o = O.Oracle(chain)
    o.keygen(11)
    m, n, M = 2, plan["n"], plan["M"]
    x = W.uniform_inputs(m * o.n0 // n, n, seed=5, M=M)
    top = chain["user_top_level"]
    slots = O.pack(x, m, o.n0)
    cts = [o.encrypt(slots[i], top, (2 / M) * o.q[top], 21, i) for i in range(m)]
    o.reset_counters()
    outs = o.softmax_b(cts, plan, em)
    assert o.counters()["bts"] == 2 * plan["k"] + 2
    y = O.unpack(np.stack([o.decrypt(c_).real for c_ in outs]), n)
    assert np.abs(y - O.softmax_fp64(x)).max() < 2 ** -15


@pytest.mark.slow
@pytest.mark.skipif(os.environ.get("HE_RUN_SLOW") != "1" or not FULL_SIZE,
                    reason="N = 2^16 oracle circuit: about 17 minutes on 8 cores (HE_RUN_SLOW=1)")
@pytest.mark.parametrize("name", ["n256_M128_B", "n4096_M64_B"])
def test_full_size_ciphertext_circuit(params, name):
    """An N = 2^16 plan (k = 4) on one ciphertext of N0/n Softmax of dimension n (attention
    logits): within 2^-15 of FP64 Softmax, output at the bootstrapping input level, and only
    the auxiliary ciphertext bootstrapped (2 per iteration, 2 more for a split polynomial)."""
    chains, _, evalmod = params
    chain, em = chains["fgb16"], evalmod["fgb16"]
    plan = plans_b[name]
    o = O.Oracle(chain)
    o.keygen(11)
    n, M = plan["n"], plan["M"]
    room = chain["user_top_level"] - chain["bts_min_level"]
    split = sum(math.ceil(math.log2(it["deg"] + 1)) > room for it in plan["iters"])
    x = W.attention_logits(o.n0 // n, n, seed=5, M=M)
    top = chain["user_top_level"]
    ct = o.encrypt(O.pack(x, 1, o.n0)[0], top, (2 / M) * o.q[top], 21, 0)
    o.reset_counters()
    t0 = time.time()
    out = o.softmax_b([ct], plan, em)[0]
    dt = time.time() - t0
    assert out.level == chain["bts_min_level"]
    nbts = o.counters()["bts"]
    assert nbts == 2 * plan["k"] + 2 * split
    y = O.unpack(o.decrypt(out).real[None, :], n)
    bits = -math.log2(np.abs(y - O.softmax_fp64(x)).max())
    print("%s: %.2f bits against FP64 Softmax, %d bootstrappings, %.0f s on %d host threads"
          % (name, bits, nbts, dt, int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))))
    # measured on this seed: 18.8 bits (n = 256) and 19.7 bits (n = 4096); half a bit of margin
    assert bits > {"n256_M128_B": 18.3, "n4096_M64_B": 19.2}[name]
