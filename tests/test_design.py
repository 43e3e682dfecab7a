"""Pins for the parameter files both implementations read (prime chains, polynomials)."""
import math

import numpy as np
import pytest

sympy = pytest.importorskip("sympy")

from paper_2410_11184_gb300 import design as D  # noqa: E402


def test_chains_are_ntt_friendly_primes(params):
    chains = params[0]
    for name, ch in chains.items():
        two_n = 2 << ch["log_n"]
        q = [int(x) for x in ch["q"]]
        p = [int(x) for x in ch["p"]]
        allp = q + p
        assert len(set(allp)) == len(allp), name
        for v in allp:
            assert sympy.isprime(v), (name, v)
            assert (v - 1) % two_n == 0, (name, v)
            assert v < 2 ** 60   # the forward NTT keeps values below 16q < 2^64
        assert len(p) == ch["alpha"]
        logqp = sum(math.log2(v) for v in allp)
        assert abs(logqp - ch["log_qp"]) < 1e-6


def test_fgb16_matches_table4(params, golden):
    ch = params[0]["fgb16"]
    t4 = golden["table4_fgb"]
    assert ch["log_n"] == t4["log_n"]
    assert ch["h"] == t4["h"]
    logqp = sum(math.log2(int(v)) for v in ch["q"] + ch["p"])
    assert logqp <= t4["log_qp"]
    hi, lo = t4["user_levels"]
    assert ch["user_top_level"] == hi
    # levels 12..4 usable: 9 multiplications from the top down to the bootstrapping level 3
    assert hi - ch["bts_min_level"] == t4["levels"]
    # level map: q0 | StC | user | CtS | EvalMod
    assert len(ch["q"]) == 1 + ch["stc_levels"] + t4["levels"] + ch["cts_levels"] + ch["evalmod_levels"]


def test_miller_rabin_against_sympy():
    rng = np.random.default_rng(3)
    for v in list(rng.integers(2, 2 ** 62, 300)) + [2 ** 61 - 1, 561, 1105, 2 ** 59 - 55]:
        assert D.is_prime(int(v)) == sympy.isprime(int(v))


def test_exp_polynomials(params):
    for pl in params[1].values():
        A = pl["A"]
        c = np.array([float.fromhex(h) for h in pl["exp"]["coeffs"]])
        u = np.linspace(-1, 1, 20001)
        err = np.max(np.abs(D.cheb_vander(u, len(c) - 1) @ c - np.exp(A * (u - 1) / 2)))
        assert err < 1e-6, (pl["name"], err)
        assert A == pl["M"] / 2 ** pl["k"]


def test_invsqrt_polynomials_and_interval_chain(params):
    for pl in params[1].values():
        n = pl["n"]
        prev = None
        for j, it in enumerate(pl["iters"]):
            c = np.array([float.fromhex(h) for h in it["coeffs"]])
            v = np.linspace(it["a"], it["b"], 20001)
            u = (2 * v - it["a"] - it["b"]) / (it["b"] - it["a"])
            p = D.cheb_vander(u, len(c) - 1) @ c
            eps = np.max(np.abs(np.sqrt(v) * p - 1))
            assert eps <= it["eps"] * 1.05 + 1e-12
            # |x P(x)^2 - 1| <= alpha on the interval (Sec. 5.1.2)
            assert np.max(np.abs(v * p * p - 1)) <= it["alpha"] * 1.05 + 1e-12
            if j == 0:
                assert it["a"] <= math.exp(-2 * pl["A"]) and it["b"] >= 1.0
            else:
                # next input in [(1-a)^2/n, (1+a)^2] (Lemma 3.4 after an alpha-normalisation)
                assert it["a"] <= (1 - prev) ** 2 / n and it["b"] >= (1 + prev) ** 2
            prev = it["alpha"]
        # the last normalisation is precise (about 19.5 bits in Sec. 5.2.4)
        assert pl["iters"][-1]["alpha"] < 2 ** -18


def test_evalmod_composes_to_sine(params):
    for em in params[2].values():
        c = np.array([float.fromhex(h) for h in em["coeffs"]])
        u = np.linspace(-1, 1, 50001)
        y = D.cheb_vander(u, len(c) - 1) @ c
        for _ in range(em["r"]):
            y = 2 * y * y - 1
        err = np.max(np.abs(y - np.sin(2 * np.pi * em["K"] * u)))
        # r double angles multiply the fit error by about 4^r; the composition must stay far
        # below the bootstrapping precision target (>= 20 bits)
        assert err < 2.0 ** -32, err


def _formula(f, k):
    """evaluate the paper's '2k+4' style depth formulas"""
    a, b = f.split("k+")
    return int(a) * k + int(b)


def test_depths_match_tables_2_and_3(params, golden):
    t2 = golden["table2_main_thread"]
    t3 = golden["table3_aux_thread"]
    pl = params[1]["n256_M128"]
    k = pl["k"]
    depth = lambda d: math.ceil(math.log2(d + 1))
    assert depth(pl["exp"]["deg"]) == t2["exp_depth"]
    # main thread: exp + 2 per round
    assert depth(pl["exp"]["deg"]) + 2 * k == _formula(t2["total_depth_formula"], k)
    row = t3[str(pl["n"])]
    d = [depth(it["deg"]) for it in pl["iters"]]
    assert d[0] == row["invsqrt_depths"]["first"]
    assert all(x == row["invsqrt_depths"]["middle"] for x in d[1:-1])
    assert d[-1] == row["invsqrt_depths"]["last"]
    total = sum(d) + row["sq_mask_per_iter"] * k
    assert total == _formula(row["total_formula"], k)


def test_softmax_k_matches_theorem_3_3():
    # k = ceil(log M - log ln n)
    assert D.softmax_k(8, 16) == 2
    assert D.softmax_k(128, 256) == 5
    assert D.softmax_k(64, 128) == 4


def test_newton_inverse_root_step():
    """Newton's step for v^(-1/p) (App. A for p = 2): the exact root is a fixed point, and a
    relative error e becomes about ((p + 1)/2) e^2 (quadratic convergence from small errors);
    from a large error (e = -0.9 for p = 2) the step does not converge."""
    from paper_2410_11184_gb300 import design as D

    v = np.linspace(0.01, 2.0, 101)
    for p in (2, 4, 8):
        exact = v ** (-1.0 / p)
        assert np.allclose(D.newton_inv_root(exact, v, p, 1), exact, rtol=1e-14)
        for e in (1e-3, -1e-3, 1e-2):
            got = D.newton_inv_root(exact * (1 + e), v, p, 1) / exact - 1.0
            assert np.allclose(got, -(p + 1) / 2 * e * e, rtol=0.05, atol=1e-12)
    bad = D.newton_inv_root(v ** -0.5 * 0.1, v, 2, 1) / v ** -0.5 - 1.0
    assert np.all(np.abs(bad) > 0.8)
    assert D.newton_levels(2) == 2 and D.newton_levels(16) == 5


@pytest.mark.slow
def test_newton_refinement_loses_at_equal_depth(params):
    """Round 5 of the n = 256, M = 128 plan: its degree-127 fit of v^(-1/2) (depth 7) reaches
    1.5e-7; a degree-31 fit with one Newton step (two levels) at the same depth does far worse."""
    from paper_2410_11184_gb300 import design as D

    rows = D.newton_study({"n256_M128": params[1]["n256_M128"]})
    last = rows[-1]
    assert last[3] == last[6] == 7
    assert last[4] < 1e-6 and last[7] > 100 * last[4]


def test_inverse_root_interpolant():
    """design.inv_root_interp (the fit of the n = 32768 plan's degree-1023 rounds), at degree 63 on
    the ratio-2^15 interval of those rounds: its coefficients are numpy's Chebyshev interpolant of
    the same function at the same nodes, the error it reports is the relative error measured
    independently on a grid, and it is within a factor 4 of the weighted minimax (LP) error of
    the same degree, the best any polynomial of that degree can do on that grid."""
    n, e, d = 32768, 0.25, 63
    a, b = 0.98 / n, 1.02
    c, err = D.inv_root_interp(e, a, b, d)
    f = lambda u: (0.5 * (b - a) * u + 0.5 * (a + b)) ** -e
    ref = np.polynomial.chebyshev.chebinterpolate(f, d)
    assert np.allclose(c, ref, rtol=1e-10, atol=1e-12)
    v = np.geomspace(a, b, 50001)
    u = (2 * v - a - b) / (b - a)
    measured = np.max(np.abs(np.polynomial.chebyshev.chebval(u, ref) * v ** e - 1.0))
    assert measured <= err * (1 + 1e-6)
    _, lp = D.weighted_minimax(lambda x: x ** -e, lambda x: x ** e, a, b, d)
    assert lp <= err <= 4.0 * lp
