"""Parameter-set and polynomial design for the normalize-and-square Softmax circuit.

This module plays the role the paper gives to its external tools (the HEaaN parameter
preset and Sollya, Sec. 5.1.1-5.1.2): it fixes the RNS prime chains and computes the
polynomial approximations the circuit evaluates.  Its outputs are plain data files
under ``params/`` that the CUDA library and the independent CPU oracle both read as
inputs; neither side runs this code at evaluation time.

* Prime chains: primes q = 1 (mod 2N) near 2^b (Sec. 5.1.1, Table 4 gives only
  log(QP) <= 1555, N = 2^16, h = 192; the split into levels is this design's choice).
* exp on [-A, 0] (Sec. 3.4, Table 2): minimax in the Chebyshev basis, degree 2^t - 1.
* x^{-1/2} (Sec. 5.1.2): weighted minimax minimising max |sqrt(v) P(v) - 1|, with the
  approximate-renormalisation intervals [(1-a)^2/n, (1+a)^2] of Sec. 5.1.2 and the
  wider first interval [n exp(-M/2^(k-1)), n] of Sec. 3.4.2.
* EvalMod (bootstrapping): Chebyshev interpolant of cos(2 pi (K u - 1/4) / 2^r), followed
  by r double-angle steps, giving sin(2 pi x) for x = K u.

Minimax here is the discrete minimax on a dense Chebyshev-distributed grid, solved as a
linear program (scipy HiGHS) instead of Sollya's Remez exchange.

Run ``python -m paper_2410_11184_gb300.design`` to regenerate ``params/*.json``.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

PARAMS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "params")


# ----------------------------------------------------------------------------- primes
def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 2^64 (bases 2..37 suffice)."""
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for p in small:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def primes_below(two_n: int, bits: int, count: int, used: set) -> list:
    """Largest primes q < 2^bits with q = 1 mod 2N, not in ``used``."""
    out = []
    k = ((1 << bits) - 2) // two_n
    while len(out) < count:
        q = k * two_n + 1
        if q < (1 << bits) and q not in used and is_prime(q):
            out.append(q)
            used.add(q)
        k -= 1
    return out


def primes_alternating(two_n: int, bits: int, count: int, used: set) -> list:
    """Primes q = 1 mod 2N nearest to 2^bits, taken alternately below and above so that
    the running product stays close to 2^(bits * i) (keeps CKKS scales near 2^bits)."""
    centre = 1 << bits
    k_up = centre // two_n + 1
    k_dn = centre // two_n
    out = []
    take_up = False
    while len(out) < count:
        if take_up:
            while True:
                q = k_up * two_n + 1
                k_up += 1
                if q not in used and is_prime(q):
                    break
        else:
            while True:
                q = k_dn * two_n + 1
                k_dn -= 1
                if q not in used and is_prime(q):
                    break
        out.append(q)
        used.add(q)
        take_up = not take_up
    return out


def make_chain(name, log_n, q0_bits, groups, p_bits, alpha, h, sigma, log_scale, bts,
               max_logqp=None):
    """Build one prime chain.  ``groups`` is a list of (label, bits, count) for q1.. in
    order of level; consecutive groups with equal ``bits`` share one alternating family."""
    two_n = 2 << log_n
    used = set()
    q0 = primes_below(two_n, q0_bits, 1, used)
    qs = list(q0)
    labels = ["base"]
    i = 0
    while i < len(groups):
        bits = groups[i][1]
        j = i
        total = 0
        while j < len(groups) and groups[j][1] == bits:
            total += groups[j][2]
            j += 1
        fam = primes_alternating(two_n, bits, total, used)
        qs += fam
        for g in groups[i:j]:
            labels += [g[0]] * g[2]
        i = j
    ps = primes_below(two_n, p_bits, alpha, used)
    logqp = sum(math.log2(q) for q in qs) + sum(math.log2(p) for p in ps)
    # keep log(QP) within the security bound: swap the prime furthest above its 2^b
    # for the next free prime below 2^b of the same size until the bound holds
    while max_logqp is not None and logqp > max_logqp:
        i = max(range(1, len(qs)), key=lambda t: qs[t] / 2.0 ** round(math.log2(qs[t])))
        bits = round(math.log2(qs[i]))
        repl = primes_below(two_n, bits, 1, used)[0]
        used.discard(qs[i])
        qs[i] = repl
        logqp = sum(math.log2(q) for q in qs) + sum(math.log2(p) for p in ps)
    chain = {
        "name": name,
        "log_n": log_n,
        "q": [str(q) for q in qs],
        "p": [str(p) for p in ps],
        "q_role": labels,
        "alpha": alpha,
        "h": h,
        "sigma": sigma,
        "log_scale": log_scale,
        "log_qp": logqp,
    }
    chain.update(bts)
    return chain


def build_chains():
    chains = {}
    # Toy, insecure, test-only: 1 x 60 + 20 x 40 scaling + 3 x 60 special, no bootstrapping.
    chains["toy"] = make_chain(
        "toy", 12, 60, [("user", 40, 20)], 60, 3, 64, 3.2, 40,
        {"user_top_level": 20, "bootstrap": 0})
    # 128-bit-security size (log QP <= 1555, N = 2^16, h = 192), full-slot bootstrapping.
    # Level map (StC-first bootstrapping): q0 | StC 1..3 | user 4..12 | CtS 13..15 | EvalMod 16..24
    bts_layout = {
        "user_top_level": 12, "bootstrap": 1, "stc_levels": 3, "cts_levels": 3,
        "evalmod_levels": 9, "bts_min_level": 3,
    }
    chains["fgb16"] = make_chain(
        "fgb16", 16, 60,
        [("stc", 42, 3), ("user", 42, 9), ("cts", 58, 3), ("evalmod", 58, 9)],
        59, 5, 192, 3.2, 42, dict(bts_layout), max_logqp=1555.0)
    # Same layout at N = 2^12 (insecure, test-only) so the bootstrapping path can be
    # checked limb for limb against the oracle in seconds.
    chains["toybts"] = make_chain(
        "toybts", 12, 60,
        [("stc", 42, 3), ("user", 42, 9), ("cts", 58, 3), ("evalmod", 58, 9)],
        59, 5, 64, 3.2, 42, dict(bts_layout), max_logqp=1555.0)
    return chains


# ---------------------------------------------------------------- Chebyshev utilities
def cheb_vander(u: np.ndarray, deg: int) -> np.ndarray:
    """Matrix of T_0..T_deg evaluated at u (u in [-1, 1])."""
    V = np.empty((len(u), deg + 1))
    V[:, 0] = 1.0
    if deg >= 1:
        V[:, 1] = u
    for k in range(2, deg + 1):
        V[:, k] = 2.0 * u * V[:, k - 1] - V[:, k - 2]
    return V


def cheb_grid(npts: int) -> np.ndarray:
    """Chebyshev-extrema-distributed points on [-1, 1] plus the end points."""
    return np.cos(np.pi * np.arange(npts) / (npts - 1))[::-1]


def weighted_minimax(f, w, a, b, deg, npts=None):
    """Discrete weighted minimax: minimise max_x |w(x) (sum c_i T_i(u(x)) - f(x))| over a
    dense grid of [a, b], u(x) = (2x - a - b) / (b - a); solved as an LP."""
    from scipy.optimize import linprog

    npts = npts or max(3000, 40 * (deg + 1))
    u = cheb_grid(npts)
    x = 0.5 * (b - a) * u + 0.5 * (a + b)
    V = cheb_vander(u, deg)
    wx = w(x)
    fx = f(x)
    WV = V * wx[:, None]
    wf = wx * fx
    ones = np.ones((npts, 1))
    A_ub = np.vstack([np.hstack([WV, -ones]), np.hstack([-WV, -ones])])
    b_ub = np.concatenate([wf, -wf])
    cost = np.zeros(deg + 2)
    cost[-1] = 1.0
    res = linprog(cost, A_ub=A_ub, b_ub=b_ub, bounds=[(None, None)] * (deg + 2),
                  method="highs")
    if not res.success:
        raise RuntimeError("minimax LP failed: " + res.message)
    coeffs = res.x[:-1]
    # measured error on a much finer uniform+Chebyshev grid
    uu = np.concatenate([np.linspace(-1, 1, 40001), cheb_grid(40001)])
    xx = 0.5 * (b - a) * uu + 0.5 * (a + b)
    err = np.max(np.abs(w(xx) * (cheb_vander(uu, deg) @ coeffs - f(xx))))
    return coeffs, float(err)


def cheb_interp(g, deg):
    """Chebyshev interpolant of g on [-1, 1] at the deg+1 Chebyshev nodes."""
    n = deg + 1
    theta = np.pi * (np.arange(n) + 0.5) / n
    gv = g(np.cos(theta))
    c = np.array([2.0 / n * np.sum(gv * np.cos(k * theta)) for k in range(n)])
    c[0] *= 0.5
    uu = np.linspace(-1, 1, 200001)
    err = np.max(np.abs(cheb_vander(uu, deg) @ c - g(uu)))
    return c, float(err)


def inv_root_interp(e, a, b, deg):
    """Chebyshev interpolant of v^(-e) on [a, b] at its deg + 1 Chebyshev nodes, with its
    relative error max |P(v) v^e - 1| measured on 40001 uniform and 40001 Chebyshev-spaced
    points.  For degrees whose weighted minimax LP is too large for the solver (degree 1023 on
    the ratio-2^15 intervals of n = 32768): v^(-e) is analytic on a Bernstein ellipse around
    [a, b] (its singularity at 0 lies 2a / (b - a) below the interval), so the interpolant's
    error falls geometrically with the degree, close to the minimax error."""
    n = deg + 1
    theta = np.pi * (np.arange(n) + 0.5) / n
    gv = (0.5 * (b - a) * np.cos(theta) + 0.5 * (a + b)) ** -e
    c = np.array([2.0 / n * np.dot(gv, np.cos(k * theta)) for k in range(n)])
    c[0] *= 0.5
    uu = np.concatenate([np.linspace(-1, 1, 40001), cheb_grid(40001)])
    v = 0.5 * (b - a) * uu + 0.5 * (a + b)
    err = float(np.max(np.abs(cheb_eval_rec(list(c), uu) * v ** e - 1.0)))
    return c, err


def hexlist(c):
    return [float(v).hex() for v in c]


# ------------------------------------------------------------------ Softmax plans
def softmax_k(M: float, n: int) -> int:
    """k = ceil(log M - log ln n) (Thm. 3.3)."""
    return int(math.ceil(math.log2(M) - math.log2(math.log(n))))


def design_softmax(name, chain_name, n, M, k, exp_deg, inv_degs, margin=0.02):
    """Polynomials of Alg. 2 / Alg. 3 for inputs in [-M, 0]^n with k iterations."""
    A = M / 2.0 ** k
    # y0 = exp(x / 2^k), x in [-M, 0]; Chebyshev variable u = 2x/M + 1.
    ce, ee = weighted_minimax(lambda u: np.exp(A * (u - 1.0) / 2.0), lambda u: np.ones_like(u),
                              -1.0, 1.0, exp_deg)
    polys = [{"kind": "exp", "a": -1.0, "b": 1.0, "deg": exp_deg, "coeffs": hexlist(ce),
              "err": ee}]
    iters = []
    # Iteration 1: S = sum y0^2 in [n e^{-2A}, n]; v = S / n in [e^{-2A}, 1].
    lo = math.exp(-2.0 * A) * (1.0 - ee) ** 2
    hi = (1.0 + ee) ** 2
    alpha = None
    for j, d in enumerate(inv_degs, start=1):
        if j > 1:
            lo = (1.0 - alpha) ** 2 / n
            hi = (1.0 + alpha) ** 2
        a = lo * (1.0 - margin)
        b = hi * (1.0 + margin)
        c, eps = weighted_minimax(lambda v: v ** -0.5, lambda v: v ** 0.5, a, b, d)
        alpha = 2.0 * eps + eps * eps
        gain_s = 1.0 / n if j == 1 else 1.0
        uu = np.linspace(-1, 1, 20001)
        pmax = float(np.max(np.abs(cheb_vander(uu, d) @ c)))
        iters.append({
            "deg": d, "a": a, "b": b, "coeffs": hexlist(c), "eps": eps, "alpha": alpha,
            # v = gain_s * S is the polynomial input; lambda = P(v) * sqrt(gain_s).
            "gain_s": gain_s,
            # bootstrapping input gain of P(v) (1 / max |P| on [a, b]), removed afterwards by
            # scale bookkeeping
            "gain_l": 1.0 / pmax,
        })
    return {
        "name": name, "chain": chain_name, "n": n, "M": M, "k": k, "A": A,
        "exp": polys[0], "iters": iters,
        # every bootstrapping input is multiplied by this factor inside SlotToCoeff and the
        # factor is removed from the output by scale bookkeeping: it lowers q_0 / (scale *
        # message) and so the EvalMod error, while keeping the sin() linearisation error
        # (2 pi boost Delta / q_0)^2 / 6 below 2^-25 for messages of magnitude <= 1
        "bts_boost": 16.0,
    }


def design_softmax_b(name, chain_name, n, M, k, exp_deg, inv_degs, margin=0.02, interp_from=None):
    """Polynomials of Alg. 4 (version B) for inputs in [-M, 0]^n with k rounds.

    Round j needs lambda_j = S_j^(-1/2^j), S_j = sum (y^(j-1))^2 (the reading under which every
    round normalises), as a weighted minimax P_j of v^(-1/2^j), min ||P_j(v) v^(1/2^j) - 1||.
    A relative error eps_j of lambda_j becomes (1 + eps_j)^(2^j) - 1 =: delta_j in y^(j), since
    y^(j) = (lambda y^(0))^(2^j); the next round starts from a vector whose sum is within
    delta_j of 1, so its S lies in [(1 - delta_j)^2 / n, (1 + delta_j)^2].  Iteration 1 takes
    v = S_1 / n in [e^(-2A), 1], A = M / 2^k, and lambda_1 = P_1(v) n^(-1/2).  Rounds of degree at
    least interp_from take the Chebyshev interpolant of v^(-1/2^j) instead (inv_root_interp)."""
    A = M / 2.0 ** k
    ce, ee = weighted_minimax(lambda u: np.exp(A * (u - 1.0) / 2.0), lambda u: np.ones_like(u),
                              -1.0, 1.0, exp_deg)
    iters = []
    lo, hi = math.exp(-2.0 * A) * (1.0 - ee) ** 2, (1.0 + ee) ** 2
    delta = None
    for j, d in enumerate(inv_degs, start=1):
        e = 2.0 ** -j
        if j > 1:
            if delta >= 1.0:
                raise ValueError("round %d: delta %.3g >= 1 leaves no interval" % (j - 1, delta))
            lo, hi = (1.0 - delta) ** 2 / n, (1.0 + delta) ** 2
        a, b = lo * (1.0 - margin), hi * (1.0 + margin)
        interp = interp_from is not None and d >= interp_from
        if interp:
            c, eps = inv_root_interp(e, a, b, d)
        else:
            c, eps = weighted_minimax(lambda v, e=e: v ** -e, lambda v, e=e: v ** e, a, b, d)
        delta = (1.0 + eps) ** (2 ** j) - 1.0
        iters.append({"deg": d, "a": a, "b": b, "coeffs": hexlist(c), "eps": eps, "delta": delta,
                      "exponent": e, "gain_s": 1.0 / n if j == 1 else 1.0})
        if interp:
            iters[-1]["fit"] = "chebyshev interpolant"
    return {"name": name, "chain": chain_name, "version": "B", "n": n, "M": M, "k": k, "A": A,
            "exp": {"kind": "exp", "a": -1.0, "b": 1.0, "deg": exp_deg, "coeffs": hexlist(ce), "err": ee},
            "iters": iters}


def cheb_eval_rec(c, u):
    """sum_k c_k T_k(u) by the three-term recurrence (FP64)."""
    t0, t1 = np.ones_like(u), u
    acc = c[0] * t0
    if len(c) > 1:
        acc = acc + c[1] * t1
    for ck in c[2:]:
        t0, t1 = t1, 2.0 * u * t1 - t0
        acc = acc + ck * t1
    return acc


def bts_gains_b(plan, chain):
    """Bootstrapping gains of Alg. 4's auxiliary thread, stored in the plan so that every
    evaluator reads the same numbers: lam_max_j bounds lambda_j on its interval with a 10 %
    margin (iteration 1: n^(-1/2) e^A, the top of [n^-1/2, n^-1/2 e^A]; later ones a_j^(-1/2^j),
    the top of [b_j^(-1/2^j), a_j^(-1/2^j)]); b_max_j bounds the upper half B of a polynomial
    that is too deep to end above the bootstrapping input level and is evaluated split as
    A + T_h B (0 where no split is needed), on a grid of 20001 Chebyshev-spaced points."""
    n, A = plan["n"], plan["A"]
    top, bts_min = chain["user_top_level"], chain["bts_min_level"]
    plan["bts_boost"] = 16.0   # the input gain inside every bootstrapping (as for Alg. 2)
    uu = np.cos(np.linspace(0.0, np.pi, 20001))
    for j, it in enumerate(plan["iters"], start=1):
        e = it["exponent"]
        it["lam_max"] = 1.1 * (n ** -e * math.exp(A) if j == 1 else it["a"] ** -e)
        c = np.array([float.fromhex(h) for h in it["coeffs"]]) * it["gain_s"] ** e
        dj = int(math.ceil(math.log2(len(c))))
        it["b_max"] = 0.0
        if top - dj < bts_min:
            h, d = 1 << (dj - 1), len(c) - 1
            b_c = np.zeros(d - h + 1)
            b_c[0] = c[h]
            for i in range(1, d - h + 1):
                b_c[i] = 2.0 * c[h + i]
            it["b_max"] = 1.1 * float(np.max(np.abs(cheb_eval_rec(list(b_c), uu))))
    return plan


def build_b(write=True, names=None):
    """Alg. 4 plans (params/plans_b.json).  n = 256 on [-128, 0] with k = 4: the main thread
    uses ceil(log2 16) = 4 levels for exp, 1 for z = lambda y0 and k for z^(2^k), 9 in all,
    which the N = 2^16 chain has between its top user level 12 and its bootstrapping input
    level 3, so the main thread is never bootstrapped.  A = 8 makes iteration 1's interval
    [e^-16, 1]: degree 1023 keeps delta_1 below 1 (0.85); degree 127 then suffices."""
    specs = {
        "n256_M128_B": ("fgb16", 256, 128.0, 4, 15, [1023, 127, 127, 127]),
        # [-64, 0] (the LLaMa-shape workload's n = 128 and the serving plan's n = 256): A = 4,
        # iteration 1's interval [e^-8, 1] needs degree 255 only (depth 8: no split)
        "n128_M64_B": ("fgb16", 128, 64.0, 4, 15, [255, 127, 127, 127]),
        "n256_M64_B": ("fgb16", 256, 64.0, 4, 15, [255, 127, 127, 127]),
        # n = 1024: S_j / n spans a ratio near 1000 after iteration 1, so degree 255 throughout
        "n1024_M64_B": ("fgb16", 1024, 64.0, 4, 15, [255, 255, 255, 255]),
        # n = 4096 (which Alg. 2 cannot serve on this chain): degree 511 after iteration 1, whose
        # depth 9 just fits above the bootstrapping input because each lambda_j is bootstrapped alone
        "n4096_M64_B": ("fgb16", 4096, 64.0, 4, 15, [255, 511, 511, 511]),
        # n = 32768 (the vocabulary-sized Softmax of the serving mix): after iteration 1 the
        # interval spans a ratio near 2^15, so degree 1023 in iterations 2-4, each evaluated split
        # (A + T_512 B) since depth 10 exceeds the room above the bootstrapping input; those three
        # are Chebyshev interpolants (the weighted minimax LP of degree 1023 on these intervals
        # did not finish in two hours here; the interpolants reach eps 2e-6 and below)
        "n32768_M64_B": ("fgb16", 32768, 64.0, 4, 15, [255, 1023, 1023, 1023], 0.02, 1023),
        # the same level map at N = 2^12 (toybts: user levels 12 ... 4), for the oracle's
        # ciphertext circuit: A = 2 keeps every interval narrow enough for degree 63
        "toybts_n16_M32_B": ("toybts", 16, 32.0, 4, 15, [63, 63, 63, 63]),
    }
    path = os.path.join(PARAMS_DIR, "plans_b.json")
    plans = {}
    if os.path.exists(path):
        with open(path) as fh:
            plans = json.load(fh)
    for name, spec in specs.items():
        if names is None or name in names:
            plans[name] = design_softmax_b(name, *spec)
    chains = load_params()[0]
    for p in plans.values():
        bts_gains_b(p, chains[p["chain"]])
    if write:
        os.makedirs(PARAMS_DIR, exist_ok=True)
        with open(os.path.join(PARAMS_DIR, "plans_b.json"), "w") as fh:
            json.dump(plans, fh, indent=1)
    return plans


def newton_inv_root(y, v, p, steps):
    """Newton's iteration for v^(-1/p) (App. A for p = 2): y <- y ((p + 1) - v y^p) / p, `steps`
    times.  A relative error e of y becomes 1 - ((1 + e)(p + 1 - (1 + e)^p)) / p ~ ((p + 1)/2) e^2."""
    for _ in range(steps):
        y = y * ((p + 1.0) - v * y ** p) / p
    return y


def newton_levels(p):
    """levels of one Newton step for v^(-1/p), p = 2^j, arranged as ((p+1)/p) y - (v y) y^p / p:
    y^p takes j squarings while v y takes one product beside them, and their product one more
    level (two levels for p = 2, as in App. A; the constants are free in the scale)."""
    return int(round(math.log2(p))) + 1


def newton_study(plans, names=None):
    """Newton-refined inverse roots against the plans' single polynomials: for every round, the
    plan's degree-d minimax fit P_j of v^(-1/p) (p = 2 for Alg. 2, 2^j for Alg. 4) with its depth
    ceil(log2(d + 1)) and relative error eps = max |v^(1/p) P_j(v) - 1|, beside a lower-degree
    fit of the same function on the same interval followed by one Newton step at a depth no
    larger.  Returns rows (plan, round, p, depth, eps, newton degree, newton depth, newton eps)."""
    rows = []
    for name, pl in plans.items():
        if names and name not in names:
            continue
        alg4 = pl.get("version") == "B"
        for j, it in enumerate(pl["iters"][: pl["k"]], start=1):
            p = 2 ** j if alg4 else 2
            a, b, d = it["a"], it["b"], it["deg"]
            depth = int(math.ceil(math.log2(d + 1)))
            uu = np.cos(np.linspace(0.0, np.pi, 20001))
            vv = 0.5 * (b - a) * uu + 0.5 * (a + b)
            c = np.array([float.fromhex(h) for h in it["coeffs"]])
            eps = float(np.max(np.abs(vv ** (1.0 / p) * (cheb_vander(uu, d) @ c) - 1.0)))
            nd_depth = depth - newton_levels(p)
            if nd_depth < 1:
                rows.append((name, j, p, depth, eps, None, None, None))
                continue
            dn = 2 ** nd_depth - 1
            cn, _ = weighted_minimax(lambda v, p=p: v ** (-1.0 / p), lambda v, p=p: v ** (1.0 / p), a, b, dn)
            y = newton_inv_root(cheb_vander(uu, dn) @ cn, vv, p, 1)
            eps_n = float(np.max(np.abs(vv ** (1.0 / p) * y - 1.0)))
            rows.append((name, j, p, depth, eps, dn, nd_depth + newton_levels(p), eps_n))
    return rows


def design_evalmod(K, r, deg):
    """cos(2 pi (K u - 1/4) / 2^r) on u in [-1, 1]; r double angles give sin(2 pi K u)."""
    g = lambda u: np.cos(2.0 * np.pi * (K * u - 0.25) / 2.0 ** r)
    c, err = cheb_interp(g, deg)
    return {"K": K, "r": r, "deg": deg, "coeffs": hexlist(c), "err": err}


def build_all(write=True):
    chains = build_chains()
    plans = {
        # config: toy N=2^12, 128 Softmax of dim 16 on [-8, 0], 2 rounds, no bootstrapping
        "cfg1_n16_M8": design_softmax("cfg1_n16_M8", "toy", 16, 8.0, 2, 7, [7, 31]),
        # N=2^16, dim 256 on [-128, 0]: k = 5, exp depth 4, x^{-1/2} depths 6, 5x3, 7 (Table 3)
        "n256_M128": design_softmax("n256_M128", "fgb16", 256, 128.0, 5, 15, [63, 31, 31, 31, 127]),
        "n128_M64": design_softmax("n128_M64", "fgb16", 128, 64.0, softmax_k(64, 128), 15,
                                   [63] + [15] * (softmax_k(64, 128) - 2) + [127]),
        # bootstrapping-path checks at N=2^12: dim 16 on [-32, 0], k = 4
        "toybts_n16_M32": design_softmax("toybts_n16_M32", "toybts", 16, 32.0, 4, 15,
                                         [15, 15, 15, 31]),
        # a second dimension at N=2^12 for the mixed-dimension serving checks: dim 64, k = 3
        "toybts_n64_M32": design_softmax("toybts_n64_M32", "toybts", 64, 32.0, softmax_k(32, 64), 15,
                                         [63, 31, 63]),
    }
    # serving mix at N=2^16 (inputs on [-64, 0]) besides n128_M64: k = 4 by Thm 3.3 for both;
    # at n = 1024 the last round needs degree 255 (alpha 1.4e-7; 127 leaves 2.5e-2).  Dims 4096
    # and 32768 are not designed: x^{-1/2} on [(1 - alpha)^2 / n, (1 + alpha)^2] keeps alpha
    # above 0.25 with degree-63 rounds (above 1 at n = 32768), so the iteration does not converge
    # within the chain's levels between bootstrappings
    plans["n256_M64"] = design_softmax("n256_M64", "fgb16", 256, 64.0, softmax_k(64, 256), 15, [63, 31, 31, 127])
    plans["n1024_M64"] = design_softmax("n1024_M64", "fgb16", 1024, 64.0, softmax_k(64, 1024), 15,
                                        [63, 63, 63, 255])
    # N = 2^16: a degree-31 cosine and 4 double angles (9 levels, like degree 63 with 3, but fewer
    # products at the top levels); the toy set keeps degree 63 with 3
    evalmod = {"fgb16": design_evalmod(25.0, 4, 31), "toybts": design_evalmod(25.0, 3, 63)}
    if write:
        os.makedirs(PARAMS_DIR, exist_ok=True)
        with open(os.path.join(PARAMS_DIR, "chains.json"), "w") as fh:
            json.dump(chains, fh, indent=1)
        with open(os.path.join(PARAMS_DIR, "plans.json"), "w") as fh:
            json.dump(plans, fh, indent=1)
        with open(os.path.join(PARAMS_DIR, "evalmod.json"), "w") as fh:
            json.dump(evalmod, fh, indent=1)
    return chains, plans, evalmod


def load_params():
    """Read the committed parameter files."""
    out = []
    for fn in ("chains.json", "plans.json", "evalmod.json"):
        with open(os.path.join(PARAMS_DIR, fn)) as fh:
            out.append(json.load(fh))
    return tuple(out)


if __name__ == "__main__":
    import sys

    if "--newton-study" in sys.argv:
        _, plans, _ = load_params()
        with open(os.path.join(PARAMS_DIR, "plans_b.json")) as fh:
            plans.update(json.load(fh))
        names = [a for a in sys.argv[1:] if not a.startswith("--")] or ["n256_M128", "n256_M128_B", "n4096_M64_B"]
        for r in newton_study(plans, names):
            print(r)
        sys.exit(0)
    if "--version-b" in sys.argv:
        # Alg. 4 plans only (params/plans_b.json); the other parameter files stay as they are.
        # Further arguments name the plans to (re)design; the others are kept from the file.
        names = [a for a in sys.argv[1:] if not a.startswith("--")] or None
        if "--gains-only" in sys.argv:
            names = []   # keep every polynomial, recompute only the bootstrapping gains
        for p in build_b(write=True, names=names).values():
            print(p["name"], "k=%d exp_err=%.3g" % (p["k"], p["exp"]["err"]),
                  [("%d" % it["deg"], "%.3g" % it["eps"], "%.3g" % it["delta"]) for it in p["iters"]])
        sys.exit(0)
    chains, plans, evalmod = build_all(write=True)
    for c in chains.values():
        print(c["name"], "logQP=%.2f" % c["log_qp"], "nq=%d np=%d" % (len(c["q"]), len(c["p"])))
    for p in plans.values():
        print(p["name"], "k=%d exp_err=%.3g" % (p["k"], p["exp"]["err"]),
              [("%d" % it["deg"], "%.3g" % it["alpha"]) for it in p["iters"]])
    for k, e in evalmod.items():
        print(k, "evalmod err=%.3g" % e["err"])
