"""Seeded synthetic Softmax inputs (numpy PCG64).  No part of the method's arithmetic lives
here; both the tests (for the CUDA path and the CPU oracle) and bench.py draw inputs from it.

The paper's inputs are LLaMa-7B attention logits (Sec. 5.2.2), which are not available; these
generators stand in for them with the shapes and ranges the paper describes."""
import numpy as np


def uniform_inputs(L, n, seed, M):
    """i.i.d. uniform on [-M, 0] (Sec. 5.2.2: 'very similar results' to the normal model)."""
    return np.random.default_rng(seed).uniform(-M, 0.0, (L, n))


def paper_normal_inputs(L, n, seed, M):
    """N(-M/2, (M/6)^2) tail-cut to [-M, 0] (Sec. 5.2.2), by redrawing out-of-range values."""
    rng = np.random.default_rng(seed)
    x = rng.normal(-M / 2, M / 6, (L, n))
    bad = (x < -M) | (x > 0)
    while bad.any():
        x[bad] = rng.normal(-M / 2, M / 6, bad.sum())
        bad = (x < -M) | (x > 0)
    return x


def attention_logits(L, n, seed, M=128.0, d=64, bound=8.0, sigma=None, rows_per_head=1):
    """q.k / sqrt(d) with q, k ~ N(0, sigma^2 I_d) (sigma = 1, or with sigma == 'per_head' one
    U[0.5, 1.5] draw per head of rows_per_head consecutive rows), minus a public bound, clipped
    to [-M, 0]."""
    rng = np.random.default_rng(seed)
    s = np.ones((L, 1))
    if sigma == "per_head":
        heads = -(-L // rows_per_head)
        s = np.repeat(rng.uniform(0.5, 1.5, (heads, 1)), rows_per_head, axis=0)[:L]
    q = rng.standard_normal((L, 1, d)) * s[:, :, None]
    k = rng.standard_normal((L, n, d)) * s[:, :, None]
    # q.k summed over the head dimension in a fixed order (elementwise products and additions,
    # no BLAS), so that the same seed gives the same bits on every host
    dot = np.zeros((L, n))
    for t in range(d):
        dot += q[:, :, t] * k[:, :, t]
    logits = dot / np.sqrt(d)
    return np.clip(logits - bound, -M, 0.0)
