"""The seeded synthetic inputs (paper_2410_11184_gb300/workloads.py) have the shapes, ranges
and distributions the paper's input model describes (Sec. 5.2.2), and are reproducible."""
import numpy as np

from paper_2410_11184_gb300 import workloads as W


def test_uniform_inputs_range_and_seed():
    x = W.uniform_inputs(64, 256, seed=3, M=128.0)
    assert x.shape == (64, 256) and x.min() >= -128.0 and x.max() <= 0.0
    assert np.array_equal(x, W.uniform_inputs(64, 256, seed=3, M=128.0))
    assert not np.array_equal(x, W.uniform_inputs(64, 256, seed=4, M=128.0))
    assert abs(x.mean() + 64.0) < 1.0          # mean -M/2


def test_paper_normal_inputs_are_tail_cut_normal():
    M = 64.0
    x = W.paper_normal_inputs(400, 256, seed=5, M=M)
    assert x.min() >= -M and x.max() <= 0.0
    # N(-M/2, (M/6)^2) cut at +-3 sigma: mean -M/2, standard deviation a little below M/6
    assert abs(x.mean() + M / 2) < 0.1
    assert 0.95 * M / 6 < x.std() < M / 6


def test_attention_logits_shape_range_and_heads():
    M, n, rows = 64.0, 128, 16
    x = W.attention_logits(4 * rows, n, seed=7, M=M, d=128, bound=16.0, sigma="per_head", rows_per_head=rows)
    assert x.shape == (4 * rows, n) and x.min() >= -M and x.max() <= 0.0
    assert np.array_equal(x, W.attention_logits(4 * rows, n, seed=7, M=M, d=128, bound=16.0, sigma="per_head",
                                                rows_per_head=rows))
    # before the shift, q.k / sqrt(d) has standard deviation sigma^2 per head: heads differ
    spread = [np.std(x[h * rows:(h + 1) * rows] + 16.0) for h in range(4)]
    assert max(spread) > 1.2 * min(spread)
    y = W.attention_logits(64, 256, seed=1)      # the 64-ciphertext workload's defaults
    assert y.min() >= -128.0 and y.max() <= 0.0 and abs(np.std(y + 8.0) - 1.0) < 0.05
