"""Full-size checks at N = 2^16 (log QP <= 1555, h = 192, bootstrapping), in the launch
configuration bench.py uses: sampled operations bit-exact with the oracle, and the Softmax
precision bar (>= 15 bits worst case against FP64 Softmax) at any batch size."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2410_11184_gb300 import he, workloads  # noqa: E402


@pytest.fixture(scope="module")
def full(params):
    ch, em = params[0]["fgb16"], params[2]["fgb16"]
    g = he.Context(ch, em)
    g.keygen(2024, rot_steps=[1])
    return g, ch, em


def test_fullsize_ops_bit_exact(full):
    g, ch, em = full
    o = O.Oracle(ch)
    o.keygen(2024)
    rng = np.random.default_rng(0)
    top = ch["user_top_level"]
    a = o.encrypt(rng.uniform(-1, 1, o.n0), top, 2.0 ** 42, 1, 0)
    b = o.encrypt(rng.uniform(-1, 1, o.n0), top, 2.0 ** 42, 1, 1)
    ga, gb = g.from_coeff(a.data, top, a.scale), g.from_coeff(b.data, top, b.scale)
    assert np.array_equal(g.to_coeff(g.hmult(ga, gb))[0], o.hmult(a, b).data)
    assert np.array_equal(g.to_coeff(g.rotate(ga, 1))[0], o.rotate(a, 1).data)


@pytest.mark.parametrize("m,kind", [(1, "uniform"), (1, "paper_normal"), (64, "attention")])
def test_fullsize_softmax_precision(full, params, m, kind):
    g, ch, em = full
    pl = params[1]["n256_M128"]
    n = pl["n"]
    g.keygen_softmax(n, m)
    L = m * g.n0 // n
    M = pl["M"]
    if kind == "uniform":
        x = workloads.uniform_inputs(L, n, 5, M)
    elif kind == "paper_normal":
        x = workloads.paper_normal_inputs(L, n, 6, M)
    else:
        x = workloads.attention_logits(L, n, 7, M=M)
    cts = g.encrypt(x, n, m, M, 99)
    c0 = g.counters()
    g.softmax(cts, pl, batched=True)
    c1 = g.counters()
    y = g.decrypt(cts, n)
    err = np.abs(y - O.softmax_fp64(x)).max()
    assert err < 2 ** -15, (kind, -math.log2(err))
    # bootstrapping calls of the planned schedule (batched: one call covers all m ciphertexts):
    # S in rounds 1, 2, 3, 5; lambda in rounds 1, 4; z once (round 3)
    assert c1["bts"] - c0["bts"] == 7


@pytest.mark.parametrize("plan", ["n128_M64", "n256_M64", "n1024_M64"])
def test_fullsize_serving_plans_grouped_precision(full, params, plan):
    """The serving mix's dimensions (inputs on [-64, 0]): two independent one-ciphertext
    requests in one grouped pass, each >= 15 bits against FP64 Softmax."""
    g, ch, em = full
    pl = params[1][plan]
    n, M = pl["n"], pl["M"]
    g.keygen_softmax(n, 1)
    L = g.n0 // n
    xs = [workloads.uniform_inputs(L, n, 40 + i, M) for i in range(2)]
    parts = [g.encrypt(x, n, 1, M, 50 + i) for i, x in enumerate(xs)]
    batch = he.Ciphertexts(g, torch.cat([p.tensor for p in parts]), parts[0].level, parts[0].scale, 2)
    g.softmax_grouped(batch, pl, 2)
    w = 2 * (batch.level + 1) * g.n
    for i, x in enumerate(xs):
        one = he.Ciphertexts(g, batch.tensor[i * w:(i + 1) * w], batch.level, batch.scale, 1)
        err = np.abs(g.decrypt(one, n) - O.softmax_fp64(x)).max()
        assert err < 2 ** -15, (plan, i, -math.log2(err))
