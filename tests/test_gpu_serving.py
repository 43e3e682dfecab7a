"""Grouped Softmax batches and the serving loop on the GPU.

he_softmax_grouped runs independent Softmax groups in one batched pass; every group must come
out exactly as it would alone (and as the oracle computes it).  The server mixes requests of
two dimensions and two ciphertext counts, arriving while earlier batches run, on one context or
on two (two lanes, batches running concurrently); every request's result must equal the same
request run alone, bit for bit, and decrypt to the FP64 Softmax."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2410_11184_gb300 import he, serve  # noqa: E402

SEED = 11


@pytest.fixture(scope="module")
def ctx(params):
    ch = params[0]["toybts"]
    em = params[2]["toybts"]
    g = he.Context(ch, em)
    g.keygen(SEED)
    for n, m in ((16, 1), (16, 2), (64, 1)):
        g.keygen_softmax(n, m)
    o = O.Oracle(ch)
    o.keygen(SEED)
    return g, o, em


def _inputs(g, pl, m, seed):
    L = m * g.n0 // pl["n"]
    return np.random.default_rng(seed).uniform(-pl["M"], 0, (L, pl["n"]))


def _cat(g, parts):
    t = torch.cat([p.tensor for p in parts])
    return he.Ciphertexts(g, t, parts[0].level, parts[0].scale, sum(p.n_ct for p in parts))


@pytest.mark.parametrize("plan", ["toybts_n16_M32", "toybts_n16_M32_B"])
@pytest.mark.parametrize("m,groups", [(1, 3), (2, 2)])
def test_grouped_equals_alone_and_oracle(ctx, params, m, groups, plan):
    """Alg. 2 and Alg. 4 (plan suffix _B): every group of a grouped pass equals the group alone."""
    g, o, em = ctx
    alg4 = plan.endswith("_B")
    pl = he.load_plans_b()[plan] if alg4 else params[1][plan]
    n = pl["n"]
    xs = [_inputs(g, pl, m, 100 + i) for i in range(groups)]
    parts = [g.encrypt(x, n, m, pl["M"], 200 + i) for i, x in enumerate(xs)]
    batch = _cat(g, parts)
    g.softmax_grouped(batch, pl, groups)
    w = m * 2 * (batch.level + 1) * g.n
    for i, (x, p) in enumerate(zip(xs, parts)):
        alone = g.like(p)
        alone.tensor.copy_(p.tensor)
        g.softmax(alone, pl)
        assert (alone.level, alone.scale) == (batch.level, batch.scale)
        assert torch.equal(batch.tensor[i * w:(i + 1) * w], alone.tensor[:w]), i
        assert np.abs(g.decrypt(alone, n) - O.softmax_fp64(x)).max() < 2 ** -15
    # group 0 against the oracle, limb for limb
    top = o.chain["user_top_level"]
    slots = O.pack(xs[0], m, o.n0)
    ins = [o.encrypt(slots[j], top, (2 / pl["M"]) * o.q[top], 200, j) for j in range(m)]
    outs = o.softmax_b(ins, pl, em) if alg4 else o.softmax(ins, pl, em)
    got = g.to_coeff(batch)
    for j in range(m):
        assert np.array_equal(got[j], outs[j].data), j


@pytest.mark.parametrize("lanes", [1, 2])
def test_server_mix_equals_alone(ctx, params, lanes):
    """lanes = 2: a second context with the same keys, so two batches of different shapes run
    concurrently on the device; every result must still be the one the request gets alone."""
    g, o, em = ctx
    ctxs = [g]
    if lanes == 2:
        g2 = he.Context(params[0]["toybts"], params[2]["toybts"])
        g2.keygen(SEED)
        for n, m in ((16, 1), (16, 2), (64, 1)):
            g2.keygen_softmax(n, m)
        ctxs.append(g2)
    plans = {k: params[1][k] for k in ("toybts_n16_M32", "toybts_n64_M32")}
    # (plan, ciphertexts per request): two dimensions, two shapes for n = 16
    spec = [("toybts_n16_M32", 1), ("toybts_n64_M32", 1), ("toybts_n16_M32", 2), ("toybts_n16_M32", 1),
            ("toybts_n64_M32", 1), ("toybts_n16_M32", 1), ("toybts_n16_M32", 2), ("toybts_n64_M32", 1)]
    reqs = []
    for i, (name, m) in enumerate(spec):
        pl = plans[name]
        x = _inputs(g, pl, m, 300 + i)
        ct = g.encrypt(x, pl["n"], m, pl["M"], 400 + i)
        host = torch.empty(ct.tensor.numel(), dtype=torch.int64).pin_memory()
        host.copy_(ct.tensor)
        reqs.append((name, m, x, ct, host))
    torch.cuda.synchronize()
    # a budget for six single-ciphertext requests at a time: the last ones wait for memory
    words1 = 2 * (reqs[0][3].level + 1) * g.n
    srv = serve.Server(ctxs, plans, budget_bytes=6.5 * words1 * 8 * 8.0, max_batch_ct=4, start=False)
    handles = [srv.submit(name, host, m, ct.level, ct.scale) for name, m, x, ct, host in reqs[:5]]
    srv.start()                 # the first five arrive together
    time.sleep(0.05)            # the rest arrive while the first batches run
    handles += [srv.submit(name, host, m, ct.level, ct.scale) for name, m, x, ct, host in reqs[5:]]
    for h in handles:
        h.wait(timeout=300)
    srv.close()
    st = srv.stats()
    assert st["requests"] == len(spec) and st["batches"] < len(spec)   # some requests shared a batch
    assert st["lanes"] == lanes
    for (name, m, x, ct, host), h in zip(reqs, handles):
        pl = plans[name]
        alone = g.like(ct)
        alone.tensor.copy_(ct.tensor)
        g.softmax(alone, pl)
        w = m * 2 * (alone.level + 1) * g.n
        assert (h.out_level, h.out_scale) == (alone.level, alone.scale)
        assert torch.equal(h.host_out[:w], alone.tensor[:w].cpu()), h.rid
        assert np.abs(g.decrypt(alone, pl["n"]) - O.softmax_fp64(x)).max() < 2 ** -15
