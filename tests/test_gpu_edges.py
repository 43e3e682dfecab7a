"""Edge cases of the GPU path: arguments the boundary must refuse before any launch (the
context stays usable), the degenerate input distributions of the method (all inputs equal:
Sigma y^2 at the lower end of the first x^{-1/2} interval; one input at the maximum and the
rest at -M: the upper end), and the packing with n = m (no rotate-and-sum), each limb for limb
against the oracle and within 2^-15 of FP64 Softmax."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2410_11184_gb300 import he  # noqa: E402

SEED = 13
EINVAL, ELEVEL, ENOKEY = -1, -2, -5


@pytest.fixture(scope="module")
def toy(params):
    ch = params[0]["toy"]
    g = he.Context(ch)
    g.keygen(SEED, rot_steps=[1])
    o = O.Oracle(ch)
    o.keygen(SEED)
    return g, o


def _code(fn):
    try:
        fn()
    except RuntimeError as e:
        return int(str(e).split("error ")[1].split(":")[0])
    return 0


def test_invalid_arguments_are_refused(toy, params):
    g, o = toy
    pl = params[1]["cfg1_n16_M8"]
    n = pl["n"]
    g.keygen_softmax(n, 1)
    x = np.random.default_rng(1).uniform(-pl["M"], 0, (g.n0 // n, n))
    ct = g.encrypt(x, n, 1, pl["M"], 5)
    # n not a power of two, n larger than the slot count, m not dividing n
    assert _code(lambda: g.softmax(ct, dict(pl, n=24))) == EINVAL
    assert _code(lambda: g.softmax(ct, dict(pl, n=2 * g.n0))) == EINVAL
    three = g.alloc(ct.level, 3, ct.scale)
    assert _code(lambda: g.softmax(three, pl)) == EINVAL
    assert _code(lambda: g.softmax_grouped(ct, pl, 2)) == EINVAL          # groups must divide n_ct
    # input count that does not fill the packing
    assert _code(lambda: g.encrypt(x[:-1], n, 1, pl["M"], 5)) == EINVAL
    # rescale / multiply at level 0, rotation without its key
    low = g.alloc(0, 1, 2.0 ** 40)
    low.tensor.zero_()
    assert _code(lambda: g.rescale(low)) == ELEVEL
    assert _code(lambda: g.hmult(low, low)) == ELEVEL
    assert _code(lambda: g.rotate(ct, 3)) == ENOKEY
    # NTT of more limbs than the chain has
    t = torch.zeros(g.n * 64, dtype=torch.int64, device="cuda")
    assert _code(lambda: g.ntt(t, 1, 64)) == EINVAL
    # the context is still usable: the same Softmax runs and is correct
    g.softmax(ct, pl)
    assert np.abs(g.decrypt(ct, n) - O.softmax_fp64(x)).max() < 2 ** -15


def _softmax_both(g, o, pl, x, m, seed):
    n = pl["n"]
    ct = g.encrypt(x, n, m, pl["M"], seed)
    top = o.chain["user_top_level"]
    slots = O.pack(x, m, o.n0)
    ocs = [o.encrypt(slots[i], top, (2 / pl["M"]) * o.q[top], seed, i) for i in range(m)]
    g.softmax(ct, pl)
    outs = o.softmax(ocs, pl)
    got = g.to_coeff(ct)
    for i in range(m):
        assert np.array_equal(got[i], outs[i].data), i
    return g.decrypt(ct, n)


@pytest.mark.parametrize("kind", ["all_equal_min", "all_equal_max", "one_hot"])
def test_degenerate_inputs(toy, params, kind):
    g, o = toy
    pl = params[1]["cfg1_n16_M8"]
    n, M = pl["n"], pl["M"]
    g.keygen_softmax(n, 1)
    L = g.n0 // n
    if kind == "all_equal_min":
        x = np.full((L, n), -M)
    elif kind == "all_equal_max":
        x = np.zeros((L, n))
    else:
        x = np.full((L, n), -M)
        x[np.arange(L), np.arange(L) % n] = 0.0
    y = _softmax_both(g, o, pl, x, 1, 21)
    assert np.abs(y - O.softmax_fp64(x)).max() < 2 ** -15


def test_n_equals_m_needs_no_rotation(toy, params):
    """m = n ciphertexts: each holds one coordinate of N0 Softmax, log2(n/m) = 0 rotations."""
    g, o = toy
    pl = params[1]["cfg1_n16_M8"]
    n = pl["n"]
    g.keygen_softmax(n, n)
    x = np.random.default_rng(4).uniform(-pl["M"], 0, (g.n0, n))
    rot0 = g.counters()["rot"]
    y = _softmax_both(g, o, pl, x, n, 22)
    assert g.counters()["rot"] == rot0
    assert np.abs(y - O.softmax_fp64(x)).max() < 2 ** -15


def test_softmax_by_dimension_and_range(toy, params):
    """he_softmax_nm, the problem statement's form (dimension n, inputs in [-M, 0]): with the
    plan registered for (n, M, method) it gives the words he_softmax gives with that plan, eagerly
    and by graph replay; an (n, M) with no registered plan is refused before any launch."""
    g, o = toy
    pl = params[1]["cfg1_n16_M8"]
    n, M = pl["n"], pl["M"]
    g.keygen_softmax(n, 1)
    x = np.random.default_rng(4).uniform(-M, 0, (g.n0 // n, n))
    ref = g.encrypt(x, n, 1, M, 9)
    g.softmax(ref, pl)
    assert _code(lambda: g.softmax_nm(g.encrypt(x, n, 1, M, 9), n, M, "alg2")) == EINVAL   # nothing registered
    g.softmax_register(pl)
    for graph in (False, True, True):
        ct = g.encrypt(x, n, 1, M, 9)
        g.softmax_nm(ct, n, M, "alg2", graph=graph)
        assert (ct.level, ct.scale) == (ref.level, ref.scale)
        assert torch.equal(ct.tensor[:2 * (ct.level + 1) * g.n], ref.tensor[:2 * (ref.level + 1) * g.n])
    ct = g.encrypt(x, n, 1, M, 9)
    assert _code(lambda: g.softmax_nm(ct, n, 2 * M, "alg2")) == EINVAL      # other range
    assert _code(lambda: g.softmax_nm(ct, 2 * n, M, "alg2")) == EINVAL      # other dimension
    assert _code(lambda: g.softmax_nm(ct, n, M, "alg4")) == EINVAL          # other method
