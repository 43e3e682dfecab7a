"""he_rescale_noalloc, the rescale that allocates no device memory (for callers whose device
memory is fully reserved up front), against he_rescale: the same words, on two calls in a row
that reuse its fixed scratch.  Kept in its own file, collected last."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2410_11184_gb300 import he  # noqa: E402


def _noalloc(g, a, out):
    ha, ho = a.c(), out.c()
    rc = he.lib().he_rescale_noalloc(g.h, C.byref(ha), C.byref(ho))
    out.update(ho)
    return rc


@pytest.mark.parametrize("chain,level,n_ct", [("toy", 20, 3), ("fgb16", 12, 1)])
def test_rescale_noalloc_matches_rescale(params, chain, level, n_ct):
    lib = he.lib()
    lib.he_rescale_noalloc.argtypes = [C.c_void_p, C.POINTER(he.he_ct), C.POINTER(he.he_ct)]
    lib.he_rescale_noalloc.restype = C.c_int
    ch = dict(params[0][chain], bootstrap=0)  # no bootstrapping tables needed here
    g = he.Context(ch)
    q = [int(x) for x in ch["q"]]
    rng = np.random.default_rng(level)
    for call in range(2):  # the second call reuses the scratch the first one left behind
        d = np.zeros((n_ct, 2, level + 1, g.n), dtype=np.uint64)
        for t in range(level + 1):
            d[:, :, t] = rng.integers(0, q[t], (n_ct, 2, g.n), dtype=np.uint64)
        a = g.from_coeff(d, level, 2.0 ** 40)
        want = g.rescale(a)
        out = g.alloc(level - 1, n_ct)
        out.tensor.fill_(0)
        assert _noalloc(g, a, out) == 0, he.lib().he_last_error(g.h).decode()
        assert (out.level, out.n_ct) == (want.level, want.n_ct)
        assert out.scale == want.scale
        words = n_ct * 2 * level * g.n
        assert want.tensor.numel() == words
        assert torch.equal(out.tensor, want.tensor), call  # integer work: bit for bit
    # sizes beyond the fixed scratch are refused before any launch
    big = g.alloc(level, 64)
    out = g.alloc(level - 1, 64)
    assert _noalloc(g, big, out) == -1
    assert "scratch" in he.lib().he_last_error(g.h).decode()


def test_rescale_noalloc_refusals(params):
    """Arguments that would reach a kernel wrongly are refused before any launch: a level outside
    the chain (HE_EINVAL), level 0 (HE_ELEVEL), and an output overlapping the input, exactly or at
    an offset (HE_EINVAL); the context stays usable."""
    lib = he.lib()
    lib.he_rescale_noalloc.argtypes = [C.c_void_p, C.POINTER(he.he_ct), C.POINTER(he.he_ct)]
    lib.he_rescale_noalloc.restype = C.c_int
    ch = dict(params[0]["toy"], bootstrap=0)
    g = he.Context(ch)
    nq = len(ch["q"])
    buf = torch.zeros(4 * 2 * nq * g.n, dtype=torch.int64, device="cuda")
    out = g.alloc(nq - 2, 1)
    for lv, code in ((-1, -1), (nq, -1), (0, -2)):
        a = he.Ciphertexts(g, buf, lv, 2.0 ** 40, 1)
        assert _noalloc(g, a, out) == code, lv
    lv = 5
    words = 2 * (lv + 1) * g.n
    a = he.Ciphertexts(g, buf[:words], lv, 2.0 ** 40, 1)
    for off in (0, g.n, words - 1):   # out starts inside a's bytes
        o = he.Ciphertexts(g, buf[off:off + 2 * lv * g.n], lv - 1, 1.0, 1)
        assert _noalloc(g, a, o) == -1, off
        assert "overlap" in lib.he_last_error(g.h).decode()
    # out ending inside a (it starts below a's first word)
    a2 = he.Ciphertexts(g, buf[g.n:g.n + words], lv, 2.0 ** 40, 1)
    o = he.Ciphertexts(g, buf[0:2 * lv * g.n], lv - 1, 1.0, 1)
    assert _noalloc(g, a2, o) == -1
    # adjacent, not overlapping: accepted and equal to he_rescale
    o = he.Ciphertexts(g, buf[words:words + 2 * lv * g.n], lv - 1, 1.0, 1)
    assert _noalloc(g, a, o) == 0, lib.he_last_error(g.h).decode()
    assert torch.equal(o.tensor, g.rescale(a).tensor)
