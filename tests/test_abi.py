"""The C ABI library loads and exports every entry point include/he_gb300.h declares (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "he_gb300.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    # any return type: a declaration is a line that starts with a type and names he_*( ... )
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+(?:\s*\*)?\s+\**\s*(he_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    assert len(names) == len(set(re.findall(r"\b(he_\w+)\s*\(", re.sub(r"/\*.*?\*/", "", open(
        os.path.join(ROOT, "include", "he_gb300.h")).read(), flags=re.S))))
    for want in ("he_context_create", "he_keygen", "he_encrypt", "he_softmax", "he_decrypt", "he_bootstrap",
                 "he_hmult", "he_rotate", "he_rescale", "he_ntt", "he_launch_count", "he_softmax_graph",
                 "he_softmax_grouped", "he_rescale_noalloc"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2410_11184_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2410_11184_gb300 import he

    monkeypatch.setattr(he, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(he, "_lib", None)
    try:
        he.lib()
    except RuntimeError as e:
        assert "no CPU fallback" in str(e)
    else:
        raise AssertionError("expected a failure")


def test_toy_chains_are_flagged_insecure(params):
    """The paper's parameter set (N = 2^16, log2(QP) = 1555, h = 192; Sec. 5.1.1) passes; the
    small test chains and a chain with a sparser secret or a larger modulus are flagged."""
    from paper_2410_11184_gb300 import build, he

    build.build()
    chains = params[0]
    assert not he.params_insecure(chains["fgb16"])
    assert he.params_insecure(chains["toy"]) and he.params_insecure(chains["toybts"])
    assert he.params_insecure(dict(chains["fgb16"], h=64))
    assert he.params_insecure(dict(chains["fgb16"], p=chains["fgb16"]["p"] + chains["fgb16"]["p"][:1]))
