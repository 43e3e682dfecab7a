"""Thin Python binding of the C ABI in include/he_gb300.h (argument marshalling only).

Every computation runs in libhe_gb300.so (CUDA kernels for sm_103a); PyTorch provides the
device buffers (uint64 words held in int64 tensors) and the CUDA stream.  There is no CPU
fallback: importing the library fails loudly when the compiled extension is missing.
"""
from __future__ import annotations

import ctypes as C
import json
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhe_gb300.so")
PARAMS_DIR = os.path.join(HERE, "params")

u64p = C.POINTER(C.c_uint64)
dblp = C.POINTER(C.c_double)
intp = C.POINTER(C.c_int)


class he_params(C.Structure):
    _fields_ = [("log_n", C.c_int), ("n_q", C.c_int), ("q", u64p), ("n_p", C.c_int), ("p", u64p),
                ("h", C.c_int), ("sigma", C.c_double), ("log_scale", C.c_int), ("user_top_level", C.c_int),
                ("bootstrap", C.c_int), ("stc_levels", C.c_int), ("cts_levels", C.c_int),
                ("bts_min_level", C.c_int), ("em_K", C.c_double), ("em_r", C.c_int), ("em_deg", C.c_int),
                ("em_coeffs", dblp)]


HE_SOFTMAX_ALG2, HE_SOFTMAX_ALG4 = 0, 1


class he_softmax_plan(C.Structure):
    _fields_ = [("n", C.c_int), ("k", C.c_int), ("M", C.c_double), ("exp_deg", C.c_int), ("exp_coeffs", dblp),
                ("inv_deg", intp), ("inv_coeffs", dblp), ("inv_a", dblp), ("inv_b", dblp), ("gain_s", dblp),
                ("gain_l", dblp), ("bts_boost", C.c_double), ("method", C.c_int), ("exponent", dblp),
                ("lam_max", dblp), ("b_max", dblp)]


class he_ct(C.Structure):
    _fields_ = [("data", C.c_void_p), ("level", C.c_int), ("scale", C.c_double), ("n_ct", C.c_int)]


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhe_gb300.so is not built: run paper_2410_11184_gb300/build.py "
                               "(or __graft_entry__.build()); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        sig = {
            "he_context_create": [C.POINTER(he_params), vp, C.POINTER(vp)],
            "he_params_insecure": [C.POINTER(he_params)],
            "he_context_destroy": [vp],
            "he_ring_degree": [vp],
            "he_keygen": [vp, C.c_uint64, intp, C.c_int],
            "he_keygen_softmax": [vp, C.c_int, C.c_int],
            "he_encrypt": [vp, dblp, C.c_size_t, C.c_int, C.c_int, C.c_double, C.c_uint64, C.POINTER(he_ct)],
            "he_decrypt": [vp, C.POINTER(he_ct), C.c_int, dblp, C.c_size_t],
            "he_decrypt_slots": [vp, C.POINTER(he_ct), C.c_int, dblp],
            "he_encrypt_slots": [vp, dblp, C.c_int, C.c_double, C.c_uint64, C.c_int, C.POINTER(he_ct), C.c_int],
            "he_softmax": [vp, C.POINTER(he_softmax_plan), C.POINTER(he_ct), C.c_int],
            "he_softmax_graph": [vp, C.POINTER(he_softmax_plan), C.POINTER(he_ct)],
            "he_softmax_register": [vp, C.POINTER(he_softmax_plan)],
            "he_softmax_nm": [vp, C.POINTER(he_ct), C.c_int, C.c_double, C.c_int, C.c_int],
            "he_softmax_grouped": [vp, C.POINTER(he_softmax_plan), C.POINTER(he_ct), C.c_int],
            "he_ntt": [vp, vp, C.c_int, C.c_int, C.c_int],
            "he_ct_to_coeff": [vp, C.POINTER(he_ct), u64p],
            "he_ct_from_coeff": [vp, u64p, C.POINTER(he_ct)],
            "he_encode": [vp, dblp, C.c_double, C.c_int, vp],
            "he_add": [vp, C.POINTER(he_ct), C.POINTER(he_ct)],
            "he_mul_plain": [vp, C.POINTER(he_ct), vp],
            "he_rescale": [vp, C.POINTER(he_ct), C.POINTER(he_ct)],
            "he_hmult": [vp, C.POINTER(he_ct), C.POINTER(he_ct), C.POINTER(he_ct)],
            "he_relinearize": [vp, vp, C.c_int, C.c_int, C.POINTER(he_ct)],
            "he_rotate": [vp, C.POINTER(he_ct), C.c_int, C.POINTER(he_ct)],
            "he_conjugate": [vp, C.POINTER(he_ct), C.POINTER(he_ct)],
            "he_poly_eval": [vp, C.POINTER(he_ct), dblp, C.c_int, C.c_int, C.c_double, C.POINTER(he_ct)],
            "he_lintrans": [vp, C.POINTER(he_ct), C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                            C.POINTER(he_ct)],
            "he_bootstrap": [vp, C.POINTER(he_ct), C.c_double, C.c_double, C.POINTER(he_ct)],
            "he_mod_raise": [vp, C.POINTER(he_ct), C.c_int, C.POINTER(he_ct)],
            "he_counters": [vp, C.POINTER(C.c_long)],
            "he_softmax_share_exp": [vp, C.POINTER(he_softmax_plan), C.POINTER(he_ct)],
            "he_softmax_share_square_sum": [vp, C.POINTER(he_ct), vp],
            "he_softmax_aux_round": [vp, C.POINTER(he_softmax_plan), C.c_int, C.c_int, vp, C.c_int, C.c_double,
                                     C.c_int, C.c_double, C.POINTER(he_ct), C.POINTER(he_ct)],
            "he_softmax_share_update": [vp, C.POINTER(he_softmax_plan), C.c_int, C.POINTER(he_ct), C.POINTER(he_ct),
                                        C.POINTER(he_ct)],
            "he_selftest_bounded_wait": [vp, C.c_long],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = None if name == "he_context_destroy" else C.c_int
        L.he_autotune.restype = C.c_int
        L.he_autotune.argtypes = [vp, intp, C.c_int, intp, C.c_int, C.c_int]
        L.he_tune_table.restype = C.c_int
        L.he_tune_table.argtypes = [vp, C.c_char_p, C.c_size_t]
        L.he_tune_force.restype = C.c_int
        L.he_tune_force.argtypes = [vp, C.c_int, C.c_int]
        L.he_launch_count.restype = C.c_long
        L.he_launch_count.argtypes = [vp]
        L.he_profile_kernel.restype = C.c_int
        L.he_profile_kernel.argtypes = [vp, C.c_char_p]
        L.he_profile_read.restype = C.c_int
        L.he_profile_read.argtypes = [vp, dblp, C.POINTER(C.c_long), dblp]
        L.he_profile_breakdown.restype = C.c_int
        L.he_profile_breakdown.argtypes = [vp, C.c_char_p, C.c_size_t]
        L.he_last_error.restype = C.c_char_p
        L.he_last_error.argtypes = [vp]
        _lib = L
    return _lib


def load_params():
    out = []
    for fn in ("chains.json", "plans.json", "evalmod.json"):
        with open(os.path.join(PARAMS_DIR, fn)) as fh:
            out.append(json.load(fh))
    return tuple(out)


def _hex(a):
    return np.array([float.fromhex(h) for h in a], dtype=np.float64)


class Ciphertexts:
    """A device batch [n_ct][2][level+1][N] held in a torch int64 tensor."""

    def __init__(self, ctx, tensor, level, scale, n_ct):
        self.ctx = ctx
        self.tensor = tensor
        self.level = level
        self.scale = scale
        self.n_ct = n_ct

    def c(self):
        return he_ct(self.tensor.data_ptr(), self.level, self.scale, self.n_ct)

    def update(self, h):
        self.level, self.scale, self.n_ct = h.level, h.scale, h.n_ct


def _make_params(chain, evalmod=None):
    """he_params for a chain dict (params/chains.json) and the arrays it points into (keep them
    alive as long as the struct is used)."""
    q = np.array([int(x) for x in chain["q"]], dtype=np.uint64)
    p = np.array([int(x) for x in chain["p"]], dtype=np.uint64)
    bts = int(chain.get("bootstrap", 0))
    em = _hex(evalmod["coeffs"]) if (bts and evalmod) else np.zeros(1)
    prm = he_params(chain["log_n"], len(q), q.ctypes.data_as(u64p), len(p), p.ctypes.data_as(u64p), chain["h"],
                    chain["sigma"], chain["log_scale"], chain["user_top_level"], bts, chain.get("stc_levels", 0),
                    chain.get("cts_levels", 0), chain.get("bts_min_level", 0), evalmod["K"] if evalmod else 0.0,
                    evalmod["r"] if evalmod else 0, evalmod["deg"] if evalmod else 0, em.ctypes.data_as(dblp))
    return prm, (q, p, em)


def params_insecure(chain):
    """True if the chain is below the paper's 128-bit parameter size (he_params_insecure; no GPU)."""
    prm, keep = _make_params(chain)
    rc = lib().he_params_insecure(C.byref(prm))
    if rc < 0:
        raise RuntimeError("he_params_insecure: malformed parameters (%d)" % rc)
    return bool(rc)


class Context:
    """he_ctx handle: parameters from a chain dict (params/chains.json)."""

    def __init__(self, chain, evalmod=None, stream=None, device="cuda"):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.chain = chain
        prm, (self.q, self.p, self._em) = _make_params(chain, evalmod)
        self.n = 1 << chain["log_n"]
        self.n0 = self.n // 2
        self.insecure = params_insecure(chain)   # the small test chains
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        rc = lib().he_context_create(C.byref(prm), C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc != 0:
            raise RuntimeError("he_context_create failed (%d)" % rc)
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            lib().he_context_destroy(self.h)
            self.h = None

    def check(self, rc):
        if rc != 0:
            raise RuntimeError("he_gb300 error %d: %s" % (rc, lib().he_last_error(self.h).decode()))

    # ---- buffers
    def alloc(self, level, n_ct, scale=1.0):
        t = self.torch.empty(n_ct * 2 * (level + 1) * self.n, dtype=self.torch.int64, device=self.device)
        return Ciphertexts(self, t, level, scale, n_ct)

    def like(self, x):
        return self.alloc(x.level, x.n_ct, x.scale)

    # ---- the C ABI
    def keygen(self, seed, rot_steps=()):
        r = np.array(list(rot_steps) or [0], dtype=np.int32)
        self.check(lib().he_keygen(self.h, seed, r.ctypes.data_as(intp), len(rot_steps)))

    def keygen_softmax(self, n, m):
        self.check(lib().he_keygen_softmax(self.h, n, m))

    def encrypt(self, x, n, m, M, seed, out=None):
        """he_encrypt of x [L][n] into m ciphertexts (a new buffer, or `out`'s, which must hold
        m ciphertexts at the top user level)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        if out is None:
            out = self.alloc(self.chain["user_top_level"], m)
        elif out.tensor.numel() < m * 2 * (self.chain["user_top_level"] + 1) * self.n:
            raise ValueError("encrypt: output buffer too small")
        h = out.c()
        self.check(lib().he_encrypt(self.h, x.ctypes.data_as(dblp), x.size, n, m, M, seed, C.byref(h)))
        out.update(h)
        return out

    def decrypt(self, cts, n):
        L = cts.n_ct * self.n0 // n
        y = np.zeros((L, n))
        h = cts.c()
        self.check(lib().he_decrypt(self.h, C.byref(h), n, y.ctypes.data_as(dblp), y.size))
        return y

    def encrypt_slots(self, z, level, scale, seed, ct_index=0, out=None, ct=0):
        z = np.asarray(z, dtype=np.complex128)
        buf = np.ascontiguousarray(np.stack([z.real, z.imag], axis=-1).reshape(-1))
        out = out or self.alloc(level, 1, scale)
        h = out.c()
        self.check(lib().he_encrypt_slots(self.h, buf.ctypes.data_as(dblp), level, scale, seed, ct_index,
                                          C.byref(h), ct))
        out.update(h)
        return out

    def decrypt_slots(self, cts, ct=0):
        buf = np.zeros(2 * self.n0)
        h = cts.c()
        self.check(lib().he_decrypt_slots(self.h, C.byref(h), ct, buf.ctypes.data_as(dblp)))
        return buf[0::2] + 1j * buf[1::2]

    def softmax(self, cts, plan, batched=True, graph=False):
        """he_softmax in place; graph=True: he_softmax_graph (captured once per buffer and
        shape, replayed afterwards; batched only)."""
        pl = Plan(plan)
        h = cts.c()
        if graph:
            if not batched:
                raise ValueError("graph replay runs the batched form")
            self.check(lib().he_softmax_graph(self.h, C.byref(pl.s), C.byref(h)))
        else:
            self.check(lib().he_softmax(self.h, C.byref(pl.s), C.byref(h), 1 if batched else 0))
        cts.update(h)
        return cts

    def softmax_register(self, plan):
        """he_softmax_register: the context keeps a copy of the plan for he_softmax_nm."""
        pl = Plan(plan)   # keeps the arrays the struct points into alive during the call
        self.check(lib().he_softmax_register(self.h, C.byref(pl.s)))

    def softmax_nm(self, cts, n, M, method="alg4", graph=False):
        """he_softmax_nm: Softmax of dimension n on inputs encrypted with range M, with the plan
        registered for (n, M, method); method "alg2" or "alg4"."""
        h = cts.c()
        code = {"alg2": 0, "alg4": 1}[method]
        self.check(lib().he_softmax_nm(self.h, C.byref(h), n, float(M), code, 1 if graph else 0))
        cts.update(h)
        return cts

    # ---- Alg. 4 split over shares of the main-thread ciphertexts (one share per device)
    def softmax_share_exp(self, share, plan):
        """he_softmax_share_exp: y0 = P_exp(2x/M + 1) in place on the share."""
        pl = Plan(plan)
        h = share.c()
        self.check(lib().he_softmax_share_exp(self.h, C.byref(pl.s), C.byref(h)))
        share.update(h)
        return share

    def softmax_share_square_sum(self, ys):
        """he_softmax_share_square_sum: the share's sum of y (x) y, a device tensor [3][level+1][N]."""
        d = self.torch.empty(3 * (ys.level + 1) * self.n, dtype=self.torch.int64, device=self.device)
        h = ys.c()
        self.check(lib().he_softmax_share_square_sum(self.h, C.byref(h), C.c_void_p(d.data_ptr())))
        return d

    def softmax_aux_round(self, plan, j, m_total, d_sum, level, y_scale, y0, lam, lr):
        """he_softmax_aux_round: d_sum is the elementwise integer sum of the shares' d tensors;
        lam (Lambda, updated) and lr (written) are one-ciphertext buffers at the top user level."""
        pl = Plan(plan)
        hl, hr = lam.c(), lr.c()
        self.check(lib().he_softmax_aux_round(self.h, C.byref(pl.s), j, m_total, C.c_void_p(d_sum.data_ptr()),
                                              level, y_scale, y0.level, y0.scale, C.byref(hl), C.byref(hr)))
        lam.update(hl)
        lr.update(hr)

    def softmax_share_update(self, plan, j, lr, y0, ys):
        """he_softmax_share_update: ys = (lr y0)^(2^j) for the share."""
        pl = Plan(plan)
        hl, hy, ho = lr.c(), y0.c(), ys.c()
        self.check(lib().he_softmax_share_update(self.h, C.byref(pl.s), j, C.byref(hl), C.byref(hy), C.byref(ho)))
        ys.update(ho)
        return ys

    def softmax_grouped(self, cts, plan, groups):
        """he_softmax_grouped in place: `groups` independent Softmax batches of
        cts.n_ct / groups ciphertexts each."""
        pl = Plan(plan)
        h = cts.c()
        self.check(lib().he_softmax_grouped(self.h, C.byref(pl.s), C.byref(h), groups))
        cts.update(h)
        return cts

    def to_coeff(self, cts):
        out = np.zeros((cts.n_ct, 2, cts.level + 1, self.n), dtype=np.uint64)
        h = cts.c()
        self.check(lib().he_ct_to_coeff(self.h, C.byref(h), out.ctypes.data_as(u64p)))
        return out

    def from_coeff(self, data, level, scale):
        data = np.ascontiguousarray(data, dtype=np.uint64)
        n_ct = data.size // (2 * (level + 1) * self.n)
        out = self.alloc(level, n_ct, scale)
        h = out.c()
        self.check(lib().he_ct_from_coeff(self.h, data.ctypes.data_as(u64p), C.byref(h)))
        return out

    def ntt(self, tensor, n_poly, n_limb, inverse=False):
        self.check(lib().he_ntt(self.h, C.c_void_p(tensor.data_ptr()), n_poly, n_limb, 1 if inverse else 0))

    def encode(self, z, scale, level):
        z = np.asarray(z, dtype=np.complex128)
        buf = np.ascontiguousarray(np.stack([z.real, z.imag], axis=-1).reshape(-1))
        t = self.torch.empty((level + 1) * self.n, dtype=self.torch.int64, device=self.device)
        self.check(lib().he_encode(self.h, buf.ctypes.data_as(dblp), scale, level, C.c_void_p(t.data_ptr())))
        return t

    def _unary(self, fn, a, *args, level=None):
        out = self.alloc(a.level if level is None else level, a.n_ct)
        ha, ho = a.c(), out.c()
        self.check(fn(self.h, C.byref(ha), *args, C.byref(ho)))
        out.update(ho)
        return out

    def add(self, a, b):
        ha, hb = a.c(), b.c()
        self.check(lib().he_add(self.h, C.byref(ha), C.byref(hb)))
        return a

    def mul_plain(self, a, pt):
        ha = a.c()
        self.check(lib().he_mul_plain(self.h, C.byref(ha), C.c_void_p(pt.data_ptr())))
        return a

    def rescale(self, a):
        return self._unary(lib().he_rescale, a, level=a.level - 1)

    def hmult(self, a, b):
        out = self.alloc(min(a.level, b.level), max(a.n_ct, b.n_ct))
        ha, hb, ho = a.c(), b.c(), out.c()
        self.check(lib().he_hmult(self.h, C.byref(ha), C.byref(hb), C.byref(ho)))
        out.update(ho)
        return out

    def relinearize(self, d_tensor, level, n_ct):
        out = self.alloc(level, n_ct)
        ho = out.c()
        self.check(lib().he_relinearize(self.h, C.c_void_p(d_tensor.data_ptr()), level, n_ct, C.byref(ho)))
        out.update(ho)
        return out

    def rotate(self, a, r):
        return self._unary(lib().he_rotate, a, r)

    def conjugate(self, a):
        return self._unary(lib().he_conjugate, a)

    def poly_eval(self, u, coeffs, level_out, scale_out):
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
        return self._unary(lib().he_poly_eval, u, c.ctypes.data_as(dblp), len(c) - 1, level_out, scale_out)

    def lintrans(self, a, nlev, inverse, which, gain, pt_scale):
        return self._unary(lib().he_lintrans, a, nlev, 1 if inverse else 0, which, gain, pt_scale)

    def bootstrap(self, a, gain, out_scale):
        return self._unary(lib().he_bootstrap, a, gain, out_scale, level=self.chain["user_top_level"])

    def mod_raise(self, a, top):
        return self._unary(lib().he_mod_raise, a, top, level=top)

    def counters(self):
        a = (C.c_long * 5)()
        self.check(lib().he_counters(self.h, a))
        return dict(zip(["ks", "rot", "hmult", "rescale", "bts"], list(a)))

    def launch_count(self):
        return lib().he_launch_count(self.h)

    def profile_kernel(self, name):
        self.check(lib().he_profile_kernel(self.h, (name or "").encode()))

    def profile_read(self):
        ms, n, b = C.c_double(), C.c_long(), C.c_double()
        self.check(lib().he_profile_read(self.h, C.byref(ms), C.byref(n), C.byref(b)))
        return ms.value, n.value, b.value

    def profile_breakdown(self):
        """{family: (launches, total_ms, algorithmic bytes)} since he_profile_kernel("all")
        (then resets); bytes are 0 for families without a stated byte count."""
        buf = C.create_string_buffer(1 << 14)
        self.check(lib().he_profile_breakdown(self.h, buf, len(buf)))
        out = {}
        for line in buf.value.decode().splitlines():
            name, n, ms, b = line.split()
            out[name] = (int(n), float(ms), float(b))
        return out

    # ---- autotuner (launch strategies; every variant gives the same words)
    TUNE_OPS = ("modup", "rot", "lt_small", "lt_rows", "branches", "ntt_small", "fuse_conv", "ntt_1pass")

    def autotune(self, levels, ncts, reps=2):
        lv = np.ascontiguousarray(levels, dtype=np.int32)
        nc = np.ascontiguousarray(ncts, dtype=np.int32)
        self.check(lib().he_autotune(self.h, lv.ctypes.data_as(intp), len(lv), nc.ctypes.data_as(intp), len(nc), reps))

    def tune_table(self):
        """[{op, limbs, n_ct, choice, ms: [variant 0, variant 1]}] of the autotuner's table"""
        buf = C.create_string_buffer(1 << 18)
        self.check(lib().he_tune_table(self.h, buf, len(buf)))
        out = []
        for line in buf.value.decode().splitlines():
            op, L, n, ch, m0, m1 = line.split()
            out.append({"op": self.TUNE_OPS[int(op)], "limbs": int(L), "n_ct": int(n), "choice": int(ch),
                        "ms": [float(m0), float(m1)]})
        return out

    def tune_force(self, op, choice):
        """forces variant `choice` (0 or 1) of op ("modup", "rot", "lt_small", "lt_rows", "branches",
        "ntt_small", "fuse_conv", "ntt_1pass"); -1 restores"""
        self.check(lib().he_tune_force(self.h, self.TUNE_OPS.index(op), choice))

    def selftest_bounded_wait(self, max_iter):
        return lib().he_selftest_bounded_wait(self.h, max_iter)


def load_plans_b():
    """The Alg. 4 (version B) plans, params/plans_b.json."""
    with open(os.path.join(PARAMS_DIR, "plans_b.json")) as fh:
        return json.load(fh)


class Plan:
    """he_softmax_plan built from a plan dict (params/plans.json for Alg. 2, params/plans_b.json
    for Alg. 4, version "B"); keeps the arrays alive."""

    def __init__(self, plan):
        its = plan["iters"][: plan["k"]]
        alg4 = plan.get("version") == "B"
        self.exp = _hex(plan["exp"]["coeffs"])
        self.deg = np.array([it["deg"] for it in its], dtype=np.int32)
        self.inv = np.concatenate([_hex(it["coeffs"]) for it in its])
        self.a = np.array([it["a"] for it in its])
        self.b = np.array([it["b"] for it in its])
        self.gs = np.array([it["gain_s"] for it in its])
        none = C.cast(None, dblp)
        if alg4:
            self.e = np.array([it["exponent"] for it in its])
            self.lm = np.array([it["lam_max"] for it in its])
            self.bm = np.array([it["b_max"] for it in its])
            gl, ex, lm, bm = none, self.e.ctypes.data_as(dblp), self.lm.ctypes.data_as(dblp), \
                self.bm.ctypes.data_as(dblp)
        else:
            self.gl = np.array([it["gain_l"] for it in its])
            gl, ex, lm, bm = self.gl.ctypes.data_as(dblp), none, none, none
        self.s = he_softmax_plan(plan["n"], plan["k"], plan["M"], plan["exp"]["deg"],
                                 self.exp.ctypes.data_as(dblp), self.deg.ctypes.data_as(intp),
                                 self.inv.ctypes.data_as(dblp), self.a.ctypes.data_as(dblp),
                                 self.b.ctypes.data_as(dblp), self.gs.ctypes.data_as(dblp),
                                 gl, float(plan["bts_boost"] if alg4 else plan.get("bts_boost", 1.0)),
                                 HE_SOFTMAX_ALG4 if alg4 else HE_SOFTMAX_ALG2, ex, lm, bm)
