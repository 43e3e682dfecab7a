"""Python face of the CPU oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this
module.  It wraps the plain C RNS-CKKS implementation in oracle/src (ciphertexts in
coefficient form) and adds two FP64 references written straight from the paper:

* softmax_fp64 : Softmax by definition (Def. 3.1), with the max shift of Lemma 3.2a
                 (exact in real arithmetic) to avoid overflow.
* simulate     : Alg. 2 in FP64 with the same polynomial approximations the encrypted
                 circuit evaluates (exp on [-M/2^k, 0], x^{-1/2} per iteration), i.e. the
                 circuit with every homomorphic error removed.
* pack/unpack  : the many-ciphertext packing of Sec. 4.2.
"""
from __future__ import annotations

import ctypes as C
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)
from build import build as _build  # noqa: E402

u64p = C.POINTER(C.c_uint64)
dblp = C.POINTER(C.c_double)
intp = C.POINTER(C.c_int)

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = C.CDLL(path)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int, C.c_int, u64p, C.c_int, u64p, C.c_int, C.c_double]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_error.restype = C.c_char_p
        L.orc_error.argtypes = [C.c_void_p]
        L.orc_psi.restype = C.c_uint64
        L.orc_psi.argtypes = [C.c_void_p, C.c_int]
        L.orc_rng_u64.restype = C.c_uint64
        L.orc_rng_u64.argtypes = [C.c_uint64] * 3
        L.orc_rng_uniform.restype = C.c_uint64
        L.orc_rng_uniform.argtypes = [C.c_uint64] * 4
        L.orc_rng_gauss.restype = C.c_int
        L.orc_rng_gauss.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64]
        L.orc_cdt.argtypes = [C.c_void_p, u64p]
        L.orc_hwt.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_void_p]
        L.orc_ntt.argtypes = [C.c_void_p, C.c_int, u64p, C.c_int]
        L.orc_polymul.argtypes = [C.c_void_p, C.c_int, u64p, u64p, u64p]
        L.orc_polymul_schoolbook.argtypes = [C.c_int, C.c_uint64, u64p, u64p, u64p]
        L.orc_special_fft.argtypes = [C.c_void_p, dblp, dblp, C.c_int]
        L.orc_encode.argtypes = [C.c_void_p, dblp, dblp, C.c_double, C.c_int, u64p]
        L.orc_decode.argtypes = [C.c_void_p, u64p, C.c_int, C.c_double, dblp, dblp]
        L.orc_decode_coeffs.argtypes = [C.c_void_p, u64p, C.c_int, dblp]
        L.orc_keygen.argtypes = [C.c_void_p, C.c_uint64]
        L.orc_secret.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_pk.argtypes = [C.c_void_p, u64p, u64p]
        L.orc_key_digit.argtypes = [C.c_void_p, C.c_int, C.c_int, u64p, u64p]
        L.orc_encrypt.argtypes = [C.c_void_p, dblp, dblp, C.c_int, C.c_double, C.c_uint64, C.c_int, u64p]
        L.orc_decrypt.argtypes = [C.c_void_p, u64p, C.c_int, C.c_double, dblp, dblp]
        L.orc_add.argtypes = [C.c_void_p, u64p, u64p, C.c_int, u64p]
        L.orc_mul_plain.argtypes = [C.c_void_p, u64p, C.c_int, u64p, u64p]
        L.orc_rescale.argtypes = [C.c_void_p, u64p, C.c_int, C.c_double, u64p, dblp]
        L.orc_tensor.argtypes = [C.c_void_p, u64p, u64p, C.c_int, u64p]
        L.orc_relin.argtypes = [C.c_void_p, u64p, C.c_int, u64p]
        L.orc_relin_rescale.argtypes = [C.c_void_p, u64p, C.c_int, u64p]
        L.orc_modup.argtypes = [C.c_void_p, u64p, C.c_int, u64p]
        L.orc_add_const.argtypes = [C.c_void_p, u64p, C.c_int, C.c_double]
        L.orc_hmult.argtypes = [C.c_void_p, u64p, C.c_int, C.c_double, u64p, C.c_int, C.c_double,
                                u64p, intp, dblp]
        L.orc_galois_for_rot.argtypes = [C.c_void_p, C.c_long]
        L.orc_rotate.argtypes = [C.c_void_p, u64p, C.c_int, C.c_int, u64p]
        L.orc_mod_raise.argtypes = [C.c_void_p, u64p, C.c_int, u64p]
        L.orc_poly_eval.argtypes = [C.c_void_p, u64p, C.c_int, C.c_double, dblp, C.c_int, C.c_int,
                                    C.c_double, u64p, dblp]
        L.orc_lintrans.argtypes = [C.c_void_p, u64p, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int,
                                   C.c_double, C.c_double, u64p, dblp]
        L.orc_lintrans_unrescaled.argtypes = [C.c_void_p, u64p, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int,
                                              C.c_double, C.c_double, C.c_int, u64p, dblp]
        L.orc_bootstrap.argtypes = [C.c_void_p, intp, dblp, dblp, u64p, C.c_int, C.c_double, C.c_double,
                                    u64p, intp, dblp]
        L.orc_softmax.argtypes = [C.c_void_p, intp, dblp, dblp, dblp, intp, dblp, dblp, u64p, C.c_int,
                                  C.c_int, C.c_double, intp, dblp]
        L.orc_mix.restype = C.c_uint64
        L.orc_mix.argtypes = [C.c_uint64]
        L.orc_counters.argtypes = [C.c_void_p, C.POINTER(C.c_long)]
        L.orc_reset_counters.argtypes = [C.c_void_p]
        _lib = L
    return _lib


def P(a, t=u64p):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


class Ct:
    """Oracle ciphertext: data [2][level+1][N] uint64 (coefficient form)."""

    def __init__(self, data, level, scale):
        self.data = data
        self.level = level
        self.scale = scale


class Oracle:
    def __init__(self, chain: dict):
        self.chain = chain
        self.q = [int(x) for x in chain["q"]]
        self.p = [int(x) for x in chain["p"]]
        self.log_n = chain["log_n"]
        self.n = 1 << self.log_n
        self.n0 = self.n // 2
        qa = np.array(self.q, dtype=np.uint64)
        pa = np.array(self.p, dtype=np.uint64)
        self.ptr = lib().orc_create(self.log_n, len(self.q), P(qa), len(self.p), P(pa), chain["h"],
                                    chain["sigma"])
        if not self.ptr:
            raise RuntimeError("oracle context creation failed")

    def __del__(self):
        if getattr(self, "ptr", None):
            lib().orc_destroy(self.ptr)
            self.ptr = None

    def _chk(self, rc):
        if rc != 0:
            raise RuntimeError("oracle: " + lib().orc_error(self.ptr).decode())

    # ---- keys / primitives
    def keygen(self, seed):
        self._chk(lib().orc_keygen(self.ptr, seed))

    def secret(self):
        s = np.zeros(self.n, dtype=np.int8)
        self._chk(lib().orc_secret(self.ptr, s.ctypes.data_as(C.c_void_p)))
        return s

    def key_digit(self, galois, j):
        nl = len(self.q) + len(self.p)
        b = np.zeros((nl, self.n), dtype=np.uint64)
        a = np.zeros((nl, self.n), dtype=np.uint64)
        nd = lib().orc_key_digit(self.ptr, galois, j, P(b), P(a))
        if nd < 0:
            raise ValueError("digit out of range")
        return b, a

    def ntt(self, t, a, inverse=False):
        a = _u64(a).copy()
        lib().orc_ntt(self.ptr, t, P(a), 1 if inverse else 0)
        return a

    def polymul(self, t, a, b):
        out = np.zeros(self.n, dtype=np.uint64)
        lib().orc_polymul(self.ptr, t, P(_u64(a)), P(_u64(b)), P(out))
        return out

    def special_fft(self, z, inverse=False):
        re = _f64(np.real(z)).copy()
        im = _f64(np.imag(z)).copy()
        lib().orc_special_fft(self.ptr, P(re, dblp), P(im, dblp), 1 if inverse else 0)
        return re + 1j * im

    def encode(self, z, scale, level):
        pt = np.zeros((level + 1, self.n), dtype=np.uint64)
        re = _f64(np.real(z))
        im = _f64(np.imag(z))
        self._chk(lib().orc_encode(self.ptr, P(re, dblp), P(im, dblp), scale, level, P(pt)))
        return pt

    def decode_coeffs(self, poly, level):
        out = np.zeros(self.n, dtype=np.float64)
        lib().orc_decode_coeffs(self.ptr, P(_u64(poly)), level, P(out, dblp))
        return out

    def decode(self, poly, level, scale):
        re = np.zeros(self.n0)
        im = np.zeros(self.n0)
        lib().orc_decode(self.ptr, P(_u64(poly)), level, scale, P(re, dblp), P(im, dblp))
        return re + 1j * im

    # ---- ciphertexts
    def encrypt(self, z, level, scale, seed, ct_index=0):
        out = np.zeros((2, level + 1, self.n), dtype=np.uint64)
        re = _f64(np.real(z))
        im = _f64(np.imag(z))
        self._chk(lib().orc_encrypt(self.ptr, P(re, dblp), P(im, dblp), level, scale, seed, ct_index, P(out)))
        return Ct(out, level, scale)

    def decrypt(self, ct):
        re = np.zeros(self.n0)
        im = np.zeros(self.n0)
        self._chk(lib().orc_decrypt(self.ptr, P(_u64(ct.data)), ct.level, ct.scale, P(re, dblp), P(im, dblp)))
        return re + 1j * im

    def add(self, a, b):
        out = np.zeros_like(a.data)
        lib().orc_add(self.ptr, P(a.data), P(b.data), a.level, P(out))
        return Ct(out, a.level, a.scale)

    def add_const(self, a, value):
        """a + value on every slot: round(value * scale) added to c0's constant coefficient."""
        out = a.data.copy()
        self._chk(lib().orc_add_const(self.ptr, P(out), a.level, value * a.scale))
        return Ct(out, a.level, a.scale)

    def mul_plain(self, a, pt):
        out = np.zeros_like(a.data)
        self._chk(lib().orc_mul_plain(self.ptr, P(a.data), a.level, P(_u64(pt)), P(out)))
        return Ct(out, a.level, a.scale)

    def rescale(self, a):
        out = np.zeros((2, a.level, self.n), dtype=np.uint64)
        s = C.c_double()
        self._chk(lib().orc_rescale(self.ptr, P(a.data), a.level, a.scale, P(out), C.byref(s)))
        return Ct(out, a.level - 1, s.value)

    def tensor(self, a, b):
        out = np.zeros((3, a.level + 1, self.n), dtype=np.uint64)
        self._chk(lib().orc_tensor(self.ptr, P(a.data), P(b.data), a.level, P(out)))
        return out

    def relin(self, d012, level):
        out = np.zeros((2, level + 1, self.n), dtype=np.uint64)
        self._chk(lib().orc_relin(self.ptr, P(_u64(d012)), level, P(out)))
        return out

    def modup(self, d, level):
        """ModUp of a coefficient-form polynomial d [level+1][N]: [ndigit][level+1+n_p][N]
        (extended limb level+1+k is the special prime p_k)."""
        nd = -(-(level + 1) // self.chain["alpha"])
        out = np.zeros((nd, level + 1 + len(self.chain["p"]), self.n), dtype=np.uint64)
        self._chk(lib().orc_modup(self.ptr, P(_u64(d)), level, P(out)))
        return out

    def relin_rescale(self, d012, level):
        """relinearisation and rescale in one division by P q_level: [2][level][N]"""
        out = np.zeros((2, level, self.n), dtype=np.uint64)
        self._chk(lib().orc_relin_rescale(self.ptr, P(_u64(d012)), level, P(out)))
        return out

    def hmult(self, a, b):
        lv = min(a.level, b.level) - 1
        out = np.zeros((2, lv + 1, self.n), dtype=np.uint64)
        lo = C.c_int()
        so = C.c_double()
        self._chk(lib().orc_hmult(self.ptr, P(a.data), a.level, a.scale, P(b.data), b.level, b.scale,
                                  P(out), C.byref(lo), C.byref(so)))
        return Ct(out, lo.value, so.value)

    def galois(self, r):
        return lib().orc_galois_for_rot(self.ptr, r)

    def rotate(self, a, r=None, galois=None):
        g = galois if galois is not None else self.galois(r)
        out = np.zeros_like(a.data)
        self._chk(lib().orc_rotate(self.ptr, P(a.data), a.level, g, P(out)))
        return Ct(out, a.level, a.scale)

    def conjugate(self, a):
        return self.rotate(a, galois=2 * self.n - 1)

    def mod_raise(self, a, top):
        out = np.zeros((2, top + 1, self.n), dtype=np.uint64)
        self._chk(lib().orc_mod_raise(self.ptr, P(a.data), top, P(out)))
        return Ct(out, top, a.scale)

    def poly_eval(self, a, coeffs, level_out, scale_out):
        coeffs = _f64(coeffs)
        out = np.zeros((2, level_out + 1, self.n), dtype=np.uint64)
        so = C.c_double()
        self._chk(lib().orc_poly_eval(self.ptr, P(a.data), a.level, a.scale, P(coeffs, dblp), len(coeffs) - 1,
                                      level_out, scale_out, P(out), C.byref(so)))
        return Ct(out, level_out, so.value)

    def lintrans(self, a, nlev, inverse, which, gain, pt_scale):
        out = np.zeros((2, a.level, self.n), dtype=np.uint64)
        so = C.c_double()
        self._chk(lib().orc_lintrans(self.ptr, P(a.data), a.level, a.scale, nlev, 1 if inverse else 0, which,
                                     gain, pt_scale, P(out), C.byref(so)))
        return Ct(out, a.level - 1, so.value)

    def lintrans_unrescaled(self, a, nlev, inverse, which, gain, pt_scale, textbook=False):
        """One linear-transform level without its final rescale (output at a.level): the giant
        steps' key switches share one ModDown, or (textbook) each giant step is a complete
        rotation with its own ModDown."""
        out = np.zeros_like(a.data)
        so = C.c_double()
        self._chk(lib().orc_lintrans_unrescaled(self.ptr, P(a.data), a.level, a.scale, nlev, 1 if inverse else 0,
                                                which, gain, pt_scale, 1 if textbook else 0, P(out), C.byref(so)))
        return Ct(out, a.level, so.value)

    def bts_args(self, evalmod):
        ch = self.chain
        top = len(self.q) - 1
        bi = np.array([ch["stc_levels"], ch["cts_levels"], top, ch["user_top_level"], evalmod["r"],
                       evalmod["deg"]], dtype=np.int32)
        bd = np.array([evalmod["K"], 2.0 ** ch["log_scale"]], dtype=np.float64)
        em = np.array([float.fromhex(h) for h in evalmod["coeffs"]], dtype=np.float64)
        return bi, bd, em

    def bootstrap(self, a, evalmod, gain=1.0, out_scale=None):
        """Bootstrapping to user_top_level: the output encrypts gain * message at out_scale
        (default Delta = 2^log_scale)."""
        bi, bd, em = self.bts_args(evalmod)
        if out_scale is not None:
            bd[1] = out_scale
        ut = self.chain["user_top_level"]
        out = np.zeros((2, ut + 1, self.n), dtype=np.uint64)
        lo = C.c_int()
        so = C.c_double()
        self._chk(lib().orc_bootstrap(self.ptr, P(bi, intp), P(bd, dblp), P(em, dblp), P(a.data), a.level,
                                      a.scale, gain, P(out), C.byref(lo), C.byref(so)))
        return Ct(out, lo.value, so.value)

    def softmax(self, cts, plan, evalmod=None):
        """Runs the Softmax circuit on a list of ciphertexts (all at one level/scale)."""
        m = len(cts)
        k = plan["k"]
        use_bts = 1 if self.chain.get("bootstrap") else 0
        pi = np.array([plan["n"], k, plan["exp"]["deg"], self.chain.get("bts_min_level", 0), use_bts]
                      + [it["deg"] for it in plan["iters"]], dtype=np.int32)
        pd = np.array([plan["M"], 2.0 ** self.chain["log_scale"]]
                      + [it["a"] for it in plan["iters"]] + [it["b"] for it in plan["iters"]]
                      + [it["gain_s"] for it in plan["iters"]] + [it["gain_l"] for it in plan["iters"]]
                      + [plan.get("bts_boost", 1.0)], dtype=np.float64)
        ec = np.array([float.fromhex(h) for h in plan["exp"]["coeffs"]], dtype=np.float64)
        ic = np.concatenate([[float.fromhex(h) for h in it["coeffs"]] for it in plan["iters"]]).astype(np.float64)
        if use_bts:
            bi, bd, em = self.bts_args(evalmod)
        else:
            bi, bd, em = np.zeros(6, np.int32), np.zeros(2), np.zeros(1)
        level = cts[0].level
        buf = np.ascontiguousarray(np.stack([c.data for c in cts]))
        lo = C.c_int()
        so = C.c_double()
        self._chk(lib().orc_softmax(self.ptr, P(pi, intp), P(pd, dblp), P(ec, dblp), P(ic, dblp), P(bi, intp),
                                    P(bd, dblp), P(em, dblp), P(buf), m, level, cts[0].scale, C.byref(lo),
                                    C.byref(so)))
        lv = lo.value
        out = []
        for i in range(m):
            flat = buf[i].reshape(-1)[: 2 * (lv + 1) * self.n]
            out.append(Ct(flat.reshape(2, lv + 1, self.n).copy(), lv, so.value))
        return out

    def softmax_b(self, cts, plan, evalmod):
        """Alg. 4 (version B) with the auxiliary thread of Alg. 3 on the m ciphertexts cts
        (packing of Sec. 4.2; all at user_top_level with scale (2/M) q_top).  Python over the
        oracle's operations; every scale is chosen so that the next polynomial input lands
        exactly at the scale of its level's prime and every bootstrapping input at Delta.

          u = 2x/M + 1 (scale bookkeeping and a constant), y0_c = P_exp(u) at scale
              sqrt(Delta q) so that S_1 = sum_c y0_c^2 comes out at Delta
          for j = 1..k:
            S_j  = RotSum(relinearised sum_c y_c (x) y_c), y = y0 (j = 1) or y^(j-1)
            v    = Bootstrap(gain_s S_j) at scale (2/(b_j - a_j)) q_top; u = affine(v)
            lam  = P_j(u) gain_s^(1/2^j) (the gain folded into the coefficients), bootstrapped
                   with a gain from its own range
            Lam  = lam (j = 1) or Lam * lam (compact: one value per Softmax in slots [0, L);
                   one level lower every iteration)
            lr   = RotSum(Lam (.) mask), mask = 1 on slots [0, L), encoded at the scale that
                   makes z land where the j squarings need it
            z_c  = lr * y0_c, y^(j)_c = z_c^(2^j) (j squarings)
        Returns the m output ciphertexts y^(k)."""
        ch = self.chain
        m, n, M, k = len(cts), plan["n"], plan["M"], plan["k"]
        top, bts_min = ch["user_top_level"], ch["bts_min_level"]
        delta = 2.0 ** ch["log_scale"]
        boost = plan["bts_boost"]
        stride, nrot = m * self.n0 // n, int(round(math.log2(n // m)))
        q = [float(v) for v in self.q]

        def bts(x, gain, out_scale):
            y = self.bootstrap(x, evalmod, gain * boost, out_scale / boost)
            y.scale *= boost
            return y

        def rotsum(x):
            for i in range(nrot):
                x = self.add(x, self.rotate(x, stride << i))
            return x

        def square_sum(ys):
            lv = ys[0].level
            qs = np.array(self.q[:lv + 1], dtype=object)[None, :, None]
            d = sum(self.tensor(y, y).astype(object) for y in ys) % qs
            out = self.relin_rescale(d.astype(np.uint64), lv)
            return rotsum(Ct(out, lv - 1, ys[0].scale * ys[0].scale / q[lv]))

        def cheb(c):
            return [float.fromhex(h) for h in c]

        # exp
        ec = cheb(plan["exp"]["coeffs"])
        de = int(math.ceil(math.log2(plan["exp"]["deg"] + 1)))
        ly0 = cts[0].level - de
        y0 = []
        for x in cts:
            u = Ct(x.data, x.level, x.scale / (2.0 / M))
            u = self.add_const(u, 1.0)
            y0.append(self.poly_eval(u, ec, ly0, math.sqrt(delta * q[ly0])))
        ys, lam_c = y0, None
        for j, it in enumerate(plan["iters"][:k], start=1):
            S = square_sum(ys)
            a, b = it["a"], it["b"]
            v = bts(S, it["gain_s"], (2.0 / (b - a)) * q[top])
            v = Ct(v.data, v.level, v.scale / (2.0 / (b - a)))
            v = self.add_const(v, -(a + b) / (b - a))
            c = np.array(cheb(it["coeffs"])) * it["gain_s"] ** it["exponent"]
            dj = int(math.ceil(math.log2(len(c))))
            lp = top - dj
            if lp < bts_min:
                lam = self._split_eval(v, c, dj, bts, delta, it["b_max"])
            else:
                lam = self.poly_eval(v, c, lp, delta)
            # lambda_j alone is bootstrapped, with a gain from its own range: iteration 1 spans
            # [n^-1/2, n^-1/2 e^A] (its bootstrapping error is removed by iteration 2, which
            # normalises the vector this very ciphertext produced), later ones lie within
            # [b_j^(-1/2^j), a_j^(-1/2^j)], narrow enough to keep the error that z^(2^j) amplifies
            # small.  Lam = Lam * lambda_j then loses one level per iteration and stays compact.
            # The plan holds that bound with a 10 % margin: lam_max = 1.1 n^(-1/2) e^A (j = 1),
            # 1.1 a_j^(-1/2^j) after that.
            lmax = it["lam_max"]
            lam_lv = top if lam_c is None else lam_c.level
            lb = bts(lam, 1.0 / lmax, q[lam_lv] * lmax)
            lb = Ct(lb.data, lb.level, lb.scale / lmax)          # lambda_j at scale q[lam_lv]
            lam_c = lb if lam_c is None else self.hmult(lam_c, lb)   # Lam keeps the scale q_top
            # where z lands and the scale it needs there: j squarings then (j < k) one more for S
            lz = ly0 - 1
            s = delta
            for i in range(j if j == k else j + 1, 0, -1):
                s = math.sqrt(s * q[lz - i + 1])
            s_lr = s * q[ly0] / y0[0].scale
            mask = np.zeros(self.n0, dtype=complex)
            mask[:stride] = 1.0
            sm = s_lr * q[lam_c.level] / lam_c.scale
            pt = self.encode(mask, sm, lam_c.level)
            lr = self.mul_plain(lam_c, pt)
            lr = Ct(lr.data, lr.level, lr.scale * sm)
            lr = rotsum(self.rescale(lr))
            ys = []
            for y in y0:
                z = self.hmult(lr, y)
                for _ in range(j):
                    z = self.hmult(z, z)
                ys.append(z)
        return ys

    def _split_eval(self, v, c, dj, bts, delta, bmax):
        """p(u) = sum c_i T_i(u) of depth dj = bootstrapping input level + 1 below the top, as
        A(u) + T_h(u) B(u) with h = 2^(dj-1) and A, B of degree < h (T_h T_j = (T_(h+j) +
        T_(h-j)) / 2): A, B and T_(h/2) take dj - 1 levels each; T_(h/2) and B are bootstrapped,
        T_h = 2 T_(h/2)^2 - 1, and the product T_h B joins A at the bootstrapping input level.
        bmax (from the plan) bounds |B| on [-1, 1] with a 10 % margin: B is bootstrapped with
        gain 1 / bmax."""
        q = [float(x) for x in self.q]
        top = v.level
        h, d = 1 << (dj - 1), len(c) - 1
        a_c, b_c = c[:h].copy(), np.zeros(d - h + 1)
        b_c[0] = c[h]
        for j in range(1, d - h + 1):
            b_c[j] = 2.0 * c[h + j]
            a_c[h - j] -= c[h + j]
        lo = top - (dj - 1)
        e = np.zeros(h // 2 + 1)
        e[-1] = 1.0
        s_t = math.sqrt(2.0 * q[top] * delta)
        t = bts(self.poly_eval(v, e, lo, delta), 1.0, s_t)
        th = self.hmult(t, t)                                   # t^2 at 2 delta = 2 t^2 at delta
        th = self.add_const(Ct(th.data, th.level, th.scale / 2.0), -1.0)
        bb = bts(self.poly_eval(v, b_c, lo, delta), 1.0 / bmax, q[top - 1] * bmax)
        bb = Ct(bb.data, bb.level, bb.scale / bmax)             # B at scale q_(top-1)
        prod = self.hmult(th, bb)
        a = self.poly_eval(v, a_c, lo, prod.scale)
        return self.add(Ct(prod.data[:, :lo + 1].copy(), lo, prod.scale), a)

    def counters(self):
        a = (C.c_long * 5)()
        lib().orc_counters(self.ptr, a)
        return dict(zip(["ks", "rot", "hmult", "rescale", "bts"], list(a)))

    def reset_counters(self):
        lib().orc_reset_counters(self.ptr)


# ------------------------------------------------------------------- FP64 references
def softmax_fp64(x):
    """SM(x)_i = exp(x_i) / sum_j exp(x_j) (Def. 3.1), rows of x independent."""
    x = np.asarray(x, dtype=np.float64)
    e = np.exp(x - x.max(axis=-1, keepdims=True))
    return e / e.sum(axis=-1, keepdims=True)


def cheb_eval(coeffs, u):
    """sum_k c_k T_k(u) by the three-term recurrence."""
    u = np.asarray(u, dtype=np.float64)
    t0 = np.ones_like(u)
    acc = coeffs[0] * t0
    if len(coeffs) == 1:
        return acc
    t1 = u
    acc = acc + coeffs[1] * t1
    for c in coeffs[2:]:
        t0, t1 = t1, 2.0 * u * t1 - t0
        acc = acc + c * t1
    return acc


def simulate(x, plan):
    """Alg. 2 in FP64 with the circuit's polynomials (no encryption error).
    x: [L][n] inputs in [-M, 0]; returns y^(k) and the per-iteration sums of squares."""
    x = np.asarray(x, dtype=np.float64)
    n, M, k = plan["n"], plan["M"], plan["k"]
    ec = [float.fromhex(h) for h in plan["exp"]["coeffs"]]
    y = cheb_eval(ec, 2.0 * x / M + 1.0)
    sums = []
    for it in plan["iters"][:k]:
        c = [float.fromhex(h) for h in it["coeffs"]]
        S = np.sum(y * y, axis=-1, keepdims=True)
        sums.append(S[..., 0])
        v = it["gain_s"] * S
        u = (2.0 * v - it["a"] - it["b"]) / (it["b"] - it["a"])
        lam = cheb_eval(c, u) * math.sqrt(it["gain_s"])
        z = lam * y
        y = z * z
    return y, sums


def simulate_b(x, plan):
    """Alg. 4 (version B) in FP64 with the plan's polynomials (no encryption error).
    lambda accumulates lambda_j = P_j(gain_s S_j) gain_s^(1/2^j), which is S_j^(-1/2^j) for
    exact P_j; z = lambda y^(0) and y^(j) = z^(2^j) by j squarings.  x: [L][n] inputs in
    [-M, 0]; returns y^(k) and the per-round sums of squares S_j."""
    x = np.asarray(x, dtype=np.float64)
    M, k = plan["M"], plan["k"]
    ec = [float.fromhex(h) for h in plan["exp"]["coeffs"]]
    y0 = cheb_eval(ec, 2.0 * x / M + 1.0)
    lam = np.ones(x.shape[:-1] + (1,))
    y, sums = y0, []
    for j, it in enumerate(plan["iters"][:k], start=1):
        c = [float.fromhex(h) for h in it["coeffs"]]
        S = np.sum(y * y, axis=-1, keepdims=True)
        sums.append(S[..., 0])
        v = it["gain_s"] * S
        u = (2.0 * v - it["a"] - it["b"]) / (it["b"] - it["a"])
        lam = lam * cheb_eval(c, u) * it["gain_s"] ** it["exponent"]
        y = lam * y0
        for _ in range(j):
            y = y * y
    return y, sums


def load_plans_b():
    """The Alg. 4 plans (params/plans_b.json), or {} where they have not been generated."""
    path = os.path.join(os.path.dirname(HERE), "paper_2410_11184_gb300", "params", "plans_b.json")
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        return json.load(fh)


def pack(x, m, n0):
    """Sec. 4.2 packing: x [L][n] -> m slot vectors; slot t*L + l of ct c holds x[l][c*(n/m) + t]."""
    x = np.asarray(x, dtype=np.float64)
    L, n = x.shape
    assert n % m == 0 and L * n == m * n0, "need L*n == m*N0"
    per = n // m
    out = np.zeros((m, n0))
    for c in range(m):
        for t in range(per):
            out[c, t * L:(t + 1) * L] = x[:, c * per + t]
    return out


def unpack(slots, n):
    """Inverse of pack: m slot vectors -> [L][n]."""
    slots = np.asarray(slots)
    m, n0 = slots.shape
    L = m * n0 // n
    per = n // m
    x = np.zeros((L, n))
    for c in range(m):
        for t in range(per):
            x[:, c * per + t] = slots[c, t * L:(t + 1) * L]
    return x


def load_params():
    base = os.path.join(os.path.dirname(HERE), "paper_2410_11184_gb300", "params")
    out = []
    for fn in ("chains.json", "plans.json", "evalmod.json"):
        with open(os.path.join(base, fn)) as fh:
            out.append(json.load(fh))
    return tuple(out)
