/* RNS-CKKS operations (Sec. 2.2 "Functionalities" and "Levels"), written from the public
 * definitions of the scheme.  Polynomials are in coefficient form; a product of two
 * polynomials is the negacyclic convolution per RNS limb.
 *
 * Keys (secret s: ternary, exactly h nonzeros):
 *   pk  = (-a s + e, a) over q_0..q_L.
 *   swk(s' -> s), digit j (digits: blocks of alpha consecutive Q primes from q_0):
 *       b_j = -a_j s + e_j + [t in D_j] (P mod q_t) s'   on Q limbs t,
 *       b_j = -a_j s + e_j                             on P limbs.
 *     (P Q~_j with Q~_j = (Q/Q_j)[(Q/Q_j)^{-1}]_{Q_j}, which is 1 mod q_t for t in D_j and 0
 *      mod the other Q primes.)  Relinearisation: s' = s^2; rotation: s' = s(X^g).
 * Key switching of d at level l (hybrid):
 *   ModUp   : for digit D, limbs t not in D get sum_{i in D} [d_i (Q_D/q_i)^{-1}]_{q_i} (Q_D/q_i)
 *             mod m_t, each [.]_{q_i} taken as its centred representative (no further
 *             correction; the result is d + u Q_D with |u| <= |D|/2, zero mean);
 *   product : c_0 = sum_j d~_j b_j, c_1 = sum_j d~_j a_j over Q_l u P;
 *   ModDown : c_t <- (c_t - sum_k [c_{p_k} (P/p_k)^{-1}]_{p_k} (P/p_k)) P^{-1} mod q_t, with the
 *             centred representative of each [.]_{p_k} in (-p_k/2, p_k/2]: the conversion error
 *             v P (|v| <= alpha/2) then has zero mean.  With [0, p_k) representatives v has mean
 *             about alpha/2, a constant on every coefficient, whose slot values 2v/(1 - zeta_j)
 *             are large at the slots with zeta_j near 1 and cost several bits there.
 * Rotation by galois element g: ModUp of c1 first, then X -> X^g on every extended digit and
 *   on c0, then the product with swk(s(X^g) -> s) and ModDown.  The result does not depend on
 *   whether the ModUp is shared among several rotations (hoisting).
 * Rescale: r = centred [c]_{q_l} in (-q_l/2, q_l/2]; c'_i = (c_i - r) q_l^{-1} mod q_i. */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define N_ (c->n)

uint64_t dom_key(int key_id, int digit, int which) {
    return 0x100000ULL + ((uint64_t)key_id * 256ULL + (uint64_t)digit) * 2ULL + (uint64_t)which;
}

orc_ct ct_alloc(const orc_ctx *c, int level) {
    orc_ct x;
    x.level = level;
    x.scale = 1.0;
    x.d = calloc((size_t)2 * (level + 1) * c->n, sizeof(uint64_t));
    return x;
}

void ct_free(orc_ct *x) {
    free(x->d);
    x->d = NULL;
}

orc_ct ct_copy(const orc_ctx *c, const orc_ct *x) {
    orc_ct y = ct_alloc(c, x->level);
    y.scale = x->scale;
    memcpy(y.d, x->d, sizeof(uint64_t) * 2 * (x->level + 1) * c->n);
    return y;
}

uint64_t *ct_poly(const orc_ctx *c, const orc_ct *x, int poly) {
    return x->d + (size_t)poly * (x->level + 1) * c->n;
}

/* Dropping limbs above `level` keeps the value mod the smaller Q and the scale. */
int ct_drop(const orc_ctx *c, orc_ct *x, int level) {
    if (level > x->level || level < 0) return -1;
    if (level == x->level) return 0;
    orc_ct y = ct_alloc(c, level);
    y.scale = x->scale;
    for (int p = 0; p < 2; p++)
        memcpy(ct_poly(c, &y, p), ct_poly(c, x, p), sizeof(uint64_t) * (level + 1) * c->n);
    ct_free(x);
    *x = y;
    return 0;
}

/* s as residues mod modulus t */
static void sk_limb(const orc_ctx *c, int t, const int8_t *s, uint64_t *out) {
    uint64_t q = c->mod[t];
    for (int k = 0; k < N_; k++) out[k] = s[k] >= 0 ? (uint64_t)s[k] : q - (uint64_t)(-s[k]);
}

int keygen_secret(orc_ctx *c, uint64_t seed) {
    if (c->h < 1 || c->h > N_) { snprintf(c->err, sizeof c->err, "keygen: h=%d, N=%d", c->h, N_); return -1; }
    c->seed = seed;
    c->s = calloc(N_, 1);
    sample_hwt(N_, c->h, seed, c->s);
    c->pk_b = calloc((size_t)c->nq * N_, sizeof(uint64_t));
    c->pk_a = calloc((size_t)c->nq * N_, sizeof(uint64_t));
    int *e = malloc(sizeof(int) * N_);
    for (int k = 0; k < N_; k++) e[k] = rng_gauss(c, seed, DOM_PK_E, k);
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < c->nq; t++) {
        uint64_t q = c->mod[t];
        uint64_t *a = c->pk_a + (size_t)t * N_, *b = c->pk_b + (size_t)t * N_;
        uint64_t *st = malloc(sizeof(uint64_t) * N_);
        sk_limb(c, t, c->s, st);
        for (int k = 0; k < N_; k++) a[k] = rng_uniform_mod(seed, DOM_PK_A, (uint64_t)t * N_ + k, q);
        negacyclic_mul(c, t, a, st, b);
        for (int k = 0; k < N_; k++) b[k] = addmod(submod(0, b[k], q), reduce_i128(e[k], q), q);
        free(st);
    }
    free(e);
    c->have_sk = 1;
    return 0;
}

void automorph_poly(const orc_ctx *c, int t, const uint64_t *in, int g, uint64_t *out) {
    uint64_t q = c->mod[t];
    long two_n = 2L * N_;
    for (long i = 0; i < N_; i++) {
        long j = (i * (long)g) % two_n;
        if (j < N_) out[j] = in[i];
        else out[j - N_] = (q - in[i]) % q;
    }
}

orc_key *get_key(orc_ctx *c, int galois) {
    for (orc_key *k = c->keys; k; k = k->next)
        if (k->galois == galois) return k;
    int nl = c->nq + c->np;
    int nd = (c->nq + c->alpha - 1) / c->alpha;
    orc_key *key = calloc(1, sizeof(orc_key));
    key->galois = galois;
    key->nlimb = nl;
    key->ndigit = nd;
    key->a = calloc((size_t)nd * nl * N_, sizeof(uint64_t));
    key->b = calloc((size_t)nd * nl * N_, sizeof(uint64_t));
    /* integer target secret s' */
    int *e = malloc(sizeof(int) * (size_t)nd * N_);
    for (int j = 0; j < nd; j++)
        for (int k = 0; k < N_; k++) e[(size_t)j * N_ + k] = rng_gauss(c, c->seed, dom_key(galois, j, 1), k);
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < nl; t++) {
        uint64_t q = c->mod[t];
        uint64_t *st = malloc(sizeof(uint64_t) * N_), *sp = malloc(sizeof(uint64_t) * N_);
        uint64_t *tmp = malloc(sizeof(uint64_t) * N_);
        sk_limb(c, t, c->s, st);
        if (galois == 0) negacyclic_mul(c, t, st, st, sp);
        else automorph_poly(c, t, st, galois, sp);
        uint64_t pmod = 1 % q;
        for (int k = 0; k < c->np; k++) pmod = mulmod(pmod, c->mod[c->nq + k] % q, q);
        for (int j = 0; j < nd; j++) {
            uint64_t *a = key->a + ((size_t)j * nl + t) * N_, *b = key->b + ((size_t)j * nl + t) * N_;
            for (int k = 0; k < N_; k++) a[k] = rng_uniform_mod(c->seed, dom_key(galois, j, 0), (uint64_t)t * N_ + k, q);
            negacyclic_mul(c, t, a, st, tmp);
            int in_digit = t < c->nq && t / c->alpha == j;
            for (int k = 0; k < N_; k++) {
                uint64_t v = submod(reduce_i128(e[(size_t)j * N_ + k], q), tmp[k], q);
                if (in_digit) v = addmod(v, mulmod(pmod, sp[k], q), q);
                b[k] = v;
            }
            ntt_fwd(c, t, a);
            ntt_fwd(c, t, b);
        }
        free(st);
        free(sp);
        free(tmp);
    }
    free(e);
    key->next = c->keys;
    c->keys = key;
    return key;
}

int encrypt(orc_ctx *c, const cplx *z, int level, double scale, uint64_t seed, int ct_index, orc_ct *out) {
    if (!c->have_sk) return -1;
    uint64_t *pt = calloc((size_t)(level + 1) * N_, sizeof(uint64_t));
    encode(c, z, scale, level, pt);
    int *v = malloc(sizeof(int) * N_), *e0 = malloc(sizeof(int) * N_), *e1 = malloc(sizeof(int) * N_);
    for (int k = 0; k < N_; k++) {
        uint64_t ctr = (uint64_t)ct_index * N_ + k;
        v[k] = rng_ternary(seed, DOM_ENC_V, ctr);
        e0[k] = rng_gauss(c, seed, DOM_ENC_E0, ctr);
        e1[k] = rng_gauss(c, seed, DOM_ENC_E1, ctr);
    }
    *out = ct_alloc(c, level);
    out->scale = scale;
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t <= level; t++) {
        uint64_t q = c->mod[t];
        uint64_t *vt = malloc(sizeof(uint64_t) * N_);
        for (int k = 0; k < N_; k++) vt[k] = reduce_i128(v[k], q);
        uint64_t *c0 = ct_poly(c, out, 0) + (size_t)t * N_, *c1 = ct_poly(c, out, 1) + (size_t)t * N_;
        negacyclic_mul(c, t, vt, c->pk_b + (size_t)t * N_, c0);
        negacyclic_mul(c, t, vt, c->pk_a + (size_t)t * N_, c1);
        for (int k = 0; k < N_; k++) {
            c0[k] = addmod(addmod(c0[k], reduce_i128(e0[k], q), q), pt[(size_t)t * N_ + k], q);
            c1[k] = addmod(c1[k], reduce_i128(e1[k], q), q);
        }
        free(vt);
    }
    free(pt);
    free(v);
    free(e0);
    free(e1);
    return 0;
}

int decrypt(orc_ctx *c, const orc_ct *x, cplx *z) {
    int L = x->level + 1;
    uint64_t *m = malloc(sizeof(uint64_t) * (size_t)L * N_);
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < L; t++) {
        uint64_t q = c->mod[t];
        uint64_t *st = malloc(sizeof(uint64_t) * N_);
        sk_limb(c, t, c->s, st);
        negacyclic_mul(c, t, ct_poly(c, x, 1) + (size_t)t * N_, st, m + (size_t)t * N_);
        for (int k = 0; k < N_; k++) m[(size_t)t * N_ + k] = addmod(m[(size_t)t * N_ + k], ct_poly(c, x, 0)[(size_t)t * N_ + k], q);
        free(st);
    }
    decode(c, m, x->level, x->scale, z);
    free(m);
    return 0;
}

static int scales_match(double a, double b) { return fabs(a - b) <= 1e-9 * fabs(a); }

int ct_add(orc_ctx *c, orc_ct *a, const orc_ct *b) {
    if (a->level != b->level || !scales_match(a->scale, b->scale)) {
        snprintf(c->err, sizeof c->err, "add: level %d/%d scale %.17g/%.17g", a->level, b->level, a->scale, b->scale);
        return -1;
    }
    for (int p = 0; p < 2; p++)
        for (int t = 0; t <= a->level; t++) {
            uint64_t q = c->mod[t];
            uint64_t *x = ct_poly(c, a, p) + (size_t)t * N_, *y = ct_poly(c, b, p) + (size_t)t * N_;
            for (int k = 0; k < N_; k++) x[k] = addmod(x[k], y[k], q);
        }
    return 0;
}

int ct_sub(orc_ctx *c, orc_ct *a, const orc_ct *b) {
    if (a->level != b->level || !scales_match(a->scale, b->scale)) {
        snprintf(c->err, sizeof c->err, "sub: level %d/%d scale %.17g/%.17g", a->level, b->level, a->scale, b->scale);
        return -1;
    }
    for (int p = 0; p < 2; p++)
        for (int t = 0; t <= a->level; t++) {
            uint64_t q = c->mod[t];
            uint64_t *x = ct_poly(c, a, p) + (size_t)t * N_, *y = ct_poly(c, b, p) + (size_t)t * N_;
            for (int k = 0; k < N_; k++) x[k] = submod(x[k], y[k], q);
        }
    return 0;
}

void ct_mul_int(orc_ctx *c, orc_ct *a, i128 kk) {
    for (int p = 0; p < 2; p++)
        for (int t = 0; t <= a->level; t++) {
            uint64_t q = c->mod[t], km = reduce_i128(kk, q);
            uint64_t *x = ct_poly(c, a, p) + (size_t)t * N_;
            for (int k = 0; k < N_; k++) x[k] = mulmod(x[k], km, q);
        }
}

/* adds the constant polynomial kk to c0 (the constant term of every limb) */
void ct_add_const_int(orc_ctx *c, orc_ct *a, i128 kk) {
    for (int t = 0; t <= a->level; t++) {
        uint64_t q = c->mod[t];
        uint64_t *x = ct_poly(c, a, 0) + (size_t)t * N_;
        x[0] = addmod(x[0], reduce_i128(kk, q), q);
    }
}

int ct_mul_plain(orc_ctx *c, orc_ct *a, const uint64_t *pt, int pt_level) {
    if (pt_level < a->level) return -1;
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int p = 0; p < 2; p++)
        for (int t = 0; t <= a->level; t++) {
            uint64_t *x = ct_poly(c, a, p) + (size_t)t * N_;
            negacyclic_mul(c, t, x, pt + (size_t)t * N_, x);
        }
    return 0;
}

int rescale(orc_ctx *c, orc_ct *a) {
    int l = a->level;
    if (l < 1) return -1;
    orc_ct y = ct_alloc(c, l - 1);
    uint64_t ql = c->mod[l];
    for (int p = 0; p < 2; p++) {
        const uint64_t *last = ct_poly(c, a, p) + (size_t)l * N_;
#pragma omp parallel for schedule(static)
        for (int t = 0; t < l; t++) {
            uint64_t q = c->mod[t], inv = invmod(ql % q, q);
            const uint64_t *x = ct_poly(c, a, p) + (size_t)t * N_;
            uint64_t *o = ct_poly(c, &y, p) + (size_t)t * N_;
            for (int k = 0; k < N_; k++) {
                i128 r = last[k] <= (ql - 1) / 2 ? (i128)last[k] : (i128)last[k] - (i128)ql;
                o[k] = mulmod(submod(x[k], reduce_i128(r, q), q), inv, q);
            }
        }
    }
    y.scale = a->scale / (double)ql;
    ct_free(a);
    *a = y;
    c->n_rescale++;
    return 0;
}

int tensor(orc_ctx *c, const orc_ct *a, const orc_ct *b, uint64_t *d0, uint64_t *d1, uint64_t *d2, int level) {
    if (a->level < level || b->level < level) return -1;
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t <= level; t++) {
        uint64_t q = c->mod[t];
        const uint64_t *a0 = ct_poly(c, a, 0) + (size_t)t * N_, *a1 = ct_poly(c, a, 1) + (size_t)t * N_;
        const uint64_t *b0 = ct_poly(c, b, 0) + (size_t)t * N_, *b1 = ct_poly(c, b, 1) + (size_t)t * N_;
        uint64_t *tmp = malloc(sizeof(uint64_t) * N_);
        negacyclic_mul(c, t, a0, b0, d0 + (size_t)t * N_);
        negacyclic_mul(c, t, a0, b1, d1 + (size_t)t * N_);
        negacyclic_mul(c, t, a1, b0, tmp);
        for (int k = 0; k < N_; k++) d1[(size_t)t * N_ + k] = addmod(d1[(size_t)t * N_ + k], tmp[k], q);
        negacyclic_mul(c, t, a1, b1, d2 + (size_t)t * N_);
        free(tmp);
    }
    return 0;
}

/* Output: [ndigit][(level+1)+np][N]; extended limb index l+1+k is the special prime p_k. */
uint64_t *modup(orc_ctx *c, const uint64_t *d, int level) {
    int L = level + 1, nl = L + c->np, al = c->alpha;
    int nd = (L + al - 1) / al;
    uint64_t *out = calloc((size_t)nd * nl * N_, sizeof(uint64_t));
    for (int j = 0; j < nd; j++) {
        int lo = j * al, hi = (j + 1) * al < L ? (j + 1) * al : L;
        /* [ (Q_D/q_i)^{-1} ]_{q_i} */
        uint64_t qhat_inv[ORC_MAXQ];
        for (int i = lo; i < hi; i++) {
            uint64_t qi = c->mod[i], prod = 1 % qi;
            for (int i2 = lo; i2 < hi; i2++)
                if (i2 != i) prod = mulmod(prod, c->mod[i2] % qi, qi);
            qhat_inv[i] = invmod(prod, qi);
        }
#pragma omp parallel for schedule(dynamic)
        for (int tt = 0; tt < nl; tt++) {
            int t = tt < L ? tt : c->nq + (tt - L);
            uint64_t mt = c->mod[t];
            uint64_t *o = out + ((size_t)j * nl + tt) * N_;
            if (tt < L && tt >= lo && tt < hi) {
                memcpy(o, d + (size_t)tt * N_, sizeof(uint64_t) * N_);
                continue;
            }
            uint64_t qhat_t[ORC_MAXQ];
            for (int i = lo; i < hi; i++) {
                uint64_t prod = 1 % mt;
                for (int i2 = lo; i2 < hi; i2++)
                    if (i2 != i) prod = mulmod(prod, c->mod[i2] % mt, mt);
                qhat_t[i] = prod;
            }
            for (int k = 0; k < N_; k++) {
                uint64_t acc = 0;
                for (int i = lo; i < hi; i++) {
                    uint64_t qi = c->mod[i];
                    uint64_t y = mulmod(d[(size_t)i * N_ + k], qhat_inv[i], qi);
                    /* centred representative in (-q_i/2, q_i/2] */
                    i128 yc = y <= (qi - 1) / 2 ? (i128)y : (i128)y - (i128)qi;
                    acc = addmod(acc, mulmod(reduce_i128(yc, mt), qhat_t[i], mt), mt);
                }
                o[k] = acc;
            }
        }
    }
    return out;
}

/* Inner product of the (optionally automorphed) extended digits with key: the two
 * polynomials of sum_j d~_j swk_j over Q_l u P, coefficient form, [(level+1)+np][N] each,
 * added to acc0 / acc1 (which the caller zeroes for a single key switch).
 * galois 0 or 1: no automorphism. */
int ks_inner(orc_ctx *c, uint64_t *digits, int level, int galois, orc_key *key, uint64_t *acc0, uint64_t *acc1) {
    int L = level + 1, nl = L + c->np, al = c->alpha;
    int nd = (L + al - 1) / al;
#pragma omp parallel for schedule(dynamic)
    for (int tt = 0; tt < nl; tt++) {
        int t = tt < L ? tt : c->nq + (tt - L);
        uint64_t q = c->mod[t];
        uint64_t *x = malloc(sizeof(uint64_t) * N_);
        uint64_t *s0 = calloc(N_, sizeof(uint64_t)), *s1 = calloc(N_, sizeof(uint64_t));
        for (int j = 0; j < nd; j++) {
            const uint64_t *dj = digits + ((size_t)j * nl + tt) * N_;
            if (galois > 1) automorph_poly(c, t, dj, galois, x);
            else memcpy(x, dj, sizeof(uint64_t) * N_);
            ntt_fwd(c, t, x);
            const uint64_t *kb = key->b + ((size_t)j * key->nlimb + t) * N_;
            const uint64_t *ka = key->a + ((size_t)j * key->nlimb + t) * N_;
            for (int k = 0; k < N_; k++) {
                s0[k] = addmod(s0[k], mulmod(x[k], kb[k], q), q);
                s1[k] = addmod(s1[k], mulmod(x[k], ka[k], q), q);
            }
        }
        ntt_inv(c, t, s0);
        ntt_inv(c, t, s1);
        uint64_t *a0 = acc0 + (size_t)tt * N_, *a1 = acc1 + (size_t)tt * N_;
        for (int k = 0; k < N_; k++) {
            a0[k] = addmod(a0[k], s0[k], q);
            a1[k] = addmod(a1[k], s1[k], q);
        }
        free(x);
        free(s0);
        free(s1);
    }
    c->n_ks++;
    return 0;
}

/* ModDown of the two extended polynomials acc0 / acc1 (coefficient form, Q_l u P):
 * out = (acc_Q - Conv_{P->Q}([acc]_P)) P^{-1} mod q_i, i <= level. */
int moddown(orc_ctx *c, const uint64_t *acc0, const uint64_t *acc1, int level, uint64_t *out0, uint64_t *out1) {
    int L = level + 1;
    int np = c->np;
    uint64_t phat_inv[ORC_MAXP];
    for (int k = 0; k < np; k++) {
        uint64_t pk = c->mod[c->nq + k], prod = 1 % pk;
        for (int k2 = 0; k2 < np; k2++)
            if (k2 != k) prod = mulmod(prod, c->mod[c->nq + k2] % pk, pk);
        phat_inv[k] = invmod(prod, pk);
    }
    for (int which = 0; which < 2; which++) {
        const uint64_t *acc = which ? acc1 : acc0;
        uint64_t *out = which ? out1 : out0;
#pragma omp parallel for schedule(dynamic)
        for (int t = 0; t < L; t++) {
            uint64_t q = c->mod[t];
            uint64_t phat_t[ORC_MAXP], pmod = 1 % q;
            for (int k = 0; k < np; k++) {
                uint64_t prod = 1 % q;
                for (int k2 = 0; k2 < np; k2++)
                    if (k2 != k) prod = mulmod(prod, c->mod[c->nq + k2] % q, q);
                phat_t[k] = prod;
                pmod = mulmod(pmod, c->mod[c->nq + k] % q, q);
            }
            uint64_t pinv = invmod(pmod, q);
            for (int kk = 0; kk < N_; kk++) {
                uint64_t conv = 0;
                for (int k = 0; k < np; k++) {
                    uint64_t pk = c->mod[c->nq + k];
                    uint64_t y = mulmod(acc[(size_t)(L + k) * N_ + kk], phat_inv[k], pk);
                    /* centred representative of y in (-p_k/2, p_k/2] */
                    i128 yc = y <= (pk - 1) / 2 ? (i128)y : (i128)y - (i128)pk;
                    conv = addmod(conv, mulmod(reduce_i128(yc, q), phat_t[k], q), q);
                }
                out[(size_t)t * N_ + kk] = mulmod(submod(acc[(size_t)t * N_ + kk], conv, q), pinv, q);
            }
        }
    }
    return 0;
}

/* one key switch: inner product, then ModDown */
int ks_inner_moddown(orc_ctx *c, uint64_t *digits, int level, int galois, orc_key *key, uint64_t *out0, uint64_t *out1) {
    size_t nl = (size_t)(level + 1) + c->np;
    uint64_t *acc0 = calloc(nl * N_, sizeof(uint64_t)), *acc1 = calloc(nl * N_, sizeof(uint64_t));
    ks_inner(c, digits, level, galois, key, acc0, acc1);
    moddown(c, acc0, acc1, level, out0, out1);
    free(acc0);
    free(acc1);
    return 0;
}

int relinearize(orc_ctx *c, const uint64_t *d0, const uint64_t *d1, const uint64_t *d2, int level, double scale, orc_ct *out) {
    int L = level + 1;
    uint64_t *dig = modup(c, d2, level);
    *out = ct_alloc(c, level);
    out->scale = scale;
    uint64_t *o0 = ct_poly(c, out, 0), *o1 = ct_poly(c, out, 1);
    ks_inner_moddown(c, dig, level, 0, get_key(c, 0), o0, o1);
    free(dig);
    for (int t = 0; t < L; t++) {
        uint64_t q = c->mod[t];
        for (int k = 0; k < N_; k++) {
            size_t i = (size_t)t * N_ + k;
            o0[i] = addmod(o0[i], d0[i], q);
            o1[i] = addmod(o1[i], d1[i], q);
        }
    }
    return 0;
}

/* Relinearisation and rescale as one division.  K = the key switch of d2 over Q_l u P,
 * Y = P (d0, d1) + K over Q_l u P, and the output at level l - 1 is
 *   out_i = (Y_i - Conv_{D->q_i}([Y]_D)) (P q_l)^{-1} mod q_i,   D = {q_l} u P,
 * the conversion taking centred representatives as ModDown does: Y / (P q_l) rounded up to the
 * usual small conversion error, one rounding where ModDown followed by a rescale has two. */
int relin_rescale(orc_ctx *c, const uint64_t *d0, const uint64_t *d1, const uint64_t *d2, int level, double scale,
                  orc_ct *out) {
    int l = level, L = level + 1, np = c->np, nl = L + np, nd = np + 1;
    if (l < 1) { snprintf(c->err, sizeof c->err, "relin_rescale at level 0"); return -1; }
    uint64_t *dig = modup(c, d2, level);
    uint64_t *y0 = calloc((size_t)nl * N_, sizeof(uint64_t)), *y1 = calloc((size_t)nl * N_, sizeof(uint64_t));
    ks_inner(c, dig, level, 0, get_key(c, 0), y0, y1);
    free(dig);
    /* Y = K + P d on the Q limbs (P d vanishes mod every p_k) */
    for (int t = 0; t <= l; t++) {
        uint64_t q = c->mod[t], pm = 1 % q;
        for (int k = 0; k < np; k++) pm = mulmod(pm, c->mod[c->nq + k] % q, q);
        for (int k = 0; k < N_; k++) {
            size_t i = (size_t)t * N_ + k;
            y0[i] = addmod(y0[i], mulmod(d0[i], pm, q), q);
            y1[i] = addmod(y1[i], mulmod(d1[i], pm, q), q);
        }
    }
    /* the dropped moduli D: q_l (limb l), then p_0 .. p_{np-1} (limbs L ..): limbs l .. l + np */
    uint64_t md[ORC_MAXP + 1], dhat_inv[ORC_MAXP + 1];
    md[0] = c->mod[l];
    for (int k = 0; k < np; k++) md[1 + k] = c->mod[c->nq + k];
    for (int j = 0; j < nd; j++) {
        uint64_t prod = 1 % md[j];
        for (int j2 = 0; j2 < nd; j2++)
            if (j2 != j) prod = mulmod(prod, md[j2] % md[j], md[j]);
        dhat_inv[j] = invmod(prod, md[j]);
    }
    *out = ct_alloc(c, l - 1);
    out->scale = scale / (double)c->mod[l];
    for (int which = 0; which < 2; which++) {
        const uint64_t *y = which ? y1 : y0;
        uint64_t *o = ct_poly(c, out, which);
#pragma omp parallel for schedule(dynamic)
        for (int t = 0; t < l; t++) {
            uint64_t q = c->mod[t], dhat_t[ORC_MAXP + 1], dq = 1 % q;
            for (int j = 0; j < nd; j++) {
                uint64_t prod = 1 % q;
                for (int j2 = 0; j2 < nd; j2++)
                    if (j2 != j) prod = mulmod(prod, md[j2] % q, q);
                dhat_t[j] = prod;
                dq = mulmod(dq, md[j] % q, q);
            }
            uint64_t dinv = invmod(dq, q);
            for (int k = 0; k < N_; k++) {
                uint64_t conv = 0;
                for (int j = 0; j < nd; j++) {
                    uint64_t v = mulmod(y[(size_t)(l + j) * N_ + k], dhat_inv[j], md[j]);
                    i128 vc = v <= (md[j] - 1) / 2 ? (i128)v : (i128)v - (i128)md[j];
                    conv = addmod(conv, mulmod(reduce_i128(vc, q), dhat_t[j], q), q);
                }
                o[(size_t)t * N_ + k] = mulmod(submod(y[(size_t)t * N_ + k], conv, q), dinv, q);
            }
        }
    }
    free(y0);
    free(y1);
    c->n_rescale++;
    return 0;
}

/* Tensor, then relinearisation and rescale in one division.  Operands at different levels:
 * the higher is dropped. */
int hmult(orc_ctx *c, const orc_ct *a, const orc_ct *b, orc_ct *out) {
    int level = a->level < b->level ? a->level : b->level;
    if (level < 1) { snprintf(c->err, sizeof c->err, "hmult at level %d", level); return -1; }
    size_t sz = (size_t)(level + 1) * N_;
    uint64_t *d0 = malloc(sizeof(uint64_t) * sz), *d1 = malloc(sizeof(uint64_t) * sz), *d2 = malloc(sizeof(uint64_t) * sz);
    tensor(c, a, b, d0, d1, d2, level);
    int rc = relin_rescale(c, d0, d1, d2, level, a->scale * b->scale, out);
    free(d0);
    free(d1);
    free(d2);
    c->n_hmult++;
    return rc;
}

int galois_for_rot(const orc_ctx *c, long r) {
    long n0 = c->n0, m = 2L * N_;
    r %= n0;
    if (r < 0) r += n0;
    long g = 1;
    for (long i = 0; i < r; i++) g = (g * 5) % m;
    return (int)g;
}

int rotate_hoisted(orc_ctx *c, const orc_ct *x, const int *galois, int nrot, orc_ct *out) {
    int L = x->level + 1;
    uint64_t *dig = modup(c, ct_poly(c, x, 1), x->level);
    for (int r = 0; r < nrot; r++) {
        int g = galois[r];
        out[r] = ct_alloc(c, x->level);
        out[r].scale = x->scale;
        if (g == 1) {
            memcpy(out[r].d, x->d, sizeof(uint64_t) * 2 * L * N_);
            continue;
        }
        uint64_t *o0 = ct_poly(c, &out[r], 0), *o1 = ct_poly(c, &out[r], 1);
        ks_inner_moddown(c, dig, x->level, g, get_key(c, g), o0, o1);
        uint64_t *tmp = malloc(sizeof(uint64_t) * N_);
        for (int t = 0; t < L; t++) {
            uint64_t q = c->mod[t];
            automorph_poly(c, t, ct_poly(c, x, 0) + (size_t)t * N_, g, tmp);
            for (int k = 0; k < N_; k++) o0[(size_t)t * N_ + k] = addmod(o0[(size_t)t * N_ + k], tmp[k], q);
        }
        free(tmp);
        c->n_rot++;
    }
    free(dig);
    return 0;
}

int rotate(orc_ctx *c, const orc_ct *x, int galois, orc_ct *out) {
    return rotate_hoisted(c, x, &galois, 1, out);
}

/* Level-0 ciphertext lifted to level `top`: each coefficient's centred representative
 * mod q_0 reduced mod q_0..q_top. */
int mod_raise(orc_ctx *c, const orc_ct *x, int top, orc_ct *out) {
    if (x->level != 0) return -1;
    *out = ct_alloc(c, top);
    out->scale = x->scale;
    uint64_t q0 = c->mod[0];
    for (int p = 0; p < 2; p++) {
        const uint64_t *in = ct_poly(c, x, p);
        uint64_t *o = ct_poly(c, out, p);
        for (int t = 0; t <= top; t++)
            for (int k = 0; k < N_; k++) {
                i128 r = in[k] <= (q0 - 1) / 2 ? (i128)in[k] : (i128)in[k] - (i128)q0;
                o[(size_t)t * N_ + k] = reduce_i128(r, c->mod[t]);
            }
    }
    return 0;
}
