/* Flat C entry points of the oracle for the Python test harness (ctypes).
 * Ciphertext buffers are [2][level+1][N] uint64 in coefficient form, owned by the caller. */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

orc_ctx *orc_create(int logn, int nq, const uint64_t *q, int np, const uint64_t *p, int h, double sigma) {
    if (nq > ORC_MAXQ || np > ORC_MAXP) return NULL;
    orc_ctx *c = calloc(1, sizeof(orc_ctx));
    c->logn = logn;
    c->n = 1 << logn;
    c->n0 = c->n / 2;
    c->nq = nq;
    c->np = np;
    c->alpha = np;
    c->h = h;
    c->sigma = sigma;
    int nm = nq + np;
    for (int i = 0; i < nq; i++) c->mod[i] = q[i];
    for (int i = 0; i < np; i++) c->mod[nq + i] = p[i];
    c->psi_pow = calloc(nm, sizeof(uint64_t *));
    c->psi_inv_pow = calloc(nm, sizeof(uint64_t *));
    c->omega_pow = calloc(nm, sizeof(uint64_t *));
    c->omega_inv_pow = calloc(nm, sizeof(uint64_t *));
    for (int t = 0; t < nm; t++) {
        uint64_t m = c->mod[t];
        c->psi[t] = find_psi(m, c->n);
        if (!c->psi[t]) { free(c); return NULL; }
        uint64_t pinv = invmod(c->psi[t], m), w = mulmod(c->psi[t], c->psi[t], m), winv = invmod(w, m);
        c->psi_pow[t] = malloc(sizeof(uint64_t) * c->n);
        c->psi_inv_pow[t] = malloc(sizeof(uint64_t) * c->n);
        c->omega_pow[t] = malloc(sizeof(uint64_t) * c->n / 2);
        c->omega_inv_pow[t] = malloc(sizeof(uint64_t) * c->n / 2);
        uint64_t a = 1, b = 1;
        for (int i = 0; i < c->n; i++) {
            c->psi_pow[t][i] = a;
            c->psi_inv_pow[t][i] = b;
            a = mulmod(a, c->psi[t], m);
            b = mulmod(b, pinv, m);
        }
        a = 1; b = 1;
        for (int i = 0; i < c->n / 2; i++) {
            c->omega_pow[t][i] = a;
            c->omega_inv_pow[t][i] = b;
            a = mulmod(a, w, m);
            b = mulmod(b, winv, m);
        }
    }
    fft_tables(c);
    cdt_build(c);
    return c;
}

void orc_destroy(orc_ctx *c) {
    if (!c) return;
    int nm = c->nq + c->np;
    for (int t = 0; t < nm; t++) {
        free(c->psi_pow[t]); free(c->psi_inv_pow[t]); free(c->omega_pow[t]); free(c->omega_inv_pow[t]);
    }
    free(c->psi_pow); free(c->psi_inv_pow); free(c->omega_pow); free(c->omega_inv_pow);
    free(c->zeta); free(c->rot_group);
    free(c->s); free(c->pk_a); free(c->pk_b);
    for (orc_key *k = c->keys; k;) { orc_key *nx = k->next; free(k->a); free(k->b); free(k); k = nx; }
    free(c);
}

const char *orc_error(orc_ctx *c) { return c->err; }
int orc_n(orc_ctx *c) { return c->n; }
uint64_t orc_psi(orc_ctx *c, int t) { return c->psi[t]; }

/* ---- primitives (for pinning tests) ---- */
uint64_t orc_rng_u64(uint64_t seed, uint64_t dom, uint64_t ctr) { return rng_u64(seed, dom, ctr); }
uint64_t orc_rng_uniform(uint64_t seed, uint64_t dom, uint64_t ctr, uint64_t q) { return rng_uniform_mod(seed, dom, ctr, q); }
int orc_rng_gauss(orc_ctx *c, uint64_t seed, uint64_t dom, uint64_t ctr) { return rng_gauss(c, seed, dom, ctr); }
int orc_cdt(orc_ctx *c, uint64_t *out) { memcpy(out, c->cdt, sizeof(uint64_t) * c->cdt_len); return c->cdt_len; }
void orc_hwt(int n, int h, uint64_t seed, int8_t *s) { sample_hwt(n, h, seed, s); }
void orc_ntt(orc_ctx *c, int t, uint64_t *a, int inverse) { if (inverse) ntt_inv(c, t, a); else ntt_fwd(c, t, a); }
void orc_polymul(orc_ctx *c, int t, const uint64_t *a, const uint64_t *b, uint64_t *out) { negacyclic_mul(c, t, a, b, out); }
void orc_polymul_schoolbook(int n, uint64_t q, const uint64_t *a, const uint64_t *b, uint64_t *out) { negacyclic_mul_schoolbook(n, q, a, b, out); }

static cplx *to_c(const double *re, const double *im, int n) {
    cplx *z = malloc(sizeof(cplx) * n);
    for (int i = 0; i < n; i++) { z[i].re = re[i]; z[i].im = im ? im[i] : 0.0; }
    return z;
}
static void from_c(const cplx *z, double *re, double *im, int n) {
    for (int i = 0; i < n; i++) { re[i] = z[i].re; if (im) im[i] = z[i].im; }
}

void orc_special_fft(orc_ctx *c, double *re, double *im, int inverse) {
    cplx *z = to_c(re, im, c->n0);
    if (inverse) special_fft_inv(c, z); else special_fft_fwd(c, z);
    from_c(z, re, im, c->n0);
    free(z);
}

int orc_encode(orc_ctx *c, const double *re, const double *im, double scale, int level, uint64_t *pt) {
    cplx *z = to_c(re, im, c->n0);
    int rc = encode(c, z, scale, level, pt);
    free(z);
    return rc;
}

int orc_decode(orc_ctx *c, const uint64_t *poly, int level, double scale, double *re, double *im) {
    cplx *z = malloc(sizeof(cplx) * c->n0);
    int rc = decode(c, poly, level, scale, z);
    from_c(z, re, im, c->n0);
    free(z);
    return rc;
}

int orc_decode_coeffs(orc_ctx *c, const uint64_t *poly, int level, double *out) { return decode_coeffs(c, poly, level, out); }

/* ---- keys ---- */
int orc_keygen(orc_ctx *c, uint64_t seed) { return keygen_secret(c, seed); }
int orc_secret(orc_ctx *c, int8_t *s) { if (!c->have_sk) return -1; memcpy(s, c->s, c->n); return 0; }
int orc_pk(orc_ctx *c, uint64_t *b, uint64_t *a) {
    memcpy(b, c->pk_b, sizeof(uint64_t) * (size_t)c->nq * c->n);
    memcpy(a, c->pk_a, sizeof(uint64_t) * (size_t)c->nq * c->n);
    return 0;
}
/* switching key digit j in coefficient form: [nlimb][N] for b and a */
int orc_key_digit(orc_ctx *c, int galois, int j, uint64_t *b, uint64_t *a) {
    orc_key *k = get_key(c, galois);
    if (j >= k->ndigit) return -1;
    for (int t = 0; t < k->nlimb; t++) {
        memcpy(b + (size_t)t * c->n, k->b + ((size_t)j * k->nlimb + t) * c->n, sizeof(uint64_t) * c->n);
        memcpy(a + (size_t)t * c->n, k->a + ((size_t)j * k->nlimb + t) * c->n, sizeof(uint64_t) * c->n);
        ntt_inv(c, t, b + (size_t)t * c->n);
        ntt_inv(c, t, a + (size_t)t * c->n);
    }
    return k->ndigit;
}

/* ---- ciphertext operations ---- */
static orc_ct wrap(orc_ctx *c, const uint64_t *d, int level, double scale) {
    orc_ct x = ct_alloc(c, level);
    memcpy(x.d, d, sizeof(uint64_t) * 2 * (level + 1) * c->n);
    x.scale = scale;
    return x;
}
static void unwrap(orc_ctx *c, orc_ct *x, uint64_t *out, int *level, double *scale) {
    memcpy(out, x->d, sizeof(uint64_t) * 2 * (x->level + 1) * c->n);
    if (level) *level = x->level;
    if (scale) *scale = x->scale;
    ct_free(x);
}

int orc_encrypt(orc_ctx *c, const double *re, const double *im, int level, double scale, uint64_t seed, int ct_index, uint64_t *out) {
    cplx *z = to_c(re, im, c->n0);
    orc_ct x;
    int rc = encrypt(c, z, level, scale, seed, ct_index, &x);
    free(z);
    if (rc) return rc;
    unwrap(c, &x, out, NULL, NULL);
    return 0;
}

int orc_decrypt(orc_ctx *c, const uint64_t *d, int level, double scale, double *re, double *im) {
    orc_ct x = wrap(c, d, level, scale);
    cplx *z = malloc(sizeof(cplx) * c->n0);
    int rc = decrypt(c, &x, z);
    from_c(z, re, im, c->n0);
    free(z);
    ct_free(&x);
    return rc;
}

int orc_add(orc_ctx *c, const uint64_t *a, const uint64_t *b, int level, uint64_t *out) {
    orc_ct x = wrap(c, a, level, 1.0), y = wrap(c, b, level, 1.0);
    int rc = ct_add(c, &x, &y);
    ct_free(&y);
    unwrap(c, &x, out, NULL, NULL);
    return rc;
}

int orc_mul_plain(orc_ctx *c, const uint64_t *a, int level, const uint64_t *pt, uint64_t *out) {
    orc_ct x = wrap(c, a, level, 1.0);
    int rc = ct_mul_plain(c, &x, pt, level);
    unwrap(c, &x, out, NULL, NULL);
    return rc;
}

int orc_rescale(orc_ctx *c, const uint64_t *a, int level, double scale, uint64_t *out, double *sout) {
    orc_ct x = wrap(c, a, level, scale);
    int rc = rescale(c, &x);
    if (rc) { ct_free(&x); return rc; }
    unwrap(c, &x, out, NULL, sout);
    return 0;
}

int orc_tensor(orc_ctx *c, const uint64_t *a, const uint64_t *b, int level, uint64_t *d012) {
    orc_ct x = wrap(c, a, level, 1.0), y = wrap(c, b, level, 1.0);
    size_t sz = (size_t)(level + 1) * c->n;
    int rc = tensor(c, &x, &y, d012, d012 + sz, d012 + 2 * sz, level);
    ct_free(&x);
    ct_free(&y);
    return rc;
}

int orc_relin_rescale(orc_ctx *c, const uint64_t *d012, int level, uint64_t *out) {
    size_t sz = (size_t)(level + 1) * c->n;
    orc_ct x;
    int rc = relin_rescale(c, d012, d012 + sz, d012 + 2 * sz, level, 1.0, &x);
    if (rc) return rc;
    unwrap(c, &x, out, NULL, NULL);
    return 0;
}

int orc_relin(orc_ctx *c, const uint64_t *d012, int level, uint64_t *out) {
    size_t sz = (size_t)(level + 1) * c->n;
    orc_ct x;
    int rc = relinearize(c, d012, d012 + sz, d012 + 2 * sz, level, 1.0, &x);
    if (rc) return rc;
    unwrap(c, &x, out, NULL, NULL);
    return 0;
}

/* ModUp of key switching (Sec. 2.2; see ckks.c): d [level+1][N] coefficient form ->
 * out [ndigit][(level+1) + n_p][N], extended limb index level+1+k being p_k. */
int orc_modup(orc_ctx *c, const uint64_t *d, int level, uint64_t *out) {
    if (level < 0 || level >= c->nq) return -1;
    int L = level + 1, nl = L + c->np, nd = (L + c->alpha - 1) / c->alpha;
    uint64_t *dig = modup(c, d, level);
    memcpy(out, dig, sizeof(uint64_t) * (size_t)nd * nl * c->n);
    free(dig);
    return 0;
}

/* adds round(v) to the constant coefficient of c0 (the constant v / scale on every slot) of the
 * coefficient-form ciphertext a [2][level+1][N], in place */
int orc_add_const(orc_ctx *c, uint64_t *a, int level, double v) {
    if (level < 0 || level >= c->nq) return -1;
    orc_ct x = wrap(c, a, level, 1.0);
    ct_add_const_int(c, &x, round_to_i128(v));
    unwrap(c, &x, a, NULL, NULL);
    return 0;
}

int orc_hmult(orc_ctx *c, const uint64_t *a, int la, double sa, const uint64_t *b, int lb, double sb,
              uint64_t *out, int *lout, double *sout) {
    orc_ct x = wrap(c, a, la, sa), y = wrap(c, b, lb, sb), z;
    int rc = hmult(c, &x, &y, &z);
    ct_free(&x);
    ct_free(&y);
    if (rc) return rc;
    unwrap(c, &z, out, lout, sout);
    return 0;
}

int orc_galois_for_rot(orc_ctx *c, long r) { return galois_for_rot(c, r); }

int orc_rotate(orc_ctx *c, const uint64_t *a, int level, int galois, uint64_t *out) {
    orc_ct x = wrap(c, a, level, 1.0), y;
    int rc = rotate(c, &x, galois, &y);
    ct_free(&x);
    if (rc) return rc;
    unwrap(c, &y, out, NULL, NULL);
    return 0;
}

int orc_mod_raise(orc_ctx *c, const uint64_t *a, int top, uint64_t *out) {
    orc_ct x = wrap(c, a, 0, 1.0), y;
    int rc = mod_raise(c, &x, top, &y);
    ct_free(&x);
    if (rc) return rc;
    unwrap(c, &y, out, NULL, NULL);
    return 0;
}

int orc_poly_eval(orc_ctx *c, const uint64_t *a, int level, double scale, const double *coeffs, int deg,
                  int level_out, double scale_out, uint64_t *out, double *sout) {
    orc_ct x = wrap(c, a, level, scale), y;
    int rc = poly_eval(c, &x, coeffs, deg, level_out, scale_out, &y);
    ct_free(&x);
    if (rc) return rc;
    unwrap(c, &y, out, NULL, sout);
    return 0;
}

int orc_lintrans(orc_ctx *c, const uint64_t *a, int level, double scale, int nlev, int inverse, int which,
                 double gain, double pt_scale, uint64_t *out, double *sout) {
    orc_lt_level lv[16];
    lt_levels(c, nlev, inverse, lv);
    orc_ct x = wrap(c, a, level, scale);
    cplx g; g.re = gain; g.im = 0.0;
    int rc = lt_eval_level(c, &x, &lv[which], g, pt_scale);
    if (rc) { ct_free(&x); return rc; }
    unwrap(c, &x, out, NULL, sout);
    return 0;
}

/* one linear-transform level without its final rescale: textbook = 0 as lt_eval_level (giant
 * steps share one ModDown), 1 in the textbook form (one ModDown per giant step); out at `level` */
int orc_lintrans_unrescaled(orc_ctx *c, const uint64_t *a, int level, double scale, int nlev, int inverse, int which,
                            double gain, double pt_scale, int textbook, uint64_t *out, double *sout) {
    orc_lt_level lv[16];
    lt_levels(c, nlev, inverse, lv);
    orc_ct x = wrap(c, a, level, scale);
    cplx g; g.re = gain; g.im = 0.0;
    int rc = textbook ? lt_eval_level_textbook(c, &x, &lv[which], g, pt_scale)
                      : lt_eval_level_ex(c, &x, &lv[which], g, pt_scale, 0);
    if (rc) { ct_free(&x); return rc; }
    unwrap(c, &x, out, NULL, sout);
    return 0;
}

static void fill_bts(orc_bts *b, const int *bi, const double *bd, const double *em_c) {
    b->stc_levels = bi[0];
    b->cts_levels = bi[1];
    b->top_level = bi[2];
    b->user_top = bi[3];
    b->r = bi[4];
    b->em_deg = bi[5];
    b->K = bd[0];
    b->out_scale = bd[1];
    b->em_coeffs = em_c;
}

int orc_bootstrap(orc_ctx *c, const int *bi, const double *bd, const double *em_c, const uint64_t *a, int level,
                  double scale, double gain, uint64_t *out, int *lout, double *sout) {
    orc_bts b;
    fill_bts(&b, bi, bd, em_c);
    orc_ct x = wrap(c, a, level, scale), y;
    int rc = bootstrap(c, &b, &x, gain, b.out_scale, &y);
    ct_free(&x);
    if (rc) return rc;
    unwrap(c, &y, out, lout, sout);
    return 0;
}

/* pi: n, k, exp_deg, bts_min, use_bts, inv_deg[k]; pd: M, out_scale, inv_a[k], inv_b[k],
 * gain_s[k], gain_l[k]; inv_c: concatenated coefficient arrays. cts: m buffers of the
 * input level, overwritten with the outputs. */
int orc_softmax(orc_ctx *c, const int *pi, const double *pd, const double *exp_c, const double *inv_c,
                const int *bi, const double *bd, const double *em_c,
                uint64_t *cts, int m, int level, double scale, int *lout, double *sout) {
    orc_plan p;
    memset(&p, 0, sizeof p);
    p.n = pi[0];
    p.k = pi[1];
    p.exp_deg = pi[2];
    p.bts_min = pi[3];
    p.use_bts = pi[4];
    p.M = pd[0];
    p.out_scale = pd[1];
    p.bts_boost = pd[2 + 4 * p.k];
    p.exp_c = exp_c;
    const double *cp = inv_c;
    for (int j = 0; j < p.k; j++) {
        p.inv_deg[j] = pi[5 + j];
        p.inv_c[j] = cp;
        cp += p.inv_deg[j] + 1;
        p.inv_a[j] = pd[2 + j];
        p.inv_b[j] = pd[2 + p.k + j];
        p.gain_s[j] = pd[2 + 2 * p.k + j];
        p.gain_l[j] = pd[2 + 3 * p.k + j];
    }
    orc_bts b;
    if (p.use_bts) fill_bts(&b, bi, bd, em_c);
    size_t csz = (size_t)2 * (level + 1) * c->n;
    orc_ct *x = calloc(m, sizeof(orc_ct));
    for (int i = 0; i < m; i++) x[i] = wrap(c, cts + i * csz, level, scale);
    int rc = softmax(c, &p, p.use_bts ? &b : NULL, x, m);
    if (!rc) {
        for (int i = 0; i < m; i++) unwrap(c, &x[i], cts + i * csz, lout, sout);
    } else {
        for (int i = 0; i < m; i++) ct_free(&x[i]);
    }
    free(x);
    return rc;
}

void orc_counters(orc_ctx *c, long *out) {
    out[0] = c->n_ks; out[1] = c->n_rot; out[2] = c->n_hmult; out[3] = c->n_rescale; out[4] = c->n_bts;
}
void orc_reset_counters(orc_ctx *c) { c->n_ks = c->n_rot = c->n_hmult = c->n_rescale = c->n_bts = 0; }

uint64_t orc_mix(uint64_t z) { return splitmix_mix(z); }
