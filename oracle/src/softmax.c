/* The normalize-and-square Softmax circuit on m ciphertexts (Alg. 2 with the auxiliary
 * thread of Alg. 3, many-ciphertext packing of Sec. 4.2, bootstrapping placement of
 * Sec. 5.1.3).
 *
 * Packing: L = m N0 / n Softmax; ciphertext c holds coordinate c (n/m) + t of Softmax l
 * in slot t L + l (t < n/m).  Rotations by L 2^i (i < log2(n/m)) sum over t.
 * Inputs are encrypted at level user_top with scale (2/M) q_{user_top}, so that
 * u = 2x/M + 1 is obtained by scale bookkeeping plus a constant add and lands at scale
 * q_{user_top}.
 *
 *   y_c   = P_exp(u_c)                                     (exp(x/2^k))
 *   for j = 1..k:
 *     (fallback: bootstrapping of every y_c if level(y) < bts_min + 1)
 *     S    = Relin(sum_c y_c (x) y_c), rescaled in the same division (Step 1 of Alg. 3, one key switch)
 *     S    = RotSum(S, L, log2(n/m))                      (Steps 3-5)
 *     if level(S) - depth_j - 1 >= bts_min: v = gain_s S by scale bookkeeping
 *     else                                 : v = Bootstrap(S, gain_s)
 *     lam  = P_j(u), u = (2v - a_j - b_j)/(b_j - a_j)      (Step 6)
 *     if lam would end below level(y) (and, in the last round, fewer than 2 levels remain):
 *         lam = Bootstrap(lam, gain_l)                     (gain removed by bookkeeping)
 *     lam  = lam (.) mask, mask = sqrt(gain_s) on slots [0, L), rescaled   (Step 7)
 *     lam  = RotSum(lam, L, log2(n/m))                    (Steps 8-10)
 *     z_c  = lam * y_c                                     (normalize)
 *     if another round follows and z_c^2 would sit below bts_min + 1: z_c = Bootstrap(z_c)
 *     y_c  = z_c * z_c                                     (square)
 *   return y
 *
 * Scales.  A Chebyshev evaluation needs its input at the scale of the prime at its level,
 * else T_{2^i} drift away from it.  Every free scale (polynomial outputs, the mask encoding
 * scale, bootstrapping outputs) is therefore chosen so that the next polynomial input lands
 * exactly there:
 *   y entering round j must have  sqrt(a'_j q_{l-1} q_l)   (l its level, a'_j =
 *     2 gain_s / (b_j - a_j)) when S_j is not bootstrapped, else Delta;
 *   lam must have (sqrt(T q_{lz - 1}) q_{lz}) / scale(y), lz = min(level(lam), level(y)),
 *     T the target of the next y, or (Delta q_{lz}) / scale(y) when z is bootstrapped, whose
 *     output scale is then sqrt(T q_{user_top});
 *   a bootstrapped S gets output scale (2/(b_j - a_j)) q_{user_top};
 *   inputs of bootstrapping are kept near Delta. */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static int ilog2(int x) { int r = 0; while ((1 << r) < x) r++; return r; }

static double qd(const orc_ctx *c, int l) { return (double)c->mod[l]; }

/* ORC_DEBUG=1 prints the first decrypted slots of each intermediate (diagnostics only) */
static void dbg(orc_ctx *c, const char *what, int j, const orc_ct *x) {
    if (!getenv("ORC_DEBUG")) return;
    cplx *z = malloc(sizeof(cplx) * c->n0);
    decrypt(c, x, z);
    fprintf(stderr, "[%d] %-8s lvl %2d log2(scale) %.6f : %.6g %.6g %.6g %.6g\n", j, what, x->level, log2(x->scale),
            z[0].re, z[1].re, z[2].re, z[c->n0 / 2].re);
    free(z);
}

static int rotsum(orc_ctx *c, orc_ct *x, int stride, int nrot) {
    for (int i = 0; i < nrot; i++) {
        orc_ct r;
        if (rotate(c, x, galois_for_rot(c, (long)stride << i), &r)) return -1;
        if (ct_add(c, x, &r)) return -1;
        ct_free(&r);
    }
    return 0;
}

/* x holds v in [a, b]; scale bookkeeping plus a constant turn it into u = (2v - a - b)/(b - a) */
static void affine_to_unit(orc_ctx *c, orc_ct *x, double a, double b) {
    double alpha = 2.0 / (b - a), beta = -(a + b) / (b - a);
    x->scale = x->scale / alpha;
    ct_add_const_int(c, x, round_to_i128(beta * x->scale));
}

/* bootstrapping with the plan's input boost B: StC multiplies the message by gain B and the
 * result (which encrypts gain B x at scale out_scale / B) is read as gain x at scale out_scale */
static int bts(orc_ctx *c, const orc_plan *p, const orc_bts *b, const orc_ct *x, double gain, double out_scale, orc_ct *out) {
    int rc = bootstrap(c, b, x, gain * p->bts_boost, out_scale / p->bts_boost, out);
    if (!rc) out->scale = out->scale * p->bts_boost;
    return rc;
}

/* fallback: y cannot feed S = sum y^2 into a bootstrappable level */
static int main_bts(const orc_plan *p, int j, int ly) {
    (void)j;
    return p->use_bts && ly < p->bts_min + 1;
}

/* z = lam y is computed at product level lz (z at lz - 1); it is bootstrapped when another round
 * follows and y = z^2 (level lz - 2) would be too low for the next round's S */
static int z_bts(const orc_plan *p, int j, int lz) {
    return p->use_bts && j < p->k - 1 && lz - 2 < p->bts_min + 1;
}

static int s_bts(const orc_plan *p, int j, int ly) {
    return p->use_bts && ((ly - 1) - ilog2(p->inv_deg[j] + 1) - 1 < p->bts_min);
}

/* scale y must have on entering round j at level ly (before a possible main bootstrap) */
static double y_target(const orc_ctx *c, const orc_plan *p, int j, int ly) {
    if (j >= p->k || main_bts(p, j, ly) || s_bts(p, j, ly)) return p->out_scale;
    double ap = (2.0 / (p->inv_b[j] - p->inv_a[j])) * p->gain_s[j];
    return sqrt((ap * qd(c, ly - 1)) * qd(c, ly));
}

int softmax(orc_ctx *c, const orc_plan *p, const orc_bts *b, orc_ct *cts, int m) {
    int n0 = c->n0, n = p->n;
    if (n % m || n0 % n) { snprintf(c->err, sizeof c->err, "softmax: bad n/m"); return -1; }
    int stride = (int)((long)m * n0 / n);
    int nrot = ilog2(n / m);
    int ut = p->use_bts ? b->user_top : 0;
    /* exp */
    for (int i = 0; i < m; i++) {
        orc_ct y;
        affine_to_unit(c, &cts[i], -p->M, 0.0);
        int lvl = cts[i].level - ilog2(p->exp_deg + 1);
        if (poly_eval(c, &cts[i], p->exp_c, p->exp_deg, lvl, y_target(c, p, 0, lvl), &y)) return -1;
        ct_free(&cts[i]);
        cts[i] = y;
    }
    dbg(c, "y0", 0, &cts[0]);
    for (int j = 0; j < p->k; j++) {
        int ly = cts[0].level;
        if (main_bts(p, j, ly)) {
            double so = y_target(c, p, j, ut);
            for (int i = 0; i < m; i++) {
                orc_ct y;
                if (bts(c, p, b, &cts[i], 1.0, so, &y)) return -1;
                ct_free(&cts[i]);
                cts[i] = y;
            }
            ly = cts[0].level;
            dbg(c, "y-bts", j, &cts[0]);
        }
        /* S = sum y^2, one relinearisation */
        size_t sz = (size_t)(ly + 1) * c->n;
        uint64_t *d0 = calloc(sz, 8), *d1 = calloc(sz, 8), *d2 = calloc(sz, 8);
        uint64_t *e0 = malloc(sz * 8), *e1 = malloc(sz * 8), *e2 = malloc(sz * 8);
        for (int i = 0; i < m; i++) {
            tensor(c, &cts[i], &cts[i], e0, e1, e2, ly);
            for (int t = 0; t <= ly; t++) {
                uint64_t q = c->mod[t];
                for (int k = 0; k < c->n; k++) {
                    size_t x = (size_t)t * c->n + k;
                    d0[x] = addmod(d0[x], e0[x], q);
                    d1[x] = addmod(d1[x], e1[x], q);
                    d2[x] = addmod(d2[x], e2[x], q);
                }
            }
        }
        free(e0); free(e1); free(e2);
        orc_ct S;
        if (relin_rescale(c, d0, d1, d2, ly, cts[0].scale * cts[0].scale, &S)) return -1;
        free(d0); free(d1); free(d2);
        c->n_hmult++;
        if (rotsum(c, &S, stride, nrot)) return -1;
        dbg(c, "S", j, &S);
        int dj = ilog2(p->inv_deg[j] + 1);
        orc_ct v;
        if (!s_bts(p, j, ly)) {
            v = S;
            v.scale = v.scale / p->gain_s[j];
        } else {
            double so = (2.0 / (p->inv_b[j] - p->inv_a[j])) * qd(c, ut);
            if (bts(c, p, b, &S, p->gain_s[j], so, &v)) return -1;
            ct_free(&S);
        }
        dbg(c, "v", j, &v);
        affine_to_unit(c, &v, p->inv_a[j], p->inv_b[j]);
        dbg(c, "u", j, &v);
        orc_ct lam;
        int lp = v.level - dj;
        if (poly_eval(c, &v, p->inv_c[j], p->inv_deg[j], lp, p->out_scale, &lam)) return -1;
        ct_free(&v);
        dbg(c, "lam", j, &lam);
        /* where lambda will meet y, and the scale it must have there */
        /* lambda is bootstrapped right after the polynomial when it would end below y (except
         * in the last round if two levels remain for z = lam y and y = z^2); masking and
         * replication follow, so every slot of a Softmax carries the same value and the same
         * error (Alg. 3, Steps 7-10), which the next normalisation removes */
        int lam_bts = p->use_bts && lp - 1 < ly && !(j == p->k - 1 && lp - 1 >= 2);
        int llam = lam_bts ? ut - 1 : lp - 1;
        int lz = llam < ly ? llam : ly;
        int zb = z_bts(p, j, lz);
        double slam;
        if (zb) {
            slam = (p->out_scale * qd(c, lz)) / cts[0].scale;
        } else {
            double tgt = y_target(c, p, j + 1, lz - 2);
            double sz_ = sqrt(tgt * qd(c, lz - 1));
            slam = (sz_ * qd(c, lz)) / cts[0].scale;
        }
        int lm = lp;
        if (lam_bts) {
            orc_ct lb;
            if (bts(c, p, b, &lam, p->gain_l[j], p->out_scale, &lb)) return -1;
            ct_free(&lam);
            lam = lb;
            lm = lam.level;
        }
        /* mask */
        cplx *mk = calloc(n0, sizeof(cplx));
        double mval = sqrt(p->gain_s[j]);
        for (int i = 0; i < stride; i++) mk[i].re = mval;
        double sm = (slam * qd(c, lm)) / lam.scale;
        if (lam_bts) sm = sm / p->gain_l[j];
        uint64_t *pt = malloc(sizeof(uint64_t) * (size_t)(lm + 1) * c->n);
        encode(c, mk, sm, lm, pt);
        ct_mul_plain(c, &lam, pt, lm);
        lam.scale = lam.scale * sm;
        free(pt);
        free(mk);
        if (rescale(c, &lam)) return -1;
        if (rotsum(c, &lam, stride, nrot)) return -1;
        if (lam_bts) lam.scale = lam.scale * p->gain_l[j];
        dbg(c, "lam-fin", j, &lam);
        double soz = zb ? sqrt(y_target(c, p, j + 1, ut - 1) * qd(c, ut)) : 0.0;
        for (int i = 0; i < m; i++) {
            orc_ct zc, yc;
            if (hmult(c, &lam, &cts[i], &zc)) return -1;
            if (zb) {
                /* z = lam y has its maximum in [n^{-1/2}, 1] (Sec. 3.2): bootstrapping it
                 * instead of y keeps the relative error small for flat distributions */
                orc_ct zz;
                if (bts(c, p, b, &zc, 1.0, soz, &zz)) return -1;
                ct_free(&zc);
                zc = zz;
            }
            if (hmult(c, &zc, &zc, &yc)) return -1;
            ct_free(&zc);
            ct_free(&cts[i]);
            cts[i] = yc;
        }
        ct_free(&lam);
        dbg(c, "y", j, &cts[0]);
    }
    return 0;
}
