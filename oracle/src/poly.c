/* Polynomial evaluation in the Chebyshev basis with exact scale targets
 * (Sec. 2.2.4: a degree-d polynomial costs ceil(log2(d+1)) levels; Table 2/3 degrees
 * 2^t - 1 use t levels).
 *
 * p(u) = sum_k c_k T_k(u), u the input ciphertext (level l_in).  eval(p, l_t, S_t) returns
 * p(u) at level l_t with scale exactly S_t (up to the rounding of the encoded constants):
 *  - leaf (deg < 8 and all T_k at level >= l_t + 1): sum_k round(c_k S_t q / S(T_k)) T_k +
 *    round(c_0 S_t q), then one rescale by q = q_{l_t+1};
 *  - otherwise, with a = 2^(ceil(log2(deg+1)) - 1), the Chebyshev division
 *    p = r + T_a q, q = c_a + sum_{i>a} 2 c_i T_{i-a}, r = sum_{i<a} c_i T_i - sum_{i>a} c_i T_{2a-i}
 *    (from T_i = 2 T_a T_{i-a} - T_{2a-i}); q is evaluated at (l_t + 1, S_t q / S(T_a)),
 *    multiplied by T_a, and r (evaluated at (l_t, S_t)) is added.
 * This uses ceil(log2(deg+1)) levels: the q-branch is one level short and recurses, the
 * r-branch has a spare level and ends in leaves.
 * Chebyshev basis: T_{2a} = 2 T_a^2 - 1; T_{a+b} = 2 T_a T_b - T_{a-b} (a the largest power of
 * two below a+b), where T_{a-b} is first brought to the scale and level of 2 T_a T_b by a
 * constant multiplication (it always has a spare level). */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define MAXT 512
#define LEAF_DEG 8

typedef struct {
    orc_ctx *c;
    orc_ct T[MAXT];
    int have[MAXT];
    int lin;
} peval;

static int ceil_log2(int x) { int r = 0; while ((1 << r) < x) r++; return r; }

static int get_T(peval *e, int k);

/* x (copy) brought to level lt and scale st by one constant product and a rescale */
static int adjust(peval *e, const orc_ct *x, int lt, double st, orc_ct *out) {
    orc_ctx *c = e->c;
    if (x->level < lt + 1) { snprintf(c->err, sizeof c->err, "adjust: level %d < %d", x->level, lt + 1); return -1; }
    *out = ct_copy(c, x);
    ct_drop(c, out, lt + 1);
    double q = (double)c->mod[lt + 1];
    ct_mul_int(c, out, round_to_i128((st * q) / x->scale));
    out->scale = st * q;
    return rescale(c, out);
}

static int get_T(peval *e, int k) {
    orc_ctx *c = e->c;
    if (k < 1 || k >= MAXT) return -1;
    if (e->have[k]) return 0;
    if ((k & (k - 1)) == 0) {
        if (get_T(e, k / 2)) return -1;
        orc_ct x;
        if (hmult(c, &e->T[k / 2], &e->T[k / 2], &x)) return -1;
        ct_mul_int(c, &x, 2);
        ct_add_const_int(c, &x, round_to_i128(-x.scale));
        e->T[k] = x;
    } else {
        int a = 1;
        while (a * 2 < k) a *= 2;
        int b = k - a;
        if (get_T(e, a) || get_T(e, b) || get_T(e, a - b)) return -1;
        orc_ct p, s;
        if (hmult(c, &e->T[a], &e->T[b], &p)) return -1;
        ct_mul_int(c, &p, 2);
        if (adjust(e, &e->T[a - b], p.level, p.scale, &s)) return -1;
        if (ct_sub(c, &p, &s)) return -1;
        ct_free(&s);
        e->T[k] = p;
    }
    e->have[k] = 1;
    return 0;
}

static int trim(const double *cf, int d) { while (d > 0 && cf[d] == 0.0) d--; return d; }

static int lincomb(peval *e, const double *cf, int d, int lt, double st, orc_ct *out) {
    orc_ctx *c = e->c;
    double q = (double)c->mod[lt + 1];
    int have = 0;
    for (int k = 1; k <= d; k++) {
        if (cf[k] == 0.0) continue;
        if (get_T(e, k)) return -1;
        orc_ct x = ct_copy(c, &e->T[k]);
        if (ct_drop(c, &x, lt + 1)) { snprintf(c->err, sizeof c->err, "lincomb: T_%d level %d", k, e->T[k].level); return -1; }
        ct_mul_int(c, &x, round_to_i128(((cf[k] * st) * q) / e->T[k].scale));
        x.scale = st * q;
        if (!have) { *out = x; have = 1; }
        else { ct_add(c, out, &x); ct_free(&x); }
    }
    if (!have) { snprintf(c->err, sizeof c->err, "lincomb: constant polynomial"); return -1; }
    ct_add_const_int(c, out, round_to_i128((cf[0] * st) * q));
    return rescale(c, out);
}

static int eval(peval *e, const double *cf_in, int d, int lt, double st, orc_ct *out) {
    orc_ctx *c = e->c;
    d = trim(cf_in, d);
    if (d < 1) { snprintf(c->err, sizeof c->err, "eval: degree 0"); return -1; }
    int avail = e->lin - lt;
    int j = ceil_log2(d + 1);
    if (avail < j) { snprintf(c->err, sizeof c->err, "eval: degree %d needs %d levels, %d left", d, j, avail); return -1; }
    if (d < LEAF_DEG && avail >= ceil_log2(d) + 1) return lincomb(e, cf_in, d, lt, st, out);
    int a = 1 << (j - 1);
    double *q = calloc(d - a + 1, sizeof(double)), *r = calloc(a, sizeof(double));
    q[0] = cf_in[a];
    for (int i = 1; i <= d - a; i++) q[i] = 2.0 * cf_in[a + i];
    for (int i = 0; i < a; i++) r[i] = cf_in[i];
    for (int i = a + 1; i <= d; i++) r[2 * a - i] = r[2 * a - i] - cf_in[i];
    if (get_T(e, a)) return -1;
    int dq = trim(q, d - a);
    int rc;
    if (dq == 0) {
        double tmp[MAXT] = {0};
        tmp[a] = q[0];
        rc = lincomb(e, tmp, a, lt, st, out);
    } else {
        double sq = (st * (double)c->mod[lt + 1]) / e->T[a].scale;
        orc_ct Q;
        rc = eval(e, q, dq, lt + 1, sq, &Q);
        if (!rc) {
            orc_ct ta = ct_copy(c, &e->T[a]);
            ct_drop(c, &ta, lt + 1);
            rc = hmult(c, &ta, &Q, out);
            ct_free(&ta);
            ct_free(&Q);
        }
    }
    if (!rc) {
        int dr = trim(r, a - 1);
        if (dr >= 1) {
            orc_ct R;
            rc = eval(e, r, dr, lt, st, &R);
            if (!rc) { rc = ct_add(c, out, &R); ct_free(&R); }
        } else {
            ct_add_const_int(c, out, round_to_i128(r[0] * out->scale));
        }
    }
    free(q);
    free(r);
    return rc;
}

int poly_eval(orc_ctx *c, const orc_ct *u, const double *coeffs, int deg, int level_out, double scale_out, orc_ct *out) {
    peval *e = calloc(1, sizeof(peval));
    e->c = c;
    e->T[1] = ct_copy(c, u);
    e->have[1] = 1;
    e->lin = u->level;
    int rc = eval(e, coeffs, deg, level_out, scale_out, out);
    for (int k = 0; k < MAXT; k++) if (e->have[k]) ct_free(&e->T[k]);
    free(e);
    return rc;
}
