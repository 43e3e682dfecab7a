/* Homomorphic slot-to-coefficient (StC) and coefficient-to-slot (CtS) transforms for
 * bootstrapping (Sec. 2.2 "Levels": bootstrapping restores the level budget; the paper
 * uses it as a black box, so this follows the standard construction).
 *
 * StC multiplies the slot vector by D = B_{N0} ... B_4 B_2, the butterfly stages of the
 * special FFT without its bit reversal; CtS multiplies by D^{-1}.  Since the bit reversal
 * is dropped on both sides, StC followed by CtS returns the slots in their order.
 * Stage B_len (half size h = len/2, twiddle t_j = zeta^{(5^j mod 4 len) (2N / 4 len)}):
 *   i mod len <  h : y_i = x_i + t_j x_{i+h},  j = i mod len
 *   i mod len >= h : y_i = x_{i-h} - t_j x_i,  j = i mod len - h
 * and its inverse x_i = (y_i + y_{i+h})/2 or (y_{i-h} - y_i) conj(t_j)/2.
 * Consecutive stages are merged into one level; each row of the merged matrix has one
 * entry per path through the butterflies, the product of the stage factors taken in the
 * order the stages apply.  A level is evaluated as sum_d diag_d (.) Rot(x, d) with the
 * baby-step/giant-step split d = e h_min, e = a g + b (0 <= b < g, g = 2^ceil((r+1)/2)):
 *   sum_a Rot( sum_b Rot(diag_{ag+b}, -a g h_min) (.) Rot(x, b h_min), a g h_min ),
 * the plaintext products summed without rescaling, one rescale at the end of the level.
 * The giant-step rotations share one ModDown: their key-switch inner products are summed
 * over Q_l u P, the c0(X^g) parts over Q_l, and the sum is brought down by P once. */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

int lt_levels(const orc_ctx *c, int nlev, int inverse, orc_lt_level *out) {
    int s = 0;
    while ((1 << s) < c->n0) s++;
    int sizes[16], base = s / nlev, rem = s % nlev;
    for (int g = 0; g < nlev; g++) sizes[g] = base + (g < rem ? 1 : 0);
    /* forward groups: stages h = 1, 2, 4, ... in order */
    orc_lt_level fwd[16];
    int h = 1;
    for (int g = 0; g < nlev; g++) {
        fwd[g].nstage = sizes[g];
        fwd[g].inverse = 0;
        for (int k = 0; k < sizes[g]; k++) { fwd[g].h[k] = h; h <<= 1; }
    }
    if (!inverse) {
        for (int g = 0; g < nlev; g++) out[g] = fwd[g];
    } else {
        for (int g = 0; g < nlev; g++) {
            const orc_lt_level *f = &fwd[nlev - 1 - g];
            out[g].nstage = f->nstage;
            out[g].inverse = 1;
            for (int k = 0; k < f->nstage; k++) out[g].h[k] = f->h[f->nstage - 1 - k];
        }
    }
    return nlev;
}

static cplx twiddle(const orc_ctx *c, int h, int j) {
    int lenq = 8 * h, m = 2 * c->n;
    return c->zeta[(c->rot_group[j] % lenq) * (m / lenq)];
}

/* the two sources of output row i in one stage: (src index, factor) */
static void stage_sources(const orc_ctx *c, int h, int inverse, int i, int *src, cplx *f) {
    int n0 = c->n0, pos = i % (2 * h);
    if (pos < h) {
        cplx t = twiddle(c, h, pos);
        src[0] = i;
        src[1] = (i + h) % n0;
        if (!inverse) {
            f[0].re = 1.0; f[0].im = 0.0;
            f[1] = t;
        } else {
            f[0].re = 0.5; f[0].im = 0.0;
            f[1].re = 0.5; f[1].im = 0.0;
        }
    } else {
        int j = pos - h;
        cplx t = twiddle(c, h, j);
        src[0] = (i - h + n0) % n0;
        src[1] = i;
        if (!inverse) {
            f[0].re = 1.0; f[0].im = 0.0;
            f[1].re = -t.re; f[1].im = -t.im;
        } else {
            f[0].re = t.re * 0.5; f[0].im = -(t.im * 0.5);
            f[1].re = -(t.re * 0.5); f[1].im = t.im * 0.5;
        }
    }
}

/* dense diagonals: diag[e + E][i] for offsets e * hmin, e in [-E, E] */
static cplx *lt_diagonals(const orc_ctx *c, const orc_lt_level *lv, cplx gain, int *E_out, int *hmin_out) {
    int n0 = c->n0, r = lv->nstage;
    int hmin = lv->h[0];
    for (int k = 1; k < r; k++) if (lv->h[k] < hmin) hmin = lv->h[k];
    int E = (1 << r) - 1;
    cplx *diag = calloc((size_t)(2 * E + 1) * n0, sizeof(cplx));
    int npath = 1 << r;
    for (int i = 0; i < n0; i++) {
        for (int path = 0; path < npath; path++) {
            /* walk backwards from the last stage; bit k of path picks the source at stage k */
            cplx fac[32];
            int idx = i;
            for (int k = r - 1; k >= 0; k--) {
                int src[2];
                cplx f[2];
                stage_sources(c, lv->h[k], lv->inverse, idx, src, f);
                int pick = (path >> k) & 1;
                fac[k] = f[pick];
                idx = src[pick];
            }
            cplx p;
            p.re = 1.0; p.im = 0.0;
            for (int k = 0; k < r; k++) cmul(p, fac[k], &p);
            cmul(p, gain, &p);
            int off = ((idx - i) % n0 + n0) % n0;
            /* offset as signed multiple of hmin */
            int e = off / hmin;
            if (e > E) e -= n0 / hmin;
            diag[(size_t)(e + E) * n0 + i] = p;
        }
    }
    *E_out = E;
    *hmin_out = hmin;
    return diag;
}

static int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

static int bsgs_g(int r) { return 1 << ((r + 2) / 2); }

static int diag_nonzero(const cplx *d, int n0) {
    for (int i = 0; i < n0; i++) if (d[i].re != 0.0 || d[i].im != 0.0) return 1;
    return 0;
}

int lt_eval_level_ex(orc_ctx *c, orc_ct *x, const orc_lt_level *lv, cplx gain, double pt_scale, int do_rescale) {
    int n0 = c->n0, E, hmin;
    cplx *diag = lt_diagonals(c, lv, gain, &E, &hmin);
    int g = bsgs_g(lv->nstage);
    int amin = floordiv(-E, g), amax = floordiv(E, g);
    /* baby rotations present */
    int need_b[64] = {0};
    for (int e = -E; e <= E; e++)
        if (diag_nonzero(diag + (size_t)(e + E) * n0, n0)) need_b[e - floordiv(e, g) * g] = 1;
    int gal[64], bidx[64], nb = 0;
    for (int b = 0; b < g; b++) {
        bidx[b] = -1;
        if (need_b[b]) { bidx[b] = nb; gal[nb++] = galois_for_rot(c, (long)b * hmin); }
    }
    orc_ct *baby = calloc(nb, sizeof(orc_ct));
    rotate_hoisted(c, x, gal, nb, baby);
    int level = x->level;
    size_t nl = (size_t)(level + 1) + c->np;
    orc_ct acc = ct_alloc(c, level);   /* zero: sum over the giant steps */
    acc.scale = x->scale * pt_scale;
    uint64_t *ext0 = calloc(nl * c->n, sizeof(uint64_t)), *ext1 = calloc(nl * c->n, sizeof(uint64_t));
    int have_ext = 0;
    uint64_t *pt = malloc(sizeof(uint64_t) * (size_t)(level + 1) * c->n);
    cplx *rd = malloc(sizeof(cplx) * n0);
    for (int a = amin; a <= amax; a++) {
        orc_ct inner;
        int have_inner = 0;
        for (int b = 0; b < g; b++) {
            int e = a * g + b;
            if (e < -E || e > E) continue;
            const cplx *dv = diag + (size_t)(e + E) * n0;
            if (!diag_nonzero(dv, n0)) continue;
            long sh = (long)a * g * hmin;
            for (int i = 0; i < n0; i++) rd[i] = dv[(((i - sh) % n0) + n0) % n0];
            encode(c, rd, pt_scale, level, pt);
            orc_ct tmp = ct_copy(c, &baby[bidx[b]]);
            ct_mul_plain(c, &tmp, pt, level);
            if (!have_inner) { inner = tmp; have_inner = 1; }
            else {
                for (int p = 0; p < 2; p++)
                    for (int t = 0; t <= level; t++) {
                        uint64_t q = c->mod[t];
                        uint64_t *u = ct_poly(c, &inner, p) + (size_t)t * c->n, *v = ct_poly(c, &tmp, p) + (size_t)t * c->n;
                        for (int k = 0; k < c->n; k++) u[k] = addmod(u[k], v[k], q);
                    }
                ct_free(&tmp);
            }
        }
        if (!have_inner) continue;
        inner.scale = acc.scale;
        if (a == 0) {
            ct_add(c, &acc, &inner);
        } else {
            /* Rot(inner, a g h_min): c0(X^g) into acc, the key switch of c1(X^g) into ext */
            int gal_a = galois_for_rot(c, (long)a * g * hmin);
            uint64_t *dig = modup(c, ct_poly(c, &inner, 1), level);
            ks_inner(c, dig, level, gal_a, get_key(c, gal_a), ext0, ext1);
            free(dig);
            uint64_t *tmp = malloc(sizeof(uint64_t) * c->n);
            uint64_t *a0 = ct_poly(c, &acc, 0);
            for (int t = 0; t <= level; t++) {
                uint64_t q = c->mod[t];
                automorph_poly(c, t, ct_poly(c, &inner, 0) + (size_t)t * c->n, gal_a, tmp);
                for (int k = 0; k < c->n; k++) a0[(size_t)t * c->n + k] = addmod(a0[(size_t)t * c->n + k], tmp[k], q);
            }
            free(tmp);
            have_ext = 1;
            c->n_rot++;
        }
        ct_free(&inner);
    }
    if (have_ext) {
        orc_ct md = ct_alloc(c, level);
        md.scale = acc.scale;
        moddown(c, ext0, ext1, level, ct_poly(c, &md, 0), ct_poly(c, &md, 1));
        ct_add(c, &acc, &md);
        ct_free(&md);
    }
    free(ext0);
    free(ext1);
    for (int b = 0; b < nb; b++) ct_free(&baby[b]);
    free(baby);
    free(pt);
    free(rd);
    free(diag);
    ct_free(x);
    *x = acc;
    return do_rescale ? rescale(c, x) : 0;
}

int lt_eval_level(orc_ctx *c, orc_ct *x, const orc_lt_level *lv, cplx gain, double pt_scale) {
    return lt_eval_level_ex(c, x, lv, gain, pt_scale, 1);
}

/* The same level in the textbook baby-step/giant-step form, for tests of the shared ModDown:
 * every giant step is a complete rotation (its own key switch and ModDown) added to the sum,
 * and the sum is not rescaled.  Its result differs from lt_eval_level_ex's (unrescaled) only by
 * the rounding of the ModDowns: under decryption by at most (giant steps) (1 + h)(alpha + 1)/2
 * per coefficient. */
int lt_eval_level_textbook(orc_ctx *c, orc_ct *x, const orc_lt_level *lv, cplx gain, double pt_scale) {
    int n0 = c->n0, E, hmin;
    cplx *diag = lt_diagonals(c, lv, gain, &E, &hmin);
    int g = bsgs_g(lv->nstage);
    int level = x->level;
    orc_ct acc = ct_alloc(c, level);
    acc.scale = x->scale * pt_scale;
    uint64_t *pt = malloc(sizeof(uint64_t) * (size_t)(level + 1) * c->n);
    cplx *rd = malloc(sizeof(cplx) * n0);
    int rc = 0;
    for (int a = floordiv(-E, g); a <= floordiv(E, g) && !rc; a++) {
        orc_ct inner = ct_alloc(c, level);
        inner.scale = acc.scale;
        int have_inner = 0;
        for (int b = 0; b < g && !rc; b++) {
            int e = a * g + b;
            if (e < -E || e > E) continue;
            const cplx *dv = diag + (size_t)(e + E) * n0;
            if (!diag_nonzero(dv, n0)) continue;
            long sh = (long)a * g * hmin;
            for (int i = 0; i < n0; i++) rd[i] = dv[(((i - sh) % n0) + n0) % n0];
            encode(c, rd, pt_scale, level, pt);
            orc_ct r;
            if (b == 0) r = ct_copy(c, x);
            else rc = rotate(c, x, galois_for_rot(c, (long)b * hmin), &r);
            if (rc) break;
            ct_mul_plain(c, &r, pt, level);
            r.scale = acc.scale;
            ct_add(c, &inner, &r);
            ct_free(&r);
            have_inner = 1;
        }
        if (have_inner && !rc) {
            if (a == 0) {
                ct_add(c, &acc, &inner);
            } else {
                orc_ct r;
                rc = rotate(c, &inner, galois_for_rot(c, (long)a * g * hmin), &r);
                if (!rc) {
                    r.scale = acc.scale;
                    ct_add(c, &acc, &r);
                    ct_free(&r);
                }
            }
        }
        ct_free(&inner);
    }
    free(pt);
    free(rd);
    free(diag);
    ct_free(x);
    *x = acc;
    return rc;
}

int lt_rotations(const orc_ctx *c, const orc_lt_level *lv, int *gal, int max) {
    int r = lv->nstage, E = (1 << r) - 1, g = bsgs_g(r);
    int hmin = lv->h[0];
    for (int k = 1; k < r; k++) if (lv->h[k] < hmin) hmin = lv->h[k];
    int n = 0;
    for (int b = 1; b < g && n < max; b++) gal[n++] = galois_for_rot(c, (long)b * hmin);
    for (int a = floordiv(-E, g); a <= floordiv(E, g) && n < max; a++)
        if (a != 0) gal[n++] = galois_for_rot(c, (long)a * g * hmin);
    return n;
}
