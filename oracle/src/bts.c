/* Full-slot CKKS bootstrapping, slot-to-coefficient first (Sec. 2.2 "Levels" uses it as a
 * black box; the paper's Table 4 gives only its precision and cost).
 *
 *   x (level >= stc_levels, scale D_in, message z)
 *   -> drop to level stc_levels
 *   -> StC: slots (gain z) become the coefficients, in bit-reversed order (stc_levels levels)
 *   -> ModRaise to the top level: the plaintext becomes t = D_in gain z + q_0 I
 *   -> CtS: slots t_k / (2 K q_0) + i (...) (cts_levels levels, output scale S_em)
 *   -> u = ct + conj(ct): real part, t_k / (K q_0) in [-1, 1]
 *   -> EvalMod: c = cos(2 pi (K u - 1/4) / 2^r) (Chebyshev), then r times c <- 2c^2 - 1,
 *      giving sin(2 pi t / q_0) ~ 2 pi D_in gain z / q_0
 *   -> the result encrypts gain z with scale S_out 2 pi D_in / q_0.
 * The target scales of the double-angle steps are chosen backwards so that the output
 * scale is the requested out_scale. */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define ORC_PI 3.14159265358979323846

int bootstrap(orc_ctx *c, const orc_bts *b, const orc_ct *x, double gain, double out_scale, orc_ct *out) {
    if (x->level < b->stc_levels) { snprintf(c->err, sizeof c->err, "bootstrap: level %d", x->level); return -1; }
    orc_ct y = ct_copy(c, x);
    ct_drop(c, &y, b->stc_levels);
    orc_lt_level lv[16];
    /* SlotToCoeff */
    lt_levels(c, b->stc_levels, 0, lv);
    for (int g = 0; g < b->stc_levels; g++) {
        cplx gn;
        gn.re = g == 0 ? gain : 1.0;
        gn.im = 0.0;
        if (lt_eval_level(c, &y, &lv[g], gn, (double)c->mod[y.level])) return -1;
    }
    double d_in = y.scale;
    /* ModRaise */
    orc_ct z;
    if (mod_raise(c, &y, b->top_level, &z)) return -1;
    ct_free(&y);
    z.scale = (double)c->mod[0];
    /* CoeffToSlot, last level lands on the EvalMod input scale */
    int em_in_level = b->top_level - b->cts_levels;
    double s_em = (double)c->mod[em_in_level];
    lt_levels(c, b->cts_levels, 1, lv);
    for (int g = 0; g < b->cts_levels; g++) {
        cplx gn;
        gn.re = g == b->cts_levels - 1 ? 1.0 / (2.0 * b->K) : 1.0;
        gn.im = 0.0;
        double qs = (double)c->mod[z.level];
        double pts = g == b->cts_levels - 1 ? (qs * s_em) / z.scale : qs;
        if (lt_eval_level(c, &z, &lv[g], gn, pts)) return -1;
    }
    /* real part */
    orc_ct cj;
    if (rotate(c, &z, 2 * c->n - 1, &cj)) return -1;
    if (ct_add(c, &z, &cj)) return -1;
    ct_free(&cj);
    /* EvalMod */
    int lp = b->user_top + b->r;
    double s_f = (out_scale * (double)c->mod[0]) / (2.0 * ORC_PI * d_in);
    double s_in = s_f;
    for (int i = b->r; i >= 1; i--) s_in = sqrt(s_in * (double)c->mod[lp - i + 1]);
    orc_ct cc;
    if (poly_eval(c, &z, b->em_coeffs, b->em_deg, lp, s_in, &cc)) return -1;
    ct_free(&z);
    for (int i = 0; i < b->r; i++) {
        orc_ct sq;
        if (hmult(c, &cc, &cc, &sq)) return -1;
        ct_free(&cc);
        ct_mul_int(c, &sq, 2);
        ct_add_const_int(c, &sq, round_to_i128(-sq.scale));
        cc = sq;
    }
    cc.scale = ((cc.scale * (2.0 * ORC_PI)) * d_in) / (double)c->mod[0];
    *out = cc;
    c->n_bts++;
    return 0;
}
