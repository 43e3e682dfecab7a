/* Canonical embedding (Sec. 2.2: messages are vectors of N0 = N/2 complex slots).
 *
 * A real polynomial t(X) of degree < N is paired with w in C^{N0}, w_k = t_k + i t_{k+N0},
 * and its slots are z_j = t(zeta^{5^j}) = sum_{k<N0} w_k zeta^{5^j k}, zeta = exp(i pi/N)
 * (because zeta_j^{N0} = i).  special_fft_fwd computes z from w in O(N0 log N0) through
 * the even/odd split t(x) = E(x^2) + x O(x^2) and zeta_{j+N0/2} = -zeta_j; the inverse
 * undoes each stage and divides by N0.  Tests pin both against the O(N0^2) sums.
 *
 * Encoding rounds scale * t_k to the nearest integer (ties to even); decoding lifts each
 * coefficient from RNS to the centred integer by Garner's mixed-radix form.  All double
 * arithmetic is written as separate IEEE operations (compiled with -ffp-contract=off). */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define ORC_PI 3.14159265358979323846

void cmul(cplx a, cplx b, cplx *out) {
    double re = a.re * b.re - a.im * b.im;
    double im = a.re * b.im + a.im * b.re;
    out->re = re;
    out->im = im;
}

void fft_tables(orc_ctx *c) {
    int m = 2 * c->n;
    c->zeta = malloc(sizeof(cplx) * m);
    for (int j = 0; j < m; j++) {
        double ang = (2.0 * ORC_PI * (double)j) / (double)m;
        c->zeta[j].re = cos(ang);
        c->zeta[j].im = sin(ang);
    }
    c->rot_group = malloc(sizeof(int) * c->n0);
    long g = 1;
    for (int j = 0; j < c->n0; j++) {
        c->rot_group[j] = (int)g;
        g = (g * 5) % m;
    }
}

static void bitrev_c(cplx *v, int n) {
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = v[i]; v[i] = v[j]; v[j] = t; }
    }
}

void special_fft_fwd(const orc_ctx *c, cplx *v) {
    int n0 = c->n0, m = 2 * c->n;
    bitrev_c(v, n0);
    for (int len = 2; len <= n0; len <<= 1) {
        int lenh = len >> 1, lenq = len << 2, gap = m / lenq;
        for (int i = 0; i < n0; i += len)
            for (int j = 0; j < lenh; j++) {
                int idx = (c->rot_group[j] % lenq) * gap;
                cplx u = v[i + j], t;
                cmul(v[i + j + lenh], c->zeta[idx], &t);
                v[i + j].re = u.re + t.re;
                v[i + j].im = u.im + t.im;
                v[i + j + lenh].re = u.re - t.re;
                v[i + j + lenh].im = u.im - t.im;
            }
    }
}

void special_fft_inv(const orc_ctx *c, cplx *v) {
    int n0 = c->n0, m = 2 * c->n;
    for (int len = n0; len >= 2; len >>= 1) {
        int lenh = len >> 1, lenq = len << 2, gap = m / lenq;
        for (int i = 0; i < n0; i += len)
            for (int j = 0; j < lenh; j++) {
                int idx = (lenq - (c->rot_group[j] % lenq)) * gap;
                cplx a = v[i + j], b = v[i + j + lenh], d, t;
                cplx s;
                s.re = a.re + b.re;
                s.im = a.im + b.im;
                d.re = a.re - b.re;
                d.im = a.im - b.im;
                cmul(d, c->zeta[idx], &t);
                v[i + j] = s;
                v[i + j + lenh] = t;
            }
    }
    bitrev_c(v, n0);
    for (int i = 0; i < n0; i++) {
        v[i].re = v[i].re / (double)n0;
        v[i].im = v[i].im / (double)n0;
    }
}

/* pt = RNS form (limbs 0..level) of round(scale * t), t the coefficients of z. */
int encode(const orc_ctx *c, const cplx *z, double scale, int level, uint64_t *pt) {
    int n0 = c->n0, n = c->n;
    cplx *w = malloc(sizeof(cplx) * n0);
    memcpy(w, z, sizeof(cplx) * n0);
    special_fft_inv(c, w);
    for (int k = 0; k < n; k++) {
        double t = k < n0 ? w[k].re : w[k - n0].im;
        i128 v = round_to_i128(scale * t);
        for (int i = 0; i <= level; i++) pt[(size_t)i * n + k] = reduce_i128(v, c->mod[i]);
    }
    free(w);
    return 0;
}

/* Centred integer value of each coefficient of an RNS polynomial, as a double. */
int decode_coeffs(const orc_ctx *c, const uint64_t *poly, int level, double *coeff) {
    int n = c->n, L = level + 1;
    uint64_t a[ORC_MAXQ], b[ORC_MAXQ];
    for (int k = 0; k < n; k++) {
        /* mixed-radix digits of x and of Q - x */
        for (int pass = 0; pass < 2; pass++) {
            uint64_t *dig = pass ? b : a;
            for (int i = 0; i < L; i++) {
                uint64_t q = c->mod[i];
                uint64_t xi = poly[(size_t)i * n + k] % q;
                if (pass) xi = (q - xi) % q;
                /* value of the digits found so far, mod q_i */
                uint64_t acc = 0, rad = 1 % q;
                for (int j = 0; j < i; j++) {
                    acc = addmod(acc, mulmod(dig[j] % q, rad, q), q);
                    rad = mulmod(rad, c->mod[j] % q, q);
                }
                dig[i] = mulmod(submod(xi, acc, q), invmod(rad, q), q);
            }
        }
        int neg = 0;
        for (int i = L - 1; i >= 0; i--) {
            if (a[i] != b[i]) { neg = a[i] > b[i]; break; }
        }
        uint64_t *d = neg ? b : a;
        double v = 0.0;
        for (int i = L - 1; i >= 0; i--) v = v * (double)c->mod[i] + (double)d[i];
        coeff[k] = neg ? -v : v;
    }
    return 0;
}

int decode(const orc_ctx *c, const uint64_t *poly, int level, double scale, cplx *z) {
    int n0 = c->n0;
    double *t = malloc(sizeof(double) * c->n);
    decode_coeffs(c, poly, level, t);
    for (int k = 0; k < n0; k++) {
        z[k].re = t[k] / scale;
        z[k].im = t[k + n0] / scale;
    }
    special_fft_fwd(c, z);
    free(t);
    return 0;
}
