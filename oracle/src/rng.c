/* Counter-based randomness.
 *
 * The mixing function is the SplitMix64 output function (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014): with
 * GAMMA = 0x9e3779b97f4a7c15,
 *     mix(z): z ^= z >> 30; z *= 0xbf58476d1ce4e5b9; z ^= z >> 27; z *= 0x94d049bb133111eb;
 *             z ^= z >> 31.
 * A draw is addressed by (seed, domain, counter):
 *     key = mix(seed + GAMMA (2 domain + 1)),  out = mix(key + GAMMA (counter + 1)).
 * Samplers built on it (the CKKS distributions, Sec. 2.2 "Key generation"):
 *   uniform mod q   : (w0 * 2^64 + w1) mod q from two consecutive counters 2c, 2c+1;
 *   ternary         : two low bits, 0/1 -> 0, 2 -> +1, 3 -> -1;
 *   Gaussian sigma  : cumulative table of rho(k) = exp(-k^2 / (2 sigma^2)) cut at
 *                     ceil(6 sigma), compared against the upper 63 bits; low bit = sign;
 *   HWT(h) secret   : the h coefficients with the smallest (draw, index), sign from a
 *                     second domain. */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

#define GAMMA 0x9e3779b97f4a7c15ULL

uint64_t splitmix_mix(uint64_t z) {
    z ^= z >> 30;
    z *= 0xbf58476d1ce4e5b9ULL;
    z ^= z >> 27;
    z *= 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return z;
}

uint64_t rng_u64(uint64_t seed, uint64_t dom, uint64_t ctr) {
    uint64_t key = splitmix_mix(seed + GAMMA * (2 * dom + 1));
    return splitmix_mix(key + GAMMA * (ctr + 1));
}

uint64_t rng_uniform_mod(uint64_t seed, uint64_t dom, uint64_t ctr, uint64_t q) {
    u128 w0 = rng_u64(seed, dom, 2 * ctr), w1 = rng_u64(seed, dom, 2 * ctr + 1);
    return (uint64_t)(((w0 << 64) | w1) % q);
}

int rng_ternary(uint64_t seed, uint64_t dom, uint64_t ctr) {
    uint64_t b = rng_u64(seed, dom, ctr) & 3;
    return b < 2 ? 0 : (b == 2 ? 1 : -1);
}

void cdt_build(orc_ctx *c) {
    int kmax = (int)ceil(6.0 * c->sigma);
    double s2 = 2.0 * c->sigma * c->sigma;
    double z = exp(-0.0 / s2);
    for (int k = 1; k <= kmax; k++) z += 2.0 * exp(-(double)(k * k) / s2);
    double acc = 0.0;
    for (int k = 0; k < kmax; k++) {
        double pk = (k == 0 ? exp(-0.0 / s2) : 2.0 * exp(-(double)(k * k) / s2)) / z;
        acc += pk;
        c->cdt[k] = (uint64_t)(acc * 9223372036854775808.0);
    }
    c->cdt_len = kmax;
}

int rng_gauss(const orc_ctx *c, uint64_t seed, uint64_t dom, uint64_t ctr) {
    uint64_t r = rng_u64(seed, dom, ctr);
    uint64_t u = r >> 1;
    int mag = 0;
    for (int k = 0; k < c->cdt_len; k++)
        if (u >= c->cdt[k]) mag++;
    return (r & 1) ? -mag : mag;
}

typedef struct { uint64_t key; int idx; } keyed;

static int cmp_keyed(const void *a, const void *b) {
    const keyed *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx - y->idx;
}

void sample_hwt(int n, int h, uint64_t seed, int8_t *s) {
    keyed *k = malloc(sizeof(keyed) * n);
    for (int i = 0; i < n; i++) {
        k[i].key = rng_u64(seed, DOM_SK, i);
        k[i].idx = i;
        s[i] = 0;
    }
    qsort(k, n, sizeof(keyed), cmp_keyed);
    for (int j = 0; j < h; j++) {
        int i = k[j].idx;
        s[i] = (rng_u64(seed, DOM_SK_SIGN, i) & 1) ? -1 : 1;
    }
    free(k);
}
