/* Modular arithmetic by definition: 128-bit product, then remainder. */
#include <math.h>
#include "oracle.h"

uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }
uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a + b) % q); }
uint64_t submod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a + q - b) % q); }

uint64_t powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

/* q prime: a^{q-2} (Fermat). */
uint64_t invmod(uint64_t a, uint64_t q) { return powmod(a, q - 2, q); }

/* A primitive 2N-th root of unity mod q (q = 1 mod 2N): the first g^((q-1)/2N), g = 2,3,..,
 * whose N-th power is -1. */
uint64_t find_psi(uint64_t q, int n) {
    uint64_t e = (q - 1) / (2 * (uint64_t)n);
    for (uint64_t g = 2; g < 1000000; g++) {
        uint64_t x = powmod(g, e, q);
        if (powmod(x, (uint64_t)n, q) == q - 1) return x;
    }
    return 0;
}

/* Signed 128-bit integer to its residue in [0, q). */
uint64_t reduce_i128(i128 x, uint64_t q) {
    i128 r = x % (i128)q;
    if (r < 0) r += q;
    return (uint64_t)r;
}

/* Round to nearest, ties to even (the default IEEE rounding of nearbyint). */
i128 round_to_i128(double x) { return (i128)nearbyint(x); }
