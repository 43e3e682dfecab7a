/* Negacyclic number-theoretic transform over Z_q[X]/(X^N + 1).
 *
 * Forward: a_hat[k] = sum_i a[i] psi^{i(2k+1)}, k = 0..N-1 (natural order): the values
 * of a(X) at the N roots psi^{2k+1} of X^N + 1.  It is computed as the twist
 * a[i] <- a[i] psi^i followed by a radix-2 cyclic transform with omega = psi^2.
 * The product of two polynomials is the inverse transform of the pointwise product.
 * negacyclic_mul_schoolbook is the O(N^2) definition used to pin this in tests. */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static void bit_reverse(uint64_t *a, int n) {
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
    }
}

/* in-place cyclic DFT over Z_q with the root table w[j] = omega^j, j < n/2 */
static void cyclic_dft(uint64_t *a, int n, uint64_t q, const uint64_t *w) {
    bit_reverse(a, n);
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1, step = n / len;
        for (int i = 0; i < n; i += len)
            for (int j = 0; j < half; j++) {
                uint64_t u = a[i + j];
                uint64_t v = mulmod(a[i + j + half], w[j * step], q);
                a[i + j] = addmod(u, v, q);
                a[i + j + half] = submod(u, v, q);
            }
    }
}

void ntt_fwd(const orc_ctx *c, int t, uint64_t *a) {
    uint64_t q = c->mod[t];
    for (int i = 0; i < c->n; i++) a[i] = mulmod(a[i], c->psi_pow[t][i], q);
    cyclic_dft(a, c->n, q, c->omega_pow[t]);
}

void ntt_inv(const orc_ctx *c, int t, uint64_t *a) {
    uint64_t q = c->mod[t];
    cyclic_dft(a, c->n, q, c->omega_inv_pow[t]);
    uint64_t ninv = invmod((uint64_t)c->n, q);
    for (int i = 0; i < c->n; i++) a[i] = mulmod(mulmod(a[i], ninv, q), c->psi_inv_pow[t][i], q);
}

void negacyclic_mul(const orc_ctx *c, int t, const uint64_t *a, const uint64_t *b, uint64_t *out) {
    int n = c->n;
    uint64_t q = c->mod[t];
    uint64_t *x = malloc(sizeof(uint64_t) * n), *y = malloc(sizeof(uint64_t) * n);
    memcpy(x, a, sizeof(uint64_t) * n);
    memcpy(y, b, sizeof(uint64_t) * n);
    ntt_fwd(c, t, x);
    ntt_fwd(c, t, y);
    for (int i = 0; i < n; i++) x[i] = mulmod(x[i], y[i], q);
    ntt_inv(c, t, x);
    memcpy(out, x, sizeof(uint64_t) * n);
    free(x);
    free(y);
}

/* out = a * b mod (X^n + 1, q): X^n = -1 folds the upper half back with a sign flip. */
void negacyclic_mul_schoolbook(int n, uint64_t q, const uint64_t *a, const uint64_t *b, uint64_t *out) {
    for (int k = 0; k < n; k++) out[k] = 0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            uint64_t p = mulmod(a[i], b[j], q);
            int k = i + j;
            if (k < n) out[k] = addmod(out[k], p, q);
            else out[k - n] = submod(out[k - n], p, q);
        }
}
