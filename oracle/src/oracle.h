/*
 * CPU oracle for RNS-CKKS and the normalize-and-square Softmax circuit.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow reference implementation that the
 * CUDA library is checked against.  Only tests, the smoke check and the benchmark's CPU
 * baseline may load it; the library never calls it.  It shares no source with the CUDA
 * path.  Every modular product is a 128-bit multiply followed by '%', polynomials are
 * kept in coefficient form, and each operation follows its textbook definition.
 *
 * Ciphertext layout: [2][level+1][N] uint64, coefficient form, residues in [0, q_i).
 */
#ifndef HE_ORACLE_H
#define HE_ORACLE_H

#include <stdint.h>
#include <stddef.h>
#include <stdio.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

#define ORC_MAXQ 64
#define ORC_MAXP 16

typedef struct { double re, im; } cplx;

typedef struct orc_key {
    int galois;        /* 0 = relinearisation key (s^2 -> s), else galois element g */
    int nlimb;         /* (L+1) + alpha limbs per polynomial */
    int ndigit;        /* digits at the top level */
    uint64_t *b;       /* [ndigit][nlimb][N], NTT form (cached transform) */
    uint64_t *a;       /* [ndigit][nlimb][N], NTT form */
    struct orc_key *next;
} orc_key;

typedef struct orc_ctx {
    int logn, n, n0;       /* N, N0 = N/2 slots */
    int nq, np, alpha;     /* Q primes q_0..q_{nq-1}; P primes p_0..p_{np-1}; alpha = np */
    uint64_t mod[ORC_MAXQ + ORC_MAXP];   /* limb t: t < nq -> q_t, else p_{t-nq} */
    uint64_t psi[ORC_MAXQ + ORC_MAXP];   /* primitive 2N-th root per modulus */
    uint64_t **psi_pow, **psi_inv_pow;   /* [modulus][N] powers of psi, psi^{-1} */
    uint64_t **omega_pow, **omega_inv_pow; /* [modulus][N/2] powers of psi^2, psi^{-2} */
    int h;
    double sigma;
    /* secret key */
    int8_t *s;             /* ternary coefficients */
    uint64_t seed;         /* key-generation seed */
    int have_sk;
    uint64_t *pk_b, *pk_a; /* [nq][N] coefficient form */
    orc_key *keys;         /* lazily generated switching keys */
    /* FFT tables for the canonical embedding */
    cplx *zeta;            /* [2N] zeta^j = exp(2 pi i j / 2N) */
    int *rot_group;        /* [N0] 5^j mod 2N */
    /* Gaussian CDT */
    uint64_t cdt[64];
    int cdt_len;
    /* operation counters (for level/op accounting tests) */
    long n_ks, n_rot, n_hmult, n_rescale, n_bts;
    char err[256];
} orc_ctx;

/* arith.c */
uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q);
uint64_t addmod(uint64_t a, uint64_t b, uint64_t q);
uint64_t submod(uint64_t a, uint64_t b, uint64_t q);
uint64_t powmod(uint64_t a, uint64_t e, uint64_t q);
uint64_t invmod(uint64_t a, uint64_t q);
uint64_t find_psi(uint64_t q, int n);
uint64_t reduce_i128(i128 x, uint64_t q);
i128 round_to_i128(double x);

/* ntt.c */
void ntt_fwd(const orc_ctx *c, int t, uint64_t *a);
void ntt_inv(const orc_ctx *c, int t, uint64_t *a);
void negacyclic_mul(const orc_ctx *c, int t, const uint64_t *a, const uint64_t *b, uint64_t *out);
void negacyclic_mul_schoolbook(int n, uint64_t q, const uint64_t *a, const uint64_t *b, uint64_t *out);

/* rng.c */
uint64_t splitmix_mix(uint64_t z);
uint64_t rng_u64(uint64_t seed, uint64_t dom, uint64_t ctr);
uint64_t rng_uniform_mod(uint64_t seed, uint64_t dom, uint64_t ctr, uint64_t q);
void cdt_build(orc_ctx *c);
int rng_gauss(const orc_ctx *c, uint64_t seed, uint64_t dom, uint64_t ctr);
int rng_ternary(uint64_t seed, uint64_t dom, uint64_t ctr);
void sample_hwt(int n, int h, uint64_t seed, int8_t *s);

/* fft.c */
void fft_tables(orc_ctx *c);
void special_fft_fwd(const orc_ctx *c, cplx *v);   /* coefficients (w) -> slots */
void special_fft_inv(const orc_ctx *c, cplx *v);   /* slots -> coefficients (w) */
void cmul(cplx a, cplx b, cplx *out);
int encode(const orc_ctx *c, const cplx *z, double scale, int level, uint64_t *pt);
int decode_coeffs(const orc_ctx *c, const uint64_t *poly, int level, double *coeff);
int decode(const orc_ctx *c, const uint64_t *poly, int level, double scale, cplx *z);

/* ckks.c */
#define DOM_SK 1
#define DOM_SK_SIGN 2
#define DOM_PK_A 3
#define DOM_PK_E 4
#define DOM_ENC_V 5
#define DOM_ENC_E0 6
#define DOM_ENC_E1 7
uint64_t dom_key(int key_id, int digit, int which);

typedef struct {
    uint64_t *d;     /* [2][level+1][N] */
    int level;
    double scale;
} orc_ct;

orc_ct ct_alloc(const orc_ctx *c, int level);
void ct_free(orc_ct *x);
orc_ct ct_copy(const orc_ctx *c, const orc_ct *x);
uint64_t *ct_poly(const orc_ctx *c, const orc_ct *x, int poly);
int ct_drop(const orc_ctx *c, orc_ct *x, int level);

int keygen_secret(orc_ctx *c, uint64_t seed);
orc_key *get_key(orc_ctx *c, int galois);
int encrypt(orc_ctx *c, const cplx *z, int level, double scale, uint64_t seed, int ct_index, orc_ct *out);
int decrypt(orc_ctx *c, const orc_ct *x, cplx *z);
int ct_add(orc_ctx *c, orc_ct *a, const orc_ct *b);
int ct_sub(orc_ctx *c, orc_ct *a, const orc_ct *b);
void ct_mul_int(orc_ctx *c, orc_ct *a, i128 k);
void ct_add_const_int(orc_ctx *c, orc_ct *a, i128 k);
int ct_mul_plain(orc_ctx *c, orc_ct *a, const uint64_t *pt, int pt_level);
int rescale(orc_ctx *c, orc_ct *a);
int tensor(orc_ctx *c, const orc_ct *a, const orc_ct *b, uint64_t *d0, uint64_t *d1, uint64_t *d2, int level);
uint64_t *modup(orc_ctx *c, const uint64_t *d, int level);
int ks_inner_moddown(orc_ctx *c, uint64_t *digits, int level, int galois, orc_key *k, uint64_t *out0, uint64_t *out1);
int ks_inner(orc_ctx *c, uint64_t *digits, int level, int galois, orc_key *k, uint64_t *acc0, uint64_t *acc1);
int moddown(orc_ctx *c, const uint64_t *acc0, const uint64_t *acc1, int level, uint64_t *out0, uint64_t *out1);
int relin_rescale(orc_ctx *c, const uint64_t *d0, const uint64_t *d1, const uint64_t *d2, int level, double scale,
                  orc_ct *out);
int relinearize(orc_ctx *c, const uint64_t *d0, const uint64_t *d1, const uint64_t *d2, int level, double scale, orc_ct *out);
int hmult(orc_ctx *c, const orc_ct *a, const orc_ct *b, orc_ct *out);
int rotate_hoisted(orc_ctx *c, const orc_ct *x, const int *galois, int nrot, orc_ct *out);
int rotate(orc_ctx *c, const orc_ct *x, int galois, orc_ct *out);
int galois_for_rot(const orc_ctx *c, long r);
void automorph_poly(const orc_ctx *c, int t, const uint64_t *in, int g, uint64_t *out);
int mod_raise(orc_ctx *c, const orc_ct *x, int top, orc_ct *out);
int ct_rescale_to(orc_ctx *c, orc_ct *x, int level, double scale);

/* lintrans.c */
typedef struct {
    int nstage;              /* stages in this level (applied in order) */
    int h[32];               /* half block size of each stage */
    int inverse;             /* 0 = forward (StC), 1 = inverse (CtS) */
} orc_lt_level;
int lt_levels(const orc_ctx *c, int nlev, int inverse, orc_lt_level *out);
int lt_eval_level(orc_ctx *c, orc_ct *x, const orc_lt_level *lv, cplx gain, double pt_scale);
int lt_eval_level_ex(orc_ctx *c, orc_ct *x, const orc_lt_level *lv, cplx gain, double pt_scale, int do_rescale);
int lt_eval_level_textbook(orc_ctx *c, orc_ct *x, const orc_lt_level *lv, cplx gain, double pt_scale);
int lt_rotations(const orc_ctx *c, const orc_lt_level *lv, int *gal, int max);

/* poly.c */
int poly_eval(orc_ctx *c, const orc_ct *u, const double *coeffs, int deg, int level_out, double scale_out, orc_ct *out);

/* bts.c */
typedef struct {
    int stc_levels, cts_levels;
    int top_level;           /* level after ModRaise */
    int user_top;            /* level of bootstrapped output */
    double K;                /* EvalMod range */
    int r;                   /* double-angle steps */
    int em_deg;
    const double *em_coeffs;
    double out_scale;        /* nominal scale (the user-level Delta) */
} orc_bts;
int bootstrap(orc_ctx *c, const orc_bts *b, const orc_ct *x, double gain, double out_scale, orc_ct *out);

/* softmax.c */
typedef struct {
    int n, k;
    double M;
    double out_scale;
    int exp_deg; const double *exp_c;
    int inv_deg[16]; const double *inv_c[16]; double inv_a[16], inv_b[16];
    double gain_s[16], gain_l[16];
    int bts_min;             /* lowest level from which bootstrapping is possible */
    int use_bts;
    double bts_boost;        /* bootstrapping input gain, removed by scale bookkeeping */
} orc_plan;
int softmax(orc_ctx *c, const orc_plan *p, const orc_bts *b, orc_ct *cts, int m);

#endif
