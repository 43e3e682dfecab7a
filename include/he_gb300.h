/*
 * he_gb300 -- C ABI of the GB300 (sm_103a) RNS-CKKS library for the normalize-and-square
 * homomorphic Softmax of Cho, Hanrot, Kim, Park, Stehle (arXiv 2410.11184).
 *
 * Conventions
 *   - Return value: 0 on success, a negative HE_E* code on failure; he_last_error() gives a
 *     message.  Invalid arguments never reach a kernel.
 *   - Ciphertexts (he_ct) live in device memory owned by the caller (e.g. torch tensors):
 *     data = [n_ct][2][level+1][N] uint64, RNS limbs q_0..q_level, NTT (evaluation) form.
 *     level and scale are metadata the library reads and updates.
 *   - Everything runs on the stream given at context creation (a cudaStream_t, or NULL for
 *     the legacy default stream).  Calls return after enqueueing unless stated otherwise;
 *     host-buffer calls synchronise the stream.
 *   - The library owns the context, its tables and the evaluation keys (device memory it
 *     allocates); he_context_destroy frees them.
 *   - Section/equation references are to the paper (CCS 2024 version).
 */
#ifndef HE_GB300_H
#define HE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HE_OK 0
#define HE_EINVAL (-1)   /* bad argument (sizes, levels, n not a power of two, ...) */
#define HE_ELEVEL (-2)   /* not enough levels left for the requested operation */
#define HE_ENOMEM (-3)   /* device allocation failed */
#define HE_ECUDA (-4)    /* a CUDA call failed */
#define HE_ENOKEY (-5)   /* a needed evaluation key was not generated */
#define HE_ETIMEOUT (-6) /* a bounded device wait gave up */

typedef struct he_ctx he_ctx;

/* CKKS parameters (Sec. 2.2; Table 4 for the 128-bit-security size).  Q = q_0 ... q_{n_q-1},
 * P = p_0 ... p_{n_p-1}; alpha = n_p primes per key-switching digit. */
typedef struct {
    int log_n;                 /* ring degree N = 2^log_n, N/2 slots; 12 or 16 (HE_EINVAL otherwise) */
    int n_q;
    const uint64_t *q;         /* n_q primes, q_i = 1 mod 2N, < 2^60 */
    int n_p;
    const uint64_t *p;         /* n_p special primes */
    int h;                     /* Hamming weight of the ternary secret */
    double sigma;              /* Gaussian error parameter */
    int log_scale;             /* nominal scale Delta = 2^log_scale */
    int user_top_level;        /* level of fresh and bootstrapped ciphertexts */
    int bootstrap;             /* 1: build bootstrapping keys and tables */
    int stc_levels, cts_levels, bts_min_level;
    double em_K;               /* EvalMod range: x = t/q_0 in [-K, K] */
    int em_r;                  /* double-angle steps */
    int em_deg;                /* Chebyshev degree of cos(2 pi (K u - 1/4) / 2^r) */
    const double *em_coeffs;   /* em_deg + 1 coefficients */
} he_params;

#define HE_SOFTMAX_ALG2 0   /* Alg. 2 with the auxiliary thread of Alg. 3 (Sec. 4.2) */
#define HE_SOFTMAX_ALG4 1   /* Alg. 4, version B (Sec. 4.3), with the auxiliary thread of Alg. 3 */

/* Softmax circuit parameters (Alg. 2 / Alg. 3 / Alg. 4; Sec. 5.1.2 for the polynomials).  All
 * arrays are host memory of k entries (inv_coeffs: the k coefficient lists back to back), read
 * during the call only. */
typedef struct {
    int n;                     /* Softmax dimension (power of two dividing N/2) */
    int k;                     /* normalize-and-square rounds */
    double M;                  /* inputs in [-M, 0] (Assumption 3.5) */
    int exp_deg;
    const double *exp_coeffs;  /* exp(x/2^k) in the Chebyshev basis of u = 2x/M + 1 */
    const int *inv_deg;        /* k degrees */
    const double *inv_coeffs;  /* round j: Chebyshev coefficients of v^{-1/2} (Alg. 2) or of
                                  v^{-exponent_j} (Alg. 4) on [inv_a_j, inv_b_j], mapped to [-1, 1] */
    const double *inv_a, *inv_b;     /* interval of round j */
    const double *gain_s, *gain_l;   /* input gain of round j; bootstrapping gain of lambda_j
                                        (Alg. 2 only: gain_l may be NULL for Alg. 4) */
    double bts_boost;          /* input gain applied inside every bootstrapping */
    int method;                /* HE_SOFTMAX_ALG2 or HE_SOFTMAX_ALG4 (HE_EINVAL otherwise) */
    /* Alg. 4 only (NULL for Alg. 2): lambda_j = S_j^(-exponent_j), exponent_j = 2^-j; lambda_j is
     * bootstrapped with gain 1/lam_max_j; b_max_j > 0 bounds the upper half B of a round-j
     * polynomial too deep to end above the bootstrapping input level, which is then evaluated
     * as A + T_h B (0: no split). */
    const double *exponent, *lam_max, *b_max;
} he_softmax_plan;

typedef struct {
    uint64_t *data;            /* device pointer, [n_ct][2][level+1][N] */
    int level;
    double scale;
    int n_ct;
} he_ct;

/* Context: builds NTT, basis-conversion and embedding tables on the device.
 * cuda_stream: a cudaStream_t (or NULL).  *out receives the handle. */
int he_context_create(const he_params *p, void *cuda_stream, he_ctx **out);
void he_context_destroy(he_ctx *ctx);
const char *he_last_error(const he_ctx *ctx);
int he_ring_degree(const he_ctx *ctx);
/* 1 if p is below the paper's 128-bit-security parameter size (Sec. 5.1.1: N = 2^16,
 * log2(QP) <= 1555, ternary secret of Hamming weight h = 192; for other N the modulus bound is
 * taken as proportional to N) -- the small test chains are --, 0 otherwise, HE_EINVAL for a
 * NULL or malformed p.  Host only: needs no GPU and no context. */
int he_params_insecure(const he_params *p);

/* KeyGen (Sec. 2.2): secret, public key, relinearisation and conjugation keys, rotation keys
 * for the n_rot slot rotations in rot_steps, and (if bootstrapping) every rotation key that
 * SlotToCoeff / CoeffToSlot need.  Randomness: counter-based SplitMix64 keyed by seed.
 * Calling it again replaces the secret: every evaluation key of the previous secret is freed
 * (he_keygen_softmax must be called again) and every graph captured by he_softmax_graph is
 * dropped, so ciphertexts of the old secret no longer decrypt. */
int he_keygen(he_ctx *ctx, uint64_t seed, const int *rot_steps, int n_rot);
/* Rotation keys a Softmax of dimension n over m ciphertexts needs (strides L 2^i, Alg. 3). */
int he_keygen_softmax(he_ctx *ctx, int n, int m);

/* Enc (Sec. 2.2) of L = m N0 / n Softmax inputs x [L][n] (row-major FP64, host memory,
 * count = L n), packed as in Sec. 4.2 into m ciphertexts at user_top_level with scale
 * (2/M) q_top.  out->data must hold m * 2 * (user_top_level+1) * N words (device). */
int he_encrypt(he_ctx *ctx, const double *x, size_t count, int n, int m, double M, uint64_t seed, he_ct *out);
/* Dec of m ciphertexts into y [L][n] (host), unpacking Sec. 4.2. Synchronises. */
int he_decrypt(he_ctx *ctx, const he_ct *cts, int n, double *y, size_t count);
/* Dec of one ciphertext (index ct) into N/2 complex slots (host, interleaved re/im). */
int he_decrypt_slots(he_ctx *ctx, const he_ct *cts, int ct, double *slots);
/* Enc of N/2 complex slots (host, interleaved) into ciphertext index ct of out at level/scale. */
int he_encrypt_slots(he_ctx *ctx, const double *slots, int level, double scale, uint64_t seed, int ct_index,
                     he_ct *out, int ct);

/* Softmax (Alg. 2 with Alg. 3, or Alg. 4 with Alg. 3, as plan->method says; many-ciphertext
 * form of Sec. 4.2) on the m = cts->n_ct ciphertexts, in place: the output level is lower, data
 * is overwritten, level/scale updated.  batched = 1: every operation runs over all m ciphertexts
 * in one launch (key read once); batched = 0: the same operation list, one ciphertext at a time.
 * Alg. 4 bootstraps only the auxiliary ciphertext (2 per round, 2 more per split polynomial);
 * it needs a bootstrapping context (HE_EINVAL otherwise).  HE_EINVAL for a NULL plan array the
 * method reads, n not a power of two dividing N/2, or m not dividing n. */
int he_softmax(he_ctx *ctx, const he_softmax_plan *plan, he_ct *cts, int batched);
/* groups independent Softmax batches in one batched pass: the n_ct ciphertexts are groups
 * consecutive groups of m = n_ct / groups ciphertexts, each packed as in Sec. 4.2 (its own
 * L = m N0 / n Softmax); the sum of squares stays inside each group and the auxiliary thread
 * (Alg. 3) runs over a batch of groups ciphertexts.  Every group's result equals he_softmax on
 * that group alone, bit for bit (all groups share level and scale).  This is how a server batches
 * requests that arrive separately. */
int he_softmax_grouped(he_ctx *ctx, const he_softmax_plan *plan, he_ct *cts, int groups);
/* The problem statement's form of the call (Sec. 3, inputs in [-M, 0]^n, Assumption 3.5):
 * Softmax of dimension n over the m = cts->n_ct ciphertexts, encrypted by he_encrypt with this
 * M, by the method's circuit, with the plan registered for exactly (n, M, method).  The plans'
 * polynomials come from the design script (the paper prints none); he_softmax_register copies a
 * plan into the context (it owns the copy; registering the same (n, M, method) again replaces
 * it).  he_softmax_nm runs he_softmax (batched; graph = 0) or he_softmax_graph (graph = 1) with
 * that plan: HE_EINVAL if none is registered, otherwise as those calls.  he_softmax_register:
 * HE_EINVAL for a NULL array the method reads or a method other than the two. */
int he_softmax_register(he_ctx *ctx, const he_softmax_plan *plan);
int he_softmax_nm(he_ctx *ctx, he_ct *cts, int n, double M, int method, int graph);
/* he_softmax (batched) as one CUDA graph: the first call for a given (cts->data, level, scale,
 * n_ct, plan) runs the circuit once on a scratch copy (filling the key, diagonal and mask caches),
 * captures it on the context stream and launches the captured graph; later calls with the same
 * buffer and shape launch the graph again (no host work per kernel).  Results are those of
 * he_softmax bit for bit.  Graphs live until he_context_destroy; the buffer must stay allocated
 * while its graph may be launched. */
int he_softmax_graph(he_ctx *ctx, const he_softmax_plan *plan, he_ct *cts);

/* ---- Alg. 4 split over shares of the m main-thread ciphertexts (Sec. 4.2, Alg. 3 Step 1) ----
 * For running one many-ciphertext batch on several devices: every device holds a share (a
 * contiguous run of the m ciphertexts of the packing) and a copy of the keys; the one exchange
 * per round is the sum of squares, an elementwise integer sum of the shares' tensors (exact in
 * uint64 for up to 16 shares, since residues are below 2^60); the auxiliary thread then runs on
 * every device with identical results.  The same calls in the order
 *   he_softmax_share_exp (each share);
 *   for j = 1 .. k: he_softmax_share_square_sum (each share, from y0 in round 1, else from the
 *     previous round's ys), sum the d's, he_softmax_aux_round, he_softmax_share_update (each share)
 * give every share exactly the ciphertexts he_softmax (Alg. 4, batched) gives those ciphertexts of
 * the whole batch.  Alg. 4 plans and bootstrapping contexts only (HE_EINVAL otherwise).
 *
 * exp: the share's ciphertexts (at user_top_level, scale (2/M) q_top, as from he_encrypt) are
 * replaced by y0 = P_exp(2x/M + 1) (stored compactly at the lower level; level/scale written). */
int he_softmax_share_exp(he_ctx *ctx, const he_softmax_plan *plan, he_ct *share);
/* d (device, [3][ys->level+1][N] words, NTT form, residues in [0, q_i)): the sum over the share's
 * ciphertexts of y (x) y. */
int he_softmax_share_square_sum(he_ctx *ctx, const he_ct *ys, uint64_t *d);
/* Auxiliary thread of round j (1 .. k) for m_total ciphertexts in all: d_sum (device) is the
 * elementwise integer sum of every share's d (words below 16 q_i; reduced here), taken from
 * ciphertexts at `level` with scale y_scale; y0_level / y0_scale are those of y0 (from
 * he_softmax_share_exp).  lam: Lambda = lambda_1 ... lambda_j, one ciphertext, written in round 1
 * and read and rewritten after (caller-allocated, 2 (user_top_level+1) N words); lr: the
 * replicated Lambda that the main thread multiplies by (written; same size). */
int he_softmax_aux_round(he_ctx *ctx, const he_softmax_plan *plan, int j, int m_total, const uint64_t *d_sum,
                         int level, double y_scale, int y0_level, double y0_scale, he_ct *lam, he_ct *lr);
/* Main thread of round j: ys = (lr y0)^(2^j) for every ciphertext of the share (y0 from
 * he_softmax_share_exp; ys caller-allocated, another buffer of at least y0's size; level/scale
 * written).  After round k, ys holds the share's Softmax outputs. */
int he_softmax_share_update(he_ctx *ctx, const he_softmax_plan *plan, int j, const he_ct *lr, const he_ct *y0,
                            he_ct *ys);

/* ---- the hot-path operations, one call each ----
 * Common to the calls below: ciphertext batches are he_ct device buffers as above; a result
 * is formed in library-owned scratch and copied to out->data (caller-allocated, at least
 * n_ct * 2 * (level_out+1) * N words; it may be an input's buffer, except for
 * he_rescale_noalloc), and out->level / scale / n_ct are written.  Errors: HE_EINVAL
 * for a NULL pointer, a NULL data pointer, n_ct < 1 or a level outside the chain;
 * HE_ELEVEL where the operation needs a level the input no longer has; HE_ENOKEY where an
 * evaluation key was not generated; HE_ECUDA if a CUDA call fails.  Nothing is launched before
 * the arguments are checked. */

/* Negacyclic NTT (inverse = 0: evaluation at the odd powers psi^(2k+1) of a primitive 2N-th
 * root mod q_i, output in bit-reversed order) or its inverse, in place, on n_poly polynomials of
 * n_limb limbs each ([n_poly][n_limb][N] uint64, device; limb i is reduced mod q_i).  The
 * evaluation representation that all CKKS products below work in; the paper delegates it to its
 * library.  Inputs must be below q_i; outputs are in [0, q_i).  HE_EINVAL if n_limb > n_q. */
int he_ntt(he_ctx *ctx, uint64_t *data, int n_poly, int n_limb, int inverse);
/* coefficient-form host copy of a ciphertext batch [n_ct][2][level+1][N] (synchronises) */
int he_ct_to_coeff(he_ctx *ctx, const he_ct *x, uint64_t *host);
/* loads a coefficient-form host ciphertext batch into x (x->data, level, scale, n_ct set) */
int he_ct_from_coeff(he_ctx *ctx, const uint64_t *host, he_ct *x);
/* Ecd (Sec. 2.2): N/2 complex slots (interleaved re/im, host) scaled by `scale`, rounded to
 * integers, into a device plaintext pt [level+1][N] in NTT form. */
int he_encode(he_ctx *ctx, const double *slots, double scale, int level, uint64_t *pt);
/* Add (Sec. 2.2, Functionalities): a += b, in place.  HE_EINVAL unless both batches have the
 * same level, n_ct and scale (relative difference at most 1e-9). */
int he_add(he_ctx *ctx, he_ct *a, const he_ct *b);
/* plaintext product (Sec. 2.2, Functionalities): a *= pt with pt [a.level+1][N] from
 * he_encode at a.level; no rescale (the scale becomes a.scale times the plaintext's). */
int he_mul_plain(he_ctx *ctx, he_ct *a, const uint64_t *pt);
/* Rescale (Sec. 2.2, Levels): out = round(a / q_level) at level-1, scale / q_level.
 * HE_ELEVEL at level 0. */
int he_rescale(he_ctx *ctx, const he_ct *a, he_ct *out);
/* Rescale that allocates no device memory (no counterpart in the paper; an interface for
 * callers that cannot allocate once they are running: a server that reserved its whole HBM
 * budget at start-up and admits work against it, or a host program whose memory pool is
 * fixed and must not grow on the request path).  The caller passes the input batch a and an
 * output buffer out->data of n_ct * 2 * level * N words whose bytes must not overlap a's
 * n_ct * 2 * (level+1) * N words at all (HE_EINVAL otherwise); level, scale and n_ct of *out
 * are written.  Results equal he_rescale's bit for bit.
 * Scratch: a fixed device array of 2^21 words (16 MiB) compiled into the library, held by
 * every device that loads it until the process exits; its device address is looked up once
 * per context, at he_context_create, with the context's device current.  Inputs needing more
 * than 2 n_ct (level+1) N = 2^21 words are rejected with HE_EINVAL before any launch.  Every
 * call shares that one array and leaves its contents behind: calls whose executions overlap
 * on the GPU (several streams, or several contexts on one device) race on it, so serialise
 * them.  Errors: HE_EINVAL for a NULL pointer, n_ct < 1, a level outside [0, n_q), an
 * overlap of out with a or a size beyond the scratch; HE_ELEVEL at level 0. */
int he_rescale_noalloc(he_ctx *ctx, const he_ct *a, he_ct *out);
/* Mult (Sec. 2.2, Functionalities): tensor product, relinearisation with the hybrid key
 * switch, and rescale (relinearisation and rescale as one division by P q_level), out at
 * level min(a, b) - 1.  a and b may differ in n_ct only if one of them has n_ct = 1 (it is
 * broadcast).  HE_ELEVEL at level 0. */
int he_hmult(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct *out);
/* relinearisation (Sec. 2.2) of a degree-2 batch d [n_ct][3][level+1][N] (device, NTT form)
 * into out at the same level (no rescale). */
int he_relinearize(he_ctx *ctx, const uint64_t *d, int level, int n_ct, he_ct *out);
/* Rot(ct, r) (Sec. 2.2, Functionalities): slot j of the output holds slot (j + r) mod N/2.
 * HE_ENOKEY if the rotation key for r was not generated (he_keygen, he_keygen_softmax). */
int he_rotate(he_ctx *ctx, const he_ct *a, int r, he_ct *out);
/* complex conjugation of every slot (the Galois map X -> X^(2N-1)). */
int he_conjugate(he_ctx *ctx, const he_ct *a, he_ct *out);
/* polynomial evaluation (Sec. 2.2, Functions as polynomials; Sec. 5.1.2): p(u) =
 * sum_{k <= deg} c_k T_k(u) (Chebyshev basis, coeffs host) at level_out with scale scale_out;
 * it consumes ceil(log2(deg + 1)) levels, so u must be at level_out + that.  HE_ELEVEL
 * otherwise. */
int he_poly_eval(he_ctx *ctx, const he_ct *u, const double *coeffs, int deg, int level_out, double scale_out,
                 he_ct *out);
/* one level (which = 0 .. nlev-1) of the bootstrapping's linear transforms (Sec. 2.2, Levels):
 * SlotToCoeff (inverse = 0) or CoeffToSlot (inverse = 1) of N/2 slots factored into nlev
 * sparse levels, evaluated baby-step giant-step; gain multiplies the result, pt_scale is the
 * scale of the diagonals.  Needs the bootstrapping rotation keys (HE_ENOKEY otherwise). */
int he_lintrans(he_ctx *ctx, const he_ct *a, int nlev, int inverse, int which, double gain, double pt_scale,
                he_ct *out);
/* bootstrapping (Sec. 2.2, Levels; Sec. 5.1.1): SlotToCoeff, ModRaise, CoeffToSlot,
 * EvalMod; out at user_top_level encrypts gain * message with scale out_scale.  HE_EINVAL if the
 * context was created without bootstrapping, HE_ELEVEL below the level SlotToCoeff needs. */
int he_bootstrap(he_ctx *ctx, const he_ct *a, double gain, double out_scale, he_ct *out);
/* ModRaise (bootstrapping's first step): a level-0 batch reinterpreted modulo q_0 ... q_top
 * (centred lift).  HE_EINVAL unless a is at level 0 and top < n_q. */
int he_mod_raise(he_ctx *ctx, const he_ct *a, int top, he_ct *out);

/* ---- autotuner: launch strategies (no counterpart in the paper; every variant gives the same
 * words, so results do not depend on the choices) ----
 * op: HE_TUNE_MODUP (1: all digits of a ModUp converted in one launch and transformed in one
 * more; 0: per digit), HE_TUNE_ROT (1: the key switches of several hoisted rotations in one
 * inner-product launch and one ModDown; 0: one per rotation), HE_TUNE_LT_SMALL (1: one ModUp of all
 * giant-step sums of a bootstrapping linear-transform level; 0: one per giant step),
 * HE_TUNE_LT_ROWS (1: linear-transform inner sums without shared-memory staging; 0: staged),
 * HE_TUNE_BRANCHES (1: independent branches of a circuit -- the halves of a split polynomial, the
 * basis elements of one layer and the two halves of every Chebyshev division of a polynomial
 * evaluation -- on side streams, concurrently, and as parallel branches of a captured graph; 0:
 * one stream; he_tune_force only, on by default), HE_TUNE_NTT_SMALL (1: transforms in CTAs of 64
 * threads instead of 256; he_autotune times both on a ladder of limb counts (1 .. 2048) per
 * direction, and a transform takes the choice of the largest ladder count at or below its limb
 * count; 256 until tuned; table entries (HE_TUNE_NTT_SMALL, limbs, 0 forward / 1 inverse)),
 * HE_TUNE_FUSE_CONV (1: the fast basis conversions of ModUp and ModDown computed inside the
 * column pass of the forward transform that follows them, so the converted limbs are never
 * written to HBM; 0: a conversion kernel, then the transform; timed on one relinearisation),
 * HE_TUNE_NTT_1PASS (N = 2^16 only: 1: a transform without fused neighbours as one launch, one
 * thread-block cluster of 16 CTAs per limb exchanging between its two passes in distributed shared
 * memory; 0: the two passes; a ladder of limb counts per direction as for HE_TUNE_NTT_SMALL, off
 * until tuned).
 * Without a table entry the choice is 1 for batches of at most 4 ciphertexts (8 rows for
 * HE_TUNE_LT_ROWS), and 0 for HE_TUNE_FUSE_CONV.
 * he_autotune times both variants of every operation on the device (CUDA events on the context
 * stream, the best of reps runs after one warm-up) for ciphertexts at each of the n_levels levels and
 * each of the n_ncts batch sizes, on uniformly random residues, and keeps the faster one per
 * (operation, level + 1 limbs, batch size).  Rotation and linear-transform variants are timed
 * only in bootstrapping contexts, at the SlotToCoeff / CoeffToSlot levels.  Needs he_keygen first
 * (HE_ENOKEY).  Synchronises. */
#define HE_TUNE_MODUP 0
#define HE_TUNE_ROT 1
#define HE_TUNE_LT_SMALL 2
#define HE_TUNE_LT_ROWS 3
#define HE_TUNE_BRANCHES 4
#define HE_TUNE_NTT_SMALL 5
#define HE_TUNE_FUSE_CONV 6
#define HE_TUNE_NTT_1PASS 7
int he_autotune(he_ctx *ctx, const int *levels, int n_levels, const int *ncts, int n_ncts, int reps);
/* the table as text, one line "op limbs n_ct choice ms_variant0 ms_variant1" per entry, into buf
 * (len bytes, NUL-terminated; HE_EINVAL if too small) */
int he_tune_table(const he_ctx *ctx, char *buf, size_t len);
/* forces variant choice (0 or 1) of op everywhere, or restores the table with choice = -1 */
int he_tune_force(he_ctx *ctx, int op, int choice);

/* operation counters since creation: [ciphertext key switches (a batched key switch over n
 * ciphertexts counts n), rotation calls, hmult calls, rescale calls, bootstrapping calls] */
int he_counters(const he_ctx *ctx, long *out5);
/* number of kernel launches this context has issued since creation */
long he_launch_count(const he_ctx *ctx);
/* live timing of one kernel family ("ntt", "ks_inner", "modup", "tensor"; "" = off): CUDA
 * events on the context stream around each launch; he_profile_read synchronises, returns the
 * summed device time, the launch count and the algorithmic bytes of those launches, and resets.
 * A graph captured by he_softmax_graph while a family is profiled carries that family's events
 * inside (event-record nodes, recorded at every launch of the graph); a read counts the latest
 * launch of each graph launched since the previous read. */
int he_profile_kernel(he_ctx *ctx, const char *name);
int he_profile_read(he_ctx *ctx, double *total_ms, long *launches, double *bytes);
/* with he_profile_kernel(ctx, "all"): every launch and device copy is timed; this call
 * synchronises and writes one text line "family launches total_ms bytes" (bytes: the
 * algorithmic bytes of those launches, 0 where not stated) per kernel family (the transforms by
 * call site and direction: ntt, ntt_modup, ntt_moddown, ntt_rescale, ntt_modraise, each with an
 * _inv twin for the inverse, 16 N bytes per limb; modup, ks_inner, moddown, tensor, rescale,
 * lintrans, elementwise, automorph, modraise, encode, decode, keygen, copy) into buf (len bytes,
 * NUL-terminated), then one line "phase:P launches total_ms 0" per phase of the Softmax circuit the launches belonged to (main: the m main-thread ciphertexts;
 * aux: the auxiliary thread of Alg. 3 outside bootstrapping; bootstrap.stc, bootstrap.modraise,
 * bootstrap.cts, bootstrap.evalmod: the four steps of every bootstrapping; other: launches
 * outside a Softmax), then one line "pf:P:family launches total_ms bytes" per (phase, family)
 * pair, then resets.  HE_EINVAL if buf is too small.  The phases are
 * also NVTX ranges of the same names. */
int he_profile_breakdown(he_ctx *ctx, char *buf, size_t len);
/* bounded device wait self test: a kernel polls a flag nobody sets for at most max_iter polls
 * and returns HE_ETIMEOUT; the context stays usable. */
int he_selftest_bounded_wait(he_ctx *ctx, long max_iter);

#ifdef __cplusplus
}
#endif
#endif
