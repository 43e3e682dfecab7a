// Kernel declarations shared by the host orchestration (he_host.cu).
#pragma once
#include "he_common.cuh"

#include <utility>

// Launch helper: klaunch(kernel, grid, block, smem, stream)(args...) launches like
// kernel<<<grid, block, smem, stream>>>(args...).  While he_pdl_launch is set (the default), the
// launch carries the programmatic-stream-serialisation attribute, so the kernel may be scheduled
// while the previous kernel of the stream finishes; its grid_dep_enter() keeps the order of
// memory effects.  Measured on the Softmax step: 3-5% faster in eager streams; in a replayed
// CUDA graph, which already hides launch latency, 0.2-0.7% slower, so graph capture turns it off
// for the capturing thread.  Launch errors are left for cudaGetLastError, as with <<<>>>.
extern thread_local int he_pdl_launch;
template <typename... P>
struct KLaunch {
    void (*k)(P...);
    dim3 grid, block;
    size_t smem;
    cudaStream_t st;
    template <typename... A>
    void operator()(A &&...a) const {
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = he_pdl_launch;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        (void)cudaLaunchKernelEx(&cfg, k, std::forward<A>(a)...);
    }
};
template <typename... P>
inline KLaunch<P...> klaunch(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st) {
    return KLaunch<P...>{k, grid, block, smem, st};
}

struct Scal {
    uint64_t v[HE_MAX_LIMBS];
};

// Baby-step/giant-step inner sums of one linear-transform level (passed by value):
//   out_a = sum_b pt_{a,b} (.) baby_b   for every giant index a,
// over batches [nct][2][L][N] in NTT form; plaintexts [L][N] in Montgomery form.
#define HE_LT_MAXB 16
#define HE_LT_MAXA 16
#define HE_LT_MAXPT 128
#define HE_LT_KT 64   // coefficients per tile (plaintext tile staged in shared memory)
struct LtArgs {
    const uint64_t *baby[HE_LT_MAXB];
    uint64_t *out[HE_LT_MAXA];
    const uint64_t *pt[HE_LT_MAXPT];
    signed char ptix[HE_LT_MAXA][HE_LT_MAXB];   // plaintext of (a, b), -1 if the diagonal is zero
    int nb, na, npt;
};

// Neighbours fused into a forward NTT (passed by value; kind 0: none).  Limb i of polynomial p of
// the transformed batch (nper limbs per polynomial, coefficient index k):
//   kind 1 (ModDown): the batch is Conv_{P->Q}; the row pass writes
//       out_i = (x_i - NTT(conv)_i) pinv_i (+ add_i), x_i at x + p (nper + alpha) N + i N,
//       out / add polynomial p at base + (p / 2) stride + (p % 2) nper N, pinv = cst[2 prime], cst[2 prime + 1];
//   kind 2 (rescale): the column pass reads the centred last limb last[p] reduced mod q_i
//       instead of the batch, the row pass writes out_i = (x_i - NTT(t)_i) qlinv_i,
//       x_i at x + p (nper + 1) N + i N, out_i at out + p nper N + i N, qlinv = cst[2 i], cst[2 i + 1];
//   kind 3 (relinearise + rescale): the batch is Conv_{D->Q}, D = {q_l} u P; the row pass writes
//       out_i = (P d_i + K_i - NTT(conv)_i) (P q_l)^{-1}, K_i at x + p (nper + alpha) N + i N,
//       d_i (tensor) at add + (p / 2) sadd + (p % 2) (nper + 1) N + i N, out as in kind 1,
//       cst[4 i ..]: P mod q_i, Shoup, (P q_l)^{-1} mod q_i, Shoup.
// Kinds 4-6 compute the transformed batch itself in the column pass, as a fast basis conversion
//   conv_t = sum_s [y_s]_centred (qhat_s mod m_t) mod m_t
// of source limbs y_s in coefficient form that the inverse transform before has already
// multiplied by qhat_s^{-1} mod q_s (its N^{-1} factor folded with that constant); the weights are
// in Montgomery form, so one 128-bit sum reduced by REDC gives the residue.
//   kind 4 (ModUp): polynomial p of the batch is digit j = j0 + p % ndc of ciphertext c = p / ndc
//       (nper = L + alpha extended limbs t).  Sources: limbs dlo[j] .. dlo[j] + dds[j] - 1 of
//       src + c sstride; weights cvw[dcv[j] + s wstride + t].  The digit's own limbs are copied
//       from the NTT-form input xntt + c sxn instead (the row pass leaves them).
//   kind 5 (ModDown): as kind 1, with conv computed from the ns limbs slo .. slo + ns - 1 of
//       src + p sstride (moduli sidx[s]); weights cvw[s wstride + prime].
//   kind 6 (relinearise + rescale): as kind 3, with conv computed as in kind 5.
//   kind 7 (ModUp of all digits after k_modup_all with its NTT-form copies): a plain forward
//       transform of the batch that leaves the digits' own limbs (dlo, dds, ndc, j0 as in kind 4).
struct NttFuse {
    int kind;
    int alpha;
    const uint64_t *x;
    uint64_t *out;
    long so;
    const uint64_t *add;
    long sadd;
    const uint64_t *cst;
    const uint64_t *last;
    uint64_t ql;
    // kinds 4-6
    const uint64_t *src;
    long sstride;
    const uint64_t *cvw;
    int wstride;
    int ns, slo;
    int sidx[HE_CONV_MAXSRC];
    const uint64_t *xntt;
    long sxn;
    int ndc, j0;
    int dlo[8], dds[8];
    long dcv[8];
};

// Several key switches in one inner-product launch.  k_ks_inner: the same digits, grid.y = r,
// key[r], galois element g[r], output at acc + r acc_stride (n = 0: the single key and g
// arguments).  k_ks_inner_sum: the sum of the n key switches with digits at dig + dig_off[r].
struct KsMulti {
    const uint64_t *key[16];
    int g[16];
    long dig_off[16];
    long acc_stride;
    int n;
};

// ModUp of every digit in one launch (grid.y = digit): digit j covers limbs [lo[j], lo[j] + ds[j])
// and its constants start at cvoff[j] (the layout k_modup uses)
struct ModUpDigits {
    int lo[8], ds[8];
    long cvoff[8];
};

// Linear combination sum_t w_t x_t (+ w0 on c0) of up to HE_LC_MAXT batches at any levels
#define HE_LC_MAXT 8
struct LcArgs {
    const uint64_t *x[HE_LC_MAXT];
    long cs[HE_LC_MAXT];   // ciphertext stride of input t (words)
    long ps[HE_LC_MAXT];   // polynomial stride of input t (words)
    uint64_t w[HE_LC_MAXT + 1][HE_MAX_LIMBS];   // weights (Montgomery form); row nt: constant on c0
    int nt;
};

__global__ void k_add(uint64_t *out, long so, const uint64_t *a, long sa, const uint64_t *b, long sb,
                      int count, int nper, LimbMap map, const ModC *mods, int logN, int sub);
__global__ void k_mul(uint64_t *out, long so, const uint64_t *a, long sa, const uint64_t *b, long sb,
                      int count, int nper, LimbMap map, const ModC *mods, int logN, int accumulate);
__global__ void k_mul_scalar(uint64_t *out, long so, const uint64_t *a, long sa, Scal scal,
                             int count, int nper, LimbMap map, const ModC *mods, int logN);
__global__ void k_add_scalar(uint64_t *a, long sa, Scal scal, int count, int nper, LimbMap map,
                             const ModC *mods, int logN);
__global__ void k_tensor(uint64_t *d, long sd, const uint64_t *a, long sa, const uint64_t *b, long sb, long psb,
                         int bdiv, int nct, int nper, LimbMap map, const ModC *mods, int logN, int accumulate);
__global__ void k_automorph(uint64_t *out, long so, const uint64_t *a, long sa, int count, int nper, int g, int logN);
__global__ void k_axpy_scalar(uint64_t *out, long so, const uint64_t *a, long sa, Scal scal, int count, int nper,
                              LimbMap map, const ModC *mods, int logN);
__global__ void k_automorph_acc(uint64_t *out, long so, const uint64_t *a, long sa, int count, int nper, LimbMap map,
                                const ModC *mods, int g, int logN);
__global__ void k_lt_bsgs(LtArgs A, int npoly, int L, LimbMap qmap, const ModC *mods, int logN);
__global__ void k_lt_bsgs_direct(LtArgs A, int npoly, int L, LimbMap qmap, const ModC *mods, int logN);
// k_lt_bsgs_ct1<nb>: the unstaged sums of one ciphertext (npoly <= 2); A.nb must be 4, 8 or 16
void launch_lt_ct1(dim3 grid, cudaStream_t st, const LtArgs &A, int npoly, int L, const LimbMap &qmap, const ModC *mods,
                   int logN);
__global__ void k_lincomb(uint64_t *out, LcArgs A, int nct, int L, LimbMap qmap, const ModC *mods, int logN);
__global__ void k_modup(uint64_t *out, long so_ct, long so_digit, const uint64_t *x, long sx, int nct,
                        int digit_lo, int dsize, int ntarget, LimbMap tmap, const ModC *mods, const uint64_t *cv,
                        int logN, const uint64_t *xntt, long sxn);
__global__ void k_modup_all(uint64_t *out, long so_ct, const uint64_t *x, long sx, int nct, ModUpDigits D,
                            int ntarget, LimbMap tmap, const ModC *mods, const uint64_t *cvbase, int logN,
                            const uint64_t *xntt, long sxn);
__global__ void k_moddown_conv(uint64_t *out, const uint64_t *x, int npoly, int L, int alpha, LimbMap qmap,
                               const int *pidx, const ModC *mods, const uint64_t *cv, int nqall, int logN);

__global__ void k_ks_inner_sum(uint64_t *__restrict__ acc, const uint64_t *__restrict__ dig, int nct, int ndig,
                               int L, int alpha, LimbMap tmap, const ModC *mods, int key_nlimb, int nq_all, int logN,
                               KsMulti M);
__global__ void k_rescale_spread(uint64_t *tmp, const uint64_t *last, int npoly, int Lm1, LimbMap qmap,
                                 const ModC *mods, uint64_t ql, int logN);
__global__ void k_rescale_fin(uint64_t *out, const uint64_t *x, const uint64_t *t, int npoly, int L, LimbMap qmap,
                              const ModC *mods, const uint64_t *qlinv, int logN);
__global__ void k_modraise(uint64_t *out, const uint64_t *x0, int npoly, int L, LimbMap qmap, const ModC *mods,
                           uint64_t q0, int logN);
__global__ void k_sample_uniform(uint64_t *out, long so, int count, int nper, LimbMap map,
                                 const ModC *mods, uint64_t seed, uint64_t dom, int logN);
__global__ void k_sample_small(int64_t *out, int n, uint64_t seed, uint64_t dom, uint64_t ctr0,
                               const uint64_t *cdt, int cdt_len, int kind);
__global__ void k_sample_hwt(int64_t *out, int n, int h, uint64_t seed, uint64_t dom, uint64_t dom_sign);
__global__ void k_small_to_limbs(uint64_t *out, long so, const int64_t *v, int count, int nper, LimbMap map,
                                 const ModC *mods, int logN);
__global__ void k_bitrev_c(double2 *v, int n0, int logn0);
__global__ void k_sfft_fwd_stage(double2 *v, int n0, int len, const double2 *zeta, const int *rg, int m2n);
__global__ void k_sfft_inv_stage(double2 *v, int n0, int len, const double2 *zeta, const int *rg, int m2n);
__global__ void k_scale_c(double2 *v, int n0, double div);
__global__ void k_round_to_limbs(uint64_t *out, long so, const double2 *w, double scale, int count, int nper,
                                 LimbMap map, const ModC *mods, int logN);
__global__ void k_crt_to_double(double2 *w, const uint64_t *x, int L, LimbMap qmap, const ModC *mods,
                                const uint64_t *radix, const uint64_t *radinv, const double *qd, double scale, int logN);
__global__ void k_key_combine(uint64_t *b, const uint64_t *a, const uint64_t *e, const uint64_t *s, const uint64_t *sp,
                              Scal pm, int nl, int dlo, int dhi, LimbMap map, const ModC *mods, int logN);
__global__ void k_bounded_wait(const volatile int *flag, int *status, long max_iter);
__global__ void k_reduce_limbs(uint64_t *out, const uint64_t *x, int count, int nper, LimbMap map, const ModC *mods,
                               int logN);

// key-switching inner product sum_j d~_j swk_j (k_ks_inner_t<ndig>, ndig in 1 .. 8: the key
// words of a (limb, coefficient) kept in registers); M.n > 0: grid.y key switches of the same digits
void launch_ks_inner(dim3 grid, cudaStream_t st, uint64_t *acc, const uint64_t *dig, int nct, int ndig, int L, int alpha,
                     const LimbMap &tmap, const ModC *mods, const uint64_t *key, int key_nlimb, int nq_all, int g,
                     int logN, int accumulate, const KsMulti &M);

// one-pass transform of `count` limbs of N = 2^16 (no fused neighbours): one cluster of 16 CTAs per
// limb, the exchange between the column and row passes in distributed shared memory; out of place
// from src when given (as launch_ntt_rb).  ntt_1pass_setup() raises the kernels' dynamic shared
// memory limit (once per device; 0 on success).
int ntt_1pass_setup();
void launch_ntt_1pass(bool inverse, int count, uint64_t *base, int nper, long poly_stride, const LimbMap &map,
                      const ModC *mods, const ulonglong2 *tw2, const uint64_t *ninv, int logN, cudaStream_t st,
                      const uint64_t *src, long src_stride);

// register-blocked NTT of `count` limbs (N = 2^12: logE = 3, N = 2^16: logE = 4); launches
// the column and row passes on stream st
// the first pass reads from src (limb l of polynomial i at src + i src_stride + l N) when it is
// not null, so the transform can be out of place
// tw2: per modulus p, N (psi^brv(k), Shoup companion) pairs at tw2 + 2 N p, then N inverse pairs
void launch_ntt_rb(int logE, bool inverse, int count, uint64_t *base, int nper, long poly_stride, const LimbMap &map,
                   const ModC *mods, const ulonglong2 *tw2, const uint64_t *ninv, int logN, cudaStream_t st,
                   const uint64_t *src = nullptr, long src_stride = 0, const NttFuse *fuse = nullptr,
                   bool small_cta = false);
