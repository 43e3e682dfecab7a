// CUDA kernels for RNS-CKKS on sm_103a.  Every step of the ciphertext arithmetic runs here;
// the host code in he_host.cu only sequences launches.
//
// Polynomial batches are addressed as (base, count, nper, poly_stride): limb l of the batch
// lives at base + (l / nper) * poly_stride + (l % nper) * N and uses modulus prime[l % nper].
#include "he_kernels.cuh"

#include <cooperative_groups.h>

thread_local int he_pdl_launch = 1;   // see klaunch

// ------------------------------------------------------------------------------------------
// Elementwise kernels over a batch (count limbs, addressing as above).
#define EW_PROLOGUE                                                                           \
    const int N = 1 << logN;                                                                  \
    long total = (long)count << logN;                                                         \
    for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < total; x += (long)gridDim.x * blockDim.x) { \
        int l = (int)(x >> logN), k = (int)(x & (N - 1));                                     \
        int li = l % nper;                                                                    \
        long po = (long)(l / nper);                                                           \
        const ModC m = mods[map.prime[li]];

__global__ void k_add(uint64_t *out, long so, const uint64_t *a, long sa, const uint64_t *b, long sb,
                      int count, int nper, LimbMap map, const ModC *mods, int logN, int sub) {
    grid_dep_enter();
    EW_PROLOGUE
    long off = (long)li * N + k;
    uint64_t u = a[po * sa + off], v = b[po * sb + off];
    out[po * so + off] = sub ? sub_mod(u, v, m.q) : add_mod(u, v, m.q);
    }
}

__global__ void k_mul(uint64_t *out, long so, const uint64_t *a, long sa, const uint64_t *b, long sb,
                      int count, int nper, LimbMap map, const ModC *mods, int logN, int accumulate) {
    grid_dep_enter();
    EW_PROLOGUE
    long off = (long)li * N + k;
    uint64_t r = mul_mod(a[po * sa + off], b[po * sb + off], m);
    if (accumulate) r = add_mod(out[po * so + off], r, m.q);
    out[po * so + off] = r;
    }
}

// out = a * s_l with a per-limb scalar (residue of the scalar mod each modulus, by limb index)
__global__ void k_mul_scalar(uint64_t *out, long so, const uint64_t *a, long sa, Scal scal,
                             int count, int nper, LimbMap map, const ModC *mods, int logN) {
    grid_dep_enter();
    EW_PROLOGUE
    long off = (long)li * N + k;
    out[po * so + off] = mul_mod(a[po * sa + off], scal.v[li], m);
    }
}

// out += a * scal[li] on the selected limbs
__global__ void k_axpy_scalar(uint64_t *out, long so, const uint64_t *a, long sa, Scal scal, int count, int nper,
                              LimbMap map, const ModC *mods, int logN) {
    grid_dep_enter();
    EW_PROLOGUE
    long off = (long)li * N + k;
    out[po * so + off] = add_mod(out[po * so + off], mul_mod(a[po * sa + off], scal.v[li], m), m.q);
    }
}

// adds scal[li] to every evaluation point of the selected polynomials (a constant polynomial
// has the same value at every root)
__global__ void k_add_scalar(uint64_t *a, long sa, Scal scal, int count, int nper, LimbMap map,
                             const ModC *mods, int logN) {
    grid_dep_enter();
    EW_PROLOGUE
    long off = (long)li * N + k;
    a[po * sa + off] = add_mod(a[po * sa + off], scal.v[li], m.q);
    }
}

// tensor of ciphertext batches a, b into d [ct][3][nper][N]: ciphertext c of a (stride sa, two
// polynomials of sa/2 words) with ciphertext c / bdiv of b (stride sb, polynomial stride psb):
// bdiv = 1 pairs them one to one, bdiv = m pairs every m of a with one of b (nct: one b for all);
// accumulate adds into d
__global__ void k_tensor(uint64_t *d, long sd, const uint64_t *a, long sa, const uint64_t *b, long sb, long psb,
                         int bdiv, int nct, int nper, LimbMap map, const ModC *mods, int logN, int accumulate) {
    grid_dep_enter();
    const int N = 1 << logN;
    long total = (long)nct * nper << logN;
    for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < total; x += (long)gridDim.x * blockDim.x) {
        int l = (int)(x >> logN), k = (int)(x & (N - 1));
        int li = l % nper, c = l / nper;
        const ModC m = mods[map.prime[li]];
        long off = (long)li * N + k;
        // each ciphertext holds 2 (inputs) or 3 (output) polynomials: poly stride = ct stride / #polys
        const uint64_t *pa = a + c * sa, *pb = b + (c / bdiv) * sb;
        long psa = sa / 2, ps = sd / 3;
        uint64_t a0 = pa[off], a1 = pa[psa + off], b0 = pb[off], b1 = pb[psb + off];
        uint64_t d0 = mul_mod(a0, b0, m);
        uint64_t d1 = add_mod(mul_mod(a0, b1, m), mul_mod(a1, b0, m), m.q);
        uint64_t d2 = mul_mod(a1, b1, m);
        uint64_t *pd = d + c * sd;
        if (accumulate) {
            d0 = add_mod(d0, pd[off], m.q);
            d1 = add_mod(d1, pd[ps + off], m.q);
            d2 = add_mod(d2, pd[2 * ps + off], m.q);
        }
        pd[off] = d0;
        pd[ps + off] = d1;
        pd[2 * ps + off] = d2;
    }
}

// NTT-domain automorphism X -> X^g: out[k] = in[pi(k)], e_k = 2 brv(k) + 1,
// pi(k) = brv((e_k g mod 2N - 1) / 2)
__device__ __forceinline__ int auto_index(int k, int g, int logN) {
    int e = 2 * brev_bits(k, logN) + 1;
    int e2 = (int)(((long)e * g) & ((2L << logN) - 1));
    return brev_bits((e2 - 1) >> 1, logN);
}

__global__ void k_automorph(uint64_t *out, long so, const uint64_t *a, long sa, int count, int nper, int g, int logN) {
    grid_dep_enter();
    const int N = 1 << logN;
    long total = (long)count << logN;
    for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < total; x += (long)gridDim.x * blockDim.x) {
        int l = (int)(x >> logN), k = (int)(x & (N - 1));
        int li = l % nper;
        long po = l / nper;
        out[po * so + (long)li * N + k] = a[po * sa + (long)li * N + auto_index(k, g, logN)];
    }
}

// out += a(X^g) on the selected limbs (the c0 part of a rotation, added to a key-switch result)
__global__ void k_automorph_acc(uint64_t *out, long so, const uint64_t *a, long sa, int count, int nper, LimbMap map,
                                const ModC *mods, int g, int logN) {
    grid_dep_enter();
    EW_PROLOGUE
    long o = po * so + (long)li * N + k;
    out[o] = add_mod(out[o], a[po * sa + (long)li * N + auto_index(k, g, logN)], m.q);
    }
}

// Baby-step/giant-step inner sums of a linear-transform level: every block stages the
// plaintext diagonals of one (limb, HE_LT_KT-coefficient tile) in shared memory, then each row
// (ciphertext polynomial) reads its nb baby-step values once and writes the na giant-step
// sums once; the sums are 128-bit and reduced once (plaintexts in Montgomery form, at most 16
// terms below 16 q^2 < q 2^64).  Dynamic shared memory: npt * HE_LT_KT words.
__global__ void __launch_bounds__(256) k_lt_bsgs(LtArgs A, int npoly, int L, LimbMap qmap, const ModC *mods,
                                                 int logN) {
    grid_dep_enter();
    extern __shared__ uint64_t spt[];
    constexpr int KT = HE_LT_KT, RG = 256 / KT;
    const int N = 1 << logN, ntile = N / KT;
    const int kk = threadIdx.x % KT, rg = threadIdx.x / KT;
    for (long t = blockIdx.x; t < (long)L * ntile; t += gridDim.x) {
        const int l = (int)(t / ntile), k0 = (int)(t % ntile) * KT;
        const ModC m = mods[qmap.prime[l]];
        __syncthreads();   // the previous tile's readers are done
        for (int i = threadIdx.x; i < A.npt * KT; i += blockDim.x) spt[i] = A.pt[i / KT][(long)l * N + k0 + i % KT];
        __syncthreads();
        for (int r = blockIdx.y * RG + rg; r < npoly; r += gridDim.y * RG) {
            const long off = ((long)r * L + l) * N + k0 + kk;
            uint64_t bv[HE_LT_MAXB];
#pragma unroll
            for (int b = 0; b < HE_LT_MAXB; b++) bv[b] = b < A.nb ? A.baby[b][off] : 0;
            for (int a = 0; a < A.na; a++) {
                uint64_t lo = 0, hi = 0;
#pragma unroll
                for (int b = 0; b < HE_LT_MAXB; b++) {
                    const int pi = b < A.nb ? A.ptix[a][b] : -1;
                    if (pi >= 0) mac_wide(lo, hi, bv[b], spt[pi * KT + kk]);
                }
                A.out[a][off] = redc(lo, hi, m);
            }
        }
    }
}

// The same sums for batches of a few rows (npoly <= 8): one thread per (limb, coefficient), no
// staging; the plaintext values of a giant step are loaded once and used for every row.
__global__ void k_lt_bsgs_direct(LtArgs A, int npoly, int L, LimbMap qmap, const ModC *mods, int logN) {
    grid_dep_enter();
    const int N = 1 << logN;
    long total = (long)L << logN;
    for (long id = blockIdx.x * (long)blockDim.x + threadIdx.x; id < total; id += (long)gridDim.x * blockDim.x) {
        const int l = (int)(id >> logN), k = (int)(id & (N - 1));
        const ModC m = mods[qmap.prime[l]];
        for (int a = 0; a < A.na; a++) {
            uint64_t pv[HE_LT_MAXB];
#pragma unroll
            for (int b = 0; b < HE_LT_MAXB; b++) {
                const int pi = b < A.nb ? A.ptix[a][b] : -1;
                pv[b] = pi >= 0 ? A.pt[pi][(long)l * N + k] : 0;
            }
            for (int r = 0; r < npoly; r++) {
                const long off = ((long)r * L + l) * N + k;
                uint64_t lo = 0, hi = 0;
#pragma unroll
                for (int b = 0; b < HE_LT_MAXB; b++) {
                    const int pi = b < A.nb ? A.ptix[a][b] : -1;
                    if (pi >= 0) mac_wide(lo, hi, A.baby[b][off], pv[b]);
                }
                A.out[a][off] = redc(lo, hi, m);
            }
        }
    }
}

// The same sums for one ciphertext (two rows) with NB baby steps known at compile time: a thread
// keeps both rows' NB baby-step values in registers (4 NB words) and reads every plaintext word
// once, using it for both rows, so each input of the level is read once.  (With the bound
// HE_LT_MAXB = 16 instead of NB the same idea needed 103 registers and lost occupancy.)
// grid.y splits the giant steps of a coefficient over that many threads (each reloads the baby
// steps): low levels have few limbs and otherwise too few threads to hide the plaintext loads.
template <int NB>
__global__ void __launch_bounds__(256) k_lt_bsgs_ct1(LtArgs A, int npoly, int L, LimbMap qmap, const ModC *mods,
                                                     int logN) {
    grid_dep_enter();
    const int N = 1 << logN;
    long total = (long)L << logN;
    for (long id = blockIdx.x * (long)blockDim.x + threadIdx.x; id < total; id += (long)gridDim.x * blockDim.x) {
        const int l = (int)(id >> logN), k = (int)(id & (N - 1));
        const ModC m = mods[qmap.prime[l]];
        const long o0 = (long)l * N + k, o1 = ((long)L + l) * N + k;
        uint64_t b0[NB], b1[NB];
#pragma unroll
        for (int b = 0; b < NB; b++) {
            b0[b] = A.baby[b][o0];
            b1[b] = npoly > 1 ? A.baby[b][o1] : 0;
        }
        const int ag = (A.na + gridDim.y - 1) / gridDim.y, a1 = min(A.na, (int)(blockIdx.y + 1) * ag);
        for (int a = blockIdx.y * ag; a < a1; a++) {
            uint64_t lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
#pragma unroll
            for (int b = 0; b < NB; b++) {
                const int pi = A.ptix[a][b];
                if (pi >= 0) {
                    const uint64_t pv = A.pt[pi][o0];
                    mac_wide(lo0, hi0, b0[b], pv);
                    mac_wide(lo1, hi1, b1[b], pv);
                }
            }
            A.out[a][o0] = redc(lo0, hi0, m);
            if (npoly > 1) A.out[a][o1] = redc(lo1, hi1, m);
        }
    }
}

void launch_lt_ct1(dim3 grid, cudaStream_t st, const LtArgs &A, int npoly, int L, const LimbMap &qmap, const ModC *mods,
                   int logN) {
    if (A.nb == 4) klaunch(k_lt_bsgs_ct1<4>, grid, 256, 0, st)(A, npoly, L, qmap, mods, logN);
    else if (A.nb == 8) klaunch(k_lt_bsgs_ct1<8>, grid, 256, 0, st)(A, npoly, L, qmap, mods, logN);
    else klaunch(k_lt_bsgs_ct1<16>, grid, 256, 0, st)(A, npoly, L, qmap, mods, logN);
}

// out[c][p][l] = sum_t x_t[c][p][l] w_t[l] (+ w_nt[l] when p = 0) for l < L: rows t < nt of w in
// Montgomery form (sums of at most 8 products stay below q 2^64), row nt a plain residue.
// Reads each input once (only its first L limbs).
__global__ void k_lincomb(uint64_t *out, LcArgs A, int nct, int L, LimbMap qmap, const ModC *mods, int logN) {
    grid_dep_enter();
    const int N = 1 << logN;
    long total = (long)nct * 2 * L << logN;
    for (long id = blockIdx.x * (long)blockDim.x + threadIdx.x; id < total; id += (long)gridDim.x * blockDim.x) {
        const int k = (int)(id & (N - 1));
        const long row = id >> logN;                 // (c * 2 + p) * L + l
        const int l = (int)(row % L), p = (int)((row / L) & 1);
        const long c = row / L / 2;
        const ModC m = mods[qmap.prime[l]];
        uint64_t lo = 0, hi = 0;
        for (int t = 0; t < A.nt; t++)
            mac_wide(lo, hi, A.x[t][c * A.cs[t] + p * A.ps[t] + (long)l * N + k], A.w[t][l]);
        uint64_t v = redc(lo, hi, m);
        if (p == 0) v = add_mod(v, A.w[A.nt][l], m.q);
        out[id] = v;
    }
}

// ------------------------------------------------------------------------------------------
// Basis conversion (coefficient domain).  ModUp for one digit D of a batch of polynomials:
// for every target modulus t of the extended basis,
//   out_t = sum_{i in D} [x_i * qhinv_i]_{q_i} * (qh_{i,t}) mod m_t.
// For t in D this reproduces x_t.  The input x already holds [x_i qhinv_i]_{q_i}: the inverse
// transform that produced it multiplied by N^{-1} qhinv_i instead of N^{-1}.  cv layout per
// (level, digit): qhinv[a], qhinv_shoup[a], then qh[a][ntarget] (Montgomery form).
__global__ void k_modup(uint64_t *out, long so_ct, long so_digit, const uint64_t *x, long sx, int nct,
                        int digit_lo, int dsize, int ntarget, LimbMap tmap, const ModC *mods, const uint64_t *cv,
                        int logN, const uint64_t *xntt, long sxn) {
    grid_dep_enter();
    // one thread per (ciphertext, coefficient): the digit's limbs are read once, then every
    // target limb is produced as one 128-bit sum reduced once (cv holds the products of the
    // other digit primes in Montgomery form, so redc returns the plain sum mod m_t)
    const int N = 1 << logN;
    long total = (long)nct << logN;
    for (long id = blockIdx.x * (long)blockDim.x + threadIdx.x; id < total; id += (long)gridDim.x * blockDim.x) {
        int c = (int)(id >> logN), k = (int)(id & (N - 1));
        // centred representatives (-q_i/2, q_i/2] (|y_i| and a sign bit): the result is
        // d + u Q_D with zero-mean u
        uint64_t y[HE_CONV_MAXSRC];   // (loops unrolled to the bound: y stays in registers)
        unsigned negmask = 0;
#pragma unroll
        for (int i = 0; i < HE_CONV_MAXSRC; i++) {
            if (i >= dsize) break;
            uint64_t qi = mods[tmap.prime[digit_lo + i]].q;
            uint64_t v = x[c * sx + (long)(digit_lo + i) * N + k];
            if (v > (qi - 1) / 2) {
                v = qi - v;
                negmask |= 1u << i;
            }
            y[i] = v;
        }
        uint64_t *o = out + c * so_ct + so_digit + k;
        // the digit's own limbs: the NTT-form input limbs themselves (the conversion would
        // reproduce their coefficients)
        for (int i = 0; i < dsize; i++)
            o[(long)(digit_lo + i) * N] = xntt[c * sxn + (long)(digit_lo + i) * N + k];
        // (two targets per iteration: two independent 128-bit sums in flight per thread)
#pragma unroll 2
        for (int t = 0; t < ntarget; t++) {
            if (t == digit_lo) t += dsize;
            if (t >= ntarget) break;
            const ModC mt = mods[tmap.prime[t]];
            // sum of |y_i| (c or m_t - c): below dsize 2^60 m_t < m_t 2^64
            uint64_t lo = 0, hi = 0;
#pragma unroll
            for (int i = 0; i < HE_CONV_MAXSRC; i++) {
                if (i >= dsize) break;
                uint64_t w = cv[2 * dsize + i * ntarget + t];
                mac_wide(lo, hi, y[i], (negmask >> i) & 1 ? mt.q - w : w);
            }
            o[(long)t * N] = redc(lo, hi, mt);
        }
    }
}

// ModUp of all digits of nct polynomials in one launch (grid.y = digit j): every target limb of
// the extended basis is converted, the digit's own limbs included (there the conversion is the
// CRT identity and returns x exactly), so one transform of all digits follows.  Output
// [nct][ndig][ntarget][N] (coefficient form).  With xntt given, the digit's own limbs are copied
// from the NTT-form input instead (xntt + c sxn), and the transform after skips them (kind 7).
__global__ void k_modup_all(uint64_t *out, long so_ct, const uint64_t *x, long sx, int nct, ModUpDigits D,
                            int ntarget, LimbMap tmap, const ModC *mods, const uint64_t *cvbase, int logN,
                            const uint64_t *xntt, long sxn) {
    grid_dep_enter();
    const int N = 1 << logN;
    const int j = blockIdx.y, lo = D.lo[j], ds = D.ds[j];
    const uint64_t *cv = cvbase + D.cvoff[j];
    long total = (long)nct << logN;
    for (long id = blockIdx.x * (long)blockDim.x + threadIdx.x; id < total; id += (long)gridDim.x * blockDim.x) {
        int c = (int)(id >> logN), k = (int)(id & (N - 1));
        uint64_t y[HE_CONV_MAXSRC];   // (loops unrolled to the bound: y stays in registers)
        unsigned negmask = 0;
#pragma unroll
        for (int i = 0; i < HE_CONV_MAXSRC; i++) {
            if (i >= ds) break;
            uint64_t qi = mods[tmap.prime[lo + i]].q;
            uint64_t v = x[c * sx + (long)(lo + i) * N + k];
            if (v > (qi - 1) / 2) {
                v = qi - v;
                negmask |= 1u << i;
            }
            y[i] = v;
        }
        uint64_t *o = out + c * so_ct + (long)j * ntarget * N + k;
        for (int t = 0; t < ntarget; t++) {
            if (xntt && t >= lo && t < lo + ds) {   // the digit's own limb: the NTT-form input
                o[(long)t * N] = xntt[c * sxn + (long)t * N + k];
                continue;
            }
            const ModC mt = mods[tmap.prime[t]];
            uint64_t l0 = 0, h0 = 0;
#pragma unroll
            for (int i = 0; i < HE_CONV_MAXSRC; i++) {
                if (i >= ds) break;
                uint64_t w = cv[2 * ds + i * ntarget + t];
                mac_wide(l0, h0, y[i], (negmask >> i) & 1 ? mt.q - w : w);
            }
            o[(long)t * N] = redc(l0, h0, mt);
        }
    }
}

// ModDown conversion: conv_i = sum_k [y_k * phinv_k]_{p_k} (phat_k mod q_i); writes conv into
// out (coefficient domain) for the Q limbs.  x: [npoly][L + alpha][N] with the coefficient-domain
// P limbs at offset L, already multiplied by phinv_k (folded into the inverse transform's N^{-1}).
// cv: phinv[alpha], phinv_shoup[alpha], phat[alpha][nqall] (by Q index).
// One thread per (polynomial, coefficient): the alpha P limbs are read once.
__global__ void k_moddown_conv(uint64_t *out, const uint64_t *x, int npoly, int L, int alpha, LimbMap qmap,
                               const int *pidx, const ModC *mods, const uint64_t *cv, int nqall, int logN) {
    grid_dep_enter();
    const int N = 1 << logN;
    long total = (long)npoly << logN;
    for (long id = blockIdx.x * (long)blockDim.x + threadIdx.x; id < total; id += (long)gridDim.x * blockDim.x) {
        int pl = (int)(id >> logN), k = (int)(id & (N - 1));
        const uint64_t *xp = x + (long)pl * (L + alpha) * N + (long)L * N + k;
        // y_j in centred form (-p_j/2, p_j/2]: keep |y_j| and its sign, so that the conversion
        // error v P has zero mean (a biased v is a constant on every coefficient, whose slot
        // values concentrate where the evaluation point is near 1)
        // (loops unrolled to the largest source count, so that y stays in registers)
        uint64_t y[HE_CONV_MAXSRC];
        unsigned negmask = 0;
#pragma unroll
        for (int j = 0; j < HE_CONV_MAXSRC; j++) {
            if (j >= alpha) break;
            uint64_t pj = mods[pidx[j]].q;
            uint64_t v = xp[(long)j * N];
            if (v > (pj - 1) / 2) {
                v = pj - v;
                negmask |= 1u << j;
            }
            y[j] = v;
        }
        uint64_t *o = out + (long)pl * L * N + k;
#pragma unroll 2
        for (int i = 0; i < L; i++) {
            const ModC mi = mods[qmap.prime[i]];
            // one 128-bit sum, reduced once (phat_j mod q_i stored in Montgomery form)
            uint64_t lo = 0, hi = 0;
#pragma unroll
            for (int j = 0; j < HE_CONV_MAXSRC; j++) {
                if (j >= alpha) break;
                uint64_t w = cv[2 * alpha + j * nqall + qmap.prime[i]];
                mac_wide(lo, hi, y[j], (negmask >> j) & 1 ? mi.q - w : w);
            }
            o[(long)i * N] = redc(lo, hi, mi);
        }
    }
}

// Key-switching inner product: for each ciphertext c and extended limb t,
//   acc_{0,1}[t] = sum_j d~_j[t][pi_g(k)] * key_j^{b,a}[kt][k],
// with the key limb kt = t for Q limbs and nq_all + (t - L) for P limbs.  The key is read once
// per (t, k) for all ciphertexts of the batch.
// NDIG digits at compile time: the key words of a (limb, coefficient) stay in registers
template <int NDIG>
__global__ void k_ks_inner_t(uint64_t *__restrict__ acc, const uint64_t *__restrict__ dig, int nct, int L, int alpha,
                             LimbMap tmap, const ModC *mods, const uint64_t *__restrict__ key, int key_nlimb,
                             int nq_all, int g, int logN, int accumulate, KsMulti M) {
    grid_dep_enter();
    const int N = 1 << logN;
    const int nl = L + alpha;
    if (M.n) {   // key switch blockIdx.y of several (same digits, own key and galois element)
        key = M.key[blockIdx.y];
        g = M.g[blockIdx.y];
        acc += blockIdx.y * M.acc_stride;
    }
    long total = (long)nl << logN;
    for (long id = blockIdx.x * (long)blockDim.x + threadIdx.x; id < total; id += (long)gridDim.x * blockDim.x) {
        int t = (int)(id >> logN), k = (int)(id & (N - 1));
        const ModC m = mods[tmap.prime[t]];
        int kt = t < L ? t : nq_all + (t - L);
        int src = g > 1 ? auto_index(k, g, logN) : k;
        uint64_t kb[NDIG], ka[NDIG];
#pragma unroll
        for (int j = 0; j < NDIG; j++) {
            kb[j] = key[((long)(2 * j) * key_nlimb + kt) * N + k];
            ka[j] = key[((long)(2 * j + 1) * key_nlimb + kt) * N + k];
        }
#pragma unroll 2
        for (int c = 0; c < nct; c++) {
            // the key is stored in Montgomery form: sum of d_j (k_j 2^64 mod m) < ndig m^2,
            // below m 2^64, reduced once
            uint64_t l0 = 0, h0 = 0, l1 = 0, h1 = 0;
#pragma unroll
            for (int j = 0; j < NDIG; j++) {
                uint64_t d = dig[(((long)c * NDIG + j) * nl + t) * N + src];
                mac_wide(l0, h0, d, kb[j]);
                mac_wide(l1, h1, d, ka[j]);
            }
            uint64_t r0 = redc(l0, h0, m), r1 = redc(l1, h1, m);
            const long o0 = ((long)(2 * c) * nl + t) * N + k, o1 = ((long)(2 * c + 1) * nl + t) * N + k;
            if (accumulate) {   // sums of several key switches over Q u P (one ModDown after)
                r0 = add_mod(acc[o0], r0, m.q);
                r1 = add_mod(acc[o1], r1, m.q);
            }
            acc[o0] = r0;
            acc[o1] = r1;
        }
    }
}

void launch_ks_inner(dim3 grid, cudaStream_t st, uint64_t *acc, const uint64_t *dig, int nct, int ndig, int L, int alpha,
                     const LimbMap &tmap, const ModC *mods, const uint64_t *key, int key_nlimb, int nq_all, int g,
                     int logN, int accumulate, const KsMulti &M) {
#define HE_KS_CASE(D)                                                                                          \
    case D:                                                                                                    \
        klaunch(k_ks_inner_t<D>, grid, 256, 0, st)(acc, dig, nct, L, alpha, tmap, mods, key, key_nlimb, nq_all, g, logN, \
                                              accumulate, M);                                                  \
        break;
    switch (ndig) {
        HE_KS_CASE(1) HE_KS_CASE(2) HE_KS_CASE(3) HE_KS_CASE(4) HE_KS_CASE(5) HE_KS_CASE(6) HE_KS_CASE(7)
        HE_KS_CASE(8)
    }
#undef HE_KS_CASE
}

// The sum of M.n key switches (key M.key[r], galois element M.g[r], digits at dig + M.dig_off[r])
// written into acc: each thread runs them in turn for its (limb, coefficient), reducing after each.
__global__ void k_ks_inner_sum(uint64_t *__restrict__ acc, const uint64_t *__restrict__ dig, int nct, int ndig,
                               int L, int alpha, LimbMap tmap, const ModC *mods, int key_nlimb, int nq_all, int logN,
                               KsMulti M) {
    grid_dep_enter();
    const int N = 1 << logN;
    const int nl = L + alpha;
    long total = (long)nl << logN;
    for (long id = blockIdx.x * (long)blockDim.x + threadIdx.x; id < total; id += (long)gridDim.x * blockDim.x) {
        int t = (int)(id >> logN), k = (int)(id & (N - 1));
        const ModC m = mods[tmap.prime[t]];
        int kt = t < L ? t : nq_all + (t - L);
        for (int r = 0; r < M.n; r++) {
            const uint64_t *kr = M.key[r];
            const uint64_t *dr = dig + M.dig_off[r];
            int src = M.g[r] > 1 ? auto_index(k, M.g[r], logN) : k;
            for (int c = 0; c < nct; c++) {
                uint64_t l0 = 0, h0 = 0, l1 = 0, h1 = 0;
                for (int j = 0; j < ndig; j++) {
                    uint64_t d = dr[(((long)c * ndig + j) * nl + t) * N + src];
                    mac_wide(l0, h0, d, kr[((long)(2 * j) * key_nlimb + kt) * N + k]);
                    mac_wide(l1, h1, d, kr[((long)(2 * j + 1) * key_nlimb + kt) * N + k]);
                }
                uint64_t r0 = redc(l0, h0, m), r1 = redc(l1, h1, m);
                const long o0 = ((long)(2 * c) * nl + t) * N + k, o1 = ((long)(2 * c + 1) * nl + t) * N + k;
                if (r > 0) {
                    r0 = add_mod(acc[o0], r0, m.q);
                    r1 = add_mod(acc[o1], r1, m.q);
                }
                acc[o0] = r0;
                acc[o1] = r1;
            }
        }
    }
}

// Rescale, step 1: r = centred last limb (coefficient form, [npoly][N]); writes r mod q_i for
// the remaining L-1 limbs into tmp [npoly][L-1][N].
__global__ void k_rescale_spread(uint64_t *tmp, const uint64_t *last, int npoly, int Lm1, LimbMap qmap,
                                 const ModC *mods, uint64_t ql, int logN) {
    grid_dep_enter();
    const int N = 1 << logN;
    long total = (long)npoly * Lm1 << logN;
    for (long id = blockIdx.x * (long)blockDim.x + threadIdx.x; id < total; id += (long)gridDim.x * blockDim.x) {
        int l = (int)(id >> logN), k = (int)(id & (N - 1));
        int i = l % Lm1, pl = l / Lm1;
        const ModC mi = mods[qmap.prime[i]];
        uint64_t r = last[(long)pl * N + k];
        uint64_t v = r <= (ql - 1) / 2 ? mul_mod(r, 1, mi) : neg_mod(mul_mod(ql - r, 1, mi), mi.q);
        tmp[(long)pl * Lm1 * N + (long)i * N + k] = v;
    }
}

// Rescale, step 2: out_i = (x_i - t_i) * qlinv_i (x: [nct][2][L][N], out: [nct][2][L-1][N])
__global__ void k_rescale_fin(uint64_t *out, const uint64_t *x, const uint64_t *t, int npoly, int L, LimbMap qmap,
                              const ModC *mods, const uint64_t *qlinv, int logN) {
    grid_dep_enter();
    const int N = 1 << logN;
    const int Lm1 = L - 1;
    long total = (long)npoly * Lm1 << logN;
    for (long id = blockIdx.x * (long)blockDim.x + threadIdx.x; id < total; id += (long)gridDim.x * blockDim.x) {
        int l = (int)(id >> logN), k = (int)(id & (N - 1));
        int i = l % Lm1, pl = l / Lm1;
        const ModC mi = mods[qmap.prime[i]];
        uint64_t v = sub_mod(x[(long)pl * L * N + (long)i * N + k], t[(long)pl * Lm1 * N + (long)i * N + k], mi.q);
        out[(long)pl * Lm1 * N + (long)i * N + k] = mul_shoup(v, qlinv[2 * i], qlinv[2 * i + 1], mi.q);
    }
}

// ModRaise: level-0 coefficients (centred mod q0) reduced into L limbs (coefficient form)
__global__ void k_modraise(uint64_t *out, const uint64_t *x0, int npoly, int L, LimbMap qmap, const ModC *mods,
                           uint64_t q0, int logN) {
    grid_dep_enter();
    const int N = 1 << logN;
    long total = (long)npoly * L << logN;
    for (long id = blockIdx.x * (long)blockDim.x + threadIdx.x; id < total; id += (long)gridDim.x * blockDim.x) {
        int l = (int)(id >> logN), k = (int)(id & (N - 1));
        int i = l % L, pl = l / L;
        const ModC mi = mods[qmap.prime[i]];
        uint64_t r = x0[(long)pl * N + k];
        uint64_t v = r <= (q0 - 1) / 2 ? mul_mod(r, 1, mi) : neg_mod(mul_mod(q0 - r, 1, mi), mi.q);
        out[(long)pl * L * N + (long)i * N + k] = v;
    }
}

// ------------------------------------------------------------------------------------------
// Counter-based randomness (SplitMix64 output function, Steele-Lea-Flood 2014):
//   key = mix(seed + G (2 dom + 1)), draw = mix(key + G (ctr + 1)), G = 0x9e3779b97f4a7c15.
__device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
    z ^= z >> 30;
    z *= 0xbf58476d1ce4e5b9ULL;
    z ^= z >> 27;
    z *= 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return z;
}

__device__ __forceinline__ uint64_t rng64(uint64_t seed, uint64_t dom, uint64_t ctr) {
    const uint64_t G = 0x9e3779b97f4a7c15ULL;
    return sm_mix(sm_mix(seed + G * (2 * dom + 1)) + G * (ctr + 1));
}

// uniform residues: limb l (modulus index p = prime[l % nper]) coefficient k from counter
// p * N + k of domain dom; value (w0 2^64 + w1) mod q_p
__global__ void k_sample_uniform(uint64_t *out, long so, int count, int nper, LimbMap map,
                                 const ModC *mods, uint64_t seed, uint64_t dom, int logN) {
    grid_dep_enter();
    const int N = 1 << logN;
    long total = (long)count << logN;
    for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < total; x += (long)gridDim.x * blockDim.x) {
        int l = (int)(x >> logN), k = (int)(x & (N - 1));
        int li = l % nper;
        uint64_t q = mods[map.prime[li]].q;
        uint64_t c = ((uint64_t)map.prime[li] << logN) + k;
        unsigned __int128 w = ((unsigned __int128)rng64(seed, dom, 2 * c) << 64) | rng64(seed, dom, 2 * c + 1);
        out[(long)(l / nper) * so + (long)li * N + k] = (uint64_t)(w % q);
    }
}

// small signed samples: kind 0 = Gaussian from the cumulative table, 1 = ternary {0,0,+1,-1}
__global__ void k_sample_small(int64_t *out, int n, uint64_t seed, uint64_t dom, uint64_t ctr0,
                               const uint64_t *cdt, int cdt_len, int kind) {
    grid_dep_enter();
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        uint64_t r = rng64(seed, dom, ctr0 + k);
        int64_t v;
        if (kind == 0) {
            uint64_t u = r >> 1;
            int mag = 0;
            for (int j = 0; j < cdt_len; j++) mag += u >= cdt[j];
            v = (r & 1) ? -mag : mag;
        } else {
            uint64_t b = r & 3;
            v = b < 2 ? 0 : (b == 2 ? 1 : -1);
        }
        out[k] = v;
    }
}

// secret with exactly h nonzeros: coefficient k is nonzero iff fewer than h pairs
// (draw_j, j) are smaller than (draw_k, k); sign from a second domain
__global__ void k_sample_hwt(int64_t *out, int n, int h, uint64_t seed, uint64_t dom, uint64_t dom_sign) {
    grid_dep_enter();
    extern __shared__ uint64_t keys[];
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t mine = k < n ? rng64(seed, dom, k) : 0;
    int rank = 0;
    for (int base = 0; base < n; base += blockDim.x) {
        int j = base + threadIdx.x;
        keys[threadIdx.x] = j < n ? rng64(seed, dom, j) : ~0ULL;
        __syncthreads();
        int lim = min((int)blockDim.x, n - base);
        for (int jj = 0; jj < lim; jj++) {
            uint64_t o = keys[jj];
            int j2 = base + jj;
            rank += (o < mine) || (o == mine && j2 < k);
        }
        __syncthreads();
    }
    if (k < n) out[k] = rank < h ? ((rng64(seed, dom_sign, k) & 1) ? -1 : 1) : 0;
}

// signed small coefficients into residues for every limb
__global__ void k_small_to_limbs(uint64_t *out, long so, const int64_t *v, int count, int nper, LimbMap map,
                                 const ModC *mods, int logN) {
    grid_dep_enter();
    EW_PROLOGUE
    out[po * so + (long)li * N + k] = reduce_i64(v[k], m);
    }
}

// ------------------------------------------------------------------------------------------
// Canonical embedding: special FFT stages on complex doubles (re, im interleaved).
// Forward (coefficients -> slots) stage of length len on the bit-reversed array,
// inverse stage undoes one forward stage (the 1/2 factors are applied at the end).
// Built with --fmad=false: every double operation is a single IEEE operation, in the
// order the definition writes it.
__global__ void k_bitrev_c(double2 *v, int n0, int logn0) {
    grid_dep_enter();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += gridDim.x * blockDim.x) {
        int j = brev_bits(i, logn0);
        if (i < j) {
            double2 t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    }
}

__global__ void k_sfft_fwd_stage(double2 *v, int n0, int len, const double2 *zeta, const int *rg, int m2n) {
    grid_dep_enter();
    int lenh = len >> 1, lenq = len << 2, gap = m2n / lenq;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < (n0 >> 1); b += gridDim.x * blockDim.x) {
        int i = (b / lenh) * len, j = b % lenh;
        double2 z = zeta[(rg[j] % lenq) * gap];
        double2 u = v[i + j], x = v[i + j + lenh], t;
        t.x = x.x * z.x - x.y * z.y;
        t.y = x.x * z.y + x.y * z.x;
        v[i + j] = make_double2(u.x + t.x, u.y + t.y);
        v[i + j + lenh] = make_double2(u.x - t.x, u.y - t.y);
    }
}

__global__ void k_sfft_inv_stage(double2 *v, int n0, int len, const double2 *zeta, const int *rg, int m2n) {
    grid_dep_enter();
    int lenh = len >> 1, lenq = len << 2, gap = m2n / lenq;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < (n0 >> 1); b += gridDim.x * blockDim.x) {
        int i = (b / lenh) * len, j = b % lenh;
        double2 z = zeta[(lenq - (rg[j] % lenq)) * gap];
        double2 a = v[i + j], c = v[i + j + lenh], s, d, t;
        s.x = a.x + c.x;
        s.y = a.y + c.y;
        d.x = a.x - c.x;
        d.y = a.y - c.y;
        t.x = d.x * z.x - d.y * z.y;
        t.y = d.x * z.y + d.y * z.x;
        v[i + j] = s;
        v[i + j + lenh] = t;
    }
}

__global__ void k_scale_c(double2 *v, int n0, double div) {
    grid_dep_enter();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += gridDim.x * blockDim.x) {
        v[i].x = v[i].x / div;
        v[i].y = v[i].y / div;
    }
}

// nearest integer (ties to even) of a double, as a signed 128-bit value, reduced mod q
__device__ __forceinline__ uint64_t round_reduce(double x, const ModC &m) {
    double r = rint(x);
    if (fabs(r) < 9.2e18) return reduce_i64((int64_t)r, m);
    // |r| >= 2^63: r is an integer m 2^e with a 53-bit m
    unsigned long long bits = (unsigned long long)__double_as_longlong(r);
    int e = (int)((bits >> 52) & 0x7ff) - 1075;
    unsigned long long man = (bits & ((1ULL << 52) - 1)) | (1ULL << 52);
    unsigned __int128 mag = (unsigned __int128)man << e;
    uint64_t v = (uint64_t)(mag % m.q);
    return (bits >> 63) ? neg_mod(v, m.q) : v;
}

// coefficient k of round(scale * t): t_k = Re w_k (k < N0), Im w_{k-N0} (k >= N0)
__global__ void k_round_to_limbs(uint64_t *out, long so, const double2 *w, double scale, int count, int nper,
                                 LimbMap map, const ModC *mods, int logN) {
    grid_dep_enter();
    EW_PROLOGUE
    int n0 = N >> 1;
    double t = k < n0 ? w[k].x : w[k - n0].y;
    out[po * so + (long)li * N + k] = round_reduce(scale * t, m);
    }
}

// Garner: centred value of each coefficient from L residues, as a double divided by scale,
// written as w_k = t_k + i t_{k+N0}.  gc: per level constants [L][L] of (prod_{j<i} q_j mod q_i)
// and inverses; computed on the host.
__global__ void k_crt_to_double(double2 *w, const uint64_t *x, int L, LimbMap qmap, const ModC *mods,
                                const uint64_t *radix, const uint64_t *radinv, const double *qd, double scale, int logN) {
    grid_dep_enter();
    const int N = 1 << logN, n0 = N >> 1;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        uint64_t a[HE_MAX_LIMBS], b[HE_MAX_LIMBS];
        for (int pass = 0; pass < 2; pass++) {
            uint64_t *dg = pass ? b : a;
            for (int i = 0; i < L; i++) {
                const ModC mi = mods[qmap.prime[i]];
                uint64_t xi = x[(long)i * N + k];
                if (pass) xi = neg_mod(xi, mi.q);
                uint64_t acc = 0;
                for (int j = 0; j < i; j++) acc = add_mod(acc, mul_mod(reduce_u64(dg[j], mi), radix[i * HE_MAX_LIMBS + j], mi), mi.q);
                dg[i] = mul_mod(sub_mod(xi, acc, mi.q), radinv[i], mi);
            }
        }
        int neg = 0;
        for (int i = L - 1; i >= 0; i--)
            if (a[i] != b[i]) { neg = a[i] > b[i]; break; }
        const uint64_t *d = neg ? b : a;
        double v = 0.0;
        for (int i = L - 1; i >= 0; i--) v = v * qd[i] + (double)d[i];
        v = (neg ? -v : v) / scale;
        if (k < n0) w[k].x = v;
        else w[k - n0].y = v;
    }
}

// switching-key rows: b = e - a s + [limb in digit] pmod_t s'  (all NTT form, limbs of Q u P)
__global__ void k_key_combine(uint64_t *b, const uint64_t *a, const uint64_t *e, const uint64_t *s, const uint64_t *sp,
                              Scal pm, int nl, int dlo, int dhi, LimbMap map, const ModC *mods, int logN) {
    grid_dep_enter();
    const int N = 1 << logN;
    long total = (long)nl << logN;
    for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < total; x += (long)gridDim.x * blockDim.x) {
        int t = (int)(x >> logN);
        const ModC m = mods[map.prime[t]];
        uint64_t v = sub_mod(e[x], mul_mod(a[x], s[x], m), m.q);
        if (t >= dlo && t < dhi && sp) v = add_mod(v, mul_mod(pm.v[t], sp[x], m), m.q);
        b[x] = v;
    }
}

// x_i mod q_i for `count` limbs of N words (limb l uses modulus map.prime[l % nper]), any uint64
__global__ void k_reduce_limbs(uint64_t *out, const uint64_t *x, int count, int nper, LimbMap map, const ModC *mods,
                               int logN) {
    grid_dep_enter();
    const long N = 1L << logN, total = (long)count << logN;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int l = (int)(i >> logN);
        out[i] = reduce_u64(x[i], mods[map.prime[l % nper]]);
    }
    (void)N;
}

// bounded spin used only by the device-wait self test: waits for *flag != 0 at most max_iter
// polls, then records a timeout in *status (1 = flag seen, 2 = gave up) and returns
__global__ void k_bounded_wait(const volatile int *flag, int *status, long max_iter) {
    grid_dep_enter();
    if (threadIdx.x || blockIdx.x) return;
    for (long i = 0; i < max_iter; i++) {
        if (*flag) { *status = 1; return; }
    }
    *status = 2;
}

// ------------------------------------------------------------------------------------------
// Negacyclic NTT (Cooley-Tukey with merged psi twist; output in bit-reversed order:
// a_hat[k] = a(psi^(2 brv(k) + 1))) and its Gentleman-Sande inverse, for N = 2^12 and 2^16.
// Twiddles per modulus p: N (psi^brv(k), Shoup companion) pairs at tw2 + 2 N p, then the N
// inverse pairs.
// Register-blocked NTT passes.  A pass runs LOGS = 2*LOGE stages on sub-transforms of size
// S = 2^LOGS; each thread holds E = 2^LOGE elements of one sub-transform in registers.
// First LOGE stages: thread lane k holds elements k + E*j (pairs (j, j + 2^p) are its own);
// one exchange through shared memory; last LOGE stages: lane k holds E*k + j.
// "cols" passes act on the N2 columns {c + N2 r} (first log2(N1) stages of the transform),
// "rows" passes on rows of N2 contiguous coefficients (the remaining stages).  The twiddle of
// the butterfly pair (j, j + t) in stage m is psi_rev[m + group] exactly as in the radix-2
// definition, so the result equals the one-stage-at-a-time transform.
template <int LOGE>
__device__ __forceinline__ void ct_stages_strided(uint64_t *v, int m0, int gbase, int gmul, const ulonglong2 *psi,
                                                  uint64_t q) {
    // elements j (index k + E j); stages with half-distance t = E/2, E/4, ..., 1 in units of j
    constexpr int E = 1 << LOGE;
    const uint64_t nq = 0 - q, red = (LOGE % 2 == 0 ? 8 : 4) * q;
#pragma unroll
    for (int p = 0; p < LOGE; p++) {
        const int t = E >> (p + 1);          // distance in j
        const int m = m0 << p;               // stage parameter
#pragma unroll
        for (int b = 0; b < E / 2; b++) {
            // Harvey's lazy butterfly with a 3-product Shoup quotient (x < 4q).  With an even
            // number of stages per half-pass, u is reduced by 8q only in odd stages: stages
            // without the reduction map [0, 12q) to [0, 16q), those with it map [0, 16q) back to
            // [0, 12q); q < 2^60 keeps 16q < 2^64.  Otherwise every stage reduces by 4q and
            // values stay in [0, 8q).
            const int grp = b / t, jj = 2 * grp * t + (b % t);
            const int idx = m + gbase * (1 << p) * gmul + grp;   // m / m0 = 2^p
            const ulonglong2 tw = __ldg(psi + idx);   // (w, w') in one 16-byte load
            uint64_t u = v[jj];
            if ((LOGE % 2 != 0 || (p & 1)) && u >= red) u -= red;
            const uint64_t x = mul_shoup_lazy(v[jj + t], tw.x, tw.y, nq);   // in [0, 4q)
            v[jj] = u + x;
            v[jj + t] = u - x + 4 * q;
        }
    }
}

template <int LOGE>
__device__ __forceinline__ void gs_stages_strided(uint64_t *v, int m0, int gbase, int gmul, const ulonglong2 *ipsi,
                                                  uint64_t q) {
    // inverse of ct_stages_strided: stages in reverse order (t = 1, 2, ..., E/2 in units of j)
    constexpr int E = 1 << LOGE;
    const uint64_t nq = 0 - q;
#pragma unroll
    for (int p = LOGE - 1; p >= 0; p--) {
        const int t = E >> (p + 1);
        const int m = m0 << p;
#pragma unroll
        for (int b = 0; b < E / 2; b++) {
            // lazy Gentleman-Sande butterfly: inputs and outputs in [0, 4q)
            const int grp = b / t, jj = 2 * grp * t + (b % t);
            const int idx = m + gbase * (1 << p) * gmul + grp;   // m / m0 = 2^p
            const ulonglong2 tw = __ldg(ipsi + idx);
            const uint64_t u = v[jj], x = v[jj + t];
            uint64_t s = u + x;
            if (s >= 4 * q) s -= 4 * q;
            const uint64_t d = u - x + 4 * q;
            v[jj] = s;
            v[jj + t] = mul_shoup_lazy(d, tw.x, tw.y, nq);
        }
    }
}

// Fast basis conversion of the E coefficients off + E N2 j (j < E) of one target limb (modulus mt),
// from ns source limbs at s0 + s N (moduli qsrc(s)) whose values already carry the factor
// qhat_s^{-1} mod q_s: v_j = sum_s [y_s]_centred w_s mod m_t with w_s = qhat_s 2^64 mod m_t read at
// w[s wstride].  A centred value y > (q_s - 1) / 2 enters as -(q_s - y), i.e. (q_s - y)(m_t - w_s);
// the sum stays below ns 2^59 m_t < m_t 2^64, so one REDC gives the residue (as in k_modup).
template <int E, class QF>
__device__ __forceinline__ void conv_column(uint64_t *v, const uint64_t *s0, long N, int ns, QF qsrc,
                                            const uint64_t *w, long wstride, const ModC &mt, long off, long step) {
    uint64_t qs[HE_CONV_MAXSRC], ws[HE_CONV_MAXSRC];
#pragma unroll
    for (int s = 0; s < HE_CONV_MAXSRC; s++) {
        if (s >= ns) break;
        qs[s] = qsrc(s);
        ws[s] = __ldg(w + s * wstride);
    }
#pragma unroll
    for (int j = 0; j < E; j++) {
        uint64_t lo = 0, hi = 0;
#pragma unroll
        for (int s = 0; s < HE_CONV_MAXSRC; s++) {
            if (s >= ns) break;
            uint64_t y = s0[s * N + off + j * step], ww = ws[s];
            if (2 * y >= qs[s]) {   // y > (q_s - 1) / 2
                y = qs[s] - y;
                ww = mt.q - ww;
            }
            mac_wide(lo, hi, y, ww);
        }
        v[j] = redc(lo, hi, mt);
    }
}

// Forward column pass: LOGS = log2(N1) stages, m = 1 .. N1/2.  CTA: SUB columns, E*... threads.
template <int LOGE, int KIND, int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 3 : 12) k_ntt_cols_fwd_rb(uint64_t *base, int nper, long poly_stride, LimbMap map,
                                                         const ModC *mods, const ulonglong2 *tw2, int logN,
                                                         const uint64_t *src, long src_stride, NttFuse F) {
    grid_dep_enter();
    constexpr int E = 1 << LOGE, S = E * E, TPS = S / E;   // threads per sub-transform = E
    constexpr int SUB = NT / TPS;                         // columns per CTA
    __shared__ uint64_t sm[S * SUB];
    const int N = 1 << logN, N2 = N / S;
    const int l = blockIdx.y, p = map.prime[l % nper];
    uint64_t *a = base + (long)(l / nper) * poly_stride + (long)(l % nper) * N;
    const uint64_t q = mods[p].q;
    const ulonglong2 *psi = tw2 + (long)p * 2 * N;
    const int c = threadIdx.x % SUB, k = threadIdx.x / SUB, col = blockIdx.x * SUB + c;
    // out of place when src is given: read limb l of src, write base
    const uint64_t *in = src ? src + (long)(l / nper) * src_stride + (long)(l % nper) * N : a;
    uint64_t v[E];
    if (KIND == 7) {
        // ModUp of all digits: the digit's own limbs are already in NTT form (copied by the
        // conversion), the transform leaves them
        const int t = l % nper, dj = F.j0 + (l / nper) % F.ndc;
        if (t >= F.dlo[dj] && t < F.dlo[dj] + F.dds[dj]) return;   // uniform over the CTA
    }
    if (KIND == 2) {
        // rescale: t_i = centred last limb mod q_i
        const ModC mi = mods[p];
        const uint64_t *lp = F.last + (long)(l / nper) * N;
#pragma unroll
        for (int j = 0; j < E; j++) {
            const uint64_t r = lp[(long)(k + E * j) * N2 + col];
            v[j] = r <= (F.ql - 1) / 2 ? mul_mod(r, 1, mi) : neg_mod(mul_mod(F.ql - r, 1, mi), mi.q);
        }
    } else if (KIND == 4) {
        // ModUp: polynomial l / nper is digit j of ciphertext c; limb t of the extended basis
        const int poly = l / nper, t = l % nper, dj = F.j0 + poly % F.ndc, ci = poly / F.ndc;
        const int lo = F.dlo[dj], ds = F.dds[dj];
        if (t >= lo && t < lo + ds) {
            // the digit's own limb: the NTT-form input itself (the row pass leaves this limb)
            const uint64_t *xi = F.xntt + (long)ci * F.sxn + (long)t * N;
#pragma unroll
            for (int j = 0; j < E; j++) a[(long)(k + E * j) * N2 + col] = xi[(long)(k + E * j) * N2 + col];
            return;   // uniform over the CTA: no barrier is skipped by part of it
        }
        conv_column<E>(v, F.src + (long)ci * F.sstride + (long)lo * N, N, ds,
                       [&](int s) { return mods[lo + s].q; }, F.cvw + F.dcv[dj] + t, F.wstride, mods[p],
                       (long)k * N2 + col, (long)E * N2);
    } else if (KIND == 5 || KIND == 6) {
        // ModDown: conv of limb i of polynomial l / nper from the dropped limbs of that polynomial
        conv_column<E>(v, F.src + (long)(l / nper) * F.sstride + (long)F.slo * N, N, F.ns,
                       [&](int s) { return mods[F.sidx[s]].q; }, F.cvw + p, F.wstride, mods[p],
                       (long)k * N2 + col, (long)E * N2);
    } else {
#pragma unroll
        for (int j = 0; j < E; j++) v[j] = in[(long)(k + E * j) * N2 + col];
    }
    // stages m = 1 .. E/2: element index r = k + E j, group = j / (2t) (independent of k)
    ct_stages_strided<LOGE>(v, 1, 0, 0, psi, q);
#pragma unroll
    for (int j = 0; j < E; j++) sm[(k + E * j) * SUB + c] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; j++) v[j] = sm[(E * k + j) * SUB + c];
    // stages m = E .. S/2 on r = E k + j: group = (E k + j) / (2t) = k * (m / E) + j / (2t)
    ct_stages_strided<LOGE>(v, E, k, 1, psi, q);
#pragma unroll
    for (int j = 0; j < E; j++) a[(long)(E * k + j) * N2 + col] = v[j];
}

// Forward row pass: stages m = N1 .. N/2 on rows of S = N2 contiguous coefficients.
template <int LOGE, int KIND, int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 3 : 12) k_ntt_rows_fwd_rb(uint64_t *base, int nper, long poly_stride, LimbMap map,
                                                         const ModC *mods, const ulonglong2 *tw2, int logN,
                                                         NttFuse F) {
    grid_dep_enter();
    constexpr int E = 1 << LOGE, S = E * E, TPS = E;
    constexpr int SUB = NT / TPS;                         // rows per CTA
    // one pad word per E: the E k + j accesses (stride E words) spread over all banks
    constexpr int SP = S + S / E;
    __shared__ uint64_t sm[SP * SUB];
    const int N = 1 << logN, N1 = N / S;
    const int l = blockIdx.y, p = map.prime[l % nper];
    uint64_t *a = base + (long)(l / nper) * poly_stride + (long)(l % nper) * N;
    const uint64_t q = mods[p].q;
    const ulonglong2 *psi = tw2 + (long)p * 2 * N;
    const int k = threadIdx.x % TPS, rr = threadIdx.x / TPS, row = blockIdx.x * SUB + rr;
    if (KIND == 4 || KIND == 7) {   // ModUp: the digit's own limbs are in NTT form already
        const int t = l % nper, dj = F.j0 + (l / nper) % F.ndc;
        if (t >= F.dlo[dj] && t < F.dlo[dj] + F.dds[dj]) return;   // uniform over the CTA
    }
    uint64_t *g = a + (long)row * S;
    uint64_t v[E];
#pragma unroll
    for (int j = 0; j < E; j++) v[j] = g[k + E * j];
    // stages m = N1 .. N1 E/2: group = row (m / N1) + j / (2t)
    ct_stages_strided<LOGE>(v, N1, row, 1, psi, q);
#pragma unroll
    for (int j = 0; j < E; j++) sm[rr * SP + k + (E + 1) * j] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; j++) v[j] = sm[rr * SP + (E + 1) * k + j];
    // stages m = N1 E .. N/2: group = row (m / N1) + k (m / (N1 E)) + j / (2t)
    ct_stages_strided<LOGE>(v, N1 * E, row * E + k, 1, psi, q);
    // back to the k + E j layout through shared memory so the store is coalesced; the lazy
    // butterflies left values r < 16q < 2^(s+4) (s = bit length of q): reduce to [0, q) with a
    // small-quotient Barrett step.  With t = floor(r / 2^(s-6)) < 2^10 and
    // mu6 = floor(2^(s+6) / q) = floor(mu / 2^57), k = floor(t mu6 / 2^12) underestimates r / q
    // by less than 2^(10-12) + 2^(s-6) / q < 1, so r - k q lies in [0, 2q).
    const uint32_t mu6 = (uint32_t)(mods[p].mu >> 57);
    const int sh = mods[p].s - 6;
    const uint64_t nq = 0 - q;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; j++) {
        const uint32_t kq = ((uint32_t)(v[j] >> sh) * mu6) >> 12;
        uint64_t r = v[j] + (uint64_t)kq * nq;   // v - kq q
        if (r >= q) r -= q;
        sm[rr * SP + (E + 1) * k + j] = r;
    }
    __syncthreads();
    if (KIND == 0 || KIND == 4 || KIND == 7) {
#pragma unroll
        for (int j = 0; j < E; j++) g[k + E * j] = sm[rr * SP + k + (E + 1) * j];
        return;
    }
    // fused epilogue (ModDown or rescale): out from x and the transformed values
    const int pl = l / nper, i = l % nper;
    const long at = (long)i * N + (long)row * S + k;
    if (KIND == 1 || KIND == 5) {
        const uint64_t w = F.cst[2 * p], wp = F.cst[2 * p + 1];
        const uint64_t *xp = F.x + (long)pl * (nper + F.alpha) * N + at;
        const long o = (long)(pl / 2) * F.so + (long)(pl % 2) * nper * N + at;
        const long oa = (long)(pl / 2) * F.sadd + (long)(pl % 2) * nper * N + at;
#pragma unroll
        for (int j = 0; j < E; j++) {
            uint64_t r = mul_shoup(sub_mod(xp[E * j], sm[rr * SP + k + (E + 1) * j], q), w, wp, q);
            if (F.add) r = add_mod(F.add[oa + E * j], r, q);
            F.out[o + E * j] = r;
        }
    } else if (KIND == 2) {
        const uint64_t w = F.cst[2 * i], wp = F.cst[2 * i + 1];
        const uint64_t *xp = F.x + (long)pl * (nper + 1) * N + at;
        uint64_t *op = F.out + (long)pl * nper * N + at;
#pragma unroll
        for (int j = 0; j < E; j++) op[E * j] = mul_shoup(sub_mod(xp[E * j], sm[rr * SP + k + (E + 1) * j], q), w, wp, q);
    } else {
        const uint64_t pm = F.cst[4 * i], pmp = F.cst[4 * i + 1], w = F.cst[4 * i + 2], wp = F.cst[4 * i + 3];
        const uint64_t *kp = F.x + (long)pl * (nper + F.alpha) * N + at;
        const uint64_t *dp = F.add + (long)(pl / 2) * F.sadd + (long)(pl % 2) * (nper + 1) * N + at;
        uint64_t *op = F.out + (long)(pl / 2) * F.so + (long)(pl % 2) * nper * N + at;
#pragma unroll
        for (int j = 0; j < E; j++) {
            const uint64_t y = add_mod(mul_shoup(dp[E * j], pm, pmp, q), kp[E * j], q);
            op[E * j] = mul_shoup(sub_mod(y, sm[rr * SP + k + (E + 1) * j], q), w, wp, q);
        }
    }
}

// Inverse row pass: stages h = N/2 .. N1 (t = 1 .. N2/2).
template <int LOGE, int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 3 : 12) k_ntt_rows_inv_rb(uint64_t *base, int nper, long poly_stride, LimbMap map,
                                                         const ModC *mods, const ulonglong2 *tw2, int logN,
                                                         const uint64_t *src, long src_stride) {
    grid_dep_enter();
    constexpr int E = 1 << LOGE, S = E * E, TPS = E;
    constexpr int SUB = NT / TPS;
    // one pad word per E: the E k + j accesses (stride E words) spread over all banks
    constexpr int SP = S + S / E;
    __shared__ uint64_t sm[SP * SUB];
    const int N = 1 << logN, N1 = N / S;
    const int l = blockIdx.y, p = map.prime[l % nper];
    uint64_t *a = base + (long)(l / nper) * poly_stride + (long)(l % nper) * N;
    const uint64_t q = mods[p].q;
    const ulonglong2 *ipsi = tw2 + (long)p * 2 * N + N;
    const int k = threadIdx.x % TPS, rr = threadIdx.x / TPS, row = blockIdx.x * SUB + rr;
    uint64_t *g = a + (long)row * S;
    // out of place when src is given: read limb l of src, write base
    const uint64_t *gi = (src ? src + (long)(l / nper) * src_stride + (long)(l % nper) * N : a) + (long)row * S;
    uint64_t v[E];
    // coalesced load, then regroup to the E k + j layout through shared memory
#pragma unroll
    for (int j = 0; j < E; j++) sm[rr * SP + k + (E + 1) * j] = gi[k + E * j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; j++) v[j] = sm[rr * SP + (E + 1) * k + j];
    __syncthreads();
    gs_stages_strided<LOGE>(v, N1 * E, row * E + k, 1, ipsi, q);
#pragma unroll
    for (int j = 0; j < E; j++) sm[rr * SP + (E + 1) * k + j] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; j++) v[j] = sm[rr * SP + k + (E + 1) * j];
    gs_stages_strided<LOGE>(v, N1, row, 1, ipsi, q);
#pragma unroll
    for (int j = 0; j < E; j++) g[k + E * j] = v[j];
}

// Inverse column pass: stages h = N1/2 .. 1, then the N^{-1} factor.
template <int LOGE, int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 3 : 12) k_ntt_cols_inv_rb(uint64_t *base, int nper, long poly_stride, LimbMap map,
                                                         const ModC *mods, const ulonglong2 *tw2, const uint64_t *ninv,
                                                         int logN) {
    grid_dep_enter();
    constexpr int E = 1 << LOGE, S = E * E, TPS = E;
    constexpr int SUB = NT / TPS;
    __shared__ uint64_t sm[S * SUB];
    const int N = 1 << logN, N2 = N / S;
    const int l = blockIdx.y, p = map.prime[l % nper];
    uint64_t *a = base + (long)(l / nper) * poly_stride + (long)(l % nper) * N;
    const uint64_t q = mods[p].q;
    const ulonglong2 *ipsi = tw2 + (long)p * 2 * N + N;
    const int c = threadIdx.x % SUB, k = threadIdx.x / SUB, col = blockIdx.x * SUB + c;
    uint64_t v[E];
#pragma unroll
    for (int j = 0; j < E; j++) v[j] = a[(long)(E * k + j) * N2 + col];
    gs_stages_strided<LOGE>(v, E, k, 1, ipsi, q);
#pragma unroll
    for (int j = 0; j < E; j++) sm[(E * k + j) * SUB + c] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; j++) v[j] = sm[(k + E * j) * SUB + c];
    gs_stages_strided<LOGE>(v, 1, 0, 0, ipsi, q);
    const uint64_t ni = ninv[2 * p], nip = ninv[2 * p + 1];
#pragma unroll
    for (int j = 0; j < E; j++) a[(long)(k + E * j) * N2 + col] = mul_shoup(v[j], ni, nip, q);
}

// NT threads per CTA: 256 (16 sub-transforms per CTA at N = 2^16), or 64 for transforms of few
// limbs, whose 256-thread grids leave SMs idle (four times as many, smaller CTAs)
template <int LOGE, int NT>
static void launch_rb(bool inverse, int count, uint64_t *base, int nper, long poly_stride, const LimbMap &map,
                      const ModC *mods, const ulonglong2 *tw2, const uint64_t *ninv, int logN, cudaStream_t st,
                      const uint64_t *src, long src_stride, const NttFuse &F) {
    constexpr int E = 1 << LOGE, S = E * E, SUB = NT / E;
    dim3 g(((1 << logN) / S) / SUB, count);
#define HE_FWD_KIND(KD)                                                                                        \
    if (!inverse && F.kind == KD) {                                                                            \
        klaunch(k_ntt_cols_fwd_rb<LOGE, KD, NT>, g, NT, 0, st)(base, nper, poly_stride, map, mods, tw2, logN, src, src_stride, F); \
        klaunch(k_ntt_rows_fwd_rb<LOGE, KD, NT>, g, NT, 0, st)(base, nper, poly_stride, map, mods, tw2, logN, F); \
        return;                                                                                                \
    }
    HE_FWD_KIND(4)
    HE_FWD_KIND(5)
    HE_FWD_KIND(6)
    HE_FWD_KIND(7)
#undef HE_FWD_KIND
    if (!inverse && F.kind == 1) {
        klaunch(k_ntt_cols_fwd_rb<LOGE, 1, NT>, g, NT, 0, st)(base, nper, poly_stride, map, mods, tw2, logN, src, src_stride, F);
        klaunch(k_ntt_rows_fwd_rb<LOGE, 1, NT>, g, NT, 0, st)(base, nper, poly_stride, map, mods, tw2, logN, F);
    } else if (!inverse && F.kind == 3) {
        klaunch(k_ntt_cols_fwd_rb<LOGE, 3, NT>, g, NT, 0, st)(base, nper, poly_stride, map, mods, tw2, logN, src, src_stride, F);
        klaunch(k_ntt_rows_fwd_rb<LOGE, 3, NT>, g, NT, 0, st)(base, nper, poly_stride, map, mods, tw2, logN, F);
    } else if (!inverse && F.kind == 2) {
        klaunch(k_ntt_cols_fwd_rb<LOGE, 2, NT>, g, NT, 0, st)(base, nper, poly_stride, map, mods, tw2, logN, src, src_stride, F);
        klaunch(k_ntt_rows_fwd_rb<LOGE, 2, NT>, g, NT, 0, st)(base, nper, poly_stride, map, mods, tw2, logN, F);
    } else if (!inverse) {
        klaunch(k_ntt_cols_fwd_rb<LOGE, 0, NT>, g, NT, 0, st)(base, nper, poly_stride, map, mods, tw2, logN, src, src_stride, F);
        klaunch(k_ntt_rows_fwd_rb<LOGE, 0, NT>, g, NT, 0, st)(base, nper, poly_stride, map, mods, tw2, logN, F);
    } else {
        klaunch(k_ntt_rows_inv_rb<LOGE, NT>, g, NT, 0, st)(base, nper, poly_stride, map, mods, tw2, logN, src, src_stride);
        klaunch(k_ntt_cols_inv_rb<LOGE, NT>, g, NT, 0, st)(base, nper, poly_stride, map, mods, tw2, ninv, logN);
    }
}

void launch_ntt_rb(int logE, bool inverse, int count, uint64_t *base, int nper, long poly_stride, const LimbMap &map,
                   const ModC *mods, const ulonglong2 *tw2, const uint64_t *ninv, int logN, cudaStream_t st,
                   const uint64_t *src, long src_stride, const NttFuse *fuse, bool small_cta) {
    NttFuse F{};
    if (fuse) F = *fuse;
    if (logE == 4) {
        if (small_cta) launch_rb<4, 64>(inverse, count, base, nper, poly_stride, map, mods, tw2, ninv, logN, st, src, src_stride, F);
        else launch_rb<4, 256>(inverse, count, base, nper, poly_stride, map, mods, tw2, ninv, logN, st, src, src_stride, F);
    } else {
        if (small_cta) launch_rb<3, 64>(inverse, count, base, nper, poly_stride, map, mods, tw2, ninv, logN, st, src, src_stride, F);
        else launch_rb<3, 256>(inverse, count, base, nper, poly_stride, map, mods, tw2, ninv, logN, st, src, src_stride, F);
    }
}

// ------------------------------------------------------------------------------------------
// One-pass transforms of N = 2^16 limbs: one thread-block cluster of CL = 4096 / NT CTAs of NT
// threads per limb (NT = 256: 16 CTAs, a non-portable cluster size).  CTA q of the cluster runs
// the column pass on columns SUB q .. SUB q + SUB - 1 and the row pass on rows SUB q .. SUB q +
// SUB - 1, SUB = NT / 16 (the two passes of the register-blocked transform above, same
// butterflies and twiddles); the column pass's output goes to the row owners' shared memory
// through distributed shared memory instead of HBM.  One launch and one read and one write of
// the limb in HBM, instead of two of each.  The cluster barriers are reached by every thread of
// every CTA (one limb per cluster, no early exit).
namespace cg = cooperative_groups;

#define HE_1P_NT 256
#define HE_1P_SUB (HE_1P_NT / 16)
#define HE_1P_CL (256 / HE_1P_SUB)
#define HE_1P_RS (256 + 8)            // forward: row stride (words) of the received rows
#define HE_1P_CS (HE_1P_SUB + 2)      // inverse: row stride (words) of the received columns
// shared memory: transposes (SP * SUB words, SP = 272 >= S) and the exchange buffer
// (max(SUB * RS, 256 * CS) words); three CTAs per SM
#define HE_1P_T_WORDS (272 * HE_1P_SUB)
#define HE_1P_X_WORDS (HE_1P_SUB * HE_1P_RS > 256 * HE_1P_CS ? HE_1P_SUB * HE_1P_RS : 256 * HE_1P_CS)
#define HE_1P_SMEM ((HE_1P_T_WORDS + HE_1P_X_WORDS) * 8)

__global__ void __cluster_dims__(HE_1P_CL, 1, 1) __launch_bounds__(HE_1P_NT, 3)
    k_ntt_fwd_1pass(uint64_t *base, int nper, long poly_stride, LimbMap map, const ModC *mods, const ulonglong2 *tw2,
                    int logN, const uint64_t *src, long src_stride) {
    grid_dep_enter();
    constexpr int LOGE = 4, E = 16, S = 256, SUB = HE_1P_NT / E, SP = S + S / E;
    extern __shared__ uint64_t dsm[];
    uint64_t *T = dsm, *RB = dsm + HE_1P_T_WORDS;
    cg::cluster_group cl = cg::this_cluster();
    const int q = (int)cl.block_rank();
    const int N = 1 << logN, N2 = N / S, N1 = N / S;
    const int l = blockIdx.y, p = map.prime[l % nper];
    uint64_t *a = base + (long)(l / nper) * poly_stride + (long)(l % nper) * N;
    const uint64_t *in = src ? src + (long)(l / nper) * src_stride + (long)(l % nper) * N : a;
    const uint64_t mq = mods[p].q;
    const ulonglong2 *psi = tw2 + (long)p * 2 * N;
    uint64_t v[E];
    {   // column pass (stages m = 1 .. N1/2) on columns SUB q + c
        const int c = threadIdx.x % SUB, k = threadIdx.x / SUB, col = q * SUB + c;
#pragma unroll
        for (int j = 0; j < E; j++) v[j] = in[(long)(k + E * j) * N2 + col];
        ct_stages_strided<LOGE>(v, 1, 0, 0, psi, mq);
#pragma unroll
        for (int j = 0; j < E; j++) T[(k + E * j) * SUB + c] = v[j];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < E; j++) v[j] = T[(E * k + j) * SUB + c];
        ct_stages_strided<LOGE>(v, E, k, 1, psi, mq);
        // element of row r = E k + j goes to the row owner r / SUB (the same CTA for all j)
        cl.sync();   // every CTA of the cluster runs and has finished reading T
        const int r0 = E * k;
        uint64_t *dst = cl.map_shared_rank(RB, r0 / SUB);
#pragma unroll
        for (int j = 0; j < E; j++) dst[((r0 + j) % SUB) * HE_1P_RS + col] = v[j];
        cl.sync();   // every row of this CTA has arrived
    }
    {   // row pass (stages m = N1 .. N/2) on rows SUB q + rr
        const int k = threadIdx.x % E, rr = threadIdx.x / E, row = q * SUB + rr;
#pragma unroll
        for (int j = 0; j < E; j++) v[j] = RB[rr * HE_1P_RS + k + E * j];
        ct_stages_strided<LOGE>(v, N1, row, 1, psi, mq);
#pragma unroll
        for (int j = 0; j < E; j++) T[rr * SP + k + (E + 1) * j] = v[j];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < E; j++) v[j] = T[rr * SP + (E + 1) * k + j];
        ct_stages_strided<LOGE>(v, N1 * E, row * E + k, 1, psi, mq);
        // final reduction to [0, q) as in k_ntt_rows_fwd_rb
        const uint32_t mu6 = (uint32_t)(mods[p].mu >> 57);
        const int sh = mods[p].s - 6;
        const uint64_t nq = 0 - mq;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < E; j++) {
            const uint32_t kq = ((uint32_t)(v[j] >> sh) * mu6) >> 12;
            uint64_t r = v[j] + (uint64_t)kq * nq;
            if (r >= mq) r -= mq;
            T[rr * SP + (E + 1) * k + j] = r;
        }
        __syncthreads();
        uint64_t *g = a + (long)row * S;
#pragma unroll
        for (int j = 0; j < E; j++) g[k + E * j] = T[rr * SP + k + (E + 1) * j];
    }
}

__global__ void __cluster_dims__(HE_1P_CL, 1, 1) __launch_bounds__(HE_1P_NT, 3)
    k_ntt_inv_1pass(uint64_t *base, int nper, long poly_stride, LimbMap map, const ModC *mods, const ulonglong2 *tw2,
                    const uint64_t *ninv, int logN, const uint64_t *src, long src_stride) {
    grid_dep_enter();
    constexpr int LOGE = 4, E = 16, S = 256, SUB = HE_1P_NT / E, SP = S + S / E;
    extern __shared__ uint64_t dsm[];
    uint64_t *T = dsm, *CB = dsm + HE_1P_T_WORDS;
    cg::cluster_group cl = cg::this_cluster();
    const int q = (int)cl.block_rank();
    const int N = 1 << logN, N2 = N / S, N1 = N / S;
    const int l = blockIdx.y, p = map.prime[l % nper];
    uint64_t *a = base + (long)(l / nper) * poly_stride + (long)(l % nper) * N;
    const uint64_t *in = src ? src + (long)(l / nper) * src_stride + (long)(l % nper) * N : a;
    const uint64_t mq = mods[p].q;
    const ulonglong2 *ipsi = tw2 + (long)p * 2 * N + N;
    uint64_t v[E];
    {   // row pass (stages h = N/2 .. N1) on rows SUB q + rr
        const int k = threadIdx.x % E, rr = threadIdx.x / E, row = q * SUB + rr;
        const uint64_t *gi = in + (long)row * S;
#pragma unroll
        for (int j = 0; j < E; j++) T[rr * SP + k + (E + 1) * j] = gi[k + E * j];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < E; j++) v[j] = T[rr * SP + (E + 1) * k + j];
        __syncthreads();
        gs_stages_strided<LOGE>(v, N1 * E, row * E + k, 1, ipsi, mq);
#pragma unroll
        for (int j = 0; j < E; j++) T[rr * SP + (E + 1) * k + j] = v[j];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < E; j++) v[j] = T[rr * SP + k + (E + 1) * j];
        gs_stages_strided<LOGE>(v, N1, row, 1, ipsi, mq);
        // element of column col = k + E j goes to the column owner col / SUB
        cl.sync();   // every CTA of the cluster runs and has finished reading T
#pragma unroll
        for (int j = 0; j < E; j++) {
            const int col = k + E * j;
            uint64_t *dst = cl.map_shared_rank(CB, col / SUB);
            dst[row * HE_1P_CS + col % SUB] = v[j];
        }
        cl.sync();   // every column of this CTA has arrived
    }
    {   // column pass (stages h = N1/2 .. 1), then the N^{-1} factor, on columns SUB q + c
        const int c = threadIdx.x % SUB, k = threadIdx.x / SUB, col = q * SUB + c;
#pragma unroll
        for (int j = 0; j < E; j++) v[j] = CB[(E * k + j) * HE_1P_CS + c];
        gs_stages_strided<LOGE>(v, E, k, 1, ipsi, mq);
#pragma unroll
        for (int j = 0; j < E; j++) T[(E * k + j) * SUB + c] = v[j];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < E; j++) v[j] = T[(k + E * j) * SUB + c];
        gs_stages_strided<LOGE>(v, 1, 0, 0, ipsi, mq);
        const uint64_t ni = ninv[2 * p], nip = ninv[2 * p + 1];
#pragma unroll
        for (int j = 0; j < E; j++) a[(long)(k + E * j) * N2 + col] = mul_shoup(v[j], ni, nip, mq);
    }
}

int ntt_1pass_setup() {
    if (cudaFuncSetAttribute(k_ntt_fwd_1pass, cudaFuncAttributeMaxDynamicSharedMemorySize, HE_1P_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(k_ntt_inv_1pass, cudaFuncAttributeMaxDynamicSharedMemorySize, HE_1P_SMEM) != cudaSuccess)
        return -1;
    if (HE_1P_CL > 8 &&
        (cudaFuncSetAttribute(k_ntt_fwd_1pass, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
         cudaFuncSetAttribute(k_ntt_inv_1pass, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess))
        return -1;
    return 0;
}

void launch_ntt_1pass(bool inverse, int count, uint64_t *base, int nper, long poly_stride, const LimbMap &map,
                      const ModC *mods, const ulonglong2 *tw2, const uint64_t *ninv, int logN, cudaStream_t st,
                      const uint64_t *src, long src_stride) {
    dim3 g(HE_1P_CL, count);
    if (inverse)
        klaunch(k_ntt_inv_1pass, g, HE_1P_NT, HE_1P_SMEM, st)(base, nper, poly_stride, map, mods, tw2, ninv, logN, src,
                                                          src_stride);
    else
        klaunch(k_ntt_fwd_1pass, g, HE_1P_NT, HE_1P_SMEM, st)(base, nper, poly_stride, map, mods, tw2, logN, src,
                                                          src_stride);
}
