// Device-side building blocks for the RNS-CKKS kernels (sm_103a).
//
// Residues are uint64 in [0, q) with q < 2^60 (NTT-friendly primes q = 1 mod 2N).
//  - mul_mod   : Barrett reduction of the 128-bit product with mu = floor(2^(s+63) / q),
//                s = bitlen(q): the quotient estimate is at most 2 below the true one.
//  - mul_shoup : Shoup's multiplication by a fixed w with w' = floor(w 2^64 / q);
//                mul_shoup_lazy leaves the product in [0, 4q) for the NTT butterflies.
//  - mac_wide / redc : sums of products kept as 128-bit integers and reduced once by
//                Montgomery's REDC (R = 2^64): redc(T) = T R^{-1} mod q for T < q 2^64, so
//                a sum of products whose constant factors are stored as c R mod q comes out
//                as the exact sum mod q.
// Limb maps describe a batch of polynomials stored as [poly][limb][N]: limb l of the batch
// uses modulus index prime[l % nper].
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define HE_MAX_LIMBS 64
#define HE_CONV_MAXSRC 9   // basis conversions: at most alpha + 1 source moduli (alpha <= 8)
#define HE_MAX_MODS 64

struct ModC {
    uint64_t q;
    uint64_t mu;   // floor(2^(s+63) / q)
    uint64_t qinv; // -q^{-1} mod 2^64
    int s;         // bit length of q
    int pad;
};

struct LimbMap {
    int nper;                       // limbs per polynomial
    int prime[HE_MAX_LIMBS];        // modulus index of limb i of each polynomial
};

// Programmatic dependent launch.  Every kernel of the library starts with grid_dep_enter():
// it waits until the grid it follows in its stream has completed and its writes are visible
// (griddepcontrol.wait; a no-op when the launch carries no programmatic dependency), and only
// then lets the next kernel of the stream be scheduled (griddepcontrol.launch_dependents).
// No kernel touches memory before the wait, so every launch sees the same memory as in plain
// stream order; the next grid's launch and the first CTAs it places on SMs that this grid's
// last wave has left overlap the end of this grid.
__device__ __forceinline__ void grid_dep_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ uint64_t he_mulhi(uint64_t a, uint64_t b) {
    return (uint64_t)__umul64hi((unsigned long long)a, (unsigned long long)b);
}

__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q) {
    uint64_t c = a + b;
    return c >= q ? c - q : c;
}

__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q) {
    return a >= b ? a - b : a + q - b;
}

__device__ __forceinline__ uint64_t neg_mod(uint64_t a, uint64_t q) { return a ? q - a : 0; }

__device__ __forceinline__ uint64_t mul_shoup(uint64_t a, uint64_t w, uint64_t wp, uint64_t q) {
    uint64_t h = he_mulhi(a, wp);
    uint64_t r = a * w - h * q;
    return r >= q ? r - q : r;
}

// a w mod q in [0, 4q), for any a < 2^64, with nq = 2^64 - q.  The Shoup quotient
// floor(a w' / 2^64) is estimated from three of the four 32x32 partial products: dropping
// a0 w'0 and the low halves of a0 w'1 and a1 w'0 loses less than 3 * 2^32 of a w', so the
// estimate is at most 2 below the exact quotient and a w - h q < 2q + 2q.  The low word
// a w + h nq = a w - h q is exact mod 2^64 because the true value is below 4q < 2^63.
// Written as 32-bit multiply-adds only: with h = H + t2, H = a1 w'1 + hi(a0 w'1) (exact in
// 64 bits) and t2 = hi(a1 w'0), h nq = H nq + t2 nq, so no 64-bit addition is needed.  The
// 64-bit sums are explicit carry chains (mad.lo.cc / madc.hi), which the compiler otherwise
// lowers with separate adds.
__device__ __forceinline__ uint64_t mul_shoup_lazy(uint64_t a, uint64_t w, uint64_t wp, uint64_t nq) {
    uint32_t a0, a1, p0, p1, w0, w1, n0, n1, r0, r1;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(a0), "=r"(a1) : "l"(a));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(p0), "=r"(p1) : "l"(wp));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(w0), "=r"(w1) : "l"(w));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(n0), "=r"(n1) : "l"(nq));
    asm("{\n\t.reg .u32 t, t2, h0, h1;\n\t"
        "mul.hi.u32 t, %2, %5;\n\t"            // hi(a0 w'1)
        "mul.hi.u32 t2, %3, %4;\n\t"           // t2 = hi(a1 w'0)
        "mad.lo.cc.u32 h0, %3, %5, t;\n\t"     // H = a1 w'1 + hi(a0 w'1)
        "madc.hi.u32 h1, %3, %5, 0;\n\t"
        "mul.lo.u32 %0, %2, %6;\n\t"           // acc = a0 w0 + h0 n0 + t2 n0 (mod 2^64)
        "mul.hi.u32 %1, %2, %6;\n\t"
        "mad.lo.cc.u32 %0, h0, %8, %0;\n\t"
        "madc.hi.u32 %1, h0, %8, %1;\n\t"
        "mad.lo.cc.u32 %0, t2, %8, %0;\n\t"
        "madc.hi.u32 %1, t2, %8, %1;\n\t"
        "mad.lo.u32 %1, %2, %7, %1;\n\t"       // high word: + a0 w1 + a1 w0 + h0 n1 + h1 n0 + t2 n1
        "mad.lo.u32 %1, %3, %6, %1;\n\t"
        "mad.lo.u32 %1, h0, %9, %1;\n\t"
        "mad.lo.u32 %1, h1, %8, %1;\n\t"
        "mad.lo.u32 %1, t2, %9, %1;\n\t}"
        : "=&r"(r0), "=&r"(r1)
        : "r"(a0), "r"(a1), "r"(p0), "r"(p1), "r"(w0), "r"(w1), "r"(n0), "r"(n1));
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(r0), "r"(r1));
    return r;
}

// valid for a < 2^62 and b < q (the quotient estimate stays within 2 of the true one)
__device__ __forceinline__ uint64_t mul_mod(uint64_t a, uint64_t b, const ModC &m) {
    uint64_t lo = a * b, hi = he_mulhi(a, b);
    uint64_t x1 = (lo >> (m.s - 2)) | (hi << (66 - m.s));
    uint64_t qe = he_mulhi(x1, m.mu) >> 1;
    uint64_t r = lo - qe * m.q;
    if (r >= m.q) r -= m.q;
    if (r >= m.q) r -= m.q;
    return r;
}

// (hi:lo) += a b as one 128-bit integer
__device__ __forceinline__ void mac_wide(uint64_t &lo, uint64_t &hi, uint64_t a, uint64_t b) {
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\tmadc.hi.u64 %1, %2, %3, %1;" : "+l"(lo), "+l"(hi) : "l"(a), "l"(b));
}

// Montgomery reduction of T = (hi:lo) < q 2^64: returns T 2^{-64} mod q in [0, q).
// u = lo (-q^{-1}) makes T + u q divisible by 2^64; its low word is 0 and carries out
// exactly when lo != 0; the quotient is below 2q.
__device__ __forceinline__ uint64_t redc(uint64_t lo, uint64_t hi, const ModC &m) {
    uint64_t u = lo * m.qinv;
    uint64_t t = hi + he_mulhi(u, m.q) + (lo != 0);
    return t >= m.q ? t - m.q : t;
}

// x (any uint64) mod q
__device__ __forceinline__ uint64_t reduce_u64(uint64_t x, const ModC &m) {
    return x >= m.q ? x % m.q : x;
}

// signed 64-bit value mod q
__device__ __forceinline__ uint64_t reduce_i64(int64_t x, const ModC &m) {
    if (x >= 0) return reduce_u64((uint64_t)x, m);
    uint64_t r = reduce_u64((uint64_t)(-(x + 1)), m);   // -(x+1) >= 0
    // x = -(r' + 1) with r' = -(x+1); x mod q = q - 1 - (r' mod q)
    return m.q - 1 - r;
}

__device__ __forceinline__ int brev_bits(int x, int bits) { return (int)(__brev((unsigned)x) >> (32 - bits)); }

#define HE_CHECK_LAUNCH() (cudaGetLastError())
