// common.cuh -- shared types and 64-bit modular arithmetic for the GB300
// (sm_103a) RNS-CKKS kernels.
//
// Words are u64.  Every modulus is a prime q = 1 + q1 * 2^32 below 2^61
// (q1 < 2^29).  sm_103a multiplies 32 x 32 bits natively, so a 64-bit product
// costs up to four 32-bit multiplies; with this form the product h * q mod 2^64
// that every reduction subtracts is h + ((h mod 2^32) * q1 mod 2^32) * 2^32, one
// 32-bit multiply, and q^{-1} mod 2^64 = 1 - q1 * 2^32.  Three reductions are used:
//  * Shoup:  x * w mod q for a fixed w with w' = floor(w * 2^64 / q); the lazy
//            form returns a value in [0, 2q) for any x < 2^64 (NTT butterflies,
//            multiplication by constants).
//  * Montgomery REDC: (hi:lo) * 2^-64 mod q for (hi:lo) < q * 2^64; used with one
//            operand pre-multiplied by 2^64 (keys, plaintexts, base-conversion
//            constants) so that sums of up to 7 products reduce once.
//  * Barrett: a * b mod q for two variable residues (ciphertext products),
//            mu = floor(2^(2k) / q), k = bit length of q.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

typedef uint64_t u64;
typedef unsigned __int128 u128;

#define HETAL_MAX_MODULI 128

// Per-modulus constants (device and host copies).
struct ModConst {
    u64 q;        // 1 + q1 * 2^32
    u64 r2;       // 2^128 mod q
    u64 mu;       // floor(2^(2k) / q) (Barrett)
    int k;        // bit length of q
    int pad;
};

// Map from the limbs of a launch to modulus indices (passed by value).
struct LimbMap {
    int n;
    unsigned char idx[HETAL_MAX_MODULI];
};

// x >= m ? x - m : x for x, m < 2^63 (the sign of x - m decides).
__device__ __forceinline__ u64 csub(u64 x, u64 m)
{
    u64 d = x - m;
    return (long long)d < 0 ? x : d;
}

// h * q mod 2^64 for q = 1 + q1 * 2^32.
__device__ __forceinline__ u64 mul_q_lo(u64 h, u64 q)
{
    return h + ((u64)((uint32_t)h * (uint32_t)(q >> 32)) << 32);
}

__device__ __forceinline__ u64 mul_shoup_lazy(u64 x, u64 w, u64 wp, u64 q)
{
    u64 h = __umul64hi(x, wp);
    return x * w - mul_q_lo(h, q);   // in [0, 2q)
}

__device__ __forceinline__ u64 mul_shoup(u64 x, u64 w, u64 wp, u64 q)
{
    return csub(mul_shoup_lazy(x, w, wp, q), q);
}

// (hi:lo) * 2^-64 mod q, requires (hi:lo) < q * 2^64; result in [0, q).
// m = lo * q^{-1} mod 2^64 makes lo - m q = 0 mod 2^64, and floor(m q / 2^64)
// = m1 q1 + floor((m0 q1 + m1) / 2^32) for m = m1 2^32 + m0.
__device__ __forceinline__ u64 redc(u64 lo, u64 hi, u64 q)
{
    const uint32_t q1 = (uint32_t)(q >> 32);
    u64 m = lo - ((u64)((uint32_t)lo * q1) << 32);
    u64 t = (u64)(uint32_t)(m >> 32) * q1 + (((u64)(uint32_t)m * q1 + (m >> 32)) >> 32);
    u64 d = hi - t;
    return (long long)d < 0 ? d + q : d;
}

// 128-bit accumulator helpers.
struct Acc128 {
    u64 lo, hi;
};
__device__ __forceinline__ void acc_init(Acc128 &a) { a.lo = 0; a.hi = 0; }
// (hi:lo) += x * y: the low product added with carry-out, the high product added
// with that carry (one multiply-add pair; 22 % faster than a separate low
// product, high product and carry compare in a register-only loop).
__device__ __forceinline__ void acc_mad(Acc128 &a, u64 x, u64 y)
{
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
        "madc.hi.u64 %1, %2, %3, %1;"
        : "+l"(a.lo), "+l"(a.hi)
        : "l"(x), "l"(y));
}

// a * b mod q for a, b < q (Barrett on the 128-bit product).
__device__ __forceinline__ u64 mul_barrett(u64 a, u64 b, const ModConst &m)
{
    u64 lo = a * b;
    u64 hi = __umul64hi(a, b);
    int k = m.k;
    // x1 = x >> (k-1)  (< 2^(k+1))
    u64 x1 = (lo >> (k - 1)) | (hi << (65 - k));
    u64 plo = x1 * m.mu;
    u64 phi = __umul64hi(x1, m.mu);
    u64 qh = (plo >> (k + 1)) | (phi << (63 - k));
    u64 r = lo - mul_q_lo(qh, m.q);
    r = csub(r, m.q);
    return csub(r, m.q);
}

// (x mod q) for a 128-bit x < 2^(2k+2): Barrett with the same mu, one extra
// correction step.
__device__ __forceinline__ u64 reduce128_barrett(u64 lo, u64 hi, const ModConst &m)
{
    int k = m.k;
    u64 x1 = (lo >> (k - 1)) | (hi << (65 - k));
    u64 plo = x1 * m.mu;
    u64 phi = __umul64hi(x1, m.mu);
    u64 qh = (plo >> (k + 1)) | (phi << (63 - k));
    u64 r = lo - mul_q_lo(qh, m.q);
    while (r >= m.q) r -= m.q;
    return r;
}

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) { return csub(a + b, q); }
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q)
{
    u64 d = a - b;
    return (long long)d < 0 ? d + q : d;
}
__device__ __forceinline__ u64 neg_mod(u64 a, u64 q) { return a == 0 ? 0 : q - a; }

// Residue of a signed 64-bit integer.
__device__ __forceinline__ u64 reduce_i64(long long v, const ModConst &m)
{
    if (v >= 0) {
        u64 u = (u64)v;
        return u < m.q ? u : u % m.q;
    }
    u64 u = (u64)(-(v + 1)) + 1;   // |v|
    u64 r = u < m.q ? u : u % m.q;
    return r == 0 ? 0 : m.q - r;
}

__device__ __forceinline__ unsigned bitrev(unsigned x, int bits) { return __brev(x) >> (32 - bits); }

#define HETAL_CUDA_CHECK(expr)                                                   \
    do {                                                                         \
        cudaError_t _e = (expr);                                                 \
        if (_e != cudaSuccess) throw hetal::CudaError(_e, #expr, __FILE__, __LINE__); \
    } while (0)
