// common.cuh -- shared types and 64-bit modular arithmetic for the GB300
// (sm_103a) RNS-CKKS kernels.
//
// Words are u64, primes q < 2^61.  Three reductions are used:
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

#define HETAL_MAX_MODULI 64

// Per-modulus constants (device and host copies).
struct ModConst {
    u64 q;
    u64 qinv;     // q^{-1} mod 2^64 (Montgomery)
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

__device__ __forceinline__ u64 mul_shoup_lazy(u64 x, u64 w, u64 wp, u64 q)
{
    u64 h = __umul64hi(x, wp);
    return x * w - h * q;   // in [0, 2q)
}

__device__ __forceinline__ u64 mul_shoup(u64 x, u64 w, u64 wp, u64 q)
{
    u64 r = mul_shoup_lazy(x, w, wp, q);
    return r >= q ? r - q : r;
}

// (hi:lo) * 2^-64 mod q, requires (hi:lo) < q * 2^64; result in [0, q).
__device__ __forceinline__ u64 redc(u64 lo, u64 hi, u64 q, u64 qinv)
{
    u64 m = lo * qinv;
    u64 t = __umul64hi(m, q);
    return hi >= t ? hi - t : hi - t + q;
}

// 128-bit accumulator helpers.
struct Acc128 {
    u64 lo, hi;
};
__device__ __forceinline__ void acc_init(Acc128 &a) { a.lo = 0; a.hi = 0; }
__device__ __forceinline__ void acc_mad(Acc128 &a, u64 x, u64 y)
{
    u64 plo = x * y;
    u64 phi = __umul64hi(x, y);
    u64 nlo = a.lo + plo;
    a.hi += phi + (nlo < plo ? 1 : 0);
    a.lo = nlo;
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
    u64 r = lo - qh * m.q;
    if (r >= m.q) r -= m.q;
    if (r >= m.q) r -= m.q;
    return r;
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
    u64 r = lo - qh * m.q;
    while (r >= m.q) r -= m.q;
    return r;
}

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q)
{
    u64 s = a + b;
    return s >= q ? s - q : s;
}
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q)
{
    return a >= b ? a - b : a + q - b;
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
