// ntt.cu -- batched negacyclic NTT / INTT for u64 RNS limbs on sm_103a.
//
// Forward transform: Cooley-Tukey with psi-powers in bit-reversed order
// (psi_rev[m + i] = psi^{brv(m + i)}), natural-order input, bit-reversed
// output: slot j holds a(psi^{2 brv(j) + 1}).  Inverse: Gentleman-Sande with
// psi^{-brv}, bit-reversed input, natural output, times N^{-1}.
//
// A limb of N = R * 256 words is viewed as R rows of 256 and transformed in two
// passes (two launches), each through shared memory:
//   column pass: the log2(R) stages whose butterfly distance is a multiple of
//                256 (a fixed column c holds the R words r*256 + c);
//   row pass:    the 8 stages inside each contiguous row of 256 words.
// Inside a pass a thread keeps E = 16 words in registers.  With the strided
// assignment (words t + T*j, j < 16, T = threads per column or row) the first
// four stages of larger distance are register-local; one exchange through
// shared memory gives the contiguous assignment (words 16*t + j) for the
// remaining stages.  All index arithmetic is compile-time shifts; twiddles of
// the column pass (indices below R) sit in shared memory.  Butterflies use
// Harvey's lazy reduction: forward values in [0, 4q), inverse in [0, 2q),
// with q < 2^61, so every comparison is the sign of a 64-bit difference.
#include "context.h"

namespace hetal {

namespace {

constexpr int LOG_N2 = 8;
constexpr int N2 = 1 << LOG_N2;
constexpr int THREADS = 256;

__device__ __forceinline__ void ct_bfly(u64 &x, u64 &y, u64 w, u64 wp, u64 q, u64 two_q)
{
    u64 a = csub(x, two_q);
    u64 t = mul_shoup_lazy(y, w, wp, q);
    x = a + t;
    y = a - t + two_q;
}

__device__ __forceinline__ void gs_bfly(u64 &x, u64 &y, u64 w, u64 wp, u64 q, u64 two_q)
{
    u64 s = csub(x + y, two_q);
    u64 d = x - y + two_q;
    x = s;
    y = mul_shoup_lazy(d, w, wp, q);
}

// ---------------------------------------------------------------------------
// Column pass.  LOGR = log2(rows); E = min(16, R) words per thread; TPC = R / E
// threads per column; COLS = 256 / TPC columns per CTA.
// ---------------------------------------------------------------------------
template <int LOGR>
struct ColShape {
    static constexpr int R = 1 << LOGR;
    static constexpr int LOGE = LOGR < 4 ? LOGR : 4;
    static constexpr int E = 1 << LOGE;
    static constexpr int LOGT = LOGR - LOGE;   // log2(threads per column)
    static constexpr int TPC = 1 << LOGT;
    static constexpr int COLS = THREADS / TPC;
};

// NA > 0: the input words are formed by a fast base conversion from NA source
// limbs of cv.src (same poly, same coefficient) instead of being loaded from b.
template <int LOGR, int NA>
__global__ void __launch_bounds__(THREADS) ntt_fwd_cols(PolyBatch b, const __grid_constant__ LimbMap mods,
                                                        const __grid_constant__ LimbMap pos,
                                                        const ModConst *__restrict__ mc,
                                                        const ulonglong2 *__restrict__ psi, int logN,
                                                        const __grid_constant__ ConvSrc cv)
{
    using S = ColShape<LOGR>;
    extern __shared__ u64 sm[];          // [R][COLS] data, then R (twiddle, Shoup twiddle) pairs
    ulonglong2 *tw = reinterpret_cast<ulonglong2 *>(sm + S::R * S::COLS);
    const int N = 1 << logN;
    const int l = blockIdx.y;
    const int midx = mods.idx[l];
    const u64 q = mc[midx].q, two_q = 2 * q;
    u64 *base = b.ptr + (size_t)blockIdx.z * b.stride + (size_t)pos.idx[l] * N + blockIdx.x * S::COLS;
    const int cc = threadIdx.x % S::COLS, t = threadIdx.x / S::COLS;
    for (int i = threadIdx.x; i < S::R; i += THREADS) tw[i] = psi[(size_t)midx * N + i];
    u64 v[S::E];
    if (NA == 0) {
#pragma unroll
        for (int j = 0; j < S::E; j++) v[j] = base[(size_t)(t + S::TPC * j) * N2 + cc];
    } else {
        const u64 *src[NA > 0 ? NA : 1];
        u64 hat[NA > 0 ? NA : 1];
#pragma unroll
        for (int a = 0; a < NA; a++) {
            src[a] = cv.src.ptr + (size_t)blockIdx.z * cv.src.stride + (size_t)cv.src_pos.idx[a] * N +
                     blockIdx.x * S::COLS;
            hat[a] = cv.hat[l * NA + a];
        }
#pragma unroll
        for (int j = 0; j < S::E; j++) {
            Acc128 acc;
            acc_init(acc);
#pragma unroll
            for (int a = 0; a < NA; a++) acc_mad(acc, src[a][(size_t)(t + S::TPC * j) * N2 + cc], hat[a]);
            v[j] = redc(acc.lo, acc.hi, q);
        }
    }
    __syncthreads();
    // stages s < LOGE: rows t + TPC*j, distance E/2^{s+1} in j, twiddle index 2^s + (j >> (LOGE - s))
#pragma unroll
    for (int s = 0; s < S::LOGE; s++) {
        const int d = S::E >> (s + 1);
#pragma unroll
        for (int j = 0; j < S::E; j++) {
            if (j & d) continue;
            const ulonglong2 w = tw[(1 << s) + (j >> (S::LOGE - s))];
            ct_bfly(v[j], v[j + d], w.x, w.y, q, two_q);
        }
    }
    if (S::LOGT > 0) {
#pragma unroll
        for (int j = 0; j < S::E; j++) sm[(t + S::TPC * j) * S::COLS + cc] = v[j];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < S::E; j++) v[j] = sm[(S::E * t + j) * S::COLS + cc];
        // stages s = LOGE .. LOGR-1: rows E*t + j, distance 2^{LOGR-1-s}, twiddle 2^s + (row >> (LOGR - s))
#pragma unroll
        for (int s = S::LOGE; s < LOGR; s++) {
            const int d = 1 << (LOGR - 1 - s);
#pragma unroll
            for (int j = 0; j < S::E; j++) {
                if (j & d) continue;
                const ulonglong2 w = tw[(1 << s) + ((S::E * t + j) >> (LOGR - s))];
                ct_bfly(v[j], v[j + d], w.x, w.y, q, two_q);
            }
        }
#pragma unroll
        for (int j = 0; j < S::E; j++) base[(size_t)(S::E * t + j) * N2 + cc] = v[j];
    } else {
#pragma unroll
        for (int j = 0; j < S::E; j++) base[(size_t)(t + S::TPC * j) * N2 + cc] = v[j];
    }
}

template <int LOGR>
__global__ void __launch_bounds__(THREADS, 4) ntt_inv_cols(PolyBatch b, const __grid_constant__ LimbMap mods,
                                                        const __grid_constant__ LimbMap pos,
                                                        const ModConst *__restrict__ mc,
                                                        const ulonglong2 *__restrict__ ipsi,
                                                        const u64 *__restrict__ ninv,
                                                        const u64 *__restrict__ ninv_sh,
                                                        const u64 *__restrict__ lsc,
                                                        const u64 *__restrict__ lsc_sh, int logN)
{
    using S = ColShape<LOGR>;
    extern __shared__ u64 sm[];
    ulonglong2 *tw = reinterpret_cast<ulonglong2 *>(sm + S::R * S::COLS);
    const int N = 1 << logN;
    const int l = blockIdx.y;
    const int midx = mods.idx[l];
    const u64 q = mc[midx].q, two_q = 2 * q;
    u64 *base = b.ptr + (size_t)blockIdx.z * b.stride + (size_t)pos.idx[l] * N + blockIdx.x * S::COLS;
    const int cc = threadIdx.x % S::COLS, t = threadIdx.x / S::COLS;
    for (int i = threadIdx.x; i < S::R; i += THREADS) tw[i] = ipsi[(size_t)midx * N + i];
    u64 v[S::E];
    if (S::LOGT > 0) {
#pragma unroll
        for (int j = 0; j < S::E; j++) v[j] = base[(size_t)(S::E * t + j) * N2 + cc];
        __syncthreads();
        // row distances 1 .. TPC/2 (rows E*t + j): h = R / (2 tr), group = row / (2 tr)
#pragma unroll
        for (int lt = 0; lt < S::LOGT; lt++) {
            const int d = 1 << lt;
#pragma unroll
            for (int j = 0; j < S::E; j++) {
                if (j & d) continue;
                const ulonglong2 w = tw[(S::R >> (lt + 1)) + ((S::E * t + j) >> (lt + 1))];
                gs_bfly(v[j], v[j + d], w.x, w.y, q, two_q);
            }
        }
#pragma unroll
        for (int j = 0; j < S::E; j++) sm[(S::E * t + j) * S::COLS + cc] = v[j];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < S::E; j++) v[j] = sm[(t + S::TPC * j) * S::COLS + cc];
    } else {
#pragma unroll
        for (int j = 0; j < S::E; j++) v[j] = base[(size_t)(t + S::TPC * j) * N2 + cc];
        __syncthreads();
    }
    // row distances TPC .. R/2 (rows t + TPC*j, distance 2^le in j): group = j >> (le + 1)
#pragma unroll
    for (int le = 0; le < S::LOGE; le++) {
        const int d = 1 << le;
#pragma unroll
        for (int j = 0; j < S::E; j++) {
            if (j & d) continue;
            const ulonglong2 w = tw[(S::E >> (le + 1)) + (j >> (le + 1))];
            gs_bfly(v[j], v[j + d], w.x, w.y, q, two_q);
        }
    }
    // final factor: N^{-1}, or a per-limb factor that includes it
    const u64 ni = lsc ? lsc[l] : ninv[midx], nis = lsc ? lsc_sh[l] : ninv_sh[midx];
#pragma unroll
    for (int j = 0; j < S::E; j++) base[(size_t)(t + S::TPC * j) * N2 + cc] = mul_shoup(v[j], ni, nis, q);
}

// ---------------------------------------------------------------------------
// Row pass: 16 threads per row of 256, 16 rows per CTA.  Global group index of
// a butterfly at stage m = R * 2^s is row * 2^s + (word >> (8 - s)).
// ---------------------------------------------------------------------------
constexpr int RPB = THREADS / 16;   // rows per CTA
// Shared row buffer: word e of a row at e + (e >> 4), row stride 272.  Words
// 16t + j then sit 17 apart across t (banks 2t, 2t+1 distinct for t < 16) and
// words t + 16j stay contiguous across t: both layouts are conflict-free.
constexpr int RS = N2 + N2 / 16;

// MD: the ModDown tail (see ntt_forward_moddown) replaces the plain store.
template <bool MD>
__global__ void __launch_bounds__(THREADS, 4) ntt_fwd_rows(PolyBatch b, const __grid_constant__ LimbMap mods,
                                                        const __grid_constant__ LimbMap pos,
                                                        const ModConst *__restrict__ mc,
                                                        const ulonglong2 *__restrict__ rowtw, int logN,
                                                        const __grid_constant__ ModDownTail tail,
                                                        const u64 *__restrict__ pinv,
                                                        const u64 *__restrict__ pinv_sh)
{
    __shared__ u64 sm[RPB * RS];
    const int N = 1 << logN;
    const int R = N >> LOG_N2;
    const int l = blockIdx.y;
    const int midx = mods.idx[l];
    const u64 q = mc[midx].q, two_q = 2 * q;
    const int rr = threadIdx.x >> 4, t = threadIdx.x & 15;
    const int row = blockIdx.x * RPB + rr;
    u64 *base = b.ptr + (size_t)blockIdx.z * b.stride + (size_t)pos.idx[l] * N;
    const ulonglong2 *tw = rowtw + ((size_t)midx * R + row) * 255;   // this row's twiddles, in read order
    __shared__ ulonglong2 stw[RPB * 16];   // the 15 pairs of the strided stages, per row
    u64 v[16];
    if (row < R) {
        if (t < 15) stw[rr * 16 + t] = __ldg(tw + t);
        const u64 *src = base + (size_t)row * N2;
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = src[t + 16 * j];
        __syncwarp(0xffffu << (threadIdx.x & 16));   // the row's 16 threads
        // stages s = 0..3: words t + 16j, distance 8 >> s in j
#pragma unroll
        for (int s = 0; s < 4; s++) {
            const int d = 8 >> s;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                if (j & d) continue;
                const ulonglong2 w = stw[rr * 16 + (1 << s) - 1 + (j >> (4 - s))];   // psi2[m + (row << s) + k]
                ct_bfly(v[j], v[j + d], w.x, w.y, q, two_q);
            }
        }
#pragma unroll
        for (int j = 0; j < 16; j++) sm[rr * RS + t + 17 * j] = v[j];
    }
    __syncthreads();
    if (row < R) {
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = sm[rr * RS + 17 * t + j];
        // stages s = 4..7: words 16t + j, distance 8 >> (s - 4)
#pragma unroll
        for (int s = 4; s < 8; s++) {
            const int d = 8 >> (s - 4);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                if (j & d) continue;
                // psi2[m + (row << s) + 2^(s-4) t + k], k = j >> (8 - s)
                const ulonglong2 w = __ldg(tw + 15 + 16 * ((1 << (s - 4)) - 1 + (j >> (8 - s))) + t);
                ct_bfly(v[j], v[j + d], w.x, w.y, q, two_q);
            }
        }
#pragma unroll
        for (int j = 0; j < 16; j++) {
            sm[rr * RS + 17 * t + j] = csub(csub(v[j], two_q), q);
        }
    }
    __syncthreads();
    if (row < R) {
        if (!MD) {
            u64 *dst = base + (size_t)row * N2;
#pragma unroll
            for (int j = 0; j < 16; j++) dst[t + 16 * j] = sm[rr * RS + t + 17 * j];
        } else {
            const int half = (int)blockIdx.z >= tail.B, pp = blockIdx.z - half * tail.B, i = pos.idx[l];
            const size_t off = (size_t)i * N + (size_t)row * N2;
            const PolyBatch o = tail.out[half], a = tail.acc[half], ad = tail.add[half];
            u64 *dst = o.ptr + (size_t)pp * o.stride + off;
            const u64 *src = a.ptr + (size_t)pp * a.stride + off;
            const u64 *adp = ad.ptr ? ad.ptr + (size_t)pp * ad.stride + off : nullptr;
            const u64 w = pinv[midx], wp = pinv_sh[midx];
#pragma unroll
            for (int j = 0; j < 16; j++) {
                u64 r = mul_shoup(sub_mod(src[t + 16 * j], sm[rr * RS + t + 17 * j], q), w, wp, q);
                if (adp) r = add_mod(r, adp[t + 16 * j], q);
                dst[t + 16 * j] = r;
            }
        }
    }
}

__global__ void __launch_bounds__(THREADS, 4) ntt_inv_rows(PolyBatch b, PolyBatch in,
                                                        const __grid_constant__ LimbMap mods,
                                                        const __grid_constant__ LimbMap pos,
                                                        const ModConst *__restrict__ mc,
                                                        const ulonglong2 *__restrict__ irowtw, int logN)
{
    __shared__ u64 sm[RPB * RS];
    const int N = 1 << logN;
    const int R = N >> LOG_N2;
    const int l = blockIdx.y;
    const int midx = mods.idx[l];
    const u64 q = mc[midx].q, two_q = 2 * q;
    const int rr = threadIdx.x >> 4, t = threadIdx.x & 15;
    const int row = blockIdx.x * RPB + rr;
    u64 *base = b.ptr + (size_t)blockIdx.z * b.stride + (size_t)pos.idx[l] * N;
    const u64 *ibase = in.ptr + (size_t)blockIdx.z * in.stride + (size_t)pos.idx[l] * N;
    const ulonglong2 *tw = irowtw + ((size_t)midx * R + row) * 255;   // this row's twiddles, in read order
    __shared__ ulonglong2 stw[RPB * 16];   // the 15 pairs of the strided stages, per row
    u64 v[16];
    if (row < R) {
        if (t < 15) stw[rr * 16 + t] = __ldg(tw + 240 + t);
        const u64 *src = ibase + (size_t)row * N2;
#pragma unroll
        for (int j = 0; j < 16; j++) sm[rr * RS + t + 17 * j] = src[t + 16 * j];
    }
    __syncthreads();
    if (row < R) {
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = sm[rr * RS + 17 * t + j];
        // distances 1..8 (words 16t + j): stage with distance 2^lt has h = N / 2^{lt+1},
        // group index row * (128 >> lt) + (word >> (lt + 1))
#pragma unroll
        for (int lt = 0; lt < 4; lt++) {
            const int d = 1 << lt;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                if (j & d) continue;
                // ipsi2[h + row 2^(7-lt) + 2^(3-lt) t + k], h = N / 2^(lt+1), k = j >> (lt + 1)
                const ulonglong2 w = __ldg(tw + 16 * (16 - (16 >> lt) + (j >> (lt + 1))) + t);
                gs_bfly(v[j], v[j + d], w.x, w.y, q, two_q);
            }
        }
#pragma unroll
        for (int j = 0; j < 16; j++) sm[rr * RS + 17 * t + j] = v[j];
    }
    __syncthreads();
    if (row < R) {
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = sm[rr * RS + t + 17 * j];
        // distances 16..128 (words t + 16j, distance 2^(lt-4) in j)
#pragma unroll
        for (int lt = 4; lt < 8; lt++) {
            const int d = 1 << (lt - 4);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                if (j & d) continue;
                // ipsi2[h + row 2^(7-lt) + k], k = j >> (lt - 3)
                const ulonglong2 w = stw[rr * 16 + (16 - (16 >> (lt - 4))) + (j >> (lt - 3))];
                gs_bfly(v[j], v[j + d], w.x, w.y, q, two_q);
            }
        }
        u64 *dst = base + (size_t)row * N2;
#pragma unroll
        for (int j = 0; j < 16; j++) dst[t + 16 * j] = v[j];
    }
}

// Row passes over groups of polynomials.  A CTA stages the 255 twiddle pairs of each
// of its 16 rows (consecutive in the row tables) in shared memory once, then
// transforms those rows of `ppc` polynomials of the same limb one after another:
// the twiddles come from L2 once per group instead of once per polynomial, and the
// per-stage reads are shared-memory reads.  Same butterflies, same bits.
constexpr int TWR = 255;
constexpr size_t GRP_SMEM = (size_t)RPB * TWR * sizeof(ulonglong2) + (size_t)RPB * RS * sizeof(u64);

template <bool MD>
__global__ void __launch_bounds__(THREADS, 2) ntt_fwd_rows_grp(PolyBatch b, const __grid_constant__ LimbMap mods,
                                                            const __grid_constant__ LimbMap pos,
                                                            const ModConst *__restrict__ mc,
                                                            const ulonglong2 *__restrict__ rowtw, int logN,
                                                            const __grid_constant__ ModDownTail tail,
                                                            const u64 *__restrict__ pinv,
                                                            const u64 *__restrict__ pinv_sh, int ppc)
{
    extern __shared__ ulonglong2 grp_tw[];                             // [RPB][255], then the row buffer
    u64 *sm = reinterpret_cast<u64 *>(grp_tw + RPB * TWR);
    const int N = 1 << logN;
    const int R = N >> LOG_N2;
    const int l = blockIdx.y;
    const int midx = mods.idx[l];
    const u64 q = mc[midx].q, two_q = 2 * q;
    const int rr = threadIdx.x >> 4, t = threadIdx.x & 15;
    const int row0 = blockIdx.x * RPB, row = row0 + rr;
    const int nrows = min(RPB, R - row0);
    const ulonglong2 *gsrc = rowtw + ((size_t)midx * R + row0) * TWR;
    for (int i = threadIdx.x; i < nrows * TWR; i += THREADS) grp_tw[i] = __ldg(gsrc + i);
    __syncthreads();
    const ulonglong2 *tw = grp_tw + rr * TWR;   // this row's twiddles, in read order
    const int z1 = min(b.count, (int)(blockIdx.z + 1) * ppc);
    for (int z = blockIdx.z * ppc; z < z1; z++) {
        u64 *base = b.ptr + (size_t)z * b.stride + (size_t)pos.idx[l] * N;
        u64 v[16];
        if (row < R) {
            const u64 *src = base + (size_t)row * N2;
#pragma unroll
            for (int j = 0; j < 16; j++) v[j] = src[t + 16 * j];
#pragma unroll
            for (int s = 0; s < 4; s++) {
                const int d = 8 >> s;
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    if (j & d) continue;
                    const ulonglong2 w = tw[(1 << s) - 1 + (j >> (4 - s))];
                    ct_bfly(v[j], v[j + d], w.x, w.y, q, two_q);
                }
            }
#pragma unroll
            for (int j = 0; j < 16; j++) sm[rr * RS + t + 17 * j] = v[j];
        }
        __syncthreads();
        if (row < R) {
#pragma unroll
            for (int j = 0; j < 16; j++) v[j] = sm[rr * RS + 17 * t + j];
#pragma unroll
            for (int s = 4; s < 8; s++) {
                const int d = 8 >> (s - 4);
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    if (j & d) continue;
                    const ulonglong2 w = tw[15 + 16 * ((1 << (s - 4)) - 1 + (j >> (8 - s))) + t];
                    ct_bfly(v[j], v[j + d], w.x, w.y, q, two_q);
                }
            }
#pragma unroll
            for (int j = 0; j < 16; j++) sm[rr * RS + 17 * t + j] = csub(csub(v[j], two_q), q);
        }
        __syncthreads();
        if (row < R) {
            if (!MD) {
                u64 *dst = base + (size_t)row * N2;
#pragma unroll
                for (int j = 0; j < 16; j++) dst[t + 16 * j] = sm[rr * RS + t + 17 * j];
            } else {
                const int half = z >= tail.B, pp = z - half * tail.B, i = pos.idx[l];
                const size_t off = (size_t)i * N + (size_t)row * N2;
                const PolyBatch o = tail.out[half], a = tail.acc[half], ad = tail.add[half];
                u64 *dst = o.ptr + (size_t)pp * o.stride + off;
                const u64 *src = a.ptr + (size_t)pp * a.stride + off;
                const u64 *adp = ad.ptr ? ad.ptr + (size_t)pp * ad.stride + off : nullptr;
                const u64 w = pinv[midx], wp = pinv_sh[midx];
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    u64 r = mul_shoup(sub_mod(src[t + 16 * j], sm[rr * RS + t + 17 * j], q), w, wp, q);
                    if (adp) r = add_mod(r, adp[t + 16 * j], q);
                    dst[t + 16 * j] = r;
                }
            }
        }
        __syncthreads();   // the next polynomial reuses the row buffer
    }
}

__global__ void __launch_bounds__(THREADS, 2) ntt_inv_rows_grp(PolyBatch b, PolyBatch in,
                                                            const __grid_constant__ LimbMap mods,
                                                            const __grid_constant__ LimbMap pos,
                                                            const ModConst *__restrict__ mc,
                                                            const ulonglong2 *__restrict__ irowtw, int logN, int ppc)
{
    extern __shared__ ulonglong2 grp_tw[];
    u64 *sm = reinterpret_cast<u64 *>(grp_tw + RPB * TWR);
    const int N = 1 << logN;
    const int R = N >> LOG_N2;
    const int l = blockIdx.y;
    const int midx = mods.idx[l];
    const u64 q = mc[midx].q, two_q = 2 * q;
    const int rr = threadIdx.x >> 4, t = threadIdx.x & 15;
    const int row0 = blockIdx.x * RPB, row = row0 + rr;
    const int nrows = min(RPB, R - row0);
    const ulonglong2 *gsrc = irowtw + ((size_t)midx * R + row0) * TWR;
    for (int i = threadIdx.x; i < nrows * TWR; i += THREADS) grp_tw[i] = __ldg(gsrc + i);
    __syncthreads();
    const ulonglong2 *tw = grp_tw + rr * TWR;
    const int z1 = min(b.count, (int)(blockIdx.z + 1) * ppc);
    for (int z = blockIdx.z * ppc; z < z1; z++) {
        u64 *base = b.ptr + (size_t)z * b.stride + (size_t)pos.idx[l] * N;
        const u64 *ibase = in.ptr + (size_t)z * in.stride + (size_t)pos.idx[l] * N;
        u64 v[16];
        if (row < R) {
            const u64 *src = ibase + (size_t)row * N2;
#pragma unroll
            for (int j = 0; j < 16; j++) sm[rr * RS + t + 17 * j] = src[t + 16 * j];
        }
        __syncthreads();
        if (row < R) {
#pragma unroll
            for (int j = 0; j < 16; j++) v[j] = sm[rr * RS + 17 * t + j];
#pragma unroll
            for (int lt = 0; lt < 4; lt++) {
                const int d = 1 << lt;
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    if (j & d) continue;
                    const ulonglong2 w = tw[16 * (16 - (16 >> lt) + (j >> (lt + 1))) + t];
                    gs_bfly(v[j], v[j + d], w.x, w.y, q, two_q);
                }
            }
#pragma unroll
            for (int j = 0; j < 16; j++) sm[rr * RS + 17 * t + j] = v[j];
        }
        __syncthreads();
        if (row < R) {
#pragma unroll
            for (int j = 0; j < 16; j++) v[j] = sm[rr * RS + t + 17 * j];
#pragma unroll
            for (int lt = 4; lt < 8; lt++) {
                const int d = 1 << (lt - 4);
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    if (j & d) continue;
                    const ulonglong2 w = tw[240 + (16 - (16 >> (lt - 4))) + (j >> (lt - 3))];
                    gs_bfly(v[j], v[j + d], w.x, w.y, q, two_q);
                }
            }
            u64 *dst = base + (size_t)row * N2;
#pragma unroll
            for (int j = 0; j < 16; j++) dst[t + 16 * j] = v[j];
        }
        __syncthreads();
    }
}

// Polys per CTA of a row pass over `count` polys and `limbs` limbs: the context's
// grouping, lowered so that the grid still fills the GPU with at least two waves.
int row_group(const Context &c, int count, int limbs)
{
    if (c.row_group <= 1 || count < 2) return 1;
    const long long ctas_1 = (long long)((c.p.N >> LOG_N2) + RPB - 1) / RPB * limbs * count;
    int g = std::min(c.row_group, count);
    while (g > 1 && ctas_1 / g < 2LL * 2 * c.sm_count) g /= 2;
    return g;
}

template <bool MD>
void launch_fwd_rows(Context &c, PolyBatch b, const LimbMap &mods, const LimbMap &pos, const ModDownTail &tail,
                     const u64 *pinv, const u64 *pinv_sh)
{
    const int R = c.p.N >> LOG_N2;
    const int g = row_group(c, b.count, mods.n);
    if (g <= 1) {
        dim3 g2((R + RPB - 1) / RPB, mods.n, b.count);
        ntt_fwd_rows<MD><<<g2, THREADS, 0, c.stream>>>(b, mods, pos, c.d_mc, c.d_rowtw, c.p.logN, tail, pinv, pinv_sh);
        return;
    }
    static bool attr = false;
    if (!attr) {
        HETAL_CUDA_CHECK(
            cudaFuncSetAttribute(ntt_fwd_rows_grp<MD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GRP_SMEM));
        attr = true;
    }
    dim3 g2((R + RPB - 1) / RPB, mods.n, (b.count + g - 1) / g);
    ntt_fwd_rows_grp<MD><<<g2, THREADS, GRP_SMEM, c.stream>>>(b, mods, pos, c.d_mc, c.d_rowtw, c.p.logN, tail, pinv,
                                                             pinv_sh, g);
}

void launch_inv_rows(Context &c, PolyBatch b, PolyBatch in, const LimbMap &mods, const LimbMap &pos)
{
    const int R = c.p.N >> LOG_N2;
    const int g = row_group(c, b.count, mods.n);
    if (g <= 1) {
        dim3 g2((R + RPB - 1) / RPB, mods.n, b.count);
        ntt_inv_rows<<<g2, THREADS, 0, c.stream>>>(b, in, mods, pos, c.d_mc, c.d_irowtw, c.p.logN);
        return;
    }
    static bool attr = false;
    if (!attr) {
        HETAL_CUDA_CHECK(
            cudaFuncSetAttribute(ntt_inv_rows_grp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GRP_SMEM));
        attr = true;
    }
    dim3 g2((R + RPB - 1) / RPB, mods.n, (b.count + g - 1) / g);
    ntt_inv_rows_grp<<<g2, THREADS, GRP_SMEM, c.stream>>>(b, in, mods, pos, c.d_mc, c.d_irowtw, c.p.logN, g);
}

template <int LOGR, int NA>
void launch_fwd_cols_na(Context &c, PolyBatch b, const LimbMap &mods, const LimbMap &pos, const ConvSrc &cv)
{
    using S = ColShape<LOGR>;
    size_t smem = (size_t)S::R * S::COLS * sizeof(u64) + (size_t)S::R * sizeof(ulonglong2);
    static bool attr = false;
    if (!attr) {
        HETAL_CUDA_CHECK(cudaFuncSetAttribute(ntt_fwd_cols<LOGR, NA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        attr = true;
    }
    dim3 g(N2 / S::COLS, mods.n, b.count);
    ntt_fwd_cols<LOGR, NA><<<g, THREADS, smem, c.stream>>>(b, mods, pos, c.d_mc, c.d_psi2, c.p.logN, cv);
}

template <int LOGR>
void launch_fwd_cols(Context &c, PolyBatch b, const LimbMap &mods, const LimbMap &pos, const ConvSrc *cv)
{
    static_assert(MAX_FUSED_CONV == 8, "one instantiation per fused source-limb count");
    switch (cv ? cv->na : 0) {
    case 0: launch_fwd_cols_na<LOGR, 0>(c, b, mods, pos, ConvSrc{}); break;
    case 1: launch_fwd_cols_na<LOGR, 1>(c, b, mods, pos, *cv); break;
    case 2: launch_fwd_cols_na<LOGR, 2>(c, b, mods, pos, *cv); break;
    case 3: launch_fwd_cols_na<LOGR, 3>(c, b, mods, pos, *cv); break;
    case 4: launch_fwd_cols_na<LOGR, 4>(c, b, mods, pos, *cv); break;
    case 5: launch_fwd_cols_na<LOGR, 5>(c, b, mods, pos, *cv); break;
    case 6: launch_fwd_cols_na<LOGR, 6>(c, b, mods, pos, *cv); break;
    case 7: launch_fwd_cols_na<LOGR, 7>(c, b, mods, pos, *cv); break;
    case 8: launch_fwd_cols_na<LOGR, 8>(c, b, mods, pos, *cv); break;
    default: throw Error(ERR_INVALID_ARG, "fused base conversion from more than MAX_FUSED_CONV limbs");
    }
}

template <int LOGR>
void launch_inv_cols(Context &c, PolyBatch b, const LimbMap &mods, const LimbMap &pos, const u64 *sc,
                     const u64 *sc_sh)
{
    using S = ColShape<LOGR>;
    size_t smem = (size_t)S::R * S::COLS * sizeof(u64) + (size_t)S::R * sizeof(ulonglong2);
    static bool attr = false;
    if (!attr) {
        HETAL_CUDA_CHECK(cudaFuncSetAttribute(ntt_inv_cols<LOGR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        attr = true;
    }
    dim3 g(N2 / S::COLS, mods.n, b.count);
    ntt_inv_cols<LOGR><<<g, THREADS, smem, c.stream>>>(b, mods, pos, c.d_mc, c.d_ipsi2, c.d_ninv, c.d_ninv_sh, sc,
                                                       sc_sh, c.p.logN);
}

void fwd_cols(Context &c, PolyBatch b, const LimbMap &mods, const LimbMap &pos, const ConvSrc *cv)
{
    switch (c.p.logN - LOG_N2) {
    case 2: launch_fwd_cols<2>(c, b, mods, pos, cv); break;
    case 3: launch_fwd_cols<3>(c, b, mods, pos, cv); break;
    case 4: launch_fwd_cols<4>(c, b, mods, pos, cv); break;
    case 5: launch_fwd_cols<5>(c, b, mods, pos, cv); break;
    case 6: launch_fwd_cols<6>(c, b, mods, pos, cv); break;
    case 7: launch_fwd_cols<7>(c, b, mods, pos, cv); break;
    case 8: launch_fwd_cols<8>(c, b, mods, pos, cv); break;
    default: throw Error(ERR_INVALID_ARG, "unsupported ring degree");
    }
}

void inv_cols(Context &c, PolyBatch b, const LimbMap &mods, const LimbMap &pos, const u64 *sc, const u64 *sc_sh)
{
    switch (c.p.logN - LOG_N2) {
    case 2: launch_inv_cols<2>(c, b, mods, pos, sc, sc_sh); break;
    case 3: launch_inv_cols<3>(c, b, mods, pos, sc, sc_sh); break;
    case 4: launch_inv_cols<4>(c, b, mods, pos, sc, sc_sh); break;
    case 5: launch_inv_cols<5>(c, b, mods, pos, sc, sc_sh); break;
    case 6: launch_inv_cols<6>(c, b, mods, pos, sc, sc_sh); break;
    case 7: launch_inv_cols<7>(c, b, mods, pos, sc, sc_sh); break;
    case 8: launch_inv_cols<8>(c, b, mods, pos, sc, sc_sh); break;
    default: throw Error(ERR_INVALID_ARG, "unsupported ring degree");
    }
}

}  // namespace

// The column pass, plain or with the fused base conversion (launch accounting:
// the conversion's products and source reads are added to the pass).
static void cols_pass(Context &c, PolyBatch b, const LimbMap &mods, const LimbMap &pos, const ConvSrc *cv)
{
    const int N = c.p.N, logN = c.p.logN;
    const double limbs = (double)b.count * mods.n;
    const int na = cv ? cv->na : 0;
    bool t = c.launch_begin(na ? "ntt_fwd_cols_conv" : "ntt_fwd_cols");
    fwd_cols(c, b, mods, pos, cv);
    // algorithmic bytes: every limb read and written once; with the conversion, each
    // poly's na source limbs read once (the target limbs of a poly share them) and
    // every target limb written once
    const double bytes = na ? (double)b.count * N * 8.0 * (mods.n + na) : limbs * N * 16.0;
    c.launch_end(t, limbs * ((N / 2) * (logN - LOG_N2) + (double)na * N), bytes);
    c.cnt.modmul += limbs * na * N;
}

void ntt_forward(Context &c, PolyBatch b, const LimbMap &mods, const LimbMap &pos)
{
    ntt_forward_conv(c, b, mods, pos, ConvSrc{{nullptr, 0, 0}, {}, nullptr, 0});
}

void ntt_forward_conv(Context &c, PolyBatch b, const LimbMap &mods, const LimbMap &pos, const ConvSrc &cv)
{
    if (b.count == 0 || mods.n == 0) return;
    if (cv.na < 0 || cv.na > MAX_FUSED_CONV || (cv.na && cv.src.count != b.count))
        throw Error(ERR_INVALID_ARG, "fused base conversion: source batch");
    const int N = c.p.N, logN = c.p.logN, R = N / N2;
    const double limbs = (double)b.count * mods.n;
    cols_pass(c, b, mods, pos, cv.na ? &cv : nullptr);
    bool t;
    t = c.launch_begin("ntt_fwd_rows");
    launch_fwd_rows<false>(c, b, mods, pos, ModDownTail{}, nullptr, nullptr);
    c.launch_end(t, limbs * (N / 2) * LOG_N2, limbs * N * 16.0);
    HETAL_CUDA_CHECK(cudaGetLastError());
    c.cnt.ntt_limbs += (long long)b.count * mods.n;
    c.cnt.modmul += limbs * (N / 2) * logN;
}

void ntt_forward_moddown(Context &c, PolyBatch b, int lv, const ModDownTail &tail)
{
    ntt_forward_moddown_conv(c, b, lv, tail, ConvSrc{{nullptr, 0, 0}, {}, nullptr, 0});
}

void ntt_forward_moddown_conv(Context &c, PolyBatch b, int lv, const ModDownTail &tail, const ConvSrc &cv)
{
    if (b.count == 0) return;
    if (b.count != 2 * tail.B) throw Error(ERR_INVALID_ARG, "ModDown tail: batch is not two halves");
    if (cv.na < 0 || cv.na > MAX_FUSED_CONV || (cv.na && cv.src.count != b.count))
        throw Error(ERR_INVALID_ARG, "fused base conversion: source batch");
    const int N = c.p.N, logN = c.p.logN, R = N / N2;
    const LimbMap mods = c.q_map(lv), pos = identity_pos(lv + 1);
    const double limbs = (double)b.count * mods.n;
    cols_pass(c, b, mods, pos, cv.na ? &cv : nullptr);
    bool t;
    const double adds = (tail.add[0].ptr ? 0.5 : 0.0) + (tail.add[1].ptr ? 0.5 : 0.0);   // share of polys with an addend
    t = c.launch_begin("ntt_fwd_rows_moddown");
    launch_fwd_rows<true>(c, b, mods, pos, tail, c.d_pinv_q, c.d_pinv_q_sh);
    c.launch_end(t, limbs * ((N / 2) * LOG_N2 + N), limbs * N * (24.0 + 8.0 * adds));
    HETAL_CUDA_CHECK(cudaGetLastError());
    c.cnt.ntt_limbs += (long long)b.count * mods.n;
    c.cnt.modmul += limbs * ((N / 2) * logN + N);
}

void ntt_inverse(Context &c, PolyBatch b, const LimbMap &mods, const LimbMap &pos)
{
    ntt_inverse_oop(c, b, b, mods, pos);
}

void ntt_inverse_oop(Context &c, PolyBatch b, PolyBatch in, const LimbMap &mods, const LimbMap &pos)
{
    ntt_inverse_scaled(c, b, in, mods, pos, nullptr, nullptr);
}

void ntt_inverse_scaled(Context &c, PolyBatch b, PolyBatch in, const LimbMap &mods, const LimbMap &pos,
                        const u64 *sc, const u64 *sc_sh)
{
    if (b.count == 0 || mods.n == 0) return;
    const int N = c.p.N, logN = c.p.logN, R = N / N2;
    const double limbs = (double)b.count * mods.n;
    bool t = c.launch_begin("ntt_inv_rows");
    launch_inv_rows(c, b, in, mods, pos);
    c.launch_end(t, limbs * (N / 2) * LOG_N2, limbs * N * 16.0);
    t = c.launch_begin("ntt_inv_cols");
    inv_cols(c, b, mods, pos, sc, sc_sh);
    c.launch_end(t, limbs * ((N / 2) * (logN - LOG_N2) + N), limbs * N * 16.0);
    HETAL_CUDA_CHECK(cudaGetLastError());
    c.cnt.ntt_limbs += (long long)b.count * mods.n;
    c.cnt.modmul += limbs * ((N / 2) * logN + N);
}

}  // namespace hetal
