// ntt.cu -- batched negacyclic NTT / INTT for u64 RNS limbs on sm_103a.
//
// Forward transform: Cooley-Tukey with psi-powers in bit-reversed order
// (psi_rev[m + i] = psi^{brv(m + i)}), natural-order input, bit-reversed
// output: slot j holds a(psi^{2 brv(j) + 1}).  Inverse: Gentleman-Sande with
// psi^{-brv}, bit-reversed input, natural output, times N^{-1}.
//
// A limb of N = N1 * N2 words (N2 = 256) is transformed in two passes through
// shared memory:
//   columns: the log2(N1) stages whose butterfly distance is a multiple of N2
//            (the element set r*N2 + c, r < N1, for a fixed column c); a CTA
//            stages COLS adjacent columns so that every global access is a
//            full 128-byte line;
//   rows:    the log2(N2) stages inside contiguous runs of N2 words.
// Butterflies use Harvey's lazy reduction: forward values stay in [0, 4q),
// inverse values in [0, 2q), with q < 2^61.
#include "context.h"

namespace hetal {

namespace {

constexpr int N2 = 256;
constexpr int LOG_N2 = 8;
constexpr int COLS = 16;          // columns per CTA in the column pass
constexpr int ROWS = 8;           // rows of N2 per CTA in the row pass
constexpr int THREADS = 256;

__device__ __forceinline__ void ct_bfly(u64 &x, u64 &y, u64 w, u64 wp, u64 q, u64 two_q)
{
    u64 a = x >= two_q ? x - two_q : x;
    u64 t = mul_shoup_lazy(y, w, wp, q);
    x = a + t;
    y = a - t + two_q;
}

__device__ __forceinline__ void gs_bfly(u64 &x, u64 &y, u64 w, u64 wp, u64 q, u64 two_q)
{
    u64 s = x + y;
    s = s >= two_q ? s - two_q : s;
    u64 d = x - y + two_q;
    x = s;
    y = mul_shoup_lazy(d, w, wp, q);
}

// Forward, column pass: stages m = 1 .. N1/2.
__global__ void __launch_bounds__(THREADS) ntt_fwd_cols(PolyBatch b, LimbMap mods, LimbMap pos,
                                                        const ModConst *__restrict__ mc,
                                                        const u64 *__restrict__ psi,
                                                        const u64 *__restrict__ psi_sh, int logN)
{
    extern __shared__ u64 sm[];
    const int N = 1 << logN;
    const int N1 = N >> LOG_N2;
    const int l = blockIdx.y;
    const int midx = mods.idx[l];
    const u64 q = mc[midx].q, two_q = 2 * q;
    u64 *base = b.ptr + (size_t)blockIdx.z * b.stride + (size_t)pos.idx[l] * N;
    const int c0 = blockIdx.x * COLS;
    const u64 *tw = psi + (size_t)midx * N;
    const u64 *tws = psi_sh + (size_t)midx * N;
    const int total = N1 * COLS;
    for (int i = threadIdx.x; i < total; i += THREADS) {
        int r = i / COLS, cc = i % COLS;
        sm[i] = base[(size_t)r * N2 + c0 + cc];
    }
    __syncthreads();
    for (int m = 1, tr = N1 >> 1; m < N1; m <<= 1, tr >>= 1) {
        for (int i = threadIdx.x; i < (N1 >> 1) * COLS; i += THREADS) {
            int bi = i / COLS, cc = i % COLS;
            int grp = bi / tr;
            int r = grp * 2 * tr + (bi % tr);
            u64 w = tw[m + grp], wp = tws[m + grp];
            u64 x = sm[r * COLS + cc], y = sm[(r + tr) * COLS + cc];
            ct_bfly(x, y, w, wp, q, two_q);
            sm[r * COLS + cc] = x;
            sm[(r + tr) * COLS + cc] = y;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < total; i += THREADS) {
        int r = i / COLS, cc = i % COLS;
        base[(size_t)r * N2 + c0 + cc] = sm[i];
    }
}

// Forward, row pass: stages m = N1 .. N/2; final reduction to [0, q).
__global__ void __launch_bounds__(THREADS) ntt_fwd_rows(PolyBatch b, LimbMap mods, LimbMap pos,
                                                        const ModConst *__restrict__ mc,
                                                        const u64 *__restrict__ psi,
                                                        const u64 *__restrict__ psi_sh, int logN)
{
    __shared__ u64 sm[ROWS * N2];
    const int N = 1 << logN;
    const int N1 = N >> LOG_N2;
    const int l = blockIdx.y;
    const int midx = mods.idx[l];
    const u64 q = mc[midx].q, two_q = 2 * q;
    const int row0 = blockIdx.x * ROWS;
    const int nrows = min(ROWS, N1 - row0);
    u64 *base = b.ptr + (size_t)blockIdx.z * b.stride + (size_t)pos.idx[l] * N + (size_t)row0 * N2;
    const u64 *tw = psi + (size_t)midx * N;
    const u64 *tws = psi_sh + (size_t)midx * N;
    const int total = nrows * N2;
    for (int i = threadIdx.x; i < total; i += THREADS) sm[i] = base[i];
    __syncthreads();
    for (int m = N1, t = N2 >> 1; t >= 1; m <<= 1, t >>= 1) {
        for (int i = threadIdx.x; i < total / 2; i += THREADS) {
            int rr = i / (N2 / 2), k = i % (N2 / 2);
            int lg = k / t;
            int j = rr * N2 + lg * 2 * t + (k % t);
            int grp = (row0 + rr) * (N2 / (2 * t)) + lg;     // global group index
            u64 w = tw[m + grp], wp = tws[m + grp];
            u64 x = sm[j], y = sm[j + t];
            ct_bfly(x, y, w, wp, q, two_q);
            sm[j] = x;
            sm[j + t] = y;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < total; i += THREADS) {
        u64 v = sm[i];
        v = v >= two_q ? v - two_q : v;
        v = v >= q ? v - q : v;
        base[i] = v;
    }
}

// Inverse, row pass: GS stages with t = 1 .. N2/2 (h = N/2 .. N1).
__global__ void __launch_bounds__(THREADS) ntt_inv_rows(PolyBatch b, LimbMap mods, LimbMap pos,
                                                        const ModConst *__restrict__ mc,
                                                        const u64 *__restrict__ ipsi,
                                                        const u64 *__restrict__ ipsi_sh, int logN)
{
    __shared__ u64 sm[ROWS * N2];
    const int N = 1 << logN;
    const int N1 = N >> LOG_N2;
    const int l = blockIdx.y;
    const int midx = mods.idx[l];
    const u64 q = mc[midx].q, two_q = 2 * q;
    const int row0 = blockIdx.x * ROWS;
    const int nrows = min(ROWS, N1 - row0);
    u64 *base = b.ptr + (size_t)blockIdx.z * b.stride + (size_t)pos.idx[l] * N + (size_t)row0 * N2;
    const u64 *tw = ipsi + (size_t)midx * N;
    const u64 *tws = ipsi_sh + (size_t)midx * N;
    const int total = nrows * N2;
    for (int i = threadIdx.x; i < total; i += THREADS) sm[i] = base[i];
    __syncthreads();
    for (int t = 1, h = N >> 1; t < N2; t <<= 1, h >>= 1) {
        for (int i = threadIdx.x; i < total / 2; i += THREADS) {
            int rr = i / (N2 / 2), k = i % (N2 / 2);
            int lg = k / t;
            int j = rr * N2 + lg * 2 * t + (k % t);
            int grp = (row0 + rr) * (N2 / (2 * t)) + lg;
            u64 w = tw[h + grp], wp = tws[h + grp];
            u64 x = sm[j], y = sm[j + t];
            gs_bfly(x, y, w, wp, q, two_q);
            sm[j] = x;
            sm[j + t] = y;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < total; i += THREADS) base[i] = sm[i];
}

// Inverse, column pass: GS stages with row distance tr = 1 .. N1/2, then N^{-1}.
__global__ void __launch_bounds__(THREADS) ntt_inv_cols(PolyBatch b, LimbMap mods, LimbMap pos,
                                                        const ModConst *__restrict__ mc,
                                                        const u64 *__restrict__ ipsi,
                                                        const u64 *__restrict__ ipsi_sh,
                                                        const u64 *__restrict__ ninv,
                                                        const u64 *__restrict__ ninv_sh, int logN)
{
    extern __shared__ u64 sm[];
    const int N = 1 << logN;
    const int N1 = N >> LOG_N2;
    const int l = blockIdx.y;
    const int midx = mods.idx[l];
    const u64 q = mc[midx].q, two_q = 2 * q;
    u64 *base = b.ptr + (size_t)blockIdx.z * b.stride + (size_t)pos.idx[l] * N;
    const int c0 = blockIdx.x * COLS;
    const u64 *tw = ipsi + (size_t)midx * N;
    const u64 *tws = ipsi_sh + (size_t)midx * N;
    const int total = N1 * COLS;
    for (int i = threadIdx.x; i < total; i += THREADS) {
        int r = i / COLS, cc = i % COLS;
        sm[i] = base[(size_t)r * N2 + c0 + cc];
    }
    __syncthreads();
    for (int tr = 1, h = N1 >> 1; tr < N1; tr <<= 1, h >>= 1) {
        for (int i = threadIdx.x; i < (N1 >> 1) * COLS; i += THREADS) {
            int bi = i / COLS, cc = i % COLS;
            int grp = bi / tr;
            int r = grp * 2 * tr + (bi % tr);
            u64 w = tw[h + grp], wp = tws[h + grp];
            u64 x = sm[r * COLS + cc], y = sm[(r + tr) * COLS + cc];
            gs_bfly(x, y, w, wp, q, two_q);
            sm[r * COLS + cc] = x;
            sm[(r + tr) * COLS + cc] = y;
        }
        __syncthreads();
    }
    const u64 ni = ninv[midx], nis = ninv_sh[midx];
    for (int i = threadIdx.x; i < total; i += THREADS) {
        int r = i / COLS, cc = i % COLS;
        base[(size_t)r * N2 + c0 + cc] = mul_shoup(sm[i], ni, nis, q);
    }
}

}  // namespace

void ntt_forward(Context &c, PolyBatch b, const LimbMap &mods, const LimbMap &pos)
{
    if (b.count == 0 || mods.n == 0) return;
    const int N = c.p.N, logN = c.p.logN, N1 = N / N2;
    const double limbs = (double)b.count * mods.n;
    if (N1 > 1) {
        dim3 g1(N2 / COLS, mods.n, b.count);
        size_t smem = (size_t)N1 * COLS * sizeof(u64);
        bool t = c.launch_begin("ntt_fwd_cols");
        ntt_fwd_cols<<<g1, THREADS, smem, c.stream>>>(b, mods, pos, c.d_mc, c.d_psi, c.d_psi_sh, logN);
        c.launch_end(t, limbs * (N / 2) * (logN - LOG_N2), limbs * N * 16.0);
    }
    dim3 g2((N1 + ROWS - 1) / ROWS, mods.n, b.count);
    bool t = c.launch_begin("ntt_fwd_rows");
    ntt_fwd_rows<<<g2, THREADS, 0, c.stream>>>(b, mods, pos, c.d_mc, c.d_psi, c.d_psi_sh, logN);
    c.launch_end(t, limbs * (N / 2) * LOG_N2, limbs * N * 16.0);
    HETAL_CUDA_CHECK(cudaGetLastError());
    c.cnt.ntt_limbs += (long long)b.count * mods.n;
    c.cnt.modmul += limbs * (N / 2) * logN;
}

void ntt_inverse(Context &c, PolyBatch b, const LimbMap &mods, const LimbMap &pos)
{
    if (b.count == 0 || mods.n == 0) return;
    const int N = c.p.N, logN = c.p.logN, N1 = N / N2;
    const double limbs = (double)b.count * mods.n;
    dim3 g2((N1 + ROWS - 1) / ROWS, mods.n, b.count);
    bool t = c.launch_begin("ntt_inv_rows");
    ntt_inv_rows<<<g2, THREADS, 0, c.stream>>>(b, mods, pos, c.d_mc, c.d_ipsi, c.d_ipsi_sh, logN);
    c.launch_end(t, limbs * (N / 2) * LOG_N2, limbs * N * 16.0);
    dim3 g1(N2 / COLS, mods.n, b.count);
    size_t smem = (size_t)N1 * COLS * sizeof(u64);
    t = c.launch_begin("ntt_inv_cols");
    ntt_inv_cols<<<g1, THREADS, smem, c.stream>>>(b, mods, pos, c.d_mc, c.d_ipsi, c.d_ipsi_sh, c.d_ninv,
                                                  c.d_ninv_sh, logN);
    c.launch_end(t, limbs * ((N / 2) * (logN - LOG_N2) + N), limbs * N * 16.0);
    HETAL_CUDA_CHECK(cudaGetLastError());
    c.cnt.ntt_limbs += (long long)b.count * mods.n;
    c.cnt.modmul += limbs * ((N / 2) * logN + N);
}

}  // namespace hetal
