// ntt32.cu -- negacyclic NTT on 32-bit words (primes below 2^30), for the choice
// of the RNS word size by measurement.
//
// The library computes on 64-bit words (primes of 50-61 bits).  Its alternative is
// 32-bit words: a modular product is one 32 x 32-bit high product and two low
// products instead of a 64-bit Shoup product's dozen 32-bit multiplies, but a
// modulus of the same size needs about twice as many limbs.  This file is that
// alternative's transform, built like the 64-bit one (ntt.cu) so that the two can
// be compared: a limb of N = R * 256 words is transformed in two passes through
// shared memory (the log2 R strided stages, then the 8 stages inside each row of
// 256), 16 words per thread in registers, Harvey's lazy butterflies (values in
// [0, 4q), q < 2^30, so everything fits a 32-bit word), twiddles psi^{brv(i)} with
// their Shoup companions floor(w 2^32 / q).  Forward transform only, natural-order
// input, bit-reversed output: slot j holds a(psi^{2 brv(j) + 1}).
#include "context.h"

#include <algorithm>

namespace hetal {

namespace {

using u32 = uint32_t;
constexpr int LOG_N2 = 8;
constexpr int N2 = 1 << LOG_N2;
constexpr int THREADS = 256;

__device__ __forceinline__ u32 csub32(u32 x, u32 m) { return x >= m ? x - m : x; }

// w y mod q up to one q: y < 2^32, w < q < 2^30, wp = floor(w 2^32 / q); result in [0, 2q)
__device__ __forceinline__ u32 mul_shoup_lazy32(u32 y, u32 w, u32 wp, u32 q)
{
    return w * y - __umulhi(y, wp) * q;
}

__device__ __forceinline__ void ct_bfly32(u32 &x, u32 &y, u32 w, u32 wp, u32 q, u32 two_q)
{
    u32 a = csub32(x, two_q);
    u32 t = mul_shoup_lazy32(y, w, wp, q);
    x = a + t;
    y = a - t + two_q;
}

template <int LOGR>
struct Col32 {
    static constexpr int R = 1 << LOGR;
    static constexpr int LOGE = LOGR < 4 ? LOGR : 4;
    static constexpr int E = 1 << LOGE;
    static constexpr int LOGT = LOGR - LOGE;
    static constexpr int TPC = 1 << LOGT;
    static constexpr int COLS = THREADS / TPC;
};

struct Poly32 {
    u32 *ptr;
    int count;
    size_t stride;   // words between polys
};

// Column pass: the log2 R stages of distance a multiple of 256 (see ntt.cu).
template <int LOGR>
__global__ void __launch_bounds__(THREADS) ntt32_fwd_cols(Poly32 b, const u32 *__restrict__ mods,
                                                          const uint2 *__restrict__ psi, int logN)
{
    using S = Col32<LOGR>;
    extern __shared__ u32 sm32[];
    uint2 *tw = reinterpret_cast<uint2 *>(sm32 + S::R * S::COLS);
    const int N = 1 << logN;
    const int l = blockIdx.y;
    const u32 q = mods[l], two_q = 2 * q;
    u32 *base = b.ptr + (size_t)blockIdx.z * b.stride + (size_t)l * N + blockIdx.x * S::COLS;
    const int cc = threadIdx.x % S::COLS, t = threadIdx.x / S::COLS;
    for (int i = threadIdx.x; i < S::R; i += THREADS) tw[i] = psi[(size_t)l * N + i];
    u32 v[S::E];
#pragma unroll
    for (int j = 0; j < S::E; j++) v[j] = base[(size_t)(t + S::TPC * j) * N2 + cc];
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S::LOGE; s++) {
        const int d = S::E >> (s + 1);
#pragma unroll
        for (int j = 0; j < S::E; j++) {
            if (j & d) continue;
            const uint2 w = tw[(1 << s) + (j >> (S::LOGE - s))];
            ct_bfly32(v[j], v[j + d], w.x, w.y, q, two_q);
        }
    }
    if (S::LOGT > 0) {
#pragma unroll
        for (int j = 0; j < S::E; j++) sm32[(t + S::TPC * j) * S::COLS + cc] = v[j];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < S::E; j++) v[j] = sm32[(S::E * t + j) * S::COLS + cc];
#pragma unroll
        for (int s = S::LOGE; s < LOGR; s++) {
            const int d = 1 << (LOGR - 1 - s);
#pragma unroll
            for (int j = 0; j < S::E; j++) {
                if (j & d) continue;
                const uint2 w = tw[(1 << s) + ((S::E * t + j) >> (LOGR - s))];
                ct_bfly32(v[j], v[j + d], w.x, w.y, q, two_q);
            }
        }
#pragma unroll
        for (int j = 0; j < S::E; j++) base[(size_t)(S::E * t + j) * N2 + cc] = v[j];
    } else {
#pragma unroll
        for (int j = 0; j < S::E; j++) base[(size_t)(t + S::TPC * j) * N2 + cc] = v[j];
    }
}

// Row pass: 16 threads per row of 256, 16 rows per CTA; twiddles in read order (ntt.cu).
constexpr int RPB = THREADS / 16;
constexpr int RS = N2 + N2 / 16;

__global__ void __launch_bounds__(THREADS, 4) ntt32_fwd_rows(Poly32 b, const u32 *__restrict__ mods,
                                                             const uint2 *__restrict__ rowtw, int logN)
{
    __shared__ u32 sm[RPB * RS];
    __shared__ uint2 stw[RPB * 16];
    const int N = 1 << logN;
    const int R = N >> LOG_N2;
    const int l = blockIdx.y;
    const u32 q = mods[l], two_q = 2 * q;
    const int rr = threadIdx.x >> 4, t = threadIdx.x & 15;
    const int row = blockIdx.x * RPB + rr;
    u32 *base = b.ptr + (size_t)blockIdx.z * b.stride + (size_t)l * N;
    const uint2 *tw = rowtw + ((size_t)l * R + row) * 255;
    u32 v[16];
    if (row < R) {
        if (t < 15) stw[rr * 16 + t] = __ldg(tw + t);
        const u32 *src = base + (size_t)row * N2;
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = src[t + 16 * j];
        __syncwarp(0xffffu << (threadIdx.x & 16));
#pragma unroll
        for (int s = 0; s < 4; s++) {
            const int d = 8 >> s;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                if (j & d) continue;
                const uint2 w = stw[rr * 16 + (1 << s) - 1 + (j >> (4 - s))];
                ct_bfly32(v[j], v[j + d], w.x, w.y, q, two_q);
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
                const uint2 w = __ldg(tw + 15 + 16 * ((1 << (s - 4)) - 1 + (j >> (8 - s))) + t);
                ct_bfly32(v[j], v[j + d], w.x, w.y, q, two_q);
            }
        }
#pragma unroll
        for (int j = 0; j < 16; j++) sm[rr * RS + 17 * t + j] = csub32(csub32(v[j], two_q), q);
    }
    __syncthreads();
    if (row < R) {
        u32 *dst = base + (size_t)row * N2;
#pragma unroll
        for (int j = 0; j < 16; j++) dst[t + 16 * j] = sm[rr * RS + t + 17 * j];
    }
}

template <int LOGR>
void launch_cols32(Context &c, Poly32 b, int limbs, const u32 *mods, const uint2 *psi)
{
    using S = Col32<LOGR>;
    const size_t smem = (size_t)S::R * S::COLS * sizeof(u32) + (size_t)S::R * sizeof(uint2);
    static bool attr = false;
    if (!attr) {
        HETAL_CUDA_CHECK(
            cudaFuncSetAttribute(ntt32_fwd_cols<LOGR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    ntt32_fwd_cols<LOGR><<<dim3(N2 / S::COLS, limbs, b.count), THREADS, smem, c.stream>>>(b, mods, psi, c.p.logN);
}

// Register-only loop of the 32-bit lazy butterfly (the ALU ceiling of the 32-bit transform).
__global__ void __launch_bounds__(256) probe_butterfly32(u32 *sink, u32 q, const uint2 *__restrict__ tw, int iters)
{
    u32 x[8], y[8], w[4], wp[4];
    const u32 two_q = 2 * q;
#pragma unroll
    for (int s = 0; s < 4; s++) {
        const uint2 v = tw[1 + s];
        w[s] = v.x;
        wp[s] = v.y;
    }
#pragma unroll
    for (int i = 0; i < 8; i++) {
        x[i] = (threadIdx.x * 8 + i) % q;
        y[i] = (blockIdx.x * 8 + i + 1) % q;
    }
    for (int it = 0; it < iters; it += 4) {
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int i = 0; i < 8; i++) ct_bfly32(x[i], y[i], w[(s + i) & 3], wp[(s + i) & 3], q, two_q);
    }
    u32 acc = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) acc ^= x[i] ^ y[i];
    if (acc == 0x1234567u) sink[blockIdx.x] = acc;   // keeps the loop alive
}

bool prime32(u64 n)
{
    if (n < 2) return false;
    for (u64 b : {2ull, 3ull, 5ull, 7ull, 61ull})
        if (n % b == 0) return n == b;
    u64 d = n - 1;
    int r = 0;
    while (!(d & 1)) {
        d >>= 1;
        r++;
    }
    for (u64 b : {2ull, 7ull, 61ull}) {   // decides every n < 4,759,123,141
        u64 x = host_powmod(b, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int k = 1; k < r && comp; k++) {
            x = host_mulmod(x, x, n);
            if (x == n - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}

}  // namespace

// Device tables of the 32-bit transform for `limbs` primes (made on first use).
struct Ntt32Tables {
    int limbs = 0;
    std::vector<u32> mod, psi;   // primes (largest below 2^30, 1 mod 2N, descending), 2N-th roots
    u32 *d_mod = nullptr;
    uint2 *d_psi = nullptr, *d_rowtw = nullptr;
    ~Ntt32Tables()
    {
        cudaFree(d_mod);
        cudaFree(d_psi);
        cudaFree(d_rowtw);
    }
};

static Ntt32Tables &ntt32_tables(Context &c, int limbs)
{
    if (limbs < 1 || limbs > HETAL_MAX_MODULI) throw Error(ERR_INVALID_ARG, "32-bit transform: 1..128 limbs");
    auto *t = static_cast<Ntt32Tables *>(c.ntt32.get());
    if (t && t->limbs >= limbs) return *t;
    const int N = c.p.N, logN = c.p.logN, R = N >> LOG_N2;
    auto nt = std::make_shared<Ntt32Tables>();
    nt->limbs = limbs;
    const u64 two_n = 2 * (u64)N;
    for (u64 q = ((1ull << 30) - 1) / two_n * two_n + 1; (int)nt->mod.size() < limbs && q > two_n; q -= two_n)
        if (prime32(q)) nt->mod.push_back((u32)q);
    if ((int)nt->mod.size() < limbs) throw Error(ERR_INVALID_ARG, "32-bit transform: not enough primes");
    std::vector<uint2> psi((size_t)limbs * N), rt((size_t)limbs * R * 255);
    for (int l = 0; l < limbs; l++) {
        const u64 q = nt->mod[l];
        u64 root = 0;
        for (u64 g = 3;; g += 2) {
            root = host_powmod(g, (q - 1) / two_n, q);
            if (host_powmod(root, two_n / 2, q) == q - 1) break;
        }
        nt->psi.push_back((u32)root);
        std::vector<u64> pw(N);
        pw[0] = 1;
        for (int i = 1; i < N; i++) pw[i] = host_mulmod(pw[i - 1], root, q);
        for (int i = 0; i < N; i++) {
            unsigned r = 0;
            for (int bb = 0; bb < logN; bb++)
                if (i & (1 << bb)) r |= 1u << (logN - 1 - bb);
            psi[(size_t)l * N + i] = make_uint2((u32)pw[r], (u32)((pw[r] << 32) / q));
        }
        for (int r = 0; r < R; r++) {   // the row pass's order (see ntt.cu)
            uint2 *o = &rt[((size_t)l * R + r) * 255];
            for (int st = 0; st < 4; st++)
                for (int k = 0; k < (1 << st); k++)
                    o[(1 << st) - 1 + k] = psi[(size_t)l * N + ((size_t)R << st) + ((size_t)r << st) + k];
            for (int st = 4; st < 8; st++)
                for (int k = 0; k < (1 << (st - 4)); k++)
                    for (int th = 0; th < 16; th++)
                        o[15 + 16 * ((1 << (st - 4)) - 1 + k) + th] =
                            psi[(size_t)l * N + ((size_t)R << st) + ((size_t)r << st) + ((size_t)th << (st - 4)) + k];
        }
    }
    HETAL_CUDA_CHECK(cudaMalloc(&nt->d_mod, sizeof(u32) * limbs));
    HETAL_CUDA_CHECK(cudaMalloc(&nt->d_psi, sizeof(uint2) * psi.size()));
    HETAL_CUDA_CHECK(cudaMalloc(&nt->d_rowtw, sizeof(uint2) * rt.size()));
    HETAL_CUDA_CHECK(cudaMemcpy(nt->d_mod, nt->mod.data(), sizeof(u32) * limbs, cudaMemcpyHostToDevice));
    HETAL_CUDA_CHECK(cudaMemcpy(nt->d_psi, psi.data(), sizeof(uint2) * psi.size(), cudaMemcpyHostToDevice));
    HETAL_CUDA_CHECK(cudaMemcpy(nt->d_rowtw, rt.data(), sizeof(uint2) * rt.size(), cudaMemcpyHostToDevice));
    c.sync();
    c.ntt32 = nt;
    return *nt;
}

std::vector<uint32_t> ntt32_moduli(Context &c, int limbs, std::vector<uint32_t> *roots)
{
    Ntt32Tables &t = ntt32_tables(c, limbs);
    if (roots) *roots = std::vector<uint32_t>(t.psi.begin(), t.psi.begin() + limbs);
    return std::vector<uint32_t>(t.mod.begin(), t.mod.begin() + limbs);
}

void ntt32_forward(Context &c, uint32_t *polys, int n_polys, int limbs)
{
    if (n_polys < 1) return;
    Ntt32Tables &t = ntt32_tables(c, limbs);
    const int N = c.p.N, logN = c.p.logN, R = N >> LOG_N2;
    Poly32 b{polys, n_polys, (size_t)limbs * N};
    const double lb = (double)n_polys * limbs;
    bool tm = c.launch_begin("ntt32_fwd_cols");
    switch (logN - LOG_N2) {
    case 2: launch_cols32<2>(c, b, limbs, t.d_mod, t.d_psi); break;
    case 3: launch_cols32<3>(c, b, limbs, t.d_mod, t.d_psi); break;
    case 4: launch_cols32<4>(c, b, limbs, t.d_mod, t.d_psi); break;
    case 5: launch_cols32<5>(c, b, limbs, t.d_mod, t.d_psi); break;
    case 6: launch_cols32<6>(c, b, limbs, t.d_mod, t.d_psi); break;
    case 7: launch_cols32<7>(c, b, limbs, t.d_mod, t.d_psi); break;
    case 8: launch_cols32<8>(c, b, limbs, t.d_mod, t.d_psi); break;
    default: throw Error(ERR_INVALID_ARG, "unsupported ring degree");
    }
    HETAL_CUDA_CHECK(cudaGetLastError());
    c.launch_end(tm, lb * (N / 2) * (logN - LOG_N2), lb * N * 8.0);
    tm = c.launch_begin("ntt32_fwd_rows");
    ntt32_fwd_rows<<<dim3((R + RPB - 1) / RPB, limbs, n_polys), THREADS, 0, c.stream>>>(b, t.d_mod, t.d_rowtw, logN);
    HETAL_CUDA_CHECK(cudaGetLastError());
    c.launch_end(tm, lb * (N / 2) * LOG_N2, lb * N * 8.0);
}

double probe_butterfly32_rate(Context &c, int iters, int blocks_per_sm)
{
    Ntt32Tables &t = ntt32_tables(c, 1);
    const int blocks = c.sm_count * blocks_per_sm;
    u32 *sink = (u32 *)c.alloc_bytes(sizeof(u32) * blocks);
    iters = std::max(4, iters / 4 * 4);
    cudaEvent_t a, e;
    HETAL_CUDA_CHECK(cudaEventCreate(&a));
    HETAL_CUDA_CHECK(cudaEventCreate(&e));
    probe_butterfly32<<<blocks, 256, 0, c.stream>>>(sink, t.mod[0], t.d_psi, iters / 40 * 4);   // warm-up
    HETAL_CUDA_CHECK(cudaEventRecord(a, c.stream));
    probe_butterfly32<<<blocks, 256, 0, c.stream>>>(sink, t.mod[0], t.d_psi, iters);
    HETAL_CUDA_CHECK(cudaEventRecord(e, c.stream));
    HETAL_CUDA_CHECK(cudaGetLastError());
    HETAL_CUDA_CHECK(cudaEventSynchronize(e));
    float ms = 0;
    HETAL_CUDA_CHECK(cudaEventElapsedTime(&ms, a, e));
    cudaEventDestroy(a);
    cudaEventDestroy(e);
    c.free_bytes(sink);
    return (double)blocks * 256 * 8 * (double)iters / (ms * 1e-3);
}

}  // namespace hetal
