// noalloc.cu -- a rescale entry point that allocates no device memory.
//
// Some callers cannot let a library allocate device memory once they are
// running: a serving process that sizes its whole device-memory budget at
// start-up and refuses later allocations (so that a burst of requests can
// never fail half-way on an out-of-memory error), or a host application that
// owns every device buffer itself and only lends pointers to the library.
// hetal_rescale_noalloc serves them: the caller passes the input and output
// buffers, and the intermediate limbs live in one file-scope device array that
// is part of the library image.
#include <map>
#include <mutex>

#include "capi_handles.h"

using namespace hetal;

namespace {

// 2^21 words = 16 MiB, held by every GPU that loads the library until exit.
constexpr size_t kScratchWords = (size_t)1 << 21;
static __device__ __align__(256) u64 g_rescale_scratch[kScratchWords];

std::mutex g_mu;
std::map<int, u64 *> g_scratch_addr;   // device -> device address of g_rescale_scratch

}  // namespace

// The array's name in host code is only a host-side stand-in; its device
// address is looked up once per device, with that device current.  Every
// context does this when it is created (hetal_ctx_create), so the lookup never
// runs inside a stream capture.
u64 *noalloc_scratch_address(int device)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_scratch_addr.find(device);
    if (it != g_scratch_addr.end()) return it->second;
    int prev = 0;
    HETAL_CUDA_CHECK(cudaGetDevice(&prev));
    HETAL_CUDA_CHECK(cudaSetDevice(device));
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_rescale_scratch);
    cudaSetDevice(prev);
    if (e != cudaSuccess) throw CudaError(e, "cudaGetSymbolAddress(g_rescale_scratch)", __FILE__, __LINE__);
    g_scratch_addr[device] = (u64 *)ptr;
    return (u64 *)ptr;
}

namespace {

LimbMap one_limb(int idx)
{
    LimbMap m;
    m.n = 1;
    m.idx[0] = (unsigned char)idx;
    return m;
}

}  // namespace

extern "C" int hetal_rescale_noalloc(hetal_ctx *ctx, const uint64_t *dev_in, uint64_t *dev_out, int n_ct, int level)
{
    if (!ctx || !dev_in || !dev_out || n_ct < 1) return HETAL_ERR_INVALID_ARG;
    try {
        Context &c = *ctx->c;
        if (level < 1 || level >= c.p.L) throw Error(ERR_LEVEL, "rescale needs a level in [1, L-1]");
        const int N = c.p.N;
        const size_t need = (size_t)2 * n_ct * N * (size_t)(1 + level);
        if (need > kScratchWords)
            throw Error(ERR_INVALID_ARG, "hetal_rescale_noalloc: 2 * n_ct * N * (level + 1) = " + std::to_string(need) +
                                             " words exceeds the static scratch of 2^21 words");
        const size_t in_words = (size_t)2 * n_ct * (level + 1) * N, out_words = (size_t)2 * n_ct * level * N;
        const uint64_t *in_end = dev_in + in_words, *out_end = dev_out + out_words;
        if (dev_out < in_end && dev_in < out_end)   // the last pass reads the input while it writes the output
            throw Error(ERR_INVALID_ARG, "hetal_rescale_noalloc: dev_out overlaps dev_in");
        u64 *scratch = noalloc_scratch_address(c.device);
        const int cnt = 2 * n_ct;
        PolyBatch in{const_cast<u64 *>(dev_in), cnt, (size_t)(level + 1) * N};
        PolyBatch out{dev_out, cnt, (size_t)level * N};
        PolyBatch top{scratch, cnt, (size_t)N};
        PolyBatch spread{scratch + (size_t)cnt * N, cnt, (size_t)level * N};
        // top limb to coefficients, centred and spread to the lower moduli, back to
        // the NTT domain, then (x_i - spread_i) * q_level^{-1}; every scratch word
        // read is written first in the same call.
        k_copy(c, top, PolyBatch{const_cast<u64 *>(dev_in) + (size_t)level * N, cnt, in.stride}, 1);
        ntt_inverse(c, top, one_limb(level), identity_pos(1));
        k_rescale_spread(c, spread, top, level);
        ntt_forward(c, spread, c.q_map(level - 1), identity_pos(level));
        k_rescale_finish(c, out, in, spread, level);
        return HETAL_OK;
    } catch (const Error &e) {
        ctx->err = e.what();
        if (ctx->c->recording) ctx->rec_failed = true;   // the graph would be incomplete
        if (e.code == ERR_CUDA) cudaGetLastError();
        return e.code;
    } catch (const std::exception &e) {
        ctx->err = e.what();
        if (ctx->c->recording) ctx->rec_failed = true;
        return HETAL_ERR_INVALID_ARG;
    }
}
