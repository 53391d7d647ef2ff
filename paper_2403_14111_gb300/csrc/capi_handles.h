// capi_handles.h -- definitions of the opaque handle types of include/hetal.h.
#pragma once
#include <functional>
#include <set>
#include "../../include/hetal.h"
#include "matmul.h"
#include "runtime.h"
#include "server.h"

// Device address of the allocation-free rescale's static scratch array on `device`
// (looked up once per device; noalloc.cu).
uint64_t *noalloc_scratch_address(int device);

struct hetal_ctx {
    hetal::Context *c = nullptr;
    std::string err;
    // worker pools by size, created by the first call that asks for that many
    // workers and kept until the context is destroyed (their outputs live on them)
    std::map<int, std::unique_ptr<hetal::WorkerPool>> pools;
    hetal::TileTuner tuner;
    // graph recording (hetal_graph_begin .. hetal_graph_end): the matrices created
    // meanwhile and still alive, whether a call failed, the launch count at the start
    std::set<hetal_mat *> recorded;
    bool rec_failed = false;
    long long rec_launches0 = 0;
    // handles made before the recording and released during it: the graph may
    // read them at every launch, so they are released with the graph
    std::vector<std::function<void()>> rec_releases;
    hetal::WorkerPool &pool(int workers)
    {
        auto &p = pools[workers];
        if (!p) p.reset(new hetal::WorkerPool(c->p, c->device, workers));
        return *p;
    }
    ~hetal_ctx()
    {
        pools.clear();
        delete c;
    }
};
struct hetal_sk {
    hetal_ctx *owner = nullptr;
    hetal::SecretKey *sk = nullptr;
};
struct hetal_evk {
    hetal_ctx *owner = nullptr;
    hetal::EvalKeys *ek = nullptr;
};
// A matrix handle carries a marker that its destructor clears, so that a handle
// passed again after hetal_mat_free is refused (HETAL_ERR_INVALID_ARG) instead of
// being dereferenced, as long as its memory has not been reused.
constexpr uint64_t kMatLive = 0x686574616c6d6174ull;
struct hetal_mat {
    uint64_t live = kMatLive;
    hetal_ctx *owner = nullptr;
    hetal::Mat m;
    ~hetal_mat() { live = 0; }
};
inline bool mat_live(const hetal_mat *p) { return p && p->live == kMatLive; }
// An instantiated CUDA graph of recorded calls.  It shares ownership of its
// output matrices' device memory with their handles, so that no output is freed
// while a later launch may still write it.
struct hetal_graph {
    hetal_ctx *ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
    std::vector<std::shared_ptr<uint64_t>> outputs;
    std::vector<std::function<void()>> releases;
};
struct hetal_ptset {
    hetal::PtSet set;
};
// A plaintext kept on the device (NTT domain, normal and Montgomery form).
constexpr uint64_t kPlainLive = 0x686574616c706c6eull;
struct hetal_plain {
    uint64_t live = kPlainLive;
    hetal_ctx *owner = nullptr;
    hetal::Plain pt;
    ~hetal_plain() { live = 0; }
};
inline bool plain_live(const hetal_plain *p) { return p && p->live == kPlainLive; }
struct hetal_server {
    hetal_ctx *parent = nullptr;
    std::unique_ptr<hetal::Server> s;
};
