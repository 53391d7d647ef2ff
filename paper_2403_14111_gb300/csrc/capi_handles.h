// capi_handles.h -- definitions of the opaque handle types of include/hetal.h.
#pragma once
#include "../../include/hetal.h"
#include "matmul.h"
#include "runtime.h"
#include "server.h"

struct hetal_ctx {
    hetal::Context *c = nullptr;
    std::string err;
    // worker pools by size, created by the first call that asks for that many
    // workers and kept until the context is destroyed (their outputs live on them)
    std::map<int, std::unique_ptr<hetal::WorkerPool>> pools;
    hetal::TileTuner tuner;
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
struct hetal_mat {
    hetal_ctx *owner = nullptr;
    hetal::Mat m;
};
struct hetal_ptset {
    hetal::PtSet set;
};
struct hetal_server {
    hetal_ctx *parent = nullptr;
    std::unique_ptr<hetal::Server> s;
};
