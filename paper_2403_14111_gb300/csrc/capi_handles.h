// capi_handles.h -- definitions of the opaque handle types of include/hetal.h.
#pragma once
#include "../../include/hetal.h"
#include "matmul.h"

struct hetal_ctx {
    hetal::Context *c = nullptr;
    std::string err;
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
