// capi.cu -- the extern "C" boundary (include/hetal.h).  Every entry point
// validates its arguments, runs on the context's stream and turns exceptions
// into status codes with a message kept on the context.
#include "capi_handles.h"

#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <tuple>

using namespace hetal;

static_assert(HETAL_MAX_MODULI == HETAL_MAX_MODULI_ABI, "the header's modulus limit and the kernels' differ");

namespace {

thread_local std::string g_err;

template <class F>
int guard(hetal_ctx *ctx, F &&f)
{
    try {
        f();
        return HETAL_OK;
    } catch (const Error &e) {
        if (ctx) ctx->err = e.what();
        if (ctx && ctx->c && ctx->c->recording) ctx->rec_failed = true;   // the graph would be incomplete
        g_err = e.what();
        if (e.code == ERR_CUDA) cudaGetLastError();
        return e.code;
    } catch (const std::exception &e) {
        if (ctx) ctx->err = e.what();
        if (ctx && ctx->c && ctx->c->recording) ctx->rec_failed = true;
        g_err = e.what();
        return HETAL_ERR_INVALID_ARG;
    }
}

// Calls that read or write host memory synchronously, create keys or run on
// other streams cannot be recorded into a graph; they are refused before any
// device work while a recording is open.
void idle(hetal_ctx *ctx)
{
    if (ctx->c->recording) throw Error(ERR_RECORDING, "this call cannot be recorded into a graph");
}

// Releasing a handle made before an open recording is deferred until the graph
// is freed (or the recording fails): the graph may read it at every launch.
bool defer_release(hetal_ctx *ctx, std::function<void()> f)
{
    if (!ctx || !ctx->c->recording) return false;
    ctx->rec_releases.push_back(std::move(f));
    return true;
}

// Host buffers a recorded copy reads or writes must stay valid and be pinned
// (page-locked): the graph copies from / to them at every launch.
void need_pinned(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) cudaGetLastError();
    if (a.type != cudaMemoryTypeHost)
        throw Error(ERR_RECORDING, "a recorded host copy needs pinned (page-locked) host memory");
}

void need(bool cond, const char *msg)
{
    if (!cond) throw Error(ERR_INVALID_ARG, msg);
}

hetal_mat *wrap(hetal_ctx *ctx, Mat &&m)
{
    hetal_mat *h = new hetal_mat();
    h->owner = ctx;
    h->m = std::move(m);
    if (ctx->c->recording) ctx->recorded.insert(h);
    return h;
}

Mat like(const Mat &src, CtBatch &&cts)
{
    Mat m;
    m.cts = std::move(cts);
    m.m = src.m;
    m.n = src.n;
    m.rows = src.rows;
    m.cols = src.cols;
    m.s0 = src.s0;
    m.s1 = src.s1;
    return m;
}

// Imported residues must be canonical (each below its limb's modulus): the kernels'
// lazy reductions assume it.  Checked on the device; the call waits for the answer.
void check_residues(Context &c, const u64 *d_coeff, int n, int lv)
{
    unsigned *bad = (unsigned *)c.alloc_bytes(sizeof(unsigned));
    unsigned h = 0;
    try {
        HETAL_CUDA_CHECK(cudaMemsetAsync(bad, 0, sizeof(unsigned), c.stream));
        k_check_range(c, PolyBatch{const_cast<u64 *>(d_coeff), 2 * n, (size_t)(lv + 1) * c.p.N}, c.q_map(lv), bad);
        HETAL_CUDA_CHECK(cudaMemcpyAsync(&h, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
        c.sync();
    } catch (...) {
        c.free_bytes(bad);
        throw;
    }
    c.free_bytes(bad);
    if (h) throw Error(ERR_INVALID_ARG, "an imported residue is not below its limb's modulus");
}

void check_desc(const Context &c, const hetal_mat_desc *d)
{
    need(d != nullptr, "desc is NULL");
    if (d->m < 1 || d->n < 1) throw Error(ERR_SHAPE, "block grid must be at least 1 x 1");
    if (d->s0 < 1 || d->s1 < 1 || (long long)d->s0 * d->s1 != c.p.N / 2)
        throw Error(ERR_SHAPE, "block shape must satisfy s0 * s1 = N/2");
    if (d->level < 0 || d->level >= c.p.L) throw Error(ERR_LEVEL, "level out of range");
}

// Groups of instances that can share launches (see hetal_run_pairs_batched).
void run_groups(Context &c, const EvalKeys &ek, const hetal_pair_job *jobs, size_t n, int flags, std::vector<Mat> &abt,
                std::vector<Mat> &atb)
{
    auto bits = [](double x) {
        u64 b;
        std::memcpy(&b, &x, sizeof b);
        return b;
    };
    using Key = std::tuple<int, int, int, int, u64, u64, int>;
    std::map<Key, std::vector<size_t>> ga, gb;
    for (size_t i = 0; i < n; i++) {
        const hetal_pair_job &j = jobs[i];
        const int f = j.flags >= 0 ? j.flags : flags;
        const Mat &x = j.x->m, &w = j.wbar->m, &u = j.a_under->m, &b = j.b->m;
        // scales within 1e-9 of each other compare equal only when their bits do: a group
        // that would mix two nearly equal scales is split, never refused
        ga[Key(x.s0, f, x.cts.lv, w.cts.lv, bits(x.cts.scale), bits(w.cts.scale), 0)].push_back(i);
        const bool rl_small = u.cts.lv >= b.cts.lv && j.c == 2;   // RotLeft branch, c/2 = 1: another level
        gb[Key(b.s0, f, u.cts.lv, b.cts.lv, bits(u.cts.scale), bits(b.cts.scale), rl_small)].push_back(i);
    }
    // A group's temporaries grow with its blocks: DiagABT holds B_cplx and its extended digits
    // (about 5.5 ciphertexts per B-bar block at the top level), DiagATB a rearranged copy of B
    // and its products (about 2 per block of B).  Groups are cut so that these stay within the
    // context's batch budget; an instance larger than the budget forms a group of its own.
    const Params &p = c.p;
    auto ct_bytes = [&](int lv) { return (double)2 * (lv + 1) * p.N * sizeof(u64); };
    auto cut = [&](const std::vector<size_t> &ids, const std::function<double(size_t)> &bytes) {
        std::vector<std::vector<size_t>> parts(1);
        double acc = 0;
        for (size_t i : ids) {
            const double b = bytes(i);
            if (!parts.back().empty() && acc + b > (double)c.batch_bytes) {
                parts.emplace_back();
                acc = 0;
            }
            parts.back().push_back(i);
            acc += b;
        }
        return parts;
    };
    for (auto &kv : ga) {
        for (auto &ids : cut(kv.second, [&](size_t i) {
                 return 5.5 * jobs[i].wbar->m.n * ct_bytes(jobs[i].wbar->m.cts.lv);
             })) {
            std::vector<AbtJob> js;
            for (size_t i : ids) js.push_back(AbtJob{&jobs[i].x->m, &jobs[i].wbar->m, jobs[i].c, jobs[i].t_abt});
            std::vector<Mat> r = diag_abt_group(c, ek, js, nullptr, std::get<1>(kv.first));
            for (size_t q = 0; q < ids.size(); q++) abt[ids[q]] = std::move(r[q]);
        }
    }
    for (auto &kv : gb) {
        for (auto &ids : cut(kv.second, [&](size_t i) {
                 return 2.0 * jobs[i].b->m.m * jobs[i].b->m.n * ct_bytes(jobs[i].b->m.cts.lv);
             })) {
            std::vector<AtbJob> js;
            for (size_t i : ids) js.push_back(AtbJob{&jobs[i].a_under->m, &jobs[i].b->m, jobs[i].c, jobs[i].t_atb});
            std::vector<Mat> r = diag_atb_group(c, ek, js, nullptr, std::get<1>(kv.first));
            for (size_t q = 0; q < ids.size(); q++) atb[ids[q]] = std::move(r[q]);
        }
    }
}

}  // namespace

extern "C" {

int hetal_ctx_create(const hetal_params *prm, int device, void *cuda_stream, hetal_ctx **out)
{
    if (!prm || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    hetal_ctx *h = new hetal_ctx();
    int st = guard(nullptr, [&] {
        Params p = make_params(prm->log_n, prm->q0_bits, prm->n_rescale, prm->rescale_bits, prm->n_special,
                               prm->special_bits, prm->alpha, prm->hamming_weight, prm->scale, prm->n_upper,
                               prm->upper_bits);
        h->c = new Context(p, device, (cudaStream_t)cuda_stream);
        noalloc_scratch_address(device);   // hetal_rescale_noalloc's scratch address, outside any capture
    });
    if (st != HETAL_OK) {
        delete h;
        return st;
    }
    *out = h;
    return HETAL_OK;
}

void hetal_ctx_destroy(hetal_ctx *ctx)
{
    if (!ctx) return;
    delete ctx;   // worker contexts first, then the main context
}

const char *hetal_last_error(const hetal_ctx *ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

int hetal_ctx_moduli(const hetal_ctx *ctx, uint64_t *host_out, int cap)
{
    if (!ctx || !host_out) return HETAL_ERR_INVALID_ARG;
    const Params &p = ctx->c->p;
    int tot = p.L + p.K;
    if (cap < tot) return HETAL_ERR_INVALID_ARG;
    for (int i = 0; i < tot; i++) host_out[i] = p.mod[i];
    return tot;
}

int hetal_ctx_info(const hetal_ctx *ctx, int *n, int *l, int *k)
{
    if (!ctx) return HETAL_ERR_INVALID_ARG;
    if (n) *n = ctx->c->p.N;
    if (l) *l = ctx->c->p.L;
    if (k) *k = ctx->c->p.K;
    return HETAL_OK;
}

int hetal_ctx_sync(hetal_ctx *ctx)
{
    if (!ctx) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        ctx->c->sync();
    });
}

int hetal_ctx_set_batch_bytes(hetal_ctx *ctx, size_t bytes)
{
    if (!ctx || bytes < ((size_t)1 << 20)) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        ctx->c->batch_bytes = bytes;
    });
}

int hetal_ctx_set_row_group(hetal_ctx *ctx, int polys)
{
    if (!ctx || polys < 1 || polys > 64) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        ctx->c->row_group = polys;
    });
}

int hetal_counters_get(const hetal_ctx *ctx, hetal_counters *out)
{
    if (!ctx || !out) return HETAL_ERR_INVALID_ARG;
    Counters k = ctx->c->cnt;   // the main context plus every worker context
    for (auto &kv : ctx->pools) {
        Counters w = kv.second->counters();
        k.cmult += w.cmult;
        k.mult += w.mult;
        k.rot += w.rot;
        k.conj += w.conj;
        k.keyswitch += w.keyswitch;
        k.modup_digits += w.modup_digits;
        k.ntt_limbs += w.ntt_limbs;
        k.rescale += w.rescale;
        k.modmul += w.modmul;
    }
    out->cmult = k.cmult;
    out->mult = k.mult;
    out->rot = k.rot;
    out->conj = k.conj;
    out->keyswitch = k.keyswitch;
    out->modup_digits = k.modup_digits;
    out->ntt_limbs = k.ntt_limbs;
    out->rescale = k.rescale;
    out->modmul = k.modmul;
    return HETAL_OK;
}

int hetal_counters_reset(hetal_ctx *ctx)
{
    if (!ctx) return HETAL_ERR_INVALID_ARG;
    ctx->c->cnt = Counters();
    for (auto &kv : ctx->pools)
        for (int i = 0; i < kv.second->size(); i++) kv.second->ctx(i).cnt = Counters();
    return HETAL_OK;
}

// ---- keys -------------------------------------------------------------------
int hetal_keygen(hetal_ctx *ctx, uint64_t seed, hetal_sk **sk_out)
{
    if (!ctx || !sk_out) return HETAL_ERR_INVALID_ARG;
    *sk_out = nullptr;
    return guard(ctx, [&] {
        idle(ctx);
        hetal_sk *h = new hetal_sk();
        h->owner = ctx;
        h->sk = keygen_secret(*ctx->c, seed);
        *sk_out = h;
    });
}

int hetal_sk_export(const hetal_sk *sk, int64_t *host_out)
{
    if (!sk || !host_out) return HETAL_ERR_INVALID_ARG;
    std::memcpy(host_out, sk->sk->coeffs.data(), sizeof(int64_t) * sk->sk->coeffs.size());
    return HETAL_OK;
}

void hetal_sk_free(hetal_sk *sk)
{
    if (!sk) return;
    auto release = [sk] {
        free_secret(*sk->owner->c, sk->sk);
        delete sk;
    };
    if (!defer_release(sk->owner, release)) release();
}

int hetal_evk_create(hetal_ctx *ctx, const hetal_sk *sk, uint64_t seed, const int32_t *rot_steps, size_t n_steps,
                     int with_conj, int with_relin, hetal_evk **out)
{
    if (!ctx || !sk || !out || (n_steps && !rot_steps)) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        idle(ctx);
        std::vector<int> rs(rot_steps, rot_steps + n_steps);
        hetal_evk *h = new hetal_evk();
        h->owner = ctx;
        h->ek = keygen_eval(*ctx->c, *sk->sk, seed, rs, with_conj != 0, with_relin != 0);
        *out = h;
    });
}

int hetal_evk_export(hetal_ctx *ctx, const hetal_evk *evk, int kind, int32_t step, uint64_t *host_out)
{
    if (!ctx || !evk || !host_out) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        Context &c = *ctx->c;
        const SwitchKey *key = nullptr;
        if (kind == 0) {
            if (!evk->ek->has_relin) throw Error(ERR_MISSING_KEY, "no relinearisation key");
            key = &evk->ek->relin;
        } else if (kind == 1) {
            if (!evk->ek->has_conj) throw Error(ERR_MISSING_KEY, "no conjugation key");
            key = &evk->ek->conj;
        } else {
            int s = c.p.slots();
            key = &rot_key(*evk->ek, ((step % s) + s) % s);
        }
        const int M = c.p.L + c.p.K, dnum = c.p.dnum_full();
        size_t words = (size_t)dnum * 2 * M * c.p.N;
        DBuf tmp(&c, words);
        LimbMap am;
        am.n = M;
        for (int i = 0; i < M; i++) am.idx[i] = (unsigned char)i;
        PolyBatch all{tmp.ptr, dnum * 2, (size_t)M * c.p.N};
        k_from_mont(c, all, PolyBatch{key->data, dnum * 2, (size_t)M * c.p.N}, am);
        ntt_inverse(c, all, am, identity_pos(M));
        HETAL_CUDA_CHECK(cudaMemcpyAsync(host_out, tmp.ptr, words * sizeof(u64), cudaMemcpyDeviceToHost, c.stream));
        c.sync();
    });
}

void hetal_evk_free(hetal_evk *evk)
{
    if (!evk) return;
    auto release = [evk] {
        free_eval(*evk->owner->c, evk->ek);
        delete evk;
    };
    if (!defer_release(evk->owner, release)) release();
}

// ---- matrices ------------------------------------------------------------------
int hetal_encrypt(hetal_ctx *ctx, const hetal_sk *sk, uint64_t seed, uint64_t nonce, const double *host_m, int rows,
                  int cols, int s0, int s1, int tiling, int tile_c, int level, double scale, hetal_mat **out)
{
    if (!ctx || !sk || !host_m || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        idle(ctx);
        Context &c = *ctx->c;
        need(rows > 0 && cols > 0, "matrix must be non-empty");
        if (s0 < 1 || s1 < 1 || (long long)s0 * s1 != c.p.N / 2) throw Error(ERR_SHAPE, "s0 * s1 must equal N/2");
        if (level < 0 || level >= c.p.L) throw Error(ERR_LEVEL, "level out of range");
        Mat m;
        m.s0 = s0;
        m.s1 = s1;
        if (tiling == HETAL_TILE_NONE) {
            m.m = (rows + s0 - 1) / s0;
            m.n = (cols + s1 - 1) / s1;
            m.rows = rows;
            m.cols = cols;
        } else if (tiling == HETAL_TILE_VERT) {
            if (tile_c < 1 || rows > tile_c || s0 % tile_c) throw Error(ERR_SHAPE, "vertical tiling needs rows <= c | s0");
            m.m = 1;
            m.n = (cols + s1 - 1) / s1;
            m.rows = s0;
            m.cols = cols;
        } else if (tiling == HETAL_TILE_HORIZ) {
            if (tile_c < 1 || cols > tile_c || s1 % tile_c)
                throw Error(ERR_SHAPE, "horizontal tiling needs cols <= c | s1");
            m.m = (rows + s0 - 1) / s0;
            m.n = 1;
            m.rows = rows;
            m.cols = s1;
        } else {
            throw Error(ERR_INVALID_ARG, "unknown tiling");
        }
        const int cnt = m.m * m.n, s = c.p.slots();
        double *d_src = (double *)c.alloc_bytes(sizeof(double) * (size_t)rows * cols);
        double *d_slots = (double *)c.alloc_bytes(sizeof(double) * (size_t)cnt * s);
        long long *d_pt = (long long *)c.alloc_bytes(sizeof(long long) * (size_t)cnt * c.p.N);
        HETAL_CUDA_CHECK(cudaMemcpyAsync(d_src, host_m, sizeof(double) * (size_t)rows * cols, cudaMemcpyHostToDevice,
                                         c.stream));
        k_block_layout(c, d_slots, d_src, rows, cols, m.m, m.n, s0, s1, tiling, tile_c);
        k_encode(c, d_pt, d_slots, nullptr, cnt, scale);
        m.cts = encrypt_int(c, *sk->sk, seed, nonce, d_pt, cnt, level, scale);
        c.free_bytes(d_src);
        c.free_bytes(d_slots);
        c.free_bytes(d_pt);
        c.sync();
        *out = wrap(ctx, std::move(m));
    });
}

int hetal_encrypt_int(hetal_ctx *ctx, const hetal_sk *sk, uint64_t seed, uint64_t nonce, const int64_t *host_pt,
                      const hetal_mat_desc *desc, hetal_mat **out)
{
    if (!ctx || !sk || !host_pt || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        idle(ctx);
        Context &c = *ctx->c;
        check_desc(c, desc);
        const int cnt = desc->m * desc->n;
        long long *d_pt = (long long *)c.alloc_bytes(sizeof(long long) * (size_t)cnt * c.p.N);
        HETAL_CUDA_CHECK(cudaMemcpyAsync(d_pt, host_pt, sizeof(long long) * (size_t)cnt * c.p.N,
                                         cudaMemcpyHostToDevice, c.stream));
        Mat m;
        m.m = desc->m;
        m.n = desc->n;
        m.rows = desc->rows;
        m.cols = desc->cols;
        m.s0 = desc->s0;
        m.s1 = desc->s1;
        m.cts = encrypt_int(c, *sk->sk, seed, nonce, d_pt, cnt, desc->level, desc->scale);
        c.free_bytes(d_pt);
        c.sync();
        *out = wrap(ctx, std::move(m));
    });
}

int hetal_decrypt(hetal_ctx *ctx, const hetal_sk *sk, const hetal_mat *mat, double *host_out)
{
    if (!ctx || !sk || !mat_live(mat) || !host_out) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        Context &c = *ctx->c;
        const Mat &m = mat->m;
        const int cnt = m.m * m.n, N = c.p.N, s = c.p.slots();
        double *d_m = (double *)c.alloc_bytes(sizeof(double) * (size_t)cnt * N);
        double *d_z = (double *)c.alloc_bytes(sizeof(double) * (size_t)cnt * s);
        double *d_out = (double *)c.alloc_bytes(sizeof(double) * (size_t)cnt * s);
        decrypt_to_double(c, *sk->sk, m.cts.view(), d_m);
        k_decode(c, d_z, nullptr, d_m, cnt, 1.0 / m.cts.scale);
        k_block_unlayout(c, d_out, d_z, m.m, m.n, m.s0, m.s1);
        HETAL_CUDA_CHECK(cudaMemcpyAsync(host_out, d_out, sizeof(double) * (size_t)cnt * s, cudaMemcpyDeviceToHost,
                                         c.stream));
        c.free_bytes(d_m);
        c.free_bytes(d_z);
        c.free_bytes(d_out);
        c.sync();
    });
}

int hetal_encode(hetal_ctx *ctx, const double *host_re, const double *host_im, int count, double scale,
                 int64_t *host_out)
{
    if (!ctx || !host_re || !host_out || count < 1) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        Context &c = *ctx->c;
        const int s = c.p.slots(), N = c.p.N;
        double *d_re = (double *)c.alloc_bytes(sizeof(double) * (size_t)count * s * 2);
        double *d_im = host_im ? d_re + (size_t)count * s : nullptr;
        long long *d_out = (long long *)c.alloc_bytes(sizeof(long long) * (size_t)count * N);
        HETAL_CUDA_CHECK(cudaMemcpyAsync(d_re, host_re, sizeof(double) * (size_t)count * s, cudaMemcpyHostToDevice,
                                         c.stream));
        if (host_im)
            HETAL_CUDA_CHECK(cudaMemcpyAsync(d_im, host_im, sizeof(double) * (size_t)count * s,
                                             cudaMemcpyHostToDevice, c.stream));
        k_encode(c, d_out, d_re, d_im, count, scale);
        HETAL_CUDA_CHECK(cudaMemcpyAsync(host_out, d_out, sizeof(long long) * (size_t)count * N,
                                         cudaMemcpyDeviceToHost, c.stream));
        c.free_bytes(d_re);
        c.free_bytes(d_out);
        c.sync();
    });
}

int hetal_mat_desc_get(const hetal_mat *mat, hetal_mat_desc *out)
{
    if (!mat_live(mat) || !out) return HETAL_ERR_INVALID_ARG;
    const Mat &m = mat->m;
    out->m = m.m;
    out->n = m.n;
    out->rows = m.rows;
    out->cols = m.cols;
    out->s0 = m.s0;
    out->s1 = m.s1;
    out->level = m.cts.lv;
    out->scale = m.cts.scale;
    return HETAL_OK;
}

int hetal_mat_export_dev(hetal_ctx *ctx, const hetal_mat *mat, uint64_t *dev_out)
{
    if (!ctx || !mat_live(mat) || !dev_out) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] { export_coeff(*ctx->c, mat->m.cts.view(), dev_out); });
}

int hetal_mat_export(hetal_ctx *ctx, const hetal_mat *mat, uint64_t *host_out)
{
    if (!ctx || !mat_live(mat) || !host_out) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        Context &c = *ctx->c;
        if (c.recording) need_pinned(host_out);
        size_t words = (size_t)mat->m.cts.n * mat->m.cts.ct_words();
        DBuf tmp(&c, words);
        export_coeff(c, mat->m.cts.view(), tmp.ptr);
        HETAL_CUDA_CHECK(cudaMemcpyAsync(host_out, tmp.ptr, words * sizeof(u64), cudaMemcpyDeviceToHost, c.stream));
        if (!c.recording) c.sync();   // recorded: complete when the launch is
    });
}

int hetal_mat_import_dev(hetal_ctx *ctx, const uint64_t *dev_in, const hetal_mat_desc *desc, hetal_mat **out)
{
    if (!ctx || !dev_in || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        Context &c = *ctx->c;
        check_desc(c, desc);
        Mat m;
        m.m = desc->m;
        m.n = desc->n;
        m.rows = desc->rows;
        m.cols = desc->cols;
        m.s0 = desc->s0;
        m.s1 = desc->s1;
        if (!c.recording) check_residues(c, dev_in, m.m * m.n, desc->level);
        m.cts = import_coeff(c, dev_in, m.m * m.n, desc->level, desc->scale);
        *out = wrap(ctx, std::move(m));
    });
}

int hetal_mat_import(hetal_ctx *ctx, const uint64_t *host_in, const hetal_mat_desc *desc, hetal_mat **out)
{
    if (!ctx || !host_in || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        Context &c = *ctx->c;
        check_desc(c, desc);
        if (c.recording) need_pinned(host_in);
        size_t words = (size_t)desc->m * desc->n * 2 * (desc->level + 1) * c.p.N;
        DBuf tmp(&c, words);
        HETAL_CUDA_CHECK(cudaMemcpyAsync(tmp.ptr, host_in, words * sizeof(u64), cudaMemcpyHostToDevice, c.stream));
        if (!c.recording) check_residues(c, tmp.ptr, desc->m * desc->n, desc->level);
        Mat m;
        m.m = desc->m;
        m.n = desc->n;
        m.rows = desc->rows;
        m.cols = desc->cols;
        m.s0 = desc->s0;
        m.s1 = desc->s1;
        m.cts = import_coeff(c, tmp.ptr, m.m * m.n, desc->level, desc->scale);
        if (!c.recording) c.sync();   // recorded: the graph reads host_in at every launch
        *out = wrap(ctx, std::move(m));
    });
}

int hetal_mat_drop(hetal_ctx *ctx, const hetal_mat *in, int level, hetal_mat **out)
{
    if (!ctx || !mat_live(in) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] { *out = wrap(ctx, like(in->m, drop_level(*ctx->c, in->m.cts.view(), level))); });
}

int hetal_mat_slice(hetal_ctx *ctx, const hetal_mat *in, int first, int count, hetal_mat **out)
{
    if (!ctx || !mat_live(in) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        const CtView v = in->m.cts.view();
        if (first < 0 || count < 1 || first > v.n - count) throw Error(ERR_SHAPE, "slice: block range outside the matrix");
        Mat m;
        m.cts = ct_copy(*ctx->c, v.sub(first, count));
        m.m = 1;
        m.n = count;
        m.rows = in->m.s0;
        m.cols = count * in->m.s1;
        m.s0 = in->m.s0;
        m.s1 = in->m.s1;
        *out = wrap(ctx, std::move(m));
    });
}

int hetal_mat_stack(hetal_ctx *ctx, const hetal_mat *const *mats, int count, const hetal_mat_desc *desc,
                    hetal_mat **out)
{
    if (!ctx || !mats || count < 1 || !desc || !out) return HETAL_ERR_INVALID_ARG;
    for (int i = 0; i < count; i++)
        if (!mat_live(mats[i])) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        Context &c = *ctx->c;
        const CtView v0 = mats[0]->m.cts.view();
        int total = 0;
        for (int i = 0; i < count; i++) {
            const CtView v = mats[i]->m.cts.view();
            if (v.lv != v0.lv) throw Error(ERR_LEVEL, "stack: inputs at different levels");
            if (v.scale != v0.scale) throw Error(ERR_SCALE, "stack: inputs at different scales");
            if (mats[i]->m.s0 != desc->s0 || mats[i]->m.s1 != desc->s1) throw Error(ERR_SHAPE, "stack: block shapes differ");
            total += v.n;
        }
        if (desc->m < 1 || desc->n < 1 || (long long)desc->m * desc->n != total)
            throw Error(ERR_SHAPE, "stack: block grid does not hold the inputs' blocks");
        Mat m;
        m.cts = CtBatch(&c, total, v0.lv, v0.scale);
        size_t at = 0;
        for (int i = 0; i < count; i++) {
            const CtView v = mats[i]->m.cts.view();
            HETAL_CUDA_CHECK(cudaMemcpyAsync(m.cts.data + at, v.data, sizeof(u64) * v.n * v.ct_words(),
                                             cudaMemcpyDeviceToDevice, c.stream));
            at += (size_t)v.n * v.ct_words();
        }
        m.m = desc->m;
        m.n = desc->n;
        m.rows = desc->rows;
        m.cols = desc->cols;
        m.s0 = desc->s0;
        m.s1 = desc->s1;
        *out = wrap(ctx, std::move(m));
    });
}

void hetal_mat_free(hetal_mat *mat)
{
    if (!mat_live(mat)) return;   // NULL, or already freed: nothing to release
    hetal_ctx *ctx = mat->owner;
    if (ctx && ctx->c->recording && !ctx->recorded.erase(mat) && defer_release(ctx, [mat] { delete mat; })) return;
    delete mat;
}

// ---- plaintext sets ----------------------------------------------------------
int hetal_ptset_create(hetal_ptset **out)
{
    if (!out) return HETAL_ERR_INVALID_ARG;
    *out = new hetal_ptset();
    return HETAL_OK;
}

int hetal_ptset_put(hetal_ptset *set, int kind, int index, int level, const int64_t *host_coeffs, int n)
{
    if (!set || !host_coeffs || n <= 0) return HETAL_ERR_INVALID_ARG;
    set->set.pts[std::make_tuple(kind, index, level)] = std::vector<long long>(host_coeffs, host_coeffs + n);
    return HETAL_OK;
}

void hetal_ptset_free(hetal_ptset *set) { delete set; }

// ---- server-side operations ----------------------------------------------------
int hetal_rotate(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *in, int32_t step, hetal_mat **out)
{
    if (!ctx || !evk || !mat_live(in) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] { *out = wrap(ctx, like(in->m, rotate(*ctx->c, *evk->ek, in->m.cts.view(), step))); });
}

int hetal_rotate_hoisted(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *in, const int32_t *steps, size_t n,
                         hetal_mat **outs)
{
    if (!ctx || !evk || !mat_live(in) || !outs || (n && !steps)) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        std::vector<int> rs(steps, steps + n);
        std::vector<CtBatch> r = rotate_hoisted(*ctx->c, *evk->ek, in->m.cts.view(), rs);
        for (size_t i = 0; i < n; i++) outs[i] = wrap(ctx, like(in->m, std::move(r[i])));
    });
}

int hetal_rotate_sum(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *in, const int32_t *steps, size_t n,
                     hetal_mat **out)
{
    if (!ctx || !evk || !mat_live(in) || !out || (n && !steps)) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        std::vector<int> rs(steps, steps + n);
        *out = wrap(ctx, like(in->m, rotate_sum(*ctx->c, *evk->ek, in->m.cts.view(), rs)));
    });
}

int hetal_conj(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *in, hetal_mat **out)
{
    if (!ctx || !evk || !mat_live(in) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] { *out = wrap(ctx, like(in->m, conjugate(*ctx->c, *evk->ek, in->m.cts.view()))); });
}

int hetal_mult(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *a, const hetal_mat *b, hetal_mat **out)
{
    if (!ctx || !evk || !mat_live(a) || !mat_live(b) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx,
                 [&] { *out = wrap(ctx, like(a->m, mult(*ctx->c, *evk->ek, a->m.cts.view(), b->m.cts.view()))); });
}

int hetal_cmult(hetal_ctx *ctx, const hetal_mat *a, const double *host_re, const double *host_im, hetal_mat **out)
{
    if (!ctx || !mat_live(a) || !host_re || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        idle(ctx);
        Context &c = *ctx->c;
        const int s = c.p.slots();
        const CtView av = a->m.cts.view();
        if (av.lv < 1) throw Error(ERR_LEVEL, "no level left for a plaintext product");
        double *d = (double *)c.alloc_bytes(sizeof(double) * 2 * s);
        HETAL_CUDA_CHECK(cudaMemcpyAsync(d, host_re, sizeof(double) * s, cudaMemcpyHostToDevice, c.stream));
        if (host_im)
            HETAL_CUDA_CHECK(cudaMemcpyAsync(d + s, host_im, sizeof(double) * s, cudaMemcpyHostToDevice, c.stream));
        Plain pt = plain_encode(c, d, host_im ? d + s : nullptr, av.lv, (double)c.p.mod[av.lv]);
        CtBatch r = mul_plain_rescale(c, av, pt, av.scale);
        c.free_bytes(d);
        c.sync();
        *out = wrap(ctx, like(a->m, std::move(r)));
    });
}

int hetal_mul_const(hetal_ctx *ctx, const hetal_mat *a, double value, double out_scale, hetal_mat **out)
{
    if (!ctx || !mat_live(a) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] { *out = wrap(ctx, like(a->m, mul_const_rescale(*ctx->c, a->m.cts.view(), value, out_scale))); });
}

int hetal_mat_set_scale(hetal_ctx *ctx, const hetal_mat *a, double scale, hetal_mat **out)
{
    if (!ctx || !mat_live(a) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        const CtView av = a->m.cts.view();
        if (!(scale > 0) || !std::isfinite(scale)) throw Error(ERR_SCALE, "hetal_mat_set_scale: scale must be positive");
        CtBatch r = ct_copy(*ctx->c, av);
        r.scale = scale;
        *out = wrap(ctx, like(a->m, std::move(r)));
    });
}

int hetal_mod_raise(hetal_ctx *ctx, const hetal_mat *a, int level, hetal_mat **out)
{
    if (!ctx || !mat_live(a) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] { *out = wrap(ctx, like(a->m, mod_raise(*ctx->c, a->m.cts.view(), level))); });
}

int hetal_mul_i(hetal_ctx *ctx, const hetal_mat *a, hetal_mat **out)
{
    if (!ctx || !mat_live(a) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] { *out = wrap(ctx, like(a->m, ct_mul_i(*ctx->c, a->m.cts.view()))); });
}

int hetal_mul_int(hetal_ctx *ctx, const hetal_mat *a, int64_t t, hetal_mat **out)
{
    if (!ctx || !mat_live(a) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] { *out = wrap(ctx, like(a->m, mul_int(*ctx->c, a->m.cts.view(), (long long)t))); });
}

int hetal_mult_scaled(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *a, const hetal_mat *b,
                      double target_scale, hetal_mat **out)
{
    if (!ctx || !evk || !mat_live(a) || !mat_live(b) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        *out = wrap(ctx, like(a->m, mult_scaled(*ctx->c, *evk->ek, a->m.cts.view(), b->m.cts.view(), target_scale)));
    });
}

namespace {

// The caller's integer plaintext (N signed coefficients, host memory) at `lv`.
Plain host_plain(Context &c, const int64_t *host_pt, int lv, double scale)
{
    long long *d = (long long *)c.alloc_bytes(sizeof(long long) * c.p.N);
    HETAL_CUDA_CHECK(cudaMemcpyAsync(d, host_pt, sizeof(long long) * c.p.N, cudaMemcpyHostToDevice, c.stream));
    Plain pt = plain_from_int(c, d, lv, scale);
    c.sync();
    c.free_bytes(d);
    return pt;
}

}  // namespace

int hetal_cmult_int(hetal_ctx *ctx, const hetal_mat *a, const int64_t *host_pt, double out_scale, hetal_mat **out)
{
    if (!ctx || !mat_live(a) || !host_pt || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        idle(ctx);
        Context &c = *ctx->c;
        const CtView av = a->m.cts.view();
        if (av.lv < 1) throw Error(ERR_LEVEL, "no level left for a plaintext product");
        if (!(out_scale > 0) || !std::isfinite(out_scale)) throw Error(ERR_INVALID_ARG, "plaintext product: out_scale");
        Plain pt = host_plain(c, host_pt, av.lv, (double)c.p.mod[av.lv]);
        CtBatch r = mul_plain_rescale(c, av, pt, out_scale);
        c.sync();
        *out = wrap(ctx, like(a->m, std::move(r)));
    });
}

int hetal_plain_create(hetal_ctx *ctx, const int64_t *host_pt, int level, double scale, hetal_plain **out)
{
    if (!ctx || !host_pt || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        idle(ctx);
        Context &c = *ctx->c;
        if (level < 0 || level >= c.p.L) throw Error(ERR_LEVEL, "plaintext level out of range");
        auto *h = new hetal_plain();
        h->owner = ctx;
        h->pt = host_plain(c, host_pt, level, scale);
        *out = h;
    });
}

void hetal_plain_free(hetal_plain *pt)
{
    if (!plain_live(pt)) return;
    hetal_ctx *ctx = pt->owner;
    if (ctx && ctx->c->recording && defer_release(ctx, [pt] { delete pt; })) return;
    delete pt;
}

int hetal_cmult_plain(hetal_ctx *ctx, const hetal_mat *a, const hetal_plain *pt, double out_scale, hetal_mat **out)
{
    if (!ctx || !mat_live(a) || !plain_live(pt) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        if (!(out_scale > 0) || !std::isfinite(out_scale)) throw Error(ERR_INVALID_ARG, "plaintext product: out_scale");
        *out = wrap(ctx, like(a->m, mul_plain_rescale(*ctx->c, a->m.cts.view(), pt->pt, out_scale)));
    });
}

int hetal_cmult_plain_sum(hetal_ctx *ctx, const hetal_mat *const *as, const hetal_plain *const *pts, int count,
                          double out_scale, hetal_mat **out)
{
    if (!ctx || !as || !pts || count < 1 || !out) return HETAL_ERR_INVALID_ARG;
    for (int i = 0; i < count; i++)
        if (!mat_live(as[i]) || !plain_live(pts[i])) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        if (!(out_scale > 0) || !std::isfinite(out_scale)) throw Error(ERR_INVALID_ARG, "plaintext product: out_scale");
        std::vector<CtView> vs;
        std::vector<const Plain *> ps;
        for (int i = 0; i < count; i++) {
            vs.push_back(as[i]->m.cts.view());
            ps.push_back(&pts[i]->pt);
        }
        *out = wrap(ctx, like(as[0]->m, mul_plain_sum_rescale(*ctx->c, vs, ps, out_scale)));
    });
}

int hetal_add_plain(hetal_ctx *ctx, const hetal_mat *a, const hetal_plain *pt, hetal_mat **out)
{
    if (!ctx || !mat_live(a) || !plain_live(pt) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] { *out = wrap(ctx, like(a->m, add_plain(*ctx->c, a->m.cts.view(), pt->pt))); });
}

int hetal_add_plain_int(hetal_ctx *ctx, const hetal_mat *a, const int64_t *host_pt, hetal_mat **out)
{
    if (!ctx || !mat_live(a) || !host_pt || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        idle(ctx);
        Context &c = *ctx->c;
        const CtView av = a->m.cts.view();
        Plain pt = host_plain(c, host_pt, av.lv, av.scale);
        CtBatch r = add_plain(c, av, pt);
        c.sync();
        *out = wrap(ctx, like(a->m, std::move(r)));
    });
}

int hetal_add(hetal_ctx *ctx, const hetal_mat *a, const hetal_mat *b, hetal_mat **out)
{
    if (!ctx || !mat_live(a) || !mat_live(b) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] { *out = wrap(ctx, like(a->m, ct_add(*ctx->c, a->m.cts.view(), b->m.cts.view()))); });
}

int hetal_sub(hetal_ctx *ctx, const hetal_mat *a, const hetal_mat *b, hetal_mat **out)
{
    if (!ctx || !mat_live(a) || !mat_live(b) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] { *out = wrap(ctx, like(a->m, ct_sub(*ctx->c, a->m.cts.view(), b->m.cts.view()))); });
}

int hetal_rescale(hetal_ctx *ctx, const hetal_mat *a, hetal_mat **out)
{
    if (!ctx || !mat_live(a) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] { *out = wrap(ctx, like(a->m, rescale(*ctx->c, a->m.cts.view()))); });
}

int hetal_diag_abt(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *a, const hetal_mat *bbar, int c, double t,
                   const hetal_ptset *pts, int flags, hetal_mat **out)
{
    if (!ctx || !evk || !mat_live(a) || !mat_live(bbar) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        Mat r = diag_abt(*ctx->c, *evk->ek, a->m, bbar->m, c, t, pts ? &pts->set : nullptr, flags);
        *out = wrap(ctx, std::move(r));
    });
}

int hetal_diag_atb(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *a_under, const hetal_mat *b, int c,
                   double t, const hetal_ptset *pts, int flags, hetal_mat **out)
{
    if (!ctx || !evk || !mat_live(a_under) || !mat_live(b) || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        Mat r = diag_atb(*ctx->c, *evk->ek, a_under->m, b->m, c, t, pts ? &pts->set : nullptr, flags);
        *out = wrap(ctx, std::move(r));
    });
}

int hetal_rotation_amounts(int s0, int s1, int c, int flags, int32_t *out, size_t cap)
{
    if (cap && !out) return HETAL_ERR_INVALID_ARG;
    try {
        std::vector<int> rs = hetal::rotation_amounts(s0, s1, c, flags);
        for (size_t i = 0; i < rs.size() && i < cap; i++) out[i] = rs[i];
        return (int)rs.size();
    } catch (const hetal::Error &e) {
        return e.code;
    } catch (...) {
        return HETAL_ERR_INVALID_ARG;
    }
}

int hetal_softmax_approx(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *m, const double *coeffs16,
                         const double *host_valid, double target_scale, const hetal_ptset *pts, hetal_mat **out)
{
    if (!ctx || !evk || !mat_live(m) || !coeffs16 || !host_valid || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        Context &c = *ctx->c;
        const int s = c.p.slots();
        // recorded: the mask's encodings must already be cached (an earlier call with
        // the same mask made them); a miss then fails instead of copying from the host
        double *d_valid = nullptr;
        if (!c.recording) {
            d_valid = (double *)c.alloc_bytes(sizeof(double) * s);
            HETAL_CUDA_CHECK(
                cudaMemcpyAsync(d_valid, host_valid, sizeof(double) * s, cudaMemcpyHostToDevice, c.stream));
        }
        u64 h = 1469598103934665603ull;   // FNV-1a of the mask bytes: the key of its cached encodings
        const unsigned char *bytes = (const unsigned char *)host_valid;
        for (size_t i = 0; i < sizeof(double) * (size_t)s; i++) h = (h ^ bytes[i]) * 1099511628211ull;
        Mat r = softmax_poly(c, *evk->ek, m->m, coeffs16, d_valid, h, target_scale, pts ? &pts->set : nullptr);
        c.free_bytes(d_valid);
        *out = wrap(ctx, std::move(r));
    });
}

// ---- raw primitives -------------------------------------------------------------
int hetal_ntt_forward(hetal_ctx *ctx, uint64_t *dev_polys, int n_polys, int n_limbs)
{
    if (!ctx || !dev_polys || n_polys < 0 || n_limbs < 1 || n_limbs > ctx->c->p.L + ctx->c->p.K)
        return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        Context &c = *ctx->c;
        LimbMap m = identity_pos(n_limbs);
        ntt_forward(c, PolyBatch{dev_polys, n_polys, (size_t)n_limbs * c.p.N}, m, m);
    });
}

int hetal_ntt_inverse(hetal_ctx *ctx, uint64_t *dev_polys, int n_polys, int n_limbs)
{
    if (!ctx || !dev_polys || n_polys < 0 || n_limbs < 1 || n_limbs > ctx->c->p.L + ctx->c->p.K)
        return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        Context &c = *ctx->c;
        LimbMap m = identity_pos(n_limbs);
        ntt_inverse(c, PolyBatch{dev_polys, n_polys, (size_t)n_limbs * c.p.N}, m, m);
    });
}

// ---- many independent instances -------------------------------------------------
int hetal_tile_choose(hetal_ctx *ctx, const hetal_evk *evk, int a, int b, int c, int *s0_out)
{
    if (!ctx || !evk || !s0_out || a < 1 || b < 1 || c < 2) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        if (!ctx->tuner.calibrated()) ctx->tuner.calibrate(*ctx->c, *evk->ek);
        *s0_out = ctx->tuner.choose_s0(ctx->c->p, a, b, c);
    });
}

int hetal_plan_choose(hetal_ctx *ctx, const hetal_evk *evk, int a, int b, int c, int *s0_out, int *flags_out)
{
    if (!ctx || !evk || !s0_out || !flags_out || a < 1 || b < 1 || c < 2) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        if (!ctx->tuner.calibrated()) ctx->tuner.calibrate(*ctx->c, *evk->ek);
        std::pair<int, int> r = ctx->tuner.choose(ctx->c->p, a, b, c);
        *s0_out = r.first;
        *flags_out = r.second;
    });
}

int hetal_run_pairs(hetal_ctx *ctx, const hetal_evk *evk, const hetal_pair_job *jobs, size_t n, int workers,
                    int flags, hetal_mat **out_abt, hetal_mat **out_atb)
{
    if (!ctx || !evk || (n && (!jobs || !out_abt || !out_atb)) || workers < 1) return HETAL_ERR_INVALID_ARG;
    for (size_t i = 0; i < n; i++) {
        out_abt[i] = nullptr;
        out_atb[i] = nullptr;
        if (!mat_live(jobs[i].x) || !mat_live(jobs[i].wbar) || !mat_live(jobs[i].a_under) || !mat_live(jobs[i].b))
            return HETAL_ERR_INVALID_ARG;
    }
    return guard(ctx, [&] {
        idle(ctx);
        Context &c = *ctx->c;
        std::vector<Mat> abt(n), atb(n);
        auto one = [&](Context &w, size_t i) {
            const hetal_pair_job &j = jobs[i];
            const int f = j.flags >= 0 ? j.flags : flags;
            abt[i] = diag_abt(w, *evk->ek, j.x->m, j.wbar->m, j.c, j.t_abt, nullptr, f);
            atb[i] = diag_atb(w, *evk->ek, j.a_under->m, j.b->m, j.c, j.t_atb, nullptr, f);
        };
        if (workers == 1) {
            for (size_t i = 0; i < n; i++) one(c, i);
            c.sync();
        } else {
            WorkerPool &wp = ctx->pool(workers);
            c.sync();   // inputs made on the main stream are complete
            wp.run(n, one);   // returns with every worker's stream synchronised
            // results belong to the caller's context: their frees are ordered on its stream,
            // after the work that reads them there, and do not depend on the pool
            for (size_t i = 0; i < n; i++) {
                abt[i].cts.rehome(&c);
                atb[i].cts.rehome(&c);
            }
        }
        for (size_t i = 0; i < n; i++) {
            out_abt[i] = wrap(ctx, std::move(abt[i]));
            out_atb[i] = wrap(ctx, std::move(atb[i]));
        }
    });
}

int hetal_run_pairs_batched(hetal_ctx *ctx, const hetal_evk *evk, const hetal_pair_job *jobs, size_t n, int flags,
                            hetal_mat **out_abt, hetal_mat **out_atb)
{
    if (!ctx || !evk || (n && (!jobs || !out_abt || !out_atb))) return HETAL_ERR_INVALID_ARG;
    for (size_t i = 0; i < n; i++) {
        out_abt[i] = nullptr;
        out_atb[i] = nullptr;
        if (!mat_live(jobs[i].x) || !mat_live(jobs[i].wbar) || !mat_live(jobs[i].a_under) || !mat_live(jobs[i].b))
            return HETAL_ERR_INVALID_ARG;
    }
    return guard(ctx, [&] {
        Context &c = *ctx->c;
        std::vector<Mat> abt(n), atb(n);
        run_groups(c, *evk->ek, jobs, n, flags, abt, atb);
        for (size_t i = 0; i < n; i++) {
            out_abt[i] = wrap(ctx, std::move(abt[i]));
            out_atb[i] = wrap(ctx, std::move(atb[i]));
        }
    });
}

// ---- serving ---------------------------------------------------------------------
int hetal_server_create(hetal_ctx *ctx, int slots, size_t budget_bytes, hetal_server **out)
{
    if (!ctx || !out || slots < 1 || budget_bytes == 0) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    return guard(ctx, [&] {
        idle(ctx);
        hetal_server *h = new hetal_server();
        h->parent = ctx;
        h->s.reset(new Server(ctx->c->p, ctx->c->device, slots, budget_bytes));
        *out = h;
    });
}

void hetal_server_destroy(hetal_server *srv) { delete srv; }

int hetal_server_add_client(hetal_server *srv, const hetal_evk *evk, int *client_id)
{
    if (!srv || !evk || !client_id) return HETAL_ERR_INVALID_ARG;
    return guard(srv->parent, [&] {
        idle(srv->parent);
        const Params &p = srv->parent->c->p;
        size_t per_key = (size_t)p.dnum_full() * 2 * (p.L + p.K) * p.N * sizeof(u64);
        size_t nkeys = evk->ek->rot.size() + (evk->ek->has_conj ? 1 : 0) + (evk->ek->has_relin ? 1 : 0);
        *client_id = srv->s->add_client(evk->ek, per_key * nkeys);
    });
}

int hetal_server_submit(hetal_server *srv, const hetal_request *req, uint64_t *ticket)
{
    if (!srv || !req || !ticket || !mat_live(req->a) || !mat_live(req->b) || (req->kind != 0 && req->kind != 1))
        return HETAL_ERR_INVALID_ARG;
    return guard(srv->parent, [&] {
        idle(srv->parent);
        srv->parent->c->sync();   // operands made on the caller's stream are complete
        ServerRequest r;
        r.client = req->client;
        r.kind = req->kind;
        r.a = &req->a->m;
        r.b = &req->b->m;
        r.c = req->c;
        r.t = req->t;
        r.flags = req->flags;
        *ticket = srv->s->submit(r);
    });
}

int hetal_server_wait(hetal_server *srv, uint64_t ticket, hetal_mat **out, double *queue_ms, double *run_ms)
{
    if (!srv || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    if (srv->parent->c->recording) {
        srv->parent->err = "this call cannot be recorded into a graph";
        return HETAL_ERR_RECORDING;
    }
    ServerResult res;
    if (!srv->s->wait(ticket, res)) {
        srv->parent->err = "unknown or already collected ticket";
        return HETAL_ERR_INVALID_ARG;
    }
    if (queue_ms) *queue_ms = res.queue_ms;
    if (run_ms) *run_ms = res.run_ms;
    if (res.status != 0) {
        srv->parent->err = res.error;
        return res.status;
    }
    // the slot synchronised its stream before posting the result; from here the result
    // belongs to the caller's context (frees ordered on its stream, no tie to the server)
    res.out.cts.rehome(srv->parent->c);
    *out = wrap(srv->parent, std::move(res.out));
    return HETAL_OK;
}

int hetal_server_cancel(hetal_server *srv, uint64_t ticket)
{
    if (!srv) return HETAL_ERR_INVALID_ARG;
    if (!srv->s->cancel(ticket)) {
        srv->parent->err = "the ticket is not queued (unknown, running, finished or collected)";
        return HETAL_ERR_INVALID_ARG;
    }
    return HETAL_OK;
}

int hetal_server_stats(const hetal_server *srv, long long *completed, size_t *resident_bytes,
                       size_t *peak_inflight_bytes)
{
    if (!srv) return HETAL_ERR_INVALID_ARG;
    if (completed) *completed = srv->s->completed();
    if (resident_bytes) *resident_bytes = srv->s->resident_bytes();
    if (peak_inflight_bytes) *peak_inflight_bytes = srv->s->peak_inflight_bytes();
    return HETAL_OK;
}

int hetal_profile_kernel(hetal_ctx *ctx, const char *kernel_name)
{
    if (!ctx) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        ctx->c->sync();
        ctx->c->prof_reset();
        ctx->c->prof_target = kernel_name ? kernel_name : "";
    });
}

int hetal_profile_read(hetal_ctx *ctx, long long *launches, double *total_ms, double *modmul, double *bytes)
{
    if (!ctx) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        Context &c = *ctx->c;
        c.sync();
        double ms = 0, mm = 0, by = 0;
        for (auto &r : c.prof) {
            float e = 0;
            HETAL_CUDA_CHECK(cudaEventElapsedTime(&e, r.a, r.b));
            ms += e;
            mm += r.modmul;
            by += r.bytes;
        }
        if (launches) *launches = (long long)c.prof.size();
        if (total_ms) *total_ms = ms;
        if (modmul) *modmul = mm;
        if (bytes) *bytes = by;
    });
}

int hetal_profile_summary(hetal_ctx *ctx, char *buf, size_t cap)
{
    if (!ctx || !buf || cap == 0) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        Context &c = *ctx->c;
        c.sync();
        struct Agg {
            long long n = 0;
            double ms = 0, mm = 0, by = 0;
        };
        std::map<std::string, Agg> agg;
        for (auto &r : c.prof) {
            float e = 0;
            HETAL_CUDA_CHECK(cudaEventElapsedTime(&e, r.a, r.b));
            Agg &a = agg[r.name];
            a.n++;
            a.ms += e;
            a.mm += r.modmul;
            a.by += r.bytes;
        }
        std::string s;
        char line[256];
        for (auto &kv : agg) {
            snprintf(line, sizeof(line), "%s\t%lld\t%.6f\t%.6e\t%.6e\n", kv.first.c_str(), kv.second.n,
                     kv.second.ms, kv.second.mm, kv.second.by);
            s += line;
        }
        if (s.size() + 1 > cap) throw Error(ERR_INVALID_ARG, "summary buffer too small");
        std::memcpy(buf, s.c_str(), s.size() + 1);
    });
}

int hetal_alloc_count(const hetal_ctx *ctx, long long *out)
{
    if (!ctx || !out) return HETAL_ERR_INVALID_ARG;
    *out = ctx->c->allocs;
    return HETAL_OK;
}

int hetal_launch_count(const hetal_ctx *ctx, long long *out)
{
    if (!ctx || !out) return HETAL_ERR_INVALID_ARG;
    long long n = ctx->c->launches;
    for (auto &kv : ctx->pools) n += kv.second->launches();
    *out = n;
    return HETAL_OK;
}

int hetal_probe_butterfly_rate(hetal_ctx *ctx, int iters, double *butterflies_per_s)
{
    if (!ctx || !butterflies_per_s || iters < 10) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        *butterflies_per_s = probe_butterfly_rate(*ctx->c, iters, 4);
    });
}

int hetal_probe_mac_rate(hetal_ctx *ctx, int iters, double *products_per_s)
{
    if (!ctx || !products_per_s || iters < 10) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        *products_per_s = probe_mac_rate(*ctx->c, iters, 4);
    });
}

int hetal_ntt32_moduli(hetal_ctx *ctx, int n_limbs, uint32_t *host_moduli, uint32_t *host_roots)
{
    if (!ctx || !host_moduli || n_limbs < 1 || n_limbs > HETAL_MAX_MODULI) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        std::vector<uint32_t> roots;
        std::vector<uint32_t> m = ntt32_moduli(*ctx->c, n_limbs, &roots);
        std::copy(m.begin(), m.end(), host_moduli);
        if (host_roots) std::copy(roots.begin(), roots.end(), host_roots);
    });
}

int hetal_ntt32_forward(hetal_ctx *ctx, uint32_t *dev_polys, int n_polys, int n_limbs)
{
    if (!ctx || !dev_polys || n_polys < 1 || n_limbs < 1 || n_limbs > HETAL_MAX_MODULI) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        auto *t = ctx->c->ntt32.get();
        if (ctx->c->recording && !t) throw Error(ERR_RECORDING, "make the 32-bit tables (hetal_ntt32_moduli) first");
        ntt32_forward(*ctx->c, dev_polys, n_polys, n_limbs);
    });
}

int hetal_probe_butterfly32_rate(hetal_ctx *ctx, int iters, double *butterflies_per_s)
{
    if (!ctx || !butterflies_per_s || iters < 10) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        *butterflies_per_s = probe_butterfly32_rate(*ctx->c, iters, 4);
    });
}

int hetal_ntt_root(const hetal_ctx *ctx, int limb, uint64_t *out)
{
    if (!ctx || !out || limb < 0 || limb >= ctx->c->p.L + ctx->c->p.K) return HETAL_ERR_INVALID_ARG;
    *out = ctx->c->p.psi[limb];
    return HETAL_OK;
}

// ---- CUDA graphs of recorded calls -------------------------------------------------
int hetal_graph_begin(hetal_ctx *ctx)
{
    if (!ctx) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        Context &c = *ctx->c;
        if (c.recording) throw Error(ERR_RECORDING, "a recording is already open");
        if (!c.prof_target.empty()) throw Error(ERR_RECORDING, "kernel timing is on: stop it before recording");
        HETAL_CUDA_CHECK(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
        c.recording = true;
        ctx->rec_failed = false;
        ctx->rec_launches0 = c.launches;
        ctx->recorded.clear();
    });
}

int hetal_graph_end(hetal_ctx *ctx, hetal_graph **out)
{
    if (!ctx || !out) return HETAL_ERR_INVALID_ARG;
    *out = nullptr;
    Context &c = *ctx->c;
    if (!c.recording) {
        ctx->err = "no recording is open";
        return HETAL_ERR_RECORDING;
    }
    c.recording = false;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamEndCapture(c.stream, &g);
    if (e == cudaSuccess && g && !ctx->rec_failed)
        e = cudaGraphInstantiateWithFlags(&exec, g, cudaGraphInstantiateFlagAutoFreeOnLaunch);
    if (e != cudaSuccess) cudaGetLastError();
    std::set<hetal_mat *> outs;
    outs.swap(ctx->recorded);
    if (e != cudaSuccess || !g || !exec) {
        // Nothing recorded ran, so the matrices made meanwhile have no device memory:
        // they are emptied (their addresses are dropped without a free).
        for (hetal_mat *m : outs) {
            CtBatch &b = m->m.cts;
            if (b.shared) new std::shared_ptr<u64>(std::move(b.shared));   // never released
            b.data = nullptr;
            b.n = 0;
        }
        if (g) cudaGraphDestroy(g);
        std::vector<std::function<void()>> rel;
        rel.swap(ctx->rec_releases);
        for (auto &f : rel) f();
        ctx->err = e != cudaSuccess ? std::string("recording failed: ") + cudaGetErrorString(e)
                                    : std::string("a recorded call failed: the recording is void");
        g_err = ctx->err;
        return HETAL_ERR_RECORDING;
    }
    hetal_graph *h = new hetal_graph();
    h->ctx = ctx;
    h->graph = g;
    h->exec = exec;
    h->kernels = c.launches - ctx->rec_launches0;
    h->releases.swap(ctx->rec_releases);
    for (hetal_mat *m : outs) {   // outputs: owned by the handle and by the graph
        CtBatch &b = m->m.cts;
        if (b.data && !b.shared) {
            Context *bc = b.ctx;
            b.shared = std::shared_ptr<u64>(b.data, FreeOn{bc});
        }
        if (b.shared) h->outputs.push_back(b.shared);
    }
    *out = h;
    // run once, so that the recorded calls' results exist as they would without a graph
    return hetal_graph_launch(ctx, h);
}

int hetal_graph_launch(hetal_ctx *ctx, hetal_graph *g)
{
    if (!ctx || !g || g->ctx != ctx) return HETAL_ERR_INVALID_ARG;
    return guard(ctx, [&] {
        idle(ctx);
        HETAL_CUDA_CHECK(cudaGraphLaunch(g->exec, ctx->c->stream));
        ctx->c->launches += g->kernels;
    });
}

int hetal_graph_kernels(const hetal_graph *g, long long *out)
{
    if (!g || !out) return HETAL_ERR_INVALID_ARG;
    *out = g->kernels;
    return HETAL_OK;
}

void hetal_graph_free(hetal_graph *g)
{
    if (!g) return;
    auto release = [g] {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        for (auto &f : g->releases) f();   // handles released while the graph was recorded
        delete g;                          // and the graph's share of its outputs
    };
    if (!defer_release(g->ctx, release)) release();
}

}  // extern "C"
