// context.cpp -- parameter generation, device tables and memory for the
// GB300 RNS-CKKS library.
#include "context.h"

#include <algorithm>
#include <cstdio>

namespace hetal {

u64 host_mulmod(u64 a, u64 b, u64 m) { return (u64)(((u128)a * b) % m); }

u64 host_powmod(u64 a, u64 e, u64 m)
{
    u64 r = 1 % m, x = a % m;
    for (; e; e >>= 1) {
        if (e & 1) r = host_mulmod(r, x, m);
        x = host_mulmod(x, x, m);
    }
    return r;
}

u64 host_invmod(u64 a, u64 m) { return host_powmod(a, m - 2, m); }   // m prime

u64 host_shoup(u64 w, u64 m) { return (u64)(((u128)w << 64) / m); }

u64 host_mont(u64 x, u64 m) { return (u64)((((u128)(x % m)) << 64) % m); }

// Strong-probable-prime test to the bases 2..37 (deterministic below 2^64).
static bool sprp(u64 n, u64 a)
{
    u64 d = n - 1;
    int s = 0;
    while (!(d & 1)) {
        d >>= 1;
        ++s;
    }
    u64 x = host_powmod(a, d, n);
    if (x == 1 || x == n - 1) return true;
    while (--s > 0) {
        x = host_mulmod(x, x, n);
        if (x == n - 1) return true;
    }
    return false;
}

static bool is_prime64(u64 n)
{
    static const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 b : small) {
        if (n % b == 0) return n == b;
    }
    for (u64 b : small)
        if (!sprp(n, b)) return false;
    return true;
}

// A primitive 2N-th root of unity: g^((q-1)/2N) for the first g where its
// N-th power is -1.
static u64 find_root(u64 q, u64 two_n)
{
    for (u64 g = 3;; g += 2) {
        u64 r = host_powmod(g, (q - 1) / two_n, q);
        if (host_powmod(r, two_n / 2, q) == q - 1) return r;
    }
}

Params make_params(int log_n, int q0_bits, int n_rescale, int rescale_bits, int n_special, int special_bits,
                   int alpha, int h, double scale, int n_upper, int upper_bits)
{
    if (log_n < 10 || log_n > 16) throw Error(ERR_INVALID_ARG, "log_n must be in [10, 16]");
    if (alpha < 1 || n_special < 1 || n_rescale < 0) throw Error(ERR_INVALID_ARG, "bad prime counts");
    if (alpha > 7 || n_special > 7) throw Error(ERR_INVALID_ARG, "alpha and the special prime count must be at most 7");
    if (n_upper < 0) throw Error(ERR_INVALID_ARG, "bad prime counts");
    for (int b : {q0_bits, rescale_bits, special_bits, n_upper ? upper_bits : 60})
        if (b < 36 || b > 61) throw Error(ERR_INVALID_ARG, "prime bit sizes must be in [36, 61]");
    Params p;
    p.logN = log_n;
    p.N = 1 << log_n;
    u64 two_n = 2 * (u64)p.N;
    // Primes q = 1 + k * 2^32 (so q = 1 mod 2N as well), the largest below
    // 2^bits first; the kernels' reductions rely on this form.
    const u64 step = (u64)1 << 32;
    std::vector<u64> taken;
    auto take = [&](int bits, int count) {
        u64 c = ((((u64)1 << bits) - 1) & ~(step - 1)) + 1;   // largest 1 + k 2^32 below 2^bits
        int got = 0;
        while (got < count) {
            if (c <= step) throw Error(ERR_INVALID_ARG, "ran out of primes 1 mod 2^32 below 2^bits");
            if (std::find(taken.begin(), taken.end(), c) == taken.end() && is_prime64(c)) {
                taken.push_back(c);
                ++got;
            }
            c -= step;
        }
    };
    take(q0_bits, 1);
    take(rescale_bits, n_rescale);
    take(upper_bits, n_upper);   // levels n_rescale + 1 .. n_rescale + n_upper
    take(special_bits, n_special);
    p.L = 1 + n_rescale + n_upper;
    p.K = n_special;
    p.alpha = alpha;
    p.h = std::min(h, p.N / 2);
    p.scale = scale;
    p.mod = taken;
    if (p.L + p.K > HETAL_MAX_MODULI) throw Error(ERR_INVALID_ARG, "too many moduli");
    // digits: at most L <= 127, so a digit index fits the 8 bits the key streams give it
    // (stream_key_a / stream_key_e); key inner products take any count, 8 digits a launch
    for (u64 q : p.mod) p.psi.push_back(find_root(q, two_n));
    return p;
}

// --------------------------------------------------------------------------
CtBatch::CtBatch(Context *c, int n_, int lv_, double scale_) : ctx(c), n(n_), lv(lv_), scale(scale_)
{
    if (n > 0) data = c->alloc((size_t)n * ct_words());
}

CtBatch &CtBatch::operator=(CtBatch &&o) noexcept
{
    if (this != &o) {
        if (data && !shared) ctx->free(data);
        ctx = o.ctx;
        data = o.data;
        n = o.n;
        lv = o.lv;
        scale = o.scale;
        shared = std::move(o.shared);
        o.data = nullptr;
        o.n = 0;
    }
    return *this;
}

CtBatch::~CtBatch()
{
    if (data && !shared) ctx->free(data);
}

std::vector<CtBatch> CtBatch::split(CtBatch &&w, int parts)
{
    if (parts < 1 || w.n % parts) throw Error(ERR_INVALID_ARG, "split: batch size not a multiple of the parts");
    Context *c = w.ctx;
    std::shared_ptr<u64> sp = w.shared;
    if (!sp && w.data) sp = std::shared_ptr<u64>(w.data, FreeOn{c});
    const int k = w.n / parts;
    std::vector<CtBatch> out(parts);
    for (int i = 0; i < parts; i++) {
        out[i].ctx = c;
        out[i].n = k;
        out[i].lv = w.lv;
        out[i].scale = w.scale;
        out[i].data = w.data ? w.data + (size_t)i * k * w.ct_words() : nullptr;
        out[i].shared = sp;
    }
    w.shared.reset();
    w.data = nullptr;
    w.n = 0;
    return out;
}

std::vector<CtBatch> CtBatch::split_sizes(CtBatch &&w, const std::vector<int> &sizes)
{
    long long total = 0;
    for (int k : sizes) {
        if (k < 0) throw Error(ERR_INVALID_ARG, "split: negative part");
        total += k;
    }
    if (total != w.n) throw Error(ERR_INVALID_ARG, "split: part sizes do not add up to the batch");
    Context *c = w.ctx;
    std::shared_ptr<u64> sp = w.shared;
    if (!sp && w.data) sp = std::shared_ptr<u64>(w.data, FreeOn{c});
    std::vector<CtBatch> out(sizes.size());
    size_t off = 0;
    for (size_t i = 0; i < sizes.size(); i++) {
        out[i].ctx = c;
        out[i].n = sizes[i];
        out[i].lv = w.lv;
        out[i].scale = w.scale;
        out[i].data = (w.data && sizes[i]) ? w.data + off * w.ct_words() : nullptr;
        out[i].shared = sizes[i] ? sp : nullptr;
        off += sizes[i];
    }
    w.shared.reset();
    w.data = nullptr;
    w.n = 0;
    return out;
}

void FreeOn::operator()(u64 *p) const { c->free(p); }

void CtBatch::rehome(Context *to)
{
    if (shared) {
        FreeOn *d = std::get_deleter<FreeOn>(shared);
        if (!d) throw Error(ERR_INVALID_ARG, "rehome: memory shared with a graph stays with its owner");
        d->c = to;
    }
    ctx = to;
}

size_t CtBatch::ct_words() const { return (size_t)2 * (lv + 1) * ctx->p.N; }

PolyBatch CtBatch::polys() const { return PolyBatch{data, 2 * n, (size_t)(lv + 1) * ctx->p.N}; }

CtView CtBatch::view() const
{
    CtView v;
    v.data = data;
    v.n = n;
    v.lv = lv;
    v.scale = scale;
    v.N = ctx ? ctx->p.N : 0;
    return v;
}

Plain &Plain::operator=(Plain &&o) noexcept
{
    if (this != &o) {
        if (data) ctx->free(data);
        if (mont) ctx->free(mont);
        ctx = o.ctx;
        data = o.data;
        mont = o.mont;
        lv = o.lv;
        scale = o.scale;
        o.data = o.mont = nullptr;
    }
    return *this;
}

Plain::~Plain()
{
    if (data) ctx->free(data);
    if (mont) ctx->free(mont);
}

PolyBatch CtBatch::comp(int c) const
{
    return PolyBatch{data + (size_t)c * (lv + 1) * ctx->p.N, n, ct_words()};
}

// --------------------------------------------------------------------------
static u64 *upload(Context &c, const std::vector<u64> &v)
{
    u64 *d = nullptr;
    HETAL_CUDA_CHECK(cudaMalloc(&d, std::max<size_t>(v.size(), 1) * sizeof(u64)));
    HETAL_CUDA_CHECK(cudaMemcpy(d, v.data(), v.size() * sizeof(u64), cudaMemcpyHostToDevice));
    return d;
}

Context::Context(const Params &prm, int dev, cudaStream_t s) : p(prm), device(dev)
{
    HETAL_CUDA_CHECK(cudaSetDevice(dev));
    HETAL_CUDA_CHECK(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));
    if (s) {
        stream = s;
    } else {
        HETAL_CUDA_CHECK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
        own_stream = true;
    }
    cudaMemPool_t pool;
    HETAL_CUDA_CHECK(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t thr = UINT64_MAX;
    HETAL_CUDA_CHECK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));

    const int M = p.L + p.K, N = p.N;
    h_mc.resize(M);
    for (int t = 0; t < M; t++) {
        u64 q = p.mod[t];
        ModConst &m = h_mc[t];
        m.q = q;
        m.r2 = (u64)((((u128)1 << 64) % q) * (u128)(((u128)1 << 64) % q) % q);
        int k = 64 - __builtin_clzll(q);
        m.k = k;
        m.mu = (u64)(((u128)1 << (2 * k)) / q);
        m.pad = 0;
    }
    HETAL_CUDA_CHECK(cudaMalloc(&d_mc, sizeof(ModConst) * M));
    HETAL_CUDA_CHECK(cudaMemcpy(d_mc, h_mc.data(), sizeof(ModConst) * M, cudaMemcpyHostToDevice));

    std::vector<u64> psi((size_t)2 * M * N), ipsi((size_t)2 * M * N);   // interleaved (w, Shoup(w))
    std::vector<u64> ninv(M), ninv_sh(M), imag(M), imag_sh(M);
    for (int t = 0; t < M; t++) {
        u64 q = p.mod[t], w = p.psi[t], wi = host_invmod(w, q);
        std::vector<u64> pw(N), ipw(N);
        pw[0] = 1;
        ipw[0] = 1;
        for (int i = 1; i < N; i++) {
            pw[i] = host_mulmod(pw[i - 1], w, q);
            ipw[i] = host_mulmod(ipw[i - 1], wi, q);
        }
        for (int i = 0; i < N; i++) {
            unsigned r = 0;
            for (int b = 0; b < p.logN; b++)
                if (i & (1 << b)) r |= 1u << (p.logN - 1 - b);
            size_t o = (size_t)t * N + i;
            psi[2 * o] = pw[r];
            psi[2 * o + 1] = host_shoup(pw[r], q);
            ipsi[2 * o] = ipw[r];
            ipsi[2 * o + 1] = host_shoup(ipw[r], q);
        }
        ninv[t] = host_invmod((u64)N % q, q);
        ninv_sh[t] = host_shoup(ninv[t], q);
        imag[t] = pw[N / 2];
        imag_sh[t] = host_shoup(imag[t], q);
    }
    d_psi2 = reinterpret_cast<ulonglong2 *>(upload(*this, psi));
    d_ipsi2 = reinterpret_cast<ulonglong2 *>(upload(*this, ipsi));
    {
        // Row pass tables.  Forward, per row r: the 15 pairs of the strided
        // stages s = 0..3 (slot 2^s - 1 + k: index R 2^s + r 2^s + k), then for the
        // contiguous stages s = 4..7 and k < 2^(s-4) the 16 pairs of threads t
        // (slot 15 + 16 (2^(s-4) - 1 + k) + t: index R 2^s + r 2^s + 2^(s-4) t + k).
        // Inverse, per row r: contiguous distances 2^lt (lt = 0..3, h = N/2^(lt+1),
        // slot 16 (o_lt + k) + t with o = 0, 8, 12, 14: index h + r 2^(7-lt) + 2^(3-lt) t + k),
        // then strided lt = 4..7 (slot 240 + o_(lt-4) + k: index h + r 2^(7-lt) + k).
        const int R = N >> 8, W = 255;
        std::vector<u64> rt((size_t)2 * M * R * W), irt((size_t)2 * M * R * W);
        const int off4[4] = {0, 8, 12, 14};
        for (int t = 0; t < M; t++)
            for (int r = 0; r < R; r++) {
                const size_t o = ((size_t)t * R + r) * W;
                auto put = [&](std::vector<u64> &dst, const std::vector<u64> &src, int slot, size_t idx) {
                    dst[2 * (o + slot)] = src[2 * ((size_t)t * N + idx)];
                    dst[2 * (o + slot) + 1] = src[2 * ((size_t)t * N + idx) + 1];
                };
                for (int st = 0; st < 4; st++)
                    for (int k = 0; k < (1 << st); k++)
                        put(rt, psi, (1 << st) - 1 + k, ((size_t)R << st) + ((size_t)r << st) + k);
                for (int st = 4; st < 8; st++)
                    for (int k = 0; k < (1 << (st - 4)); k++)
                        for (int th = 0; th < 16; th++)
                            put(rt, psi, 15 + 16 * ((1 << (st - 4)) - 1 + k) + th,
                                ((size_t)R << st) + ((size_t)r << st) + ((size_t)th << (st - 4)) + k);
                for (int lt = 0; lt < 4; lt++) {
                    const size_t h = (size_t)(N >> 1) >> lt;
                    for (int k = 0; k < (8 >> lt); k++)
                        for (int th = 0; th < 16; th++)
                            put(irt, ipsi, 16 * (off4[lt] + k) + th,
                                h + (size_t)r * (128 >> lt) + (size_t)th * (8 >> lt) + k);
                }
                for (int lt = 4; lt < 8; lt++) {
                    const size_t h = (size_t)(N >> 1) >> lt;
                    for (int k = 0; k < (128 >> lt); k++)
                        put(irt, ipsi, 240 + off4[lt - 4] + k, h + (size_t)r * (128 >> lt) + k);
                }
            }
        d_rowtw = reinterpret_cast<ulonglong2 *>(upload(*this, rt));
        d_irowtw = reinterpret_cast<ulonglong2 *>(upload(*this, irt));
    }
    d_ninv = upload(*this, ninv);
    d_ninv_sh = upload(*this, ninv_sh);
    d_imag = upload(*this, imag);
    d_imag_sh = upload(*this, imag_sh);

    // ModDown constants
    std::vector<u64> pinv(p.L), pinv_sh(p.L), phinv(p.K), phm((size_t)p.L * p.K);
    for (int k = 0; k < p.K; k++) {
        u64 pk = p.mod[p.L + k];
        u64 hat = 1;
        for (int b = 0; b < p.K; b++)
            if (b != k) hat = host_mulmod(hat, p.mod[p.L + b] % pk, pk);
        phinv[k] = host_invmod(hat, pk);
    }
    for (int i = 0; i < p.L; i++) {
        u64 qi = p.mod[i];
        u64 P = 1;
        for (int k = 0; k < p.K; k++) P = host_mulmod(P, p.mod[p.L + k] % qi, qi);
        pinv[i] = host_invmod(P, qi);
        pinv_sh[i] = host_shoup(pinv[i], qi);
        for (int k = 0; k < p.K; k++) {
            u64 hat = 1;
            for (int b = 0; b < p.K; b++)
                if (b != k) hat = host_mulmod(hat, p.mod[p.L + b] % qi, qi);
            phm[(size_t)i * p.K + k] = host_mont(hat, qi);
        }
    }
    d_pinv_q = upload(*this, pinv);
    d_pinv_q_sh = upload(*this, pinv_sh);
    std::vector<u64> mds(p.K), mds_sh(p.K);
    for (int k = 0; k < p.K; k++) {
        u64 pk = p.mod[p.L + k];
        mds[k] = host_mulmod(host_invmod((u64)N % pk, pk), phinv[k], pk);
        mds_sh[k] = host_shoup(mds[k], pk);
    }
    d_md_scale = upload(*this, mds);
    d_md_scale_sh = upload(*this, mds_sh);
    d_phat_mont = upload(*this, phm);

    // rescale constants q_l^{-1} mod q_i
    std::vector<u64> ql((size_t)p.L * p.L, 0), ql_sh((size_t)p.L * p.L, 0);
    for (int l = 1; l < p.L; l++)
        for (int i = 0; i < l; i++) {
            u64 v = host_invmod(p.mod[l] % p.mod[i], p.mod[i]);
            ql[(size_t)l * p.L + i] = v;
            ql_sh[(size_t)l * p.L + i] = host_shoup(v, p.mod[i]);
        }
    d_qlinv = upload(*this, ql);
    d_qlinv_sh = upload(*this, ql_sh);

    // slot positions for encode / decode
    std::vector<int> pos(N / 2);
    u64 e = 1;
    for (int j = 0; j < N / 2; j++) {
        pos[j] = (int)((e - 1) / 2);
        e = (e * 5) % (2 * (u64)N);
    }
    HETAL_CUDA_CHECK(cudaMalloc(&d_slot_pos, sizeof(int) * (N / 2)));
    HETAL_CUDA_CHECK(cudaMemcpy(d_slot_pos, pos.data(), sizeof(int) * (N / 2), cudaMemcpyHostToDevice));
    HETAL_CUDA_CHECK(cudaDeviceSynchronize());
}

Context::~Context()
{
    cudaStreamSynchronize(stream);
    pt_cache.clear();   // frees on the stream, before the stream goes away
    cudaStreamSynchronize(stream);
    prof_reset();
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    for (auto &kv : modup_cache) {
        cudaFree(kv.second.hat_mont);
    }
    for (auto &kv : modup_scale_cache) {
        cudaFree(kv.second.sc);
        cudaFree(kv.second.sc_sh);
    }
    void *ptrs[] = {d_mc, d_psi2, d_ipsi2, d_rowtw, d_irowtw, d_ninv, d_ninv_sh, d_imag, d_imag_sh,
                    d_pinv_q, d_pinv_q_sh, d_md_scale, d_md_scale_sh, d_phat_mont, d_qlinv, d_qlinv_sh,
                    d_slot_pos};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (own_stream) cudaStreamDestroy(stream);
}

u64 *Context::alloc(size_t words) { return (u64 *)alloc_bytes(words * sizeof(u64)); }

void Context::free(u64 *ptr) { free_bytes(ptr); }

void *Context::alloc_bytes(size_t bytes)
{
    void *ptr = nullptr;
    cudaError_t e = cudaMallocAsync(&ptr, std::max<size_t>(bytes, 16), stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(e == cudaErrorMemoryAllocation ? ERR_OOM : ERR_CUDA,
                    std::string("device allocation of ") + std::to_string(bytes) + " bytes failed: " +
                        cudaGetErrorString(e));
    }
    allocs++;
    return ptr;
}

void Context::free_bytes(void *ptr)
{
    if (ptr && cudaFreeAsync(ptr, stream) != cudaSuccess) cudaGetLastError();
}

void Context::sync()
{
    if (recording) throw Error(ERR_RECORDING, "a call that waits for the device cannot be recorded into a graph");
    HETAL_CUDA_CHECK(cudaStreamSynchronize(stream));
}

static cudaEvent_t take_event(std::vector<cudaEvent_t> &pool)
{
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    HETAL_CUDA_CHECK(cudaEventCreate(&e));
    return e;
}

bool Context::launch_begin(const char *name)
{
    ++launches;
    if (prof_target.empty() || (prof_target != "*" && prof_target != name)) return false;
    ProfRec r;
    r.a = take_event(ev_pool);
    r.b = take_event(ev_pool);
    r.modmul = r.bytes = 0;
    r.name = name;
    HETAL_CUDA_CHECK(cudaEventRecord(r.a, stream));
    prof.push_back(r);
    return true;
}

void Context::launch_end(bool timed, double modmul, double bytes)
{
    if (!timed) return;
    ProfRec &r = prof.back();
    HETAL_CUDA_CHECK(cudaEventRecord(r.b, stream));
    r.modmul = modmul;
    r.bytes = bytes;
}

void Context::prof_reset()
{
    for (auto &r : prof) {
        ev_pool.push_back(r.a);
        ev_pool.push_back(r.b);
    }
    prof.clear();
}

LimbMap Context::q_map(int lv) const
{
    LimbMap m;
    m.n = lv + 1;
    for (int i = 0; i <= lv; i++) m.idx[i] = (unsigned char)i;
    return m;
}

LimbMap Context::ext_map(int lv) const
{
    LimbMap m;
    m.n = lv + 1 + p.K;
    for (int t = 0; t < m.n; t++) m.idx[t] = (unsigned char)ext_mod(lv, t);
    return m;
}

LimbMap identity_pos(int n)
{
    LimbMap m;
    m.n = n;
    for (int i = 0; i < n; i++) m.idx[i] = (unsigned char)i;
    return m;
}

const ModUpTables &Context::modup_tables(int lv, int j)
{
    auto key = std::make_pair(lv, j);
    auto it = modup_cache.find(key);
    if (it != modup_cache.end()) return it->second;
    ModUpTables t;
    int lo = j * p.alpha, hi = std::min((j + 1) * p.alpha, lv + 1);
    t.a = hi - lo;
    t.src.n = t.a;
    for (int a = 0; a < t.a; a++) t.src.idx[a] = (unsigned char)(lo + a);
    int next = lv + 1 + p.K;
    t.dst.n = 0;
    t.dst_pos.n = 0;
    for (int pos = 0; pos < next; pos++) {
        if (pos >= lo && pos < hi) continue;
        t.dst.idx[t.dst.n++] = (unsigned char)ext_mod(lv, pos);
        t.dst_pos.idx[t.dst_pos.n++] = (unsigned char)pos;
    }
    t.nt = t.dst.n;
    std::vector<u64> ih(t.a), hm((size_t)t.nt * t.a);
    for (int a = 0; a < t.a; a++) {
        u64 qa = p.mod[lo + a];
        u64 hat = 1;
        for (int b = 0; b < t.a; b++)
            if (b != a) hat = host_mulmod(hat, p.mod[lo + b] % qa, qa);
        ih[a] = host_invmod(hat, qa);
    }
    for (int d = 0; d < t.nt; d++) {
        u64 m = p.mod[t.dst.idx[d]];
        for (int a = 0; a < t.a; a++) {
            u64 hat = 1;
            for (int b = 0; b < t.a; b++)
                if (b != a) hat = host_mulmod(hat, p.mod[lo + b] % m, m);
            hm[(size_t)d * t.a + a] = host_mont(hat, m);
        }
    }
    t.hat_mont = upload(*this, hm);
    t.h_inv_hat = ih;
    return modup_cache.emplace(key, t).first->second;
}

const Context::LimbScale &Context::modup_scale(int lv)
{
    auto it = modup_scale_cache.find(lv);
    if (it != modup_scale_cache.end()) return it->second;
    std::vector<u64> sc(lv + 1), sc_sh(lv + 1);
    for (int j = 0; j < p.dnum(lv); j++) {
        const ModUpTables &t = modup_tables(lv, j);
        for (int a = 0; a < t.a; a++) {
            const int i = t.src.idx[a];
            const u64 q = p.mod[i];
            sc[i] = host_mulmod(host_invmod((u64)p.N % q, q), t.h_inv_hat[a], q);
            sc_sh[i] = host_shoup(sc[i], q);
        }
    }
    LimbScale ls;
    ls.sc = upload(*this, sc);
    ls.sc_sh = upload(*this, sc_sh);
    return modup_scale_cache.emplace(lv, ls).first->second;
}

}  // namespace hetal
