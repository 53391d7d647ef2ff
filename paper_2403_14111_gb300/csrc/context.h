// context.h -- host-side runtime of the GB300 RNS-CKKS library: parameters,
// device tables, stream-ordered device memory, ciphertext / key containers
// and the launch wrappers of every kernel.
#pragma once
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace hetal {

enum Status {
    OK = 0,
    ERR_INVALID_ARG = -1,
    ERR_SHAPE = -2,
    ERR_LEVEL = -3,
    ERR_MISSING_KEY = -4,
    ERR_OOM = -5,
    ERR_CUDA = -6,
    ERR_SCALE = -7,
    ERR_TIMEOUT = -8,
    ERR_RECORDING = -9,
    ERR_CANCELLED = -10,
};

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

struct CudaError : Error {
    CudaError(cudaError_t e, const char *expr, const char *file, int line)
        : Error(e == cudaErrorMemoryAllocation ? ERR_OOM : ERR_CUDA,
                std::string(cudaGetErrorString(e)) + " at " + expr + " (" + file + ":" + std::to_string(line) + ")") {}
};

// Operation counters (paper-level operations and primitive work).
struct Counters {
    long long cmult = 0, mult = 0, rot = 0, conj = 0;
    long long keyswitch = 0, modup_digits = 0, ntt_limbs = 0, rescale = 0;
    double modmul = 0;          // algorithmic modular multiplies issued
    double bytes = 0;           // algorithmic bytes (ciphertexts in/out, keys)
};

struct Params {
    int logN = 0, N = 0;
    int L = 0;       // ciphertext primes q_0..q_{L-1}
    int K = 0;       // special primes p_0..p_{K-1} (modulus index L..L+K-1)
    int alpha = 0;   // primes per key-switching digit
    int h = 0;       // secret Hamming weight
    double scale = 0;
    std::vector<u64> mod;     // L + K moduli
    std::vector<u64> psi;     // primitive 2N-th roots
    int dnum_full() const { return (L + alpha - 1) / alpha; }
    int dnum(int lv) const { return (lv + 1 + alpha - 1) / alpha; }
    int slots() const { return N / 2; }
};

// Creates the prime chain of a parameter request (host, independent of any
// other implementation): q_0 = largest prime < 2^q0_bits with q = 1 mod 2N,
// then the n_rescale largest below 2^rescale_bits, then (levels above those) the
// n_upper largest below 2^upper_bits, then n_special below 2^special_bits,
// skipping primes already taken.
Params make_params(int log_n, int q0_bits, int n_rescale, int rescale_bits, int n_special,
                   int special_bits, int alpha, int h, double scale, int n_upper = 0, int upper_bits = 0);

// Device-side view of a batch of polynomials: poly p, limb l at
// ptr + p * stride + l * N.
struct PolyBatch {
    u64 *ptr;
    int count;
    size_t stride;
};

class Context;

// Non-owning view of n ciphertexts at level lv, NTT domain, packed as
// data[i][c][limb][N] (i < n, c < 2, limb <= lv).
struct CtView {
    u64 *data = nullptr;
    int n = 0;
    int lv = -1;
    double scale = 0;
    int N = 0;
    size_t ct_words() const { return (size_t)2 * (lv + 1) * N; }
    u64 *ct(int i) const { return data + (size_t)i * ct_words(); }
    PolyBatch polys() const { return PolyBatch{data, 2 * n, (size_t)(lv + 1) * N}; }
    PolyBatch comp(int c) const { return PolyBatch{data + (size_t)c * (lv + 1) * N, n, ct_words()}; }
    CtView sub(int first, int count) const
    {
        CtView v = *this;
        v.data = ct(first);
        v.n = count;
        return v;
    }
};

// Deleter of an allocation shared by the slices of one batch: frees on its context's
// stream.  The context can be changed (rehome) while slices are alive.
struct FreeOn {
    Context *c;
    void operator()(u64 *p) const;
};

// A batch of n ciphertexts at level lv, NTT domain: data[i][c][limb][N].
struct CtBatch {
    Context *ctx = nullptr;
    u64 *data = nullptr;
    int n = 0;
    int lv = -1;
    double scale = 0;
    // set on the slices of one allocation made by split(); the allocation is
    // freed (on ctx's stream) with the last slice
    std::shared_ptr<u64> shared;
    CtBatch() = default;
    CtBatch(Context *c, int n_, int lv_, double scale_);
    CtBatch(const CtBatch &) = delete;
    CtBatch &operator=(const CtBatch &) = delete;
    CtBatch(CtBatch &&o) noexcept { *this = std::move(o); }
    CtBatch &operator=(CtBatch &&o) noexcept;
    ~CtBatch();
    size_t ct_words() const;
    u64 *ct(int i) const { return data + (size_t)i * ct_words(); }
    PolyBatch polys() const;      // 2n polys
    PolyBatch comp(int c) const;  // component c of each ciphertext (n polys)
    CtView view() const;
    operator CtView() const { return view(); }
    // `parts` batches of whole.n / parts ciphertexts each, in order, sharing whole's memory
    static std::vector<CtBatch> split(CtBatch &&whole, int parts);
    // consecutive batches of sizes[i] ciphertexts (summing to whole.n), sharing whole's memory
    static std::vector<CtBatch> split_sizes(CtBatch &&whole, const std::vector<int> &sizes);
    // Hands the batch (and every slice sharing its memory) to another context of the same
    // device: later frees are ordered on that context's stream.  The caller has made sure
    // that no work of the old context uses the memory any more (its stream was synchronised).
    void rehome(Context *to);
};

// Switching key: [dnum_full][2][L+K][N], NTT domain, Montgomery form (x * 2^64 mod m).
struct SwitchKey {
    u64 *data = nullptr;
};

struct SecretKey {
    std::vector<long long> coeffs;   // host copy of the ternary secret
    u64 *ntt = nullptr;              // [L+K][N], NTT domain
};

struct EvalKeys {
    SwitchKey relin, conj;
    std::map<int, SwitchKey> rot;    // left rotation amount in [1, s)
    bool has_relin = false, has_conj = false;
};

// Plaintext over moduli 0..lv in the NTT domain: normal form (for additions)
// and Montgomery form (for products).
struct Plain {
    Context *ctx = nullptr;
    u64 *data = nullptr;
    u64 *mont = nullptr;
    int lv = -1;
    double scale = 0;
    Plain() = default;
    Plain(const Plain &) = delete;
    Plain &operator=(const Plain &) = delete;
    Plain(Plain &&o) noexcept { *this = std::move(o); }
    Plain &operator=(Plain &&o) noexcept;
    ~Plain();
};

// Integer plaintexts supplied by the caller, keyed by (kind, index, level).
struct PtSet {
    std::map<std::tuple<int, int, int>, std::vector<long long>> pts;
};

struct ModUpTables {
    // digit limbs I (count a), targets T (count nt)
    int a = 0, nt = 0;
    u64 *hat_mont = nullptr;                         // [nt][a] ((D/q_i) mod m_t) * 2^64 mod m_t
    std::vector<u64> h_inv_hat;                      // [a]  (D/q_i)^{-1} mod q_i (host)
    LimbMap src, dst;                                // moduli of digit limbs, target limbs
    LimbMap dst_pos;                                 // positions of the targets in the extended layout
};

class Context {
  public:
    Params p;
    int device = 0;
    int sm_count = 0;   // streaming multiprocessors of the device
    // true while the stream is being captured into a CUDA graph: calls that wait
    // for the device (sync) are refused
    bool recording = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string last_error;
    Counters cnt;

    // device tables
    ModConst *d_mc = nullptr;
    ulonglong2 *d_psi2 = nullptr;    // [L+K][N]  (psi^{brv(i)}, its Shoup companion)
    ulonglong2 *d_ipsi2 = nullptr;   // [L+K][N]  (psi^{-brv(i)}, its Shoup companion)
    // The row passes' twiddles (psi2 / ipsi2 entries R .. N-1, R = N/256) in the
    // order the row kernels read them: [L+K][R rows][255], see ntt.cu.
    ulonglong2 *d_rowtw = nullptr, *d_irowtw = nullptr;
    u64 *d_ninv = nullptr, *d_ninv_sh = nullptr;   // [L+K]
    u64 *d_imag = nullptr, *d_imag_sh = nullptr;   // [L+K]  psi^{N/2}
    u64 *d_pinv_q = nullptr, *d_pinv_q_sh = nullptr;     // [L]  P^{-1} mod q_i
    u64 *d_md_scale = nullptr, *d_md_scale_sh = nullptr; // [K]  N^{-1} (P/p_k)^{-1} mod p_k (ModDown INTT)
    u64 *d_phat_mont = nullptr;                          // [L][K] ((P/p_k) mod q_i) * 2^64 mod q_i
    u64 *d_qlinv = nullptr, *d_qlinv_sh = nullptr;       // [L][L] q_l^{-1} mod q_i
    int *d_slot_pos = nullptr;                           // [N/2] (5^j mod 2N - 1) / 2
    std::vector<ModConst> h_mc;
    std::map<std::pair<int, int>, ModUpTables> modup_cache;
    struct LimbScale {
        u64 *sc = nullptr, *sc_sh = nullptr;
    };
    std::map<int, LimbScale> modup_scale_cache;

    Context(const Params &prm, int dev, cudaStream_t s);
    ~Context();

    u64 *alloc(size_t words);
    void free(u64 *ptr);
    void *alloc_bytes(size_t bytes);
    void free_bytes(void *ptr);
    void sync();

    // Plaintexts the library encoded itself (masks, constants), kept across calls:
    // (kind, index, level, c, s0, s1, bits of t or coefficient, bits of scale / input hash).
    using PtKey = std::tuple<int, int, int, int, int, int, u64, u64>;
    std::map<PtKey, Plain> pt_cache;
    // NTT row passes: polynomials per CTA with the rows' twiddles staged in shared memory
    // (1: one polynomial per CTA, twiddles read from L2 per polynomial)
    int row_group = 1;
    // tables of the 32-bit-word transform (ntt32.cu), made on first use
    std::shared_ptr<void> ntt32;
    // Target size of one batched operation's ciphertexts; the matrix products
    // process their c/2 diagonals in chunks that stay near it.
    size_t batch_bytes = (size_t)8 << 30;

    const ModUpTables &modup_tables(int lv, int j);
    // [lv+1]: N^{-1} (D_j/q_i)^{-1} mod q_i for limb i of digit j (ModUp INTT scaling)
    const LimbScale &modup_scale(int lv);
    LimbMap q_map(int lv) const;            // moduli 0..lv
    LimbMap ext_map(int lv) const;          // 0..lv, L..L+K-1
    int ext_mod(int lv, int t) const { return t <= lv ? t : p.L + (t - lv - 1); }

    // Launch accounting and per-kernel timing.  Every launch wrapper calls
    // launch_begin / launch_end with the kernel's name and the algorithmic work
    // of that launch; when `name` is the profiled kernel, CUDA events are
    // recorded around it on the context's stream.
    long long launches = 0;
    long long allocs = 0;   // device allocations made through alloc / alloc_bytes
    std::string prof_target;
    struct ProfRec {
        cudaEvent_t a, b;
        double modmul, bytes;
        const char *name;   // a string literal of the launch wrapper
    };
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    bool launch_begin(const char *name);
    void launch_end(bool timed, double modmul, double bytes);
    void prof_reset();
};

// RAII device buffer on a context's stream.
struct DBuf {
    Context *ctx = nullptr;
    u64 *ptr = nullptr;
    DBuf() = default;
    DBuf(Context *c, size_t words) : ctx(c), ptr(c->alloc(words)) {}
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : ctx(o.ctx), ptr(o.ptr) { o.ptr = nullptr; }
    DBuf &operator=(DBuf &&o) noexcept
    {
        if (this != &o) {
            if (ptr) ctx->free(ptr);
            ctx = o.ctx;
            ptr = o.ptr;
            o.ptr = nullptr;
        }
        return *this;
    }
    ~DBuf()
    {
        if (ptr) ctx->free(ptr);
    }
};

// ---------------------------------------------------------------------------
// Kernel launch wrappers (kernels.cu / ntt.cu).  All run on ctx->stream.
// ---------------------------------------------------------------------------
// Forward / inverse negacyclic NTT of every limb of every poly; limb l of a
// poly is at position pos.idx[l] and uses modulus mods.idx[l].  Forward output
// is bit-reversed (slot j = value at psi^{2 brv(j) + 1}); inverse takes that order.
void ntt_forward(Context &c, PolyBatch b, const LimbMap &mods, const LimbMap &pos);
void ntt_inverse(Context &c, PolyBatch b, const LimbMap &mods, const LimbMap &pos);
LimbMap identity_pos(int n);

// Elementwise (limb l of every poly uses modulus mods.idx[l]; n_limbs = mods.n).
void k_add(Context &c, PolyBatch out, PolyBatch a, PolyBatch b, const LimbMap &mods);
void k_sub(Context &c, PolyBatch out, PolyBatch a, PolyBatch b, const LimbMap &mods);
void k_neg(Context &c, PolyBatch out, PolyBatch a, const LimbMap &mods);
void k_copy(Context &c, PolyBatch out, PolyBatch a, int n_limbs);
// out = a (.) pt, pt a single Montgomery-form poly broadcast over the batch.
void k_mul_plain(Context &c, PolyBatch out, PolyBatch a, const u64 *pt, const LimbMap &mods);
// out = a (.) pa + b (.) pb (Montgomery plaintexts [limb][N], one reduction)
// out = sum_i (poly of cts[i]) (.) pts[i] (Montgomery plaintexts [limb][N]); every term's
// polynomials at stride ps; up to PSUM_MAX terms a launch, later launches adding on.
constexpr int PSUM_MAX = 32;
void k_mul_plain_sum(Context &c, PolyBatch out, const std::vector<const u64 *> &cts, size_t ps,
                     const std::vector<const u64 *> &pts, const LimbMap &mods);
void k_mul_plain2(Context &c, PolyBatch out, PolyBatch a, const u64 *pa, PolyBatch b, const u64 *pb,
                  const LimbMap &mods);
// out = a (.) b (both normal form), Barrett.
void k_mul(Context &c, PolyBatch out, PolyBatch a, PolyBatch b, const LimbMap &mods);
// multiply by X^{N/2} in the NTT domain
void k_mul_i(Context &c, PolyBatch out, PolyBatch a, const LimbMap &mods);
// to Montgomery form (x * 2^64 mod q)
void k_to_mont(Context &c, PolyBatch out, PolyBatch a, const LimbMap &mods);
// tensor of ciphertext pairs: d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1 (count n each)
void k_tensor(Context &c, PolyBatch d0, PolyBatch d1, PolyBatch d2, PolyBatch a0, PolyBatch a1, PolyBatch b0,
              PolyBatch b1, int lv);
// X -> X^g in the NTT domain
void k_automorphism(Context &c, PolyBatch out, PolyBatch in, int n_limbs, u64 g);
// tensor products of G groups of n pairs (a_g: n ciphertexts at level lv; b_g: n, or 1 when
// bstep[g] == 0) into d = [3][total][lv+1][N], group g at polys g * n .. g * n + n - 1
void k_tensor_groups(Context &c, u64 *d, int total, const std::vector<const u64 *> &a,
                     const std::vector<const u64 *> &b, const std::vector<int> &bstep, int n, int lv);
// the same summed over each group's n pairs: d = [3][G][lv+1][N], group g's sum at poly g
void k_tensor_sum_groups(Context &c, u64 *d, int G, const std::vector<const u64 *> &a,
                         const std::vector<const u64 *> &b, const std::vector<int> &bstep, int n, int lv);
// the same with n_g pairs in group g
void k_tensor_sum_ragged(Context &c, u64 *d, int G, const std::vector<const u64 *> &a,
                         const std::vector<const u64 *> &b, const std::vector<int> &bstep, const std::vector<int> &ns,
                         int lv);
// Work lists over ragged batches (persistent grid, items = ciphertext x limb x run of coefficients):
// ciphertext z of out = ciphertext z of a (.) pts[z] (Montgomery plaintexts [limb][N]);
// out and a hold 2 * pts.size() polys (both components of each ciphertext)
void k_mul_plain_list(Context &c, PolyBatch out, PolyBatch a, const std::vector<const u64 *> &pts,
                      const LimbMap &mods);
// ciphertext z of out = (itself if accumulate) + sum_{i < len[z]} ciphertext start[z] + i of in
// (out and in are component polys, 2 per ciphertext)
void k_sum_ranges(Context &c, PolyBatch out, PolyBatch in, const std::vector<int> &start, const std::vector<int> &len,
                  bool accumulate, const LimbMap &mods);
// Same on the 2n interleaved component polys of a ciphertext batch, adding add0[i]
// (n polys, limb l mod q_l) to component 0 of ciphertext i.
void k_automorphism_add0(Context &c, PolyBatch out, PolyBatch in, PolyBatch add0, int n_limbs, u64 g);
// signed 64-bit coefficients -> residues on mods (coefficient domain), batched
void k_reduce_i64(Context &c, PolyBatch out, const long long *in, size_t in_stride, const LimbMap &mods);
// out[p][x] = residue of limb 0 of in[p] modulo q, centred into (-q/2, q/2]
void k_center_i64(Context &c, long long *out, PolyBatch in, u64 q);
// *d_bad |= 1 when a residue of limb l of any poly is not below modulus mods.idx[l]
void k_check_range(Context &c, PolyBatch in, const LimbMap &mods, unsigned *d_bad);
// sum of a batch of polys into one (out has count 1)
void k_sum_polys(Context &c, PolyBatch out, PolyBatch in, int groups, const LimbMap &mods);

// Key inner product with optional automorphism of the extended digits:
// acc_c[b][t] = sum_j ext_j[b][t](X^g) * key_{j,c}[mod(t)]  (Montgomery keys)
void k_kip(Context &c, PolyBatch acc0, PolyBatch acc1, const u64 *ext, size_t ext_digit_stride, int dnum,
           const u64 *key, int lv, u64 g, PolyBatch own);
// The same for several keys / Galois elements at once (hoisted rotations): step s
// writes acc polys s * B .. s * B + B - 1 from the B polys of own / ext.
constexpr int MAX_KS_STEPS = 64;   // steps per launch (longer lists take several)
void k_kip_steps(Context &c, PolyBatch acc0, PolyBatch acc1, const u64 *ext, size_t ext_digit_stride, int dnum,
                 const std::vector<const u64 *> &keys, const std::vector<u64> &gs, int lv, PolyBatch own);
// out[s * B + p] = in[p](X^{g_s}) for the B = in.count polys and every step s
void k_automorphism_steps(Context &c, PolyBatch out, PolyBatch in, const std::vector<u64> &gs, int n_limbs);
// One accumulator per poly for a + sum_s Lrot(a, r_s): acc_c[p] = sum_s sum_j
// ext_j[p](X^{g_s}) * key_{s,j,c}  (acc0/acc1/own: B polys; at most MAX_KS_STEPS steps)
void k_kip_sum(Context &c, PolyBatch acc0, PolyBatch acc1, const u64 *ext, size_t ext_digit_stride, int dnum,
               const std::vector<const u64 *> &keys, const std::vector<u64> &gs, int lv, PolyBatch own);
// out[p] = in[p] + sum_s in[p](X^{g_s})  (limb l mod q_l)
void k_automorphism_sum(Context &c, PolyBatch out, PolyBatch in, const std::vector<u64> &gs, int n_limbs);
// out-of-place inverse NTT (positions `pos` in both batches)
void ntt_inverse_oop(Context &c, PolyBatch out, PolyBatch in, const LimbMap &mods, const LimbMap &pos);
// Inverse NTT whose final scaling by N^{-1} is replaced by sc[l] (Shoup sc_sh[l])
// for launch limb l: a base conversion's first factor folded into the transform.
void ntt_inverse_scaled(Context &c, PolyBatch out, PolyBatch in, const LimbMap &mods, const LimbMap &pos,
                        const u64 *sc, const u64 *sc_sh);
// ModDown tail fused into the forward NTT of conv = [conv_0 (B polys), conv_1 (B polys)]
// over limbs 0..lv: out_c = (acc_c - NTT(conv_c)) * P^{-1} (+ addend_c if given),
// written in place of the transform (conv keeps the column-pass intermediate).
struct ModDownTail {
    PolyBatch out[2], acc[2], add[2];
    int B;
};
void ntt_forward_moddown(Context &c, PolyBatch conv, int lv, const ModDownTail &tail);
// Fast base conversion fused into the first pass of a forward NTT: the column pass
// reads limb l of poly p as REDC(sum_{a<na} src[p][src_pos[a]] * hat[l * na + a])
// mod m_{mods[l]} (hat in Montgomery form) instead of loading it from the output
// batch.  The result equals k_base_conv into the output followed by the transform.
struct ConvSrc {
    PolyBatch src;
    LimbMap src_pos;
    const u64 *hat;
    int na;
};
// na above this runs k_base_conv, then the transform.  The fused sum of na products below
// q^2 is reduced once (REDC needs it below q 2^64: na q < 2^64, true for q < 2^61 up to 8).
constexpr int MAX_FUSED_CONV = 8;
void ntt_forward_conv(Context &c, PolyBatch out, const LimbMap &mods, const LimbMap &pos, const ConvSrc &cv);
void ntt_forward_moddown_conv(Context &c, PolyBatch conv, int lv, const ModDownTail &tail, const ConvSrc &cv);
// Fast base conversion after the first factor: out[p][dst_pos[d]] =
// REDC(sum_{a<na} in[p][src_pos[a]] * hat[d * na + a]) mod m_{dst_mod[d]},
// hat in Montgomery form (na <= 7).
void k_base_conv(Context &c, const char *name, PolyBatch out, PolyBatch in, int na, const LimbMap &src_pos,
                 const LimbMap &dst_mod, const LimbMap &dst_pos, const u64 *hat);
// out = a + s_l * b per limb l (s given per limb, Shoup form)
struct ScalarMap {
    u64 v[HETAL_MAX_MODULI];
    u64 vs[HETAL_MAX_MODULI];
};
void k_axpy_scalar(Context &c, PolyBatch out, PolyBatch a, PolyBatch b, const ScalarMap &s, const LimbMap &mods);
// out = a * s_l per limb l (s given per limb, Shoup form)
void k_mul_scalar(Context &c, PolyBatch out, PolyBatch a, const ScalarMap &s, const LimbMap &mods);
// device-generated block masks (slot vectors, real and imaginary parts), see matmul.cpp
void k_make_mask(Context &c, double *re, double *im, int kind, int k, int cc, int s0, int s1, double t);
// out[i] = a * v[i] (real slot vectors of length n)
void k_scale_vec(Context &c, double *out, const double *v, double a, int n);
// from Montgomery form (x * 2^-64 mod q)
void k_from_mont(Context &c, PolyBatch out, PolyBatch a, const LimbMap &mods);
// block layout of a row-major rows x cols matrix into slot vectors [m*n][s0*s1]
// (tiling 0 none, 1 vertical copies of period tile_c, 2 horizontal copies)
void k_block_layout(Context &c, double *slots, const double *src, int rows, int cols, int m, int n, int s0, int s1,
                    int tiling, int tile_c);
// inverse layout: slot vectors [m*n][s0*s1] -> (m*s0) x (n*s1) row-major
void k_block_unlayout(Context &c, double *dst, const double *slots, int m, int n, int s0, int s1);
// rescale helpers
void k_rescale_spread(Context &c, PolyBatch out, PolyBatch top, int lv);   // centred top limb -> limbs 0..lv-1
void k_rescale_finish(Context &c, PolyBatch out, PolyBatch in, PolyBatch spread, int lv);

// samplers (Philox4x64-10)
void k_sample_uniform(Context &c, PolyBatch out, u64 seed, u64 stream, const LimbMap &mods);
void k_sample_cbd(Context &c, long long *out, int count, size_t stride, u64 seed, const u64 *streams_host);
void k_sample_secret(Context &c, long long *out, u64 seed, u64 stream, int h);

// FP64 canonical-embedding encode / decode
void k_encode(Context &c, long long *out, const double *z_re, const double *z_im, int count, double scale);
void k_decode(Context &c, double *z_re, double *z_im, const double *m, int count, double inv_scale);
// limb 0 of NTT-domain c0 + c1*s, then INTT, centred, as doubles: m[b][x]
void k_center_to_double(Context &c, double *out, PolyBatch in, int count);

// 32-bit-word transform (ntt32.cu): the first `limbs` primes below 2^30 that are 1 mod 2N
// (descending) and their 2N-th roots; forward NTT of polys[p][limb][N] (uint32, limb l mod
// prime l), bit-reversed output; register-only rate of its butterfly
std::vector<uint32_t> ntt32_moduli(Context &c, int limbs, std::vector<uint32_t> *roots);
void ntt32_forward(Context &c, uint32_t *polys, int n_polys, int limbs);
double probe_butterfly32_rate(Context &c, int iters, int blocks_per_sm);
// register-only loop of the NTT butterfly; returns butterflies per second
double probe_butterfly_rate(Context &c, int iters, int blocks_per_sm);
// register-only loop of the 128-bit multiply-accumulate; returns products per second
double probe_mac_rate(Context &c, int iters, int blocks_per_sm);

// Montgomery constant helper (host)
u64 host_mulmod(u64 a, u64 b, u64 m);
u64 host_powmod(u64 a, u64 e, u64 m);
u64 host_invmod(u64 a, u64 m);
u64 host_shoup(u64 w, u64 m);
u64 host_mont(u64 x, u64 m);

}  // namespace hetal
