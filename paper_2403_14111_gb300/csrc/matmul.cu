// matmul.cu -- DiagABT and DiagATB (arXiv 2403.14111, Sec. 4.2 and App. B),
// and the degree-15 softmax stand-in of the encrypted training step.
//
// The operation order of every ciphertext follows the paper's algorithms
// (Algorithm DiagABT, RotLeft, PRotUp, DiagATB in App. B.3) with the
// multi-block lifting of App. B.1.  The c/2 iterations of the k-loop are
// independent until their results are summed, so they run together: a chunk
// of k values (as many as fit a memory budget) goes through each step as one
// batched operation over all its blocks.  Every ciphertext sees the same
// operations as in the sequential loop, so the bits are the same.
#include "matmul.h"

#include <set>

#include <cmath>
#include <cstring>

namespace hetal {

static bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }
static int ilog2(int x)
{
    int r = 0;
    while ((1 << r) < x) r++;
    return r;
}

const Plain *PtProvider::lookup(int kind, int k, int lv, double scale)
{
    auto key = std::make_tuple(kind, k, lv);
    auto it = cache_.find(key);
    if (it != cache_.end()) return &it->second;
    if (set_) {
        auto s = set_->pts.find(key);
        if (s != set_->pts.end()) {
            if ((int)s->second.size() != c_.p.N) throw Error(ERR_INVALID_ARG, "supplied plaintext has wrong length");
            long long *d = (long long *)c_.alloc_bytes(sizeof(long long) * c_.p.N);
            HETAL_CUDA_CHECK(cudaMemcpyAsync(d, s->second.data(), sizeof(long long) * c_.p.N, cudaMemcpyHostToDevice,
                                             c_.stream));
            Plain pt = plain_from_int(c_, d, lv, scale);
            c_.sync();
            c_.free_bytes(d);
            return &cache_.emplace(key, std::move(pt)).first->second;
        }
    }
    return nullptr;
}

static u64 dbits(double x)
{
    u64 b;
    std::memcpy(&b, &x, sizeof b);
    return b;
}

// Plaintexts the library encodes itself are kept on the context across calls
// (a training loop multiplies by the same masks every step).
static Plain *ctx_cached(Context &c, const Context::PtKey &key)
{
    auto it = c.pt_cache.find(key);
    return it == c.pt_cache.end() ? nullptr : &it->second;
}

static const Plain &ctx_store(Context &c, const Context::PtKey &key, Plain &&pt)
{
    if (c.pt_cache.size() >= 4096) c.pt_cache.clear();
    return c.pt_cache.emplace(key, std::move(pt)).first->second;
}

const Plain &PtProvider::mask(int kind, int k, int lv, double scale, int cc, int s0, int s1, double t)
{
    if (const Plain *p = lookup(kind, k, lv, scale)) return *p;
    Context::PtKey key(kind, k, lv, cc, s0, s1, dbits(t), dbits(scale));
    if (Plain *p = ctx_cached(c_, key)) return *p;
    int s = c_.p.slots();
    double *re = (double *)c_.alloc_bytes(sizeof(double) * 2 * s);
    k_make_mask(c_, re, re + s, kind, k, cc, s0, s1, t);
    Plain pt = plain_encode(c_, re, re + s, lv, scale);
    c_.free_bytes(re);
    return ctx_store(c_, key, std::move(pt));
}

const Plain &PtProvider::scaled_vec(int kind, int k, int lv, double scale, const double *d_vec, double coeff,
                                    u64 vec_hash)
{
    if (const Plain *p = lookup(kind, k, lv, scale)) return *p;
    Context::PtKey key(kind, k, lv, 0, 0, 0, dbits(coeff), dbits(scale) ^ vec_hash);
    if (Plain *p = ctx_cached(c_, key)) return *p;
    if (!d_vec)   // a recorded call does not copy the vector from the host
        throw Error(ERR_RECORDING, "a plaintext not encoded yet cannot be recorded: run the call once first");
    int s = c_.p.slots();
    double *re = (double *)c_.alloc_bytes(sizeof(double) * s);
    k_scale_vec(c_, re, d_vec, coeff, s);
    Plain pt = plain_encode(c_, re, nullptr, lv, scale);
    c_.free_bytes(re);
    return ctx_store(c_, key, std::move(pt));
}

// CMult by a mask encoded at scale q_lv: the ciphertext keeps its scale.
static CtBatch cmult_mask(Context &c, PtProvider &pp, const CtView &a, int kind, int k, int cc, int s0, int s1,
                          double t)
{
    double q = (double)c.p.mod[a.lv];
    const Plain &pt = pp.mask(kind, k, a.lv, q, cc, s0, s1, t);
    return mul_plain_rescale(c, a, pt, a.scale);
}

static std::vector<const Plain *> masks_for(Context &c, PtProvider &pp, int kind, int k0, int count, int lv, int cc,
                                            int s0, int s1, double t)
{
    std::vector<const Plain *> v;
    for (int k = k0; k < k0 + count; k++) v.push_back(&pp.mask(kind, k, lv, (double)c.p.mod[lv], cc, s0, s1, t));
    return v;
}

// Steps of at most 3 bits, as even as possible, larger first: 10 -> {3, 3, 2, 2}.
static std::vector<int> radix_plan(int bits)
{
    std::vector<int> plan;
    if (bits <= 0) return plan;
    const int steps = (bits + 2) / 3, base = bits / steps, extra = bits % steps;
    for (int i = 0; i < steps; i++) plan.push_back(base + (i < extra ? 1 : 0));
    return plan;
}

// x summed over its rotations by sign * u * unit (u < 2^bits) in radix steps:
// x <- x + sum_{0 < j < 2^b} Lrot(x, sign * j * t * unit), t the earlier radices' product.
static CtBatch rot_sum_steps(Context &c, const EvalKeys &ek, CtBatch x, int bits, int unit, int s, int sign)
{
    int t = 1;
    for (int b : radix_plan(bits)) {
        std::vector<int> rs;
        for (int j = 1; j < (1 << b); j++) rs.push_back((int)((((long long)sign * j * t * unit) % s + s) % s));
        x = rotate_sum(c, ek, x.view(), rs);
        t <<= b;
    }
    return x;
}

std::vector<int> rotation_amounts(int s0, int s1, int cc, int flags)
{
    if (!is_pow2(cc) || cc < 2 || cc > s0 || cc > s1 || !is_pow2(s0) || !is_pow2(s1))
        throw Error(ERR_SHAPE, "rotation amounts: c must be a power of two with 2 <= c <= min(s0, s1)");
    const int s = s0 * s1, h = cc / 2;
    std::set<int> rs;
    auto add = [&](long long r) {
        const int v = (int)(((r % s) + s) % s);
        if (v) rs.insert(v);
    };
    for (int k = 1; k <= h; k++) add((long long)k * s1);   // RotUp(B-bar, k)
    for (int k = 1; k <= h; k++) add(k);                   // Lrot(A_cplx, k), RotLeft
    if (flags & FLAG_SHARED_ROT)
        for (int k = 1; k <= h; k++) add((long long)k - s1);   // RotLeft from Lrot(A, k - s1)
    else
        add(-s1);                                              // RotLeft: Rrot(., s1)
    add(s1);                                               // PRotUp: RotUp(., 1)
    auto sums = [&](int bits, int unit, int sign) {
        if (flags & FLAG_RADIX_SUM) {
            int t = 1;
            for (int b : radix_plan(bits)) {
                for (int j = 1; j < (1 << b); j++) add((long long)sign * j * t * unit);
                t <<= b;
            }
        } else {
            for (int u = 0; u < bits; u++) add((long long)sign * (1 << u) * unit);
        }
    };
    sums(ilog2(s1), 1, 1);    // SumCols, left
    sums(ilog2(s1), 1, -1);   // SumCols, right
    sums(ilog2(s0), s1, 1);   // SumRows
    return std::vector<int>(rs.begin(), rs.end());
}

// SumCols: rotate-and-add by 2^u (u < log s1), column-0 mask, rotate-and-add
// rightwards; FLAG_RADIX_SUM runs both chains as radix steps (same sums).
static CtBatch sum_cols(Context &c, const EvalKeys &ek, PtProvider &pp, CtBatch x, int s0, int s1, int flags)
{
    const int s = s0 * s1;
    if (flags & FLAG_RADIX_SUM) {
        x = rot_sum_steps(c, ek, std::move(x), ilog2(s1), 1, s, 1);
        x = cmult_mask(c, pp, x.view(), PT_COLMASK, 0, 0, s0, s1, 0.0);
        return rot_sum_steps(c, ek, std::move(x), ilog2(s1), 1, s, -1);
    }
    for (int u = 0; u < ilog2(s1); u++) x = add_rotate(c, ek, x.view(), x.view(), 1 << u);
    x = cmult_mask(c, pp, x.view(), PT_COLMASK, 0, 0, s0, s1, 0.0);
    for (int u = 0; u < ilog2(s1); u++) x = add_rotate(c, ek, x.view(), x.view(), s - (1 << u));
    return x;
}

// SumRows: rotate-and-add by 2^u * s1 for u < log s0 (radix steps with FLAG_RADIX_SUM).
static CtBatch sum_rows(Context &c, const EvalKeys &ek, CtBatch x, int s0, int s1, int flags)
{
    if (flags & FLAG_RADIX_SUM) return rot_sum_steps(c, ek, std::move(x), ilog2(s0), s1, s0 * s1, 1);
    for (int u = 0; u < ilog2(s0); u++) x = add_rotate(c, ek, x.view(), x.view(), (1 << u) * s1);
    return x;
}

static void check_shape(int cc, int s0, int s1, int N)
{
    if (!is_pow2(cc) || cc < 2 || cc > s0 || cc > s1)
        throw Error(ERR_SHAPE, "c must be a power of two with 2 <= c <= min(s0, s1)");
    if (!is_pow2(s0) || !is_pow2(s1) || (long long)s0 * s1 != N / 2)
        throw Error(ERR_SHAPE, "block shape must be powers of two with s0 * s1 = N/2");
}

static CtBatch gather(Context &c, std::vector<CtBatch> &parts)
{
    if (parts.size() == 1) return std::move(parts[0]);
    int n = 0;
    for (auto &p : parts) n += p.n;
    CtBatch out(&c, n, parts[0].lv, parts[0].scale);
    size_t off = 0;
    for (auto &p : parts) {
        if (p.lv != out.lv) throw Error(ERR_LEVEL, "blocks at different levels");
        HETAL_CUDA_CHECK(cudaMemcpyAsync(out.data + off, p.data, sizeof(u64) * p.n * p.ct_words(),
                                         cudaMemcpyDeviceToDevice, c.stream));
        off += (size_t)p.n * p.ct_words();
    }
    return out;
}

// out[g] = sum of the n consecutive ciphertexts of group g (x has G*n).
static CtBatch sum_within_groups(Context &c, const CtView &x, int G, int n)
{
    if (n == 1) return ct_copy(c, x);
    CtBatch out(&c, G, x.lv, x.scale);
    LimbMap qm = c.q_map(x.lv);
    for (int k = 0; k < 2; k++) k_sum_polys(c, out.comp(k), x.comp(k), G, qm);
    return out;
}

// out[j] = sum over groups g of x[g*n + j]  (x has G*n, layout [group][j]).
static CtBatch sum_across_groups(Context &c, const CtView &x, int G, int n)
{
    CtBatch acc = ct_copy(c, x.sub(0, n));
    for (int g = 1; g < G; g++) acc = ct_add(c, acc.view(), x.sub(g * n, n));
    return acc;
}

static size_t ct_bytes(const Context &c, int n, int lv) { return (size_t)n * 2 * (lv + 1) * c.p.N * sizeof(u64); }

// Number of k values processed together when one k costs `per_k` bytes.
static int k_chunk(const Context &c, size_t per_k, int h)
{
    size_t kc = per_k ? c.batch_bytes / per_k : (size_t)h;
    return (int)std::max<size_t>(1, std::min<size_t>(kc, (size_t)h));
}

// Lrot(a, r) for every r of rs, [r][block]: one batched hoisted key switch when a
// is hoisted, else one plain rotation per amount.
static CtBatch rotate_src(Context &c, const EvalKeys &ek, const CtView &a, const HoistedSource *hs,
                          const std::vector<int> &rs)
{
    if (hs) return hoist_rotate_batch(c, ek, *hs, rs);
    std::vector<CtBatch> outs;
    for (int r : rs) outs.push_back(rotate(c, ek, a, r));
    return gather(c, outs);
}

Mat diag_abt(Context &c, const EvalKeys &ek, const Mat &A, const Mat &Bbar, int cc, double t, const PtSet *pts,
             int flags)
{
    const int s0 = A.s0, s1 = A.s1, h = cc / 2, m = A.m, n = A.n;
    check_shape(cc, s0, s1, c.p.N);
    if (Bbar.m != 1 || Bbar.n != n || Bbar.s0 != s0 || Bbar.s1 != s1)
        throw Error(ERR_SHAPE, "B-bar must be one block row with A's column blocks and block shape");
    PtProvider pp(c, pts);
    // B_cplx = Bbar + sqrt(-1) RotUp(Bbar, c/2)
    CtBatch Bc;
    {
        CtBatch r = rotate(c, ek, Bbar.cts.view(), h * s1);
        CtBatch ri = ct_mul_i(c, r.view());
        Bc = ct_add(c, Bbar.cts.view(), ri.view());
    }
    std::unique_ptr<HoistedSource> hs;
    if ((flags & FLAG_HOIST) && h > 1) hs.reset(new HoistedSource(hoist_prepare(c, Bc.view())));
    // one k holds B_k (n blocks) and the tensor products of a block row (3 polys each)
    const int kc = k_chunk(c, ct_bytes(c, n, Bc.lv) * 3, h);
    std::vector<CtBatch> X(m);
    for (int k0 = 0; k0 < h; k0 += kc) {
        const int G = std::min(h, k0 + kc) - k0;
        std::vector<CtBatch> keep;
        keep.reserve(G);
        std::vector<CtView> Bks;
        std::vector<int> ups;
        for (int k = std::max(k0, 1); k < k0 + G; k++) ups.push_back(k * s1);   // RotUp(B_cplx, k)
        if (!ups.empty()) keep.push_back(rotate_src(c, ek, Bc.view(), hs.get(), ups));
        for (int k = k0; k < k0 + G; k++)
            Bks.push_back(k == 0 ? Bc.view() : keep.back().view().sub((k - std::max(k0, 1)) * n, n));
        for (int r = 0; r < m; r++) {
            // S_k = sum_j A_{r,j} (.) B_{k,j} for every k of the chunk
            std::vector<CtView> As(G, A.cts.view().sub(r * n, n));
            CtBatch S;
            if (flags & FLAG_LAZY_RELIN) {
                S = mult_sum_grouped(c, ek, As, Bks);
            } else {
                CtBatch R = mult_grouped(c, ek, As, Bks);
                S = sum_within_groups(c, R.view(), G, n);
            }
            CtBatch x = sum_cols(c, ek, pp, std::move(S), s0, s1, flags);
            std::vector<const Plain *> mk = masks_for(c, pp, PT_ABT_DIAG, k0, G, x.lv, cc, s0, s1, t);
            x = mul_plain_rescale_grouped(c, x.view(), mk, 1, false, x.scale);
            CtBatch part = sum_across_groups(c, x.view(), G, 1);
            X[r] = (k0 == 0) ? std::move(part) : ct_add(c, X[r].view(), part.view());
        }
    }
    CtBatch Xall = gather(c, X);
    Mat out;
    out.cts = add_conjugate(c, ek, Xall.view(), Xall.view());
    out.m = m;
    out.n = 1;
    out.rows = A.rows;
    out.cols = s1;
    out.s0 = s0;
    out.s1 = s1;
    return out;
}

Mat diag_atb(Context &c, const EvalKeys &ek, const Mat &Au, const Mat &B, int cc, double t, const PtSet *pts,
             int flags)
{
    const int s0 = B.s0, s1 = B.s1, h = cc / 2, m = B.m, n = B.n;
    check_shape(cc, s0, s1, c.p.N);
    if (Au.n != 1 || Au.m != m || Au.s0 != s0 || Au.s1 != s1)
        throw Error(ERR_SHAPE, "A-underbar must be one block column with B's row blocks and block shape");
    PtProvider pp(c, pts);
    const bool pru = Au.cts.lv < B.cts.lv;
    const bool shared = flags & FLAG_SHARED_ROT;
    const int s = s0 * s1;
    // A_cplx = A + sqrt(-1) RotLeft(A, c/2), batched over the m row blocks:
    // RotLeft(A, k) = A2 + Rrot(A1 - A2, s1), A1 = Lrot(A, k), A2 = A1 (.) D_k
    // (FLAG_SHARED_ROT: A1 (.) D_k + Lrot(A, k - s1) (.) (1 - D_k), both rotations of A hoisted)
    CtBatch Ac;
    if (shared) {
        std::unique_ptr<HoistedSource> ha;
        if (flags & FLAG_HOIST) ha.reset(new HoistedSource(hoist_prepare(c, Au.cts.view())));
        CtBatch r2 = rotate_src(c, ek, Au.cts.view(), ha.get(), {h, (h - s1 + s) % s});
        std::vector<const Plain *> dk = masks_for(c, pp, PT_DMASK, h, 1, r2.lv, 0, s0, s1, 0.0);
        std::vector<const Plain *> dc = masks_for(c, pp, PT_DMASK_C, h, 1, r2.lv, 0, s0, s1, 0.0);
        CtBatch rl = mul_plain2_rescale_grouped(c, r2.view().sub(0, m), dk, r2.view().sub(m, m), dc, m, r2.scale);
        CtBatch ri = ct_mul_i(c, rl.view());
        Ac = ct_add(c, Au.cts.view(), ri.view());
    } else {
        CtBatch a1 = rotate(c, ek, Au.cts.view(), h);
        CtBatch a2 = cmult_mask(c, pp, a1.view(), PT_DMASK, h, 0, s0, s1, 0.0);
        CtBatch d = ct_sub(c, a1.view(), a2.view());
        CtBatch rl = add_rotate(c, ek, a2.view(), d.view(), s0 * s1 - s1);
        CtBatch ri = ct_mul_i(c, rl.view());
        Ac = ct_add(c, Au.cts.view(), ri.view());
    }
    std::unique_ptr<HoistedSource> hs;
    if ((flags & FLAG_HOIST) && h > 1) hs.reset(new HoistedSource(hoist_prepare(c, Ac.view())));
    // B with the m blocks of every column contiguous: [j][r]
    CtBatch Bcm;
    CtView Bv = B.cts.view();
    if (m > 1) {
        Bcm = CtBatch(&c, m * n, Bv.lv, Bv.scale);
        for (int j = 0; j < n; j++)
            for (int r = 0; r < m; r++)
                HETAL_CUDA_CHECK(cudaMemcpyAsync(Bcm.ct(j * m + r), Bv.ct(r * n + j), sizeof(u64) * Bv.ct_words(),
                                                 cudaMemcpyDeviceToDevice, c.stream));
        Bv = Bcm.view();
    }
    // the level every product is taken at: PRotUp branch min(level(A_cplx), level(B) - 1)
    // (k = 0 included); RotLeft branch min(level(A_cplx) - 1, level(B)) when c/2 > 1
    const int lvP = pru ? std::min(Ac.lv, (h > 1 ? Bv.lv - 1 : Bv.lv))
                        : std::min(h > 1 ? Ac.lv - 1 : Ac.lv, Bv.lv);
    CtBatch Bd;   // B at the product level (for the k values that use B itself)
    CtView Bprod = Bv;
    if (Bv.lv > lvP) {
        Bd = drop_level(c, Bv, lvP);
        Bprod = Bd.view();
    }
    const int kc = k_chunk(c, ct_bytes(c, m * n, Bv.lv) * (pru ? 5 : 2), h);
    // FLAG_SHARED_ROT, PRotUp branch: RotUp(B, 1) once for every k
    CtBatch Bup;
    if (shared && pru && h > 1) Bup = rotate(c, ek, Bv, s1);
    CtBatch X;
    for (int k0 = 0; k0 < h; k0 += kc) {
        const int G = std::min(h, k0 + kc) - k0;
        const int k1s = std::max(k0, 1);                 // first k >= 1 of the chunk
        const int G1 = k0 + G - k1s;                     // number of k >= 1 in the chunk
        std::vector<CtBatch> keep;
        keep.reserve(G + 8);
        // A_k for every k of the chunk (m blocks each)
        std::vector<CtView> Aks;
        if (k0 == 0) {
            if (Ac.lv > lvP) {
                keep.push_back(drop_level(c, Ac.view(), lvP));
                Aks.push_back(keep.back().view());
            } else {
                Aks.push_back(Ac.view());
            }
        }
        if (G1 > 0) {
            std::vector<int> ks;
            for (int k = k1s; k < k0 + G; k++) ks.push_back(k);
            if (shared && !pru)   // Lrot(A_cplx, k - s1) as well, in the same hoisted batch
                for (int k = k1s; k < k0 + G; k++) ks.push_back((k - s1 + s) % s);
            CtBatch a1 = rotate_src(c, ek, Ac.view(), hs.get(), ks);   // Lrot(A_cplx, k), [k][r]
            if (shared && !pru) {
                std::vector<const Plain *> dk = masks_for(c, pp, PT_DMASK, k1s, G1, a1.lv, 0, s0, s1, 0.0);
                std::vector<const Plain *> dc = masks_for(c, pp, PT_DMASK_C, k1s, G1, a1.lv, 0, s0, s1, 0.0);
                CtBatch rl = mul_plain2_rescale_grouped(c, a1.view().sub(0, G1 * m), dk, a1.view().sub(G1 * m, G1 * m),
                                                        dc, m, a1.scale);   // RotLeft(A_cplx, k)
                if (rl.lv > lvP) rl = drop_level(c, rl.view(), lvP);
                keep.push_back(std::move(rl));
            } else if (pru) {
                if (a1.lv > lvP) a1 = drop_level(c, a1.view(), lvP);
                keep.push_back(std::move(a1));
            } else {
                std::vector<const Plain *> dk = masks_for(c, pp, PT_DMASK, k1s, G1, a1.lv, 0, s0, s1, 0.0);
                CtBatch a2 = mul_plain_rescale_grouped(c, a1.view(), dk, m, false, a1.scale);
                CtBatch d = ct_sub(c, a1.view(), a2.view());
                CtBatch rl = add_rotate(c, ek, a2.view(), d.view(), s0 * s1 - s1);   // RotLeft(A_cplx, k)
                if (rl.lv > lvP) rl = drop_level(c, rl.view(), lvP);
                keep.push_back(std::move(rl));
            }
            for (int g = 0; g < G1; g++) Aks.push_back(keep.back().view().sub(g * m, m));
        }
        // B_k for every k of the chunk (m*n blocks each, [j][r])
        std::vector<CtView> Bks;
        if (!pru) {
            for (int g = 0; g < G; g++) Bks.push_back(Bprod);
        } else {
            if (k0 == 0) Bks.push_back(Bprod);
            if (G1 > 0 && shared) {
                // PRotUp(B, k) = B (.) D_k + RotUp(B, 1) (.) (1 - D_k)
                std::vector<const Plain *> dk = masks_for(c, pp, PT_DMASK, k1s, G1, Bv.lv, 0, s0, s1, 0.0);
                std::vector<const Plain *> dc = masks_for(c, pp, PT_DMASK_C, k1s, G1, Bv.lv, 0, s0, s1, 0.0);
                CtBatch pr = mul_plain2_rescale_grouped(c, Bv, dk, Bup.view(), dc, m * n, Bv.scale);
                if (pr.lv > lvP) pr = drop_level(c, pr.view(), lvP);
                keep.push_back(std::move(pr));
                for (int g = 0; g < G1; g++) Bks.push_back(keep.back().view().sub(g * m * n, m * n));
            } else if (G1 > 0) {
                // PRotUp(B, k) = B' + RotUp(B - B', 1), B' = B (.) D_k, RotUp(., 1) = Lrot(., s1)
                std::vector<const Plain *> dk = masks_for(c, pp, PT_DMASK, k1s, G1, Bv.lv, 0, s0, s1, 0.0);
                CtBatch Bp = mul_plain_rescale_grouped(c, Bv, dk, m * n, true, Bv.scale);
                CtBatch Bl = drop_level(c, Bv, Bp.lv);
                CtBatch diff(&c, G1 * m * n, Bp.lv, Bp.scale);
                LimbMap qm = c.q_map(Bp.lv);
                for (int g = 0; g < G1; g++)
                    for (int q = 0; q < 2; q++)
                        k_sub(c, diff.view().sub(g * m * n, m * n).comp(q), Bl.comp(q),
                              Bp.view().sub(g * m * n, m * n).comp(q), qm);
                CtBatch pr = add_rotate(c, ek, Bp.view(), diff.view(), s1);
                if (pr.lv > lvP) pr = drop_level(c, pr.view(), lvP);
                keep.push_back(std::move(pr));
                for (int g = 0; g < G1; g++) Bks.push_back(keep.back().view().sub(g * m * n, m * n));
            }
        }
        // S_{k,j} = sum_r A_k[r] (.) B_k[j][r]: one group of m pairs per (k, j)
        std::vector<CtView> ga, gb;
        for (int g = 0; g < G; g++)
            for (int j = 0; j < n; j++) {
                gb.push_back(Aks[g]);
                ga.push_back(Bks[g].sub(j * m, m));
            }
        CtBatch S;
        if ((flags & FLAG_LAZY_RELIN) || m == 1) {
            S = (flags & FLAG_LAZY_RELIN) ? mult_sum_grouped(c, ek, ga, gb) : mult_grouped(c, ek, ga, gb);
        } else {
            CtBatch R = mult_grouped(c, ek, ga, gb);
            S = sum_within_groups(c, R.view(), G * n, m);
        }
        CtBatch x = sum_rows(c, ek, std::move(S), s0, s1, flags);
        std::vector<const Plain *> mk = masks_for(c, pp, PT_ATB_DIAG, k0, G, x.lv, cc, s0, s1, t);
        x = mul_plain_rescale_grouped(c, x.view(), mk, n, false, x.scale);
        CtBatch part = sum_across_groups(c, x.view(), G, n);
        X = (k0 == 0) ? std::move(part) : ct_add(c, X.view(), part.view());
    }
    Mat out;
    out.cts = add_conjugate(c, ek, X.view(), X.view());
    out.m = 1;
    out.n = n;
    out.rows = s0;
    out.cols = B.cols;
    out.s0 = s0;
    out.s1 = s1;
    return out;
}

// CMult landing on an exact target scale: the plaintext scale is
// target * q_lv / scale(a), so that after the rescale by q_lv the scale is target.
static CtBatch cmult_scaled(Context &c, PtProvider &pp, const CtView &a, int kind, int k, const double *d_valid,
                            u64 valid_hash, double coeff, double target)
{
    double pt_scale = target * (double)c.p.mod[a.lv] / a.scale;
    const Plain &pt = pp.scaled_vec(kind, k, a.lv, pt_scale, d_valid, coeff, valid_hash);
    return mul_plain_rescale(c, a, pt, target);
}

Mat softmax_poly(Context &c, const EvalKeys &ek, const Mat &Xm, const double *coeffs, const double *d_valid,
                 u64 valid_hash, double target, const PtSet *pts)
{
    PtProvider pp(c, pts);
    CtView x = Xm.cts.view();
    if (x.lv < 5) throw Error(ERR_LEVEL, "the degree-15 evaluation needs 5 levels");
    CtBatch x2 = mult(c, ek, x, x);
    CtBatch x3 = mult(c, ek, x2.view(), x);
    CtBatch x4 = mult(c, ek, x2.view(), x2.view());
    CtBatch x8 = mult(c, ek, x4.view(), x4.view());
    const int lu = x.lv - 3;
    const double s4 = x4.scale, s8 = x8.scale;
    double S[4];
    S[0] = target;
    S[1] = target * (double)c.p.mod[lu] / s4;
    S[2] = target * (double)c.p.mod[lu - 1] / s8;
    S[3] = S[2] * (double)c.p.mod[lu] / s4;
    CtView xs[4] = {x, x, x2.view(), x3.view()};
    std::vector<CtBatch> u(4);
    for (int j = 0; j < 4; j++) {
        CtBatch acc;
        for (int r = 1; r <= 3; r++) {
            CtBatch term = cmult_scaled(c, pp, xs[r], PT_SM_COEF, 4 * j + r, d_valid, valid_hash, coeffs[4 * j + r],
                                        S[j]);
            if (term.lv > lu) term = drop_level(c, term.view(), lu);
            acc = (r == 1) ? std::move(term) : ct_add(c, acc.view(), term.view());
        }
        const Plain &cst = pp.scaled_vec(PT_SM_CONST, j, acc.lv, acc.scale, d_valid, coeffs[4 * j], valid_hash);
        u[j] = add_plain(c, acc.view(), cst);
    }
    CtBatch t34 = mult(c, ek, u[3].view(), x4.view());
    CtBatch inner = ct_add(c, u[2].view(), t34.view());
    CtBatch outer = mult(c, ek, inner.view(), x8.view());
    CtBatch t14 = mult(c, ek, u[1].view(), x4.view());
    CtBatch low = ct_add(c, u[0].view(), t14.view());
    Mat out;
    out.cts = ct_add(c, low.view(), outer.view());
    out.m = Xm.m;
    out.n = Xm.n;
    out.rows = Xm.rows;
    out.cols = Xm.cols;
    out.s0 = Xm.s0;
    out.s1 = Xm.s1;
    return out;
}

}  // namespace hetal
