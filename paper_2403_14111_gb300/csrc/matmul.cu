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

#include <algorithm>
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

// Lrot of the first `cnt` blocks of a by every amount of rs, [amount][block]: one batched
// hoisted key switch over those blocks' extended digits when hs is given, else one plain
// rotation per amount.
static CtBatch rotate_prefix(Context &c, const EvalKeys &ek, const CtView &a, const HoistedSource *hs, int cnt,
                             const std::vector<int> &rs)
{
    if (hs) return hoist_rotate_batch(c, ek, hoisted_view(c, *hs, 0, cnt), rs);
    std::vector<CtBatch> outs;
    for (int r : rs) outs.push_back(rotate(c, ek, a.sub(0, cnt), r));
    return gather(c, outs);
}

static void same_scale(double a, double b)
{
    if (std::fabs(a / b - 1.0) > 1e-9) throw Error(ERR_SCALE, "instances of a group must share their inputs' scales");
}

// Consecutive ciphertext runs as one batch: the run itself when there is one, else a copy.
struct Joined {
    CtBatch own;
    CtView v;
};
static Joined join(Context &c, const std::vector<CtView> &parts)
{
    Joined j;
    if (parts.size() == 1) {
        j.v = parts[0];
        return j;
    }
    int n = 0;
    for (auto &p : parts) n += p.n;
    j.own = CtBatch(&c, n, parts[0].lv, parts[0].scale);
    size_t off = 0;
    for (auto &p : parts) {
        if (p.lv != j.own.lv) throw Error(ERR_LEVEL, "blocks at different levels");
        same_scale(p.scale, j.own.scale);
        HETAL_CUDA_CHECK(cudaMemcpyAsync(j.own.data + off, p.data, sizeof(u64) * p.n * p.ct_words(),
                                         cudaMemcpyDeviceToDevice, c.stream));
        off += (size_t)p.n * p.ct_words();
    }
    j.v = j.own.view();
    return j;
}

// CMult of ciphertext z of a by pts[z] (each its own plaintext, encoded at scale q_lv),
// then one rescale of the whole batch; the result carries out_scale.
static CtBatch mul_plain_list_rescale(Context &c, const CtView &a, const std::vector<const Plain *> &pts,
                                      double out_scale)
{
    if ((int)pts.size() != a.n) throw Error(ERR_SHAPE, "one plaintext per ciphertext");
    if (a.lv < 1) throw Error(ERR_LEVEL, "no level left for a plaintext product");
    std::vector<const u64 *> mont;
    for (const Plain *p : pts) {
        if (p->lv < a.lv) throw Error(ERR_LEVEL, "plaintext below ciphertext level");
        mont.push_back(p->mont);
    }
    CtBatch tmp(&c, a.n, a.lv, out_scale);
    k_mul_plain_list(c, tmp.polys(), a.polys(), mont, c.q_map(a.lv));
    CtBatch out = rescale(c, tmp.view());
    out.scale = out_scale;
    c.cnt.cmult += a.n;
    return out;
}

// Order of a group's instances: c/2 descending (stable), so that the instances still
// active at diagonal k (those with k < c/2) are a prefix.
static std::vector<int> by_half_desc(const std::vector<int> &h)
{
    std::vector<int> ord(h.size());
    for (size_t i = 0; i < ord.size(); i++) ord[i] = (int)i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return h[x] > h[y]; });
    return ord;
}

static int active_prefix(const std::vector<int> &hh, int k)
{
    int P = 0;
    while (P < (int)hh.size() && hh[P] > k) P++;
    return P;
}

std::vector<Mat> diag_abt_group(Context &c, const EvalKeys &ek, const std::vector<AbtJob> &jobs, const PtSet *pts,
                                int flags)
{
    const int I = (int)jobs.size();
    if (I == 0) return {};
    for (const AbtJob &j : jobs)
        if (!j.A || !j.Bbar) throw Error(ERR_INVALID_ARG, "DiagABT: missing operand");
    const Mat &A0 = *jobs[0].A, &B0 = *jobs[0].Bbar;
    const int s0 = A0.s0, s1 = A0.s1;
    for (const AbtJob &j : jobs) {
        check_shape(j.cc, s0, s1, c.p.N);
        if (j.A->s0 != s0 || j.A->s1 != s1) throw Error(ERR_SHAPE, "instances of a group must share the block shape");
        if (j.Bbar->m != 1 || j.Bbar->n != j.A->n || j.Bbar->s0 != s0 || j.Bbar->s1 != s1)
            throw Error(ERR_SHAPE, "B-bar must be one block row with A's column blocks and block shape");
        if (j.A->cts.lv != A0.cts.lv || j.Bbar->cts.lv != B0.cts.lv)
            throw Error(ERR_LEVEL, "instances of a group must share their inputs' levels");
        same_scale(j.A->cts.scale, A0.cts.scale);
        same_scale(j.Bbar->cts.scale, B0.cts.scale);
    }
    if (pts && I > 1) throw Error(ERR_INVALID_ARG, "a caller's plaintext set serves one instance at a time");
    std::vector<int> half(I);
    for (int i = 0; i < I; i++) half[i] = jobs[i].cc / 2;
    const std::vector<int> ord = by_half_desc(half);
    std::vector<int> hh(I), mm(I), nn(I), bo(I + 1, 0), xo(I + 1, 0);   // by position in ord
    for (int p = 0; p < I; p++) {
        const AbtJob &j = jobs[ord[p]];
        hh[p] = j.cc / 2;
        mm[p] = j.A->m;
        nn[p] = j.A->n;
        bo[p + 1] = bo[p] + nn[p];
        xo[p + 1] = xo[p] + mm[p];
    }
    const int hmax = hh[0];
    PtProvider pp(c, pts);
    // B_cplx = Bbar + sqrt(-1) RotUp(Bbar, c/2): one batched rotation per distinct c/2
    CtBatch Bc;
    {
        std::vector<CtBatch> parts;
        for (int p0 = 0; p0 < I;) {
            int p1 = p0;
            std::vector<CtView> run;
            while (p1 < I && hh[p1] == hh[p0]) run.push_back(jobs[ord[p1++]].Bbar->cts.view());
            Joined rb = join(c, run);
            CtBatch r = rotate(c, ek, rb.v, hh[p0] * s1);
            CtBatch ri = ct_mul_i(c, r.view());
            parts.push_back(ct_add(c, rb.v, ri.view()));
            p0 = p1;
        }
        Bc = gather(c, parts);
    }
    std::unique_ptr<HoistedSource> hs;
    if ((flags & FLAG_HOIST) && hmax > 1)
        hs.reset(new HoistedSource(hoist_prepare(c, Bc.view().sub(0, bo[active_prefix(hh, 1)]))));
    // one k holds B_k (the active blocks), the tensor products of the rows (3 polys each) and
    // SumCols over one ciphertext per row block, whose key switches hold about 7 ciphertexts'
    // worth of extended digits, accumulators and results each
    const int kc = k_chunk(c, ct_bytes(c, 3 * bo[I] + 7 * xo[I], Bc.lv), hmax);
    CtBatch X;   // [position][row block], created by the first chunk (every instance is active at k = 0)
    for (int k0 = 0; k0 < hmax; k0 += kc) {
        const int k1 = std::min(hmax, k0 + kc);
        std::vector<CtBatch> keep;
        keep.reserve(k1 - k0);
        // B_k = RotUp(B_cplx, k) for the instances active at k, one batch per run of k with the same ones
        std::vector<CtView> Bk(k1 - k0);
        for (int k = k0; k < k1;) {
            if (k == 0) {
                Bk[0] = Bc.view();
                k++;
                continue;
            }
            const int P = active_prefix(hh, k);
            int ke = k;
            std::vector<int> ups;
            while (ke < k1 && active_prefix(hh, ke) == P) ups.push_back((ke++) * s1);
            const int cnt = bo[P];
            keep.push_back(rotate_prefix(c, ek, Bc.view(), hs.get(), cnt, ups));
            for (int q = k; q < ke; q++) Bk[q - k0] = keep.back().view().sub((q - k) * cnt, cnt);
            k = ke;
        }
        // S_{p,r,k} = sum_j A_p[r][j] (.) B_k[p][j], groups [position][row][k]
        std::vector<CtView> ga, gb;
        std::vector<int> glen;   // k of the chunk per (position, row)
        const int P0 = active_prefix(hh, k0);
        for (int p = 0; p < P0; p++) {
            const int ka = std::min(k1, hh[p]);
            const Mat &A = *jobs[ord[p]].A;
            for (int r = 0; r < mm[p]; r++) {
                for (int k = k0; k < ka; k++) {
                    ga.push_back(A.cts.view().sub(r * nn[p], nn[p]));
                    gb.push_back(Bk[k - k0].sub(bo[p], nn[p]));
                }
                glen.push_back(ka - k0);
            }
        }
        CtBatch S;
        if (flags & FLAG_LAZY_RELIN) {
            S = mult_sum_grouped(c, ek, ga, gb);
        } else {
            CtBatch R = mult_grouped(c, ek, ga, gb);
            bool ones = true;
            for (auto &v : ga) ones = ones && v.n == 1;
            if (ones) {
                S = std::move(R);
            } else {
                std::vector<int> st, ln;
                int off = 0;
                for (auto &v : ga) {
                    st.push_back(off);
                    ln.push_back(v.n);
                    off += v.n;
                }
                S = CtBatch(&c, (int)ga.size(), R.lv, R.scale);
                k_sum_ranges(c, S.polys(), R.polys(), st, ln, false, c.q_map(R.lv));
            }
        }
        CtBatch x = sum_cols(c, ek, pp, std::move(S), s0, s1, flags);
        // t_p M_cplx^{(k, c_p)} for every group
        std::vector<const Plain *> mk;
        const double q = (double)c.p.mod[x.lv];
        for (int p = 0; p < P0; p++) {
            const AbtJob &j = jobs[ord[p]];
            const int ka = std::min(k1, hh[p]);
            for (int r = 0; r < mm[p]; r++)
                for (int k = k0; k < ka; k++) mk.push_back(&pp.mask(PT_ABT_DIAG, k, x.lv, q, j.cc, s0, s1, j.t));
        }
        x = mul_plain_list_rescale(c, x.view(), mk, x.scale);
        // X[p][r] (+)= the sum of its groups over the chunk's k
        std::vector<int> st;
        int off = 0;
        for (int len : glen) {
            st.push_back(off);
            off += len;
        }
        if (k0 == 0) X = CtBatch(&c, xo[I], x.lv, x.scale);
        k_sum_ranges(c, X.view().sub(0, xo[P0]).polys(), x.polys(), st, glen, k0 > 0, c.q_map(x.lv));
    }
    CtBatch Xc = add_conjugate(c, ek, X.view(), X.view());
    std::vector<CtBatch> parts;
    if (I == 1)
        parts.push_back(std::move(Xc));
    else
        parts = CtBatch::split_sizes(std::move(Xc), mm);
    std::vector<Mat> out(I);
    for (int p = 0; p < I; p++) {
        Mat &o = out[ord[p]];
        o.cts = std::move(parts[p]);
        o.m = mm[p];
        o.n = 1;
        o.rows = jobs[ord[p]].A->rows;
        o.cols = s1;
        o.s0 = s0;
        o.s1 = s1;
    }
    return out;
}

Mat diag_abt(Context &c, const EvalKeys &ek, const Mat &A, const Mat &Bbar, int cc, double t, const PtSet *pts,
             int flags)
{
    std::vector<Mat> r = diag_abt_group(c, ek, std::vector<AbtJob>{AbtJob{&A, &Bbar, cc, t}}, pts, flags);
    return std::move(r[0]);
}

std::vector<Mat> diag_atb_group(Context &c, const EvalKeys &ek, const std::vector<AtbJob> &jobs, const PtSet *pts,
                                int flags)
{
    const int I = (int)jobs.size();
    if (I == 0) return {};
    for (const AtbJob &j : jobs)
        if (!j.Au || !j.B) throw Error(ERR_INVALID_ARG, "DiagATB: missing operand");
    const Mat &U0 = *jobs[0].Au, &B0 = *jobs[0].B;
    const int s0 = B0.s0, s1 = B0.s1, s = s0 * s1;
    for (const AtbJob &j : jobs) {
        check_shape(j.cc, s0, s1, c.p.N);
        if (j.B->s0 != s0 || j.B->s1 != s1) throw Error(ERR_SHAPE, "instances of a group must share the block shape");
        if (j.Au->n != 1 || j.Au->m != j.B->m || j.Au->s0 != s0 || j.Au->s1 != s1)
            throw Error(ERR_SHAPE, "A-underbar must be one block column with B's row blocks and block shape");
        if (j.Au->cts.lv != U0.cts.lv || j.B->cts.lv != B0.cts.lv)
            throw Error(ERR_LEVEL, "instances of a group must share their inputs' levels");
        same_scale(j.Au->cts.scale, U0.cts.scale);
        same_scale(j.B->cts.scale, B0.cts.scale);
    }
    if (pts && I > 1) throw Error(ERR_INVALID_ARG, "a caller's plaintext set serves one instance at a time");
    const bool pru = U0.cts.lv < B0.cts.lv;
    const bool shared = flags & FLAG_SHARED_ROT;
    std::vector<int> half(I);
    for (int i = 0; i < I; i++) half[i] = jobs[i].cc / 2;
    const std::vector<int> ord = by_half_desc(half);
    std::vector<int> hh(I), mm(I), nn(I), ao(I + 1, 0), bo(I + 1, 0), xo(I + 1, 0);
    for (int p = 0; p < I; p++) {
        const AtbJob &j = jobs[ord[p]];
        hh[p] = j.cc / 2;
        mm[p] = j.B->m;
        nn[p] = j.B->n;
        ao[p + 1] = ao[p] + mm[p];
        bo[p + 1] = bo[p] + mm[p] * nn[p];
        xo[p + 1] = xo[p] + nn[p];
    }
    const int hmax = hh[0];
    PtProvider pp(c, pts);
    // A_cplx = A + sqrt(-1) RotLeft(A, c/2), batched over the row blocks of each run of equal c/2:
    // RotLeft(A, h) = A2 + Rrot(A1 - A2, s1), A1 = Lrot(A, h), A2 = A1 (.) D_h
    // (FLAG_SHARED_ROT: A1 (.) D_h + Lrot(A, h - s1) (.) (1 - D_h), both rotations of A hoisted)
    CtBatch Ac;
    {
        std::vector<CtBatch> parts;
        for (int p0 = 0; p0 < I;) {
            int p1 = p0;
            std::vector<CtView> run;
            while (p1 < I && hh[p1] == hh[p0]) run.push_back(jobs[ord[p1++]].Au->cts.view());
            Joined ar = join(c, run);
            const int M = ar.v.n, h = hh[p0];
            if (shared) {
                std::unique_ptr<HoistedSource> ha;
                if (flags & FLAG_HOIST) ha.reset(new HoistedSource(hoist_prepare(c, ar.v)));
                CtBatch r2 = rotate_prefix(c, ek, ar.v, ha.get(), M, {h, (h - s1 + s) % s});
                std::vector<const Plain *> dk = masks_for(c, pp, PT_DMASK, h, 1, r2.lv, 0, s0, s1, 0.0);
                std::vector<const Plain *> dc = masks_for(c, pp, PT_DMASK_C, h, 1, r2.lv, 0, s0, s1, 0.0);
                CtBatch rl = mul_plain2_rescale_grouped(c, r2.view().sub(0, M), dk, r2.view().sub(M, M), dc, M, r2.scale);
                CtBatch ri = ct_mul_i(c, rl.view());
                parts.push_back(ct_add(c, ar.v, ri.view()));
            } else {
                CtBatch a1 = rotate(c, ek, ar.v, h);
                CtBatch a2 = cmult_mask(c, pp, a1.view(), PT_DMASK, h, 0, s0, s1, 0.0);
                CtBatch d = ct_sub(c, a1.view(), a2.view());
                CtBatch rl = add_rotate(c, ek, a2.view(), d.view(), s - s1);
                CtBatch ri = ct_mul_i(c, rl.view());
                parts.push_back(ct_add(c, ar.v, ri.view()));
            }
            p0 = p1;
        }
        Ac = gather(c, parts);
    }
    // the level every product is taken at: PRotUp branch min(level(A_cplx), level(B) - 1)
    // (k = 0 included); RotLeft branch min(level(A_cplx) - 1, level(B)) when c/2 > 1
    const int Blv = B0.cts.lv;
    auto product_level = [&](int h) {
        return pru ? std::min(Ac.lv, (h > 1 ? Blv - 1 : Blv)) : std::min(h > 1 ? Ac.lv - 1 : Ac.lv, Blv);
    };
    const int lvP = product_level(hmax);
    for (int p = 0; p < I; p++)
        if (product_level(hh[p]) != lvP)
            throw Error(ERR_LEVEL, "instances of a group must take their products at one level (c = 2 with larger c)");
    std::unique_ptr<HoistedSource> hs;
    if ((flags & FLAG_HOIST) && hmax > 1)
        hs.reset(new HoistedSource(hoist_prepare(c, Ac.view().sub(0, ao[active_prefix(hh, 1)]))));
    // B of every instance with the m blocks of each column contiguous: [position][j][r]
    CtBatch Bcm;
    CtView Bv = B0.cts.view();
    if (I > 1 || mm[0] > 1) {
        Bcm = CtBatch(&c, bo[I], Blv, B0.cts.scale);
        for (int p = 0; p < I; p++) {
            const CtView src = jobs[ord[p]].B->cts.view();
            for (int j = 0; j < nn[p]; j++)
                for (int r = 0; r < mm[p]; r++)
                    HETAL_CUDA_CHECK(cudaMemcpyAsync(Bcm.ct(bo[p] + j * mm[p] + r), src.ct(r * nn[p] + j),
                                                     sizeof(u64) * src.ct_words(), cudaMemcpyDeviceToDevice, c.stream));
        }
        Bv = Bcm.view();
    }
    CtBatch Bd;   // B at the product level (for the k values that use B itself)
    CtView Bprod = Bv;
    if (Bv.lv > lvP) {
        Bd = drop_level(c, Bv, lvP);
        Bprod = Bd.view();
    }
    // one k holds B_k or PRotUp(B, k) and its products, and SumRows over one ciphertext per
    // column block (about 7 ciphertexts' worth of key-switching temporaries each)
    const int kc = k_chunk(c, ct_bytes(c, bo[I], Bv.lv) * (pru ? 5 : 2) + ct_bytes(c, 7 * xo[I], Bv.lv), hmax);
    // FLAG_SHARED_ROT, PRotUp branch: RotUp(B, 1) once for every k
    CtBatch Bup;
    if (shared && pru && hmax > 1) Bup = rotate(c, ek, Bv.sub(0, bo[active_prefix(hh, 1)]), s1);
    CtBatch X;   // [position][column block]
    for (int k0 = 0; k0 < hmax; k0 += kc) {
        const int k1 = std::min(hmax, k0 + kc);
        std::vector<CtBatch> keep;
        keep.reserve(2 * (k1 - k0) + 8);
        std::vector<CtView> Ak(k1 - k0), Bk(k1 - k0);
        if (k0 == 0) {
            if (Ac.lv > lvP) {
                keep.push_back(drop_level(c, Ac.view(), lvP));
                Ak[0] = keep.back().view();
            } else {
                Ak[0] = Ac.view();
            }
            Bk[0] = Bprod;
        }
        for (int k = std::max(k0, 1); k < k1;) {
            const int P = active_prefix(hh, k);
            int ke = k;
            while (ke < k1 && active_prefix(hh, ke) == P) ke++;
            const int G1 = ke - k, cnt = ao[P], cntB = bo[P];
            // A_k for k in [k, ke): the instances active at k
            std::vector<int> ks;
            for (int q = k; q < ke; q++) ks.push_back(q);
            if (shared && !pru)   // Lrot(A_cplx, k - s1) as well, in the same hoisted batch
                for (int q = k; q < ke; q++) ks.push_back((q - s1 + s) % s);
            CtBatch a1 = rotate_prefix(c, ek, Ac.view(), hs.get(), cnt, ks);   // Lrot(A_cplx, k), [k][r]
            if (shared && !pru) {
                std::vector<const Plain *> dk = masks_for(c, pp, PT_DMASK, k, G1, a1.lv, 0, s0, s1, 0.0);
                std::vector<const Plain *> dc = masks_for(c, pp, PT_DMASK_C, k, G1, a1.lv, 0, s0, s1, 0.0);
                CtBatch rl = mul_plain2_rescale_grouped(c, a1.view().sub(0, G1 * cnt), dk,
                                                        a1.view().sub(G1 * cnt, G1 * cnt), dc, cnt, a1.scale);
                if (rl.lv > lvP) rl = drop_level(c, rl.view(), lvP);
                keep.push_back(std::move(rl));
            } else if (pru) {
                if (a1.lv > lvP) a1 = drop_level(c, a1.view(), lvP);
                keep.push_back(std::move(a1));
            } else {
                std::vector<const Plain *> dk = masks_for(c, pp, PT_DMASK, k, G1, a1.lv, 0, s0, s1, 0.0);
                CtBatch a2 = mul_plain_rescale_grouped(c, a1.view(), dk, cnt, false, a1.scale);
                CtBatch d = ct_sub(c, a1.view(), a2.view());
                CtBatch rl = add_rotate(c, ek, a2.view(), d.view(), s - s1);   // RotLeft(A_cplx, k)
                if (rl.lv > lvP) rl = drop_level(c, rl.view(), lvP);
                keep.push_back(std::move(rl));
            }
            for (int q = k; q < ke; q++) Ak[q - k0] = keep.back().view().sub((q - k) * cnt, cnt);
            // B_k: B itself (RotLeft branch) or PRotUp(B, k)
            if (!pru) {
                for (int q = k; q < ke; q++) Bk[q - k0] = Bprod;
            } else if (shared) {
                // PRotUp(B, k) = B (.) D_k + RotUp(B, 1) (.) (1 - D_k)
                std::vector<const Plain *> dk = masks_for(c, pp, PT_DMASK, k, G1, Bv.lv, 0, s0, s1, 0.0);
                std::vector<const Plain *> dc = masks_for(c, pp, PT_DMASK_C, k, G1, Bv.lv, 0, s0, s1, 0.0);
                CtBatch pr = mul_plain2_rescale_grouped(c, Bv.sub(0, cntB), dk, Bup.view().sub(0, cntB), dc, cntB,
                                                        Bv.scale);
                if (pr.lv > lvP) pr = drop_level(c, pr.view(), lvP);
                keep.push_back(std::move(pr));
                for (int q = k; q < ke; q++) Bk[q - k0] = keep.back().view().sub((q - k) * cntB, cntB);
            } else {
                // PRotUp(B, k) = B' + RotUp(B - B', 1), B' = B (.) D_k, RotUp(., 1) = Lrot(., s1)
                std::vector<const Plain *> dk = masks_for(c, pp, PT_DMASK, k, G1, Bv.lv, 0, s0, s1, 0.0);
                CtBatch Bp = mul_plain_rescale_grouped(c, Bv.sub(0, cntB), dk, cntB, true, Bv.scale);
                CtBatch Bl = drop_level(c, Bv.sub(0, cntB), Bp.lv);
                CtBatch diff(&c, G1 * cntB, Bp.lv, Bp.scale);
                LimbMap qm = c.q_map(Bp.lv);
                for (int g = 0; g < G1; g++)
                    for (int q = 0; q < 2; q++)
                        k_sub(c, diff.view().sub(g * cntB, cntB).comp(q), Bl.comp(q),
                              Bp.view().sub(g * cntB, cntB).comp(q), qm);
                CtBatch pr = add_rotate(c, ek, Bp.view(), diff.view(), s1);
                if (pr.lv > lvP) pr = drop_level(c, pr.view(), lvP);
                keep.push_back(std::move(pr));
                for (int q = k; q < ke; q++) Bk[q - k0] = keep.back().view().sub((q - k) * cntB, cntB);
            }
            k = ke;
        }
        // S_{p,j,k} = sum_r A_k[p][r] (.) B_k[p][j][r]: groups [position][j][k] of m_p pairs
        std::vector<CtView> ga, gb;
        std::vector<int> glen;
        const int P0 = active_prefix(hh, k0);
        bool ones = true;
        for (int p = 0; p < P0; p++) {
            const int ka = std::min(k1, hh[p]);
            for (int j = 0; j < nn[p]; j++) {
                for (int k = k0; k < ka; k++) {
                    ga.push_back(Bk[k - k0].sub(bo[p] + j * mm[p], mm[p]));
                    gb.push_back(Ak[k - k0].sub(ao[p], mm[p]));
                }
                glen.push_back(ka - k0);
            }
            ones = ones && mm[p] == 1;
        }
        CtBatch S;
        if (flags & FLAG_LAZY_RELIN) {
            S = mult_sum_grouped(c, ek, ga, gb);
        } else {
            CtBatch R = mult_grouped(c, ek, ga, gb);
            if (ones) {
                S = std::move(R);
            } else {
                std::vector<int> st, ln;
                int off = 0;
                for (auto &v : ga) {
                    st.push_back(off);
                    ln.push_back(v.n);
                    off += v.n;
                }
                S = CtBatch(&c, (int)ga.size(), R.lv, R.scale);
                k_sum_ranges(c, S.polys(), R.polys(), st, ln, false, c.q_map(R.lv));
            }
        }
        CtBatch x = sum_rows(c, ek, std::move(S), s0, s1, flags);
        std::vector<const Plain *> mk;
        const double q = (double)c.p.mod[x.lv];
        for (int p = 0; p < P0; p++) {
            const AtbJob &j = jobs[ord[p]];
            const int ka = std::min(k1, hh[p]);
            for (int jj = 0; jj < nn[p]; jj++)
                for (int k = k0; k < ka; k++) mk.push_back(&pp.mask(PT_ATB_DIAG, k, x.lv, q, j.cc, s0, s1, j.t));
        }
        x = mul_plain_list_rescale(c, x.view(), mk, x.scale);
        std::vector<int> st;
        int off = 0;
        for (int len : glen) {
            st.push_back(off);
            off += len;
        }
        if (k0 == 0) X = CtBatch(&c, xo[I], x.lv, x.scale);
        k_sum_ranges(c, X.view().sub(0, xo[P0]).polys(), x.polys(), st, glen, k0 > 0, c.q_map(x.lv));
    }
    CtBatch Xc = add_conjugate(c, ek, X.view(), X.view());
    std::vector<CtBatch> parts;
    if (I == 1)
        parts.push_back(std::move(Xc));
    else
        parts = CtBatch::split_sizes(std::move(Xc), nn);
    std::vector<Mat> out(I);
    for (int p = 0; p < I; p++) {
        Mat &o = out[ord[p]];
        o.cts = std::move(parts[p]);
        o.m = 1;
        o.n = nn[p];
        o.rows = s0;
        o.cols = jobs[ord[p]].B->cols;
        o.s0 = s0;
        o.s1 = s1;
    }
    return out;
}

Mat diag_atb(Context &c, const EvalKeys &ek, const Mat &Au, const Mat &B, int cc, double t, const PtSet *pts,
             int flags)
{
    std::vector<Mat> r = diag_atb_group(c, ek, std::vector<AtbJob>{AtbJob{&Au, &B, cc, t}}, pts, flags);
    return std::move(r[0]);
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
