// matmul.cu -- DiagABT and DiagATB (arXiv 2403.14111, Sec. 4.2 and App. B),
// and the degree-15 softmax stand-in of the encrypted training step.
//
// The operation order follows the paper's algorithms (Algorithm DiagABT,
// RotLeft, PRotUp, DiagATB in App. B.3) with the multi-block lifting of
// App. B.1; every operation is batched over the blocks it applies to.
#include "matmul.h"

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

static std::vector<CtBatch> rotations(Context &c, const EvalKeys &ek, const CtView &a, const std::vector<int> &rs,
                                      int flags)
{
    if (flags & FLAG_HOIST) return rotate_hoisted(c, ek, a, rs);
    std::vector<CtBatch> out;
    for (int r : rs) out.push_back(rotate(c, ek, a, r));
    return out;
}

// SumCols: rotate-and-add by 2^u (u < log s1), column-0 mask, rotate-and-add rightwards.
static CtBatch sum_cols(Context &c, const EvalKeys &ek, PtProvider &pp, CtBatch x, int s0, int s1)
{
    const int s = s0 * s1;
    for (int u = 0; u < ilog2(s1); u++) {
        CtBatch r = rotate(c, ek, x.view(), 1 << u);
        x = ct_add(c, x.view(), r.view());
    }
    x = cmult_mask(c, pp, x.view(), PT_COLMASK, 0, 0, s0, s1, 0.0);
    for (int u = 0; u < ilog2(s1); u++) {
        CtBatch r = rotate(c, ek, x.view(), s - (1 << u));
        x = ct_add(c, x.view(), r.view());
    }
    return x;
}

// SumRows: rotate-and-add by 2^u * s1 for u < log s0.
static CtBatch sum_rows(Context &c, const EvalKeys &ek, CtBatch x, int s0, int s1)
{
    for (int u = 0; u < ilog2(s0); u++) {
        CtBatch r = rotate(c, ek, x.view(), (1 << u) * s1);
        x = ct_add(c, x.view(), r.view());
    }
    return x;
}

// RotLeft(A, k) = A2 + Rrot(A1 - A2, s1), A1 = Lrot(A, k) (given), A2 = A1 (.) D_k.
static CtBatch rot_left_from(Context &c, const EvalKeys &ek, PtProvider &pp, const CtView &a1, int k, int s0, int s1)
{
    CtBatch a2 = cmult_mask(c, pp, a1, PT_DMASK, k, 0, s0, s1, 0.0);
    CtBatch d = ct_sub(c, a1, a2.view());
    CtBatch r = rotate(c, ek, d.view(), s0 * s1 - s1);
    return ct_add(c, a2.view(), r.view());
}

// PRotUp(B, k) = B' + RotUp(B - B', 1), B' = B (.) D_k, RotUp(., 1) = Lrot(., s1).
static CtBatch prot_up(Context &c, const EvalKeys &ek, PtProvider &pp, const CtView &b, int k, int s0, int s1)
{
    CtBatch b2 = cmult_mask(c, pp, b, PT_DMASK, k, 0, s0, s1, 0.0);
    CtBatch d = ct_sub(c, b, b2.view());
    CtBatch r = rotate(c, ek, d.view(), s1);
    return ct_add(c, b2.view(), r.view());
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

static std::vector<const Plain *> masks_for(Context &c, PtProvider &pp, int kind, int k0, int count, int lv, int cc,
                                            int s0, int s1, double t)
{
    std::vector<const Plain *> v;
    for (int k = k0; k < k0 + count; k++) v.push_back(&pp.mask(kind, k, lv, (double)c.p.mod[lv], cc, s0, s1, t));
    return v;
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
    // B_k = RotUp(B_cplx, k) for k = 1 .. c/2 - 1
    std::vector<CtBatch> BR;
    if (h > 1) {
        std::vector<int> rs;
        for (int k = 1; k < h; k++) rs.push_back(k * s1);
        BR = rotations(c, ek, Bc.view(), rs, flags);
    }
    std::vector<CtView> Bks(h);
    Bks[0] = Bc.view();
    for (int k = 1; k < h; k++) Bks[k] = BR[k - 1].view();
    std::vector<CtBatch> outs;
    for (int r = 0; r < m; r++) {
        // all c/2 iterations of the k-loop at once: S_k = sum_j A_{r,j} (.) B_{k,j}
        std::vector<CtView> As(h, A.cts.view().sub(r * n, n));
        CtBatch S;
        if (flags & FLAG_LAZY_RELIN) {
            S = mult_sum_grouped(c, ek, As, Bks);
        } else {
            CtBatch R = mult_grouped(c, ek, As, Bks);
            S = sum_within_groups(c, R.view(), h, n);
        }
        CtBatch x = sum_cols(c, ek, pp, std::move(S), s0, s1);
        std::vector<const Plain *> mk = masks_for(c, pp, PT_ABT_DIAG, 0, h, x.lv, cc, s0, s1, t);
        x = mul_plain_rescale_grouped(c, x.view(), mk, 1, false, x.scale);
        CtBatch X = sum_across_groups(c, x.view(), h, 1);
        CtBatch cj = conjugate(c, ek, X.view());
        outs.push_back(ct_add(c, X.view(), cj.view()));
    }
    Mat out;
    out.cts = gather(c, outs);
    out.m = m;
    out.n = 1;
    out.rows = A.rows;
    out.cols = s1;
    out.s0 = s0;
    out.s1 = s1;
    return out;
}

static Mat diag_atb_rows(Context &c, const EvalKeys &ek, const Mat &Au, const Mat &B, int cc, double t,
                         const PtSet *pts, int flags);

Mat diag_atb(Context &c, const EvalKeys &ek, const Mat &Au, const Mat &B, int cc, double t, const PtSet *pts,
             int flags)
{
    const int s0 = B.s0, s1 = B.s1, h = cc / 2, m = B.m, n = B.n;
    check_shape(cc, s0, s1, c.p.N);
    if (Au.n != 1 || Au.m != m || Au.s0 != s0 || Au.s1 != s1)
        throw Error(ERR_SHAPE, "A-underbar must be one block column with B's row blocks and block shape");
    if (m != 1) return diag_atb_rows(c, ek, Au, B, cc, t, pts, flags);
    PtProvider pp(c, pts);
    const bool pru = Au.cts.lv < B.cts.lv;
    // A_cplx = A + sqrt(-1) RotLeft(A, c/2)
    CtBatch Ac;
    {
        CtBatch a1 = rotate(c, ek, Au.cts.view(), h);
        CtBatch rl = rot_left_from(c, ek, pp, a1.view(), h, s0, s1);
        CtBatch ri = ct_mul_i(c, rl.view());
        Ac = ct_add(c, Au.cts.view(), ri.view());
    }
    std::vector<CtBatch> AR;
    if (h > 1) {
        std::vector<int> rs;
        for (int k = 1; k < h; k++) rs.push_back(k);
        AR = rotations(c, ek, Ac.view(), rs, flags);
    }
    std::vector<CtView> Aks(h), Bks(h);
    CtBatch hold0, hold1;
    const CtView Bv = B.cts.view();
    if (pru) {
        // A_k = Lrot(A_cplx, k), B_k = PRotUp(B, k) for all k >= 1 at once
        Aks[0] = Ac.view();
        Bks[0] = Bv;
        for (int k = 1; k < h; k++) Aks[k] = AR[k - 1].view();
        if (h > 1) {
            std::vector<const Plain *> dk = masks_for(c, pp, PT_DMASK, 1, h - 1, Bv.lv, 0, s0, s1, 0.0);
            CtBatch Bp = mul_plain_rescale_grouped(c, Bv, dk, n, true, Bv.scale);   // B' = B (.) D_k
            CtBatch Bd = drop_level(c, Bv, Bv.lv - 1);
            CtBatch diff(&c, (h - 1) * n, Bp.lv, Bp.scale);
            LimbMap qm = c.q_map(Bp.lv);
            for (int g = 0; g < h - 1; g++)
                for (int k = 0; k < 2; k++)
                    k_sub(c, diff.view().sub(g * n, n).comp(k), Bd.comp(k), Bp.view().sub(g * n, n).comp(k), qm);
            CtBatch rot = rotate(c, ek, diff.view(), s1);                   // RotUp(B - B', 1)
            hold0 = ct_add(c, Bp.view(), rot.view());
            for (int k = 1; k < h; k++) Bks[k] = hold0.view().sub((k - 1) * n, n);
        }
    } else {
        // A_k = RotLeft(A_cplx, k) for all k >= 1 at once; the k = 0 term is brought
        // down to their level so that all c/2 products share one rescale prime.
        if (h > 1) {
            std::vector<CtBatch> parts;
            for (auto &a : AR) parts.push_back(ct_copy(c, a.view()));
            CtBatch a1 = gather(c, parts);                                   // Lrot(A_cplx, k), k >= 1
            std::vector<const Plain *> dk = masks_for(c, pp, PT_DMASK, 1, h - 1, a1.lv, 0, s0, s1, 0.0);
            CtBatch a2 = mul_plain_rescale_grouped(c, a1.view(), dk, 1, false, a1.scale);
            CtBatch d = ct_sub(c, a1.view(), a2.view());
            CtBatch r = rotate(c, ek, d.view(), s0 * s1 - s1);
            hold0 = ct_add(c, a2.view(), r.view());
            hold1 = drop_level(c, Ac.view(), Ac.lv - 1);
            Aks[0] = hold1.view();
            for (int k = 1; k < h; k++) Aks[k] = hold0.view().sub(k - 1, 1);
        } else {
            Aks[0] = Ac.view();
        }
        for (int k = 0; k < h; k++) Bks[k] = Bv;
    }
    // S_{k,j} = A_k (.) B_{k,j}, all k at once: layout [k][j]
    CtBatch S = mult_grouped(c, ek, Bks, Aks);
    CtBatch x = sum_rows(c, ek, std::move(S), s0, s1);
    std::vector<const Plain *> mk = masks_for(c, pp, PT_ATB_DIAG, 0, h, x.lv, cc, s0, s1, t);
    x = mul_plain_rescale_grouped(c, x.view(), mk, n, false, x.scale);
    CtBatch X = sum_across_groups(c, x.view(), h, n);
    CtBatch cj = conjugate(c, ek, X.view());
    Mat out;
    out.cts = ct_add(c, X.view(), cj.view());
    out.m = 1;
    out.n = n;
    out.rows = s0;
    out.cols = B.cols;
    out.s0 = s0;
    out.s1 = s1;
    return out;
}

// Several block rows (m > 1): row blocks summed per column block, k-loop in order.
static Mat diag_atb_rows(Context &c, const EvalKeys &ek, const Mat &Au, const Mat &B, int cc, double t,
                         const PtSet *pts, int flags)
{
    const int s0 = B.s0, s1 = B.s1, h = cc / 2, m = B.m, n = B.n;
    check_shape(cc, s0, s1, c.p.N);
    if (Au.n != 1 || Au.m != m || Au.s0 != s0 || Au.s1 != s1)
        throw Error(ERR_SHAPE, "A-underbar must be one block column with B's row blocks and block shape");
    PtProvider pp(c, pts);
    const bool pru = Au.cts.lv < B.cts.lv;
    // A_cplx = A + sqrt(-1) RotLeft(A, c/2), batched over the m row blocks
    CtBatch Ac;
    {
        CtBatch a1 = rotate(c, ek, Au.cts.view(), h);
        CtBatch rl = rot_left_from(c, ek, pp, a1.view(), h, s0, s1);
        CtBatch ri = ct_mul_i(c, rl.view());
        Ac = ct_add(c, Au.cts.view(), ri.view());
    }
    std::vector<CtBatch> AR;
    if (h > 1) {
        std::vector<int> rs;
        for (int k = 1; k < h; k++) rs.push_back(k);
        AR = rotations(c, ek, Ac.view(), rs, flags);
    }
    // RotLeft(A_cplx, k >= 1) sits one level below A_cplx; the k = 0 term is
    // brought down too so that all c/2 products share one rescale prime.
    CtBatch Ac0;
    if (!pru && h > 1) Ac0 = drop_level(c, Ac.view(), Ac.lv - 1);
    CtView Ac0v = (!pru && h > 1) ? Ac0.view() : Ac.view();
    CtBatch X;
    for (int k = 0; k < h; k++) {
        CtBatch Akb, Bkb;
        CtView Ak, Bk;
        if (pru) {
            Ak = k == 0 ? Ac.view() : AR[k - 1].view();
            if (k == 0) {
                Bk = B.cts.view();
            } else {
                Bkb = prot_up(c, ek, pp, B.cts.view(), k, s0, s1);
                Bk = Bkb.view();
            }
        } else {
            if (k == 0) {
                Ak = Ac0v;
            } else {
                Akb = rot_left_from(c, ek, pp, AR[k - 1].view(), k, s0, s1);
                Ak = Akb.view();
            }
            Bk = B.cts.view();
        }
        // S_j = sum_r A_k[r] * B_k[r][j]
        CtBatch S;
        if (m == 1) {
            S = mult(c, ek, Bk, Ak);
        } else {
            std::vector<CtBatch> cols;
            for (int j = 0; j < n; j++) {
                std::vector<CtBatch> prods;
                CtBatch acc;
                if (flags & FLAG_LAZY_RELIN) {
                    // gather column j of B_k into a batch aligned with A_k's rows
                    CtBatch colj(&c, m, Bk.lv, Bk.scale);
                    for (int r = 0; r < m; r++)
                        HETAL_CUDA_CHECK(cudaMemcpyAsync(colj.ct(r), Bk.ct(r * n + j), sizeof(u64) * Bk.ct_words(),
                                                         cudaMemcpyDeviceToDevice, c.stream));
                    acc = mult_sum(c, ek, Ak, colj.view());
                } else {
                    for (int r = 0; r < m; r++) {
                        CtBatch pr = mult(c, ek, Ak.sub(r, 1), Bk.sub(r * n + j, 1));
                        acc = r == 0 ? std::move(pr) : ct_add(c, acc.view(), pr.view());
                    }
                }
                cols.push_back(std::move(acc));
            }
            S = gather(c, cols);
        }
        CtBatch x = sum_rows(c, ek, std::move(S), s0, s1);
        x = cmult_mask(c, pp, x.view(), PT_ATB_DIAG, k, cc, s0, s1, t);
        X = (k == 0) ? std::move(x) : ct_add(c, X.view(), x.view());
    }
    CtBatch cj = conjugate(c, ek, X.view());
    Mat out;
    out.cts = ct_add(c, X.view(), cj.view());
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
