// ckks.cu -- RNS-CKKS operations on the device, orchestrated on the host.
//
// Key switching is the hybrid (digit + special primes) form:
//   ModUp   each digit j of d (limbs [j*alpha, (j+1)*alpha)) is brought from
//           coefficient form to the other lv+1+K-alpha moduli by fast base
//           conversion and transformed;
//   KIP     acc_c = sum_j ext_j * key_{j,c} on lv+1+K limbs;
//   ModDown acc_c -> (acc_c - conv_P->Q(acc_c)) * P^{-1} on the lv+1 limbs.
// Rotation by r applies X -> X^{5^r} to both components and switches the key
// of c1(X^g); the hoisted form extends c1 once and applies X -> X^g to the
// extended digits inside the key inner product.
#include "ckks.h"

#include <climits>

#include <algorithm>
#include <cmath>
#include <cstring>

namespace hetal {

u64 galois_rot(const Params &p, int r)
{
    u64 two_n = 2 * (u64)p.N, g = 1, b = 5;
    int e = ((r % p.slots()) + p.slots()) % p.slots();
    for (; e; e >>= 1) {
        if (e & 1) g = (g * b) % two_n;
        b = (b * b) % two_n;
    }
    return g;
}

u64 galois_conj(const Params &p) { return 2 * (u64)p.N - 1; }

static LimbMap all_map(const Params &p)
{
    LimbMap m;
    m.n = p.L + p.K;
    for (int i = 0; i < m.n; i++) m.idx[i] = (unsigned char)i;
    return m;
}

static LimbMap single_map(int idx)
{
    LimbMap m;
    m.n = 1;
    m.idx[0] = (unsigned char)idx;
    return m;
}

// ---------------------------------------------------------------------------
// keys
// ---------------------------------------------------------------------------
SecretKey *keygen_secret(Context &c, u64 seed)
{
    const Params &p = c.p;
    SecretKey *sk = new SecretKey();
    long long *d_s = (long long *)c.alloc_bytes(sizeof(long long) * p.N);
    k_sample_secret(c, d_s, seed, stream_secret(), p.h);
    sk->coeffs.resize(p.N);
    HETAL_CUDA_CHECK(cudaMemcpyAsync(sk->coeffs.data(), d_s, sizeof(long long) * p.N, cudaMemcpyDeviceToHost,
                                     c.stream));
    LimbMap am = all_map(p);
    sk->ntt = c.alloc((size_t)am.n * p.N);
    PolyBatch sb{sk->ntt, 1, 0};
    k_reduce_i64(c, sb, d_s, 0, am);
    ntt_forward(c, sb, am, identity_pos(am.n));
    c.free_bytes(d_s);
    c.sync();
    return sk;
}

void free_secret(Context &c, SecretKey *sk)
{
    if (!sk) return;
    if (sk->ntt) c.free(sk->ntt);
    c.sync();
    delete sk;
}

SwitchKey gen_switch_key(Context &c, const SecretKey &sk, u64 seed, u64 kid, const u64 *s_from_ntt)
{
    const Params &p = c.p;
    const int M = p.L + p.K, N = p.N, dnum = p.dnum_full();
    LimbMap am = all_map(p);
    LimbMap idm = identity_pos(M);
    SwitchKey key;
    key.data = c.alloc((size_t)dnum * 2 * M * N);
    long long *d_e = (long long *)c.alloc_bytes(sizeof(long long) * dnum * N);
    std::vector<u64> streams(dnum);
    for (int j = 0; j < dnum; j++) streams[j] = stream_key_e(kid, (u64)j);
    k_sample_cbd(c, d_e, dnum, N, seed, streams.data());
    DBuf tmp(&c, (size_t)M * N);
    PolyBatch tb{tmp.ptr, 1, 0};
    PolyBatch sb{sk.ntt, 1, 0};
    PolyBatch sf{const_cast<u64 *>(s_from_ntt), 1, 0};
    for (int j = 0; j < dnum; j++) {
        PolyBatch a{key.data + (size_t)(j * 2 + 1) * M * N, 1, 0};
        PolyBatch b{key.data + (size_t)(j * 2 + 0) * M * N, 1, 0};
        k_sample_uniform(c, a, seed, stream_key_a(kid, (u64)j), am);
        ntt_forward(c, a, am, idm);
        k_reduce_i64(c, b, d_e + (size_t)j * N, 0, am);
        ntt_forward(c, b, am, idm);
        k_mul(c, tb, a, sb, am);
        k_sub(c, b, b, tb, am);
        ScalarMap sm;
        std::memset(&sm, 0, sizeof(sm));
        for (int t = j * p.alpha; t < std::min((j + 1) * p.alpha, p.L); t++) {
            u64 q = p.mod[t], P = 1;
            for (int k = 0; k < p.K; k++) P = host_mulmod(P, p.mod[p.L + k] % q, q);
            sm.v[t] = P;
            sm.vs[t] = host_shoup(P, q);
        }
        k_axpy_scalar(c, b, b, sf, sm, am);
    }
    PolyBatch all{key.data, dnum * 2, (size_t)M * N};
    k_to_mont(c, all, all, am);
    c.free_bytes(d_e);
    return key;
}

EvalKeys *keygen_eval(Context &c, const SecretKey &sk, u64 seed, const std::vector<int> &rots, bool conj, bool relin)
{
    const Params &p = c.p;
    const int M = p.L + p.K;
    LimbMap am = all_map(p);
    EvalKeys *ek = new EvalKeys();
    DBuf sf(&c, (size_t)M * p.N);
    PolyBatch sfb{sf.ptr, 1, 0}, sb{sk.ntt, 1, 0};
    if (relin) {
        k_mul(c, sfb, sb, sb, am);
        ek->relin = gen_switch_key(c, sk, seed, KID_RELIN, sf.ptr);
        ek->has_relin = true;
    }
    if (conj) {
        k_automorphism(c, PolyBatch{sf.ptr, 1, 0}, PolyBatch{sk.ntt, 1, 0}, M, galois_conj(p));
        ek->conj = gen_switch_key(c, sk, seed, KID_CONJ, sf.ptr);
        ek->has_conj = true;
    }
    for (int r0 : rots) {
        int r = ((r0 % p.slots()) + p.slots()) % p.slots();
        if (r == 0 || ek->rot.count(r)) continue;
        k_automorphism(c, PolyBatch{sf.ptr, 1, 0}, PolyBatch{sk.ntt, 1, 0}, M, galois_rot(p, r));
        ek->rot[r] = gen_switch_key(c, sk, seed, kid_rot(r), sf.ptr);
    }
    c.sync();
    return ek;
}

void free_eval(Context &c, EvalKeys *ek)
{
    if (!ek) return;
    if (ek->relin.data) c.free(ek->relin.data);
    if (ek->conj.data) c.free(ek->conj.data);
    for (auto &kv : ek->rot) c.free(kv.second.data);
    c.sync();
    delete ek;
}

const SwitchKey &rot_key(const EvalKeys &ek, int r)
{
    auto it = ek.rot.find(r);
    if (it == ek.rot.end()) throw Error(ERR_MISSING_KEY, "no rotation key for step " + std::to_string(r));
    return it->second;
}

// ---------------------------------------------------------------------------
// encryption, decryption, import / export
// ---------------------------------------------------------------------------
CtBatch encrypt_int(Context &c, const SecretKey &sk, u64 seed, u64 nonce0, const long long *d_m, int n, int lv,
                    double scale)
{
    const Params &p = c.p;
    if (lv < 0 || lv >= p.L) throw Error(ERR_LEVEL, "encryption level out of range");
    const int N = p.N;
    LimbMap qm = c.q_map(lv);
    LimbMap id = identity_pos(lv + 1);
    CtBatch out(&c, n, lv, scale);
    for (int i = 0; i < n; i++) {
        PolyBatch c1{out.ct(i) + (size_t)(lv + 1) * N, 1, 0};
        k_sample_uniform(c, c1, seed, stream_enc_a(nonce0 + i), qm);
    }
    ntt_forward(c, out.comp(1), qm, id);
    long long *d_e = (long long *)c.alloc_bytes(sizeof(long long) * n * N);
    std::vector<u64> streams(n);
    for (int i = 0; i < n; i++) streams[i] = stream_enc_e(nonce0 + i);
    k_sample_cbd(c, d_e, n, N, seed, streams.data());
    DBuf e(&c, (size_t)n * (lv + 1) * N);
    PolyBatch eb{e.ptr, n, (size_t)(lv + 1) * N};
    k_reduce_i64(c, out.comp(0), d_m, N, qm);
    ntt_forward(c, out.comp(0), qm, id);
    k_reduce_i64(c, eb, d_e, N, qm);
    ntt_forward(c, eb, qm, id);
    k_add(c, out.comp(0), out.comp(0), eb, qm);
    k_mul(c, eb, out.comp(1), PolyBatch{sk.ntt, n, 0}, qm);
    k_sub(c, out.comp(0), out.comp(0), eb, qm);
    c.free_bytes(d_e);
    return out;
}

void decrypt_to_double(Context &c, const SecretKey &sk, const CtView &a, double *d_out)
{
    const int N = c.p.N;
    DBuf t(&c, (size_t)a.n * N);
    PolyBatch tb{t.ptr, a.n, (size_t)N};
    LimbMap m0 = single_map(0);
    k_mul(c, tb, a.comp(1), PolyBatch{sk.ntt, a.n, 0}, m0);
    k_add(c, tb, tb, a.comp(0), m0);
    ntt_inverse(c, tb, m0, identity_pos(1));
    k_center_to_double(c, d_out, tb, a.n);
}

CtBatch import_coeff(Context &c, const u64 *d_coeff, int n, int lv, double scale)
{
    if (lv < 0 || lv >= c.p.L) throw Error(ERR_LEVEL, "level out of range");
    CtBatch out(&c, n, lv, scale);
    HETAL_CUDA_CHECK(cudaMemcpyAsync(out.data, d_coeff, sizeof(u64) * n * out.ct_words(), cudaMemcpyDeviceToDevice,
                                     c.stream));
    ntt_forward(c, out.polys(), c.q_map(lv), identity_pos(lv + 1));
    return out;
}

void export_coeff(Context &c, const CtView &a, u64 *d_coeff)
{
    HETAL_CUDA_CHECK(cudaMemcpyAsync(d_coeff, a.data, sizeof(u64) * a.n * a.ct_words(), cudaMemcpyDeviceToDevice,
                                     c.stream));
    PolyBatch pb{d_coeff, 2 * a.n, (size_t)(a.lv + 1) * a.N};
    ntt_inverse(c, pb, c.q_map(a.lv), identity_pos(a.lv + 1));
}

Plain plain_from_int(Context &c, const long long *d_coeffs, int lv, double scale)
{
    const int N = c.p.N;
    LimbMap qm = c.q_map(lv);
    Plain pt;
    pt.ctx = &c;
    pt.lv = lv;
    pt.scale = scale;
    pt.data = c.alloc((size_t)(lv + 1) * N);
    pt.mont = c.alloc((size_t)(lv + 1) * N);
    PolyBatch db{pt.data, 1, 0}, mb{pt.mont, 1, 0};
    k_reduce_i64(c, db, d_coeffs, 0, qm);
    ntt_forward(c, db, qm, identity_pos(lv + 1));
    k_to_mont(c, mb, db, qm);
    return pt;
}

Plain plain_encode(Context &c, const double *d_re, const double *d_im, int lv, double scale)
{
    long long *d_m = (long long *)c.alloc_bytes(sizeof(long long) * c.p.N);
    k_encode(c, d_m, d_re, d_im, 1, scale);
    Plain pt = plain_from_int(c, d_m, lv, scale);
    c.free_bytes(d_m);
    return pt;
}

// ---------------------------------------------------------------------------
// slot-wise operations
// ---------------------------------------------------------------------------
static void check_scales(double a, double b)
{
    if (std::fabs(a / b - 1.0) > 1e-9) throw Error(ERR_SCALE, "ciphertext scales differ");
}

CtBatch ct_copy(Context &c, const CtView &a)
{
    CtBatch out(&c, a.n, a.lv, a.scale);
    HETAL_CUDA_CHECK(cudaMemcpyAsync(out.data, a.data, sizeof(u64) * a.n * a.ct_words(), cudaMemcpyDeviceToDevice,
                                     c.stream));
    return out;
}

CtBatch drop_level(Context &c, const CtView &a, int lv)
{
    if (lv > a.lv || lv < 0) throw Error(ERR_LEVEL, "cannot raise a ciphertext's level");
    if (lv == a.lv) return ct_copy(c, a);
    CtBatch out(&c, a.n, lv, a.scale);
    for (int k = 0; k < 2; k++) k_copy(c, out.comp(k), a.comp(k), lv + 1);
    return out;
}

// Bring a and b to a common level; tmp holds a dropped copy if one was needed.
static void align(Context &c, CtView &a, CtView &b, CtBatch &tmp)
{
    if (a.lv > b.lv) {
        tmp = drop_level(c, a, b.lv);
        a = tmp.view();
    } else if (b.lv > a.lv) {
        tmp = drop_level(c, b, a.lv);
        b = tmp.view();
    }
}

static CtBatch add_sub(Context &c, CtView a, CtView b, bool sub)
{
    CtBatch tmp;
    align(c, a, b, tmp);
    check_scales(a.scale, b.scale);
    if (b.n != a.n && b.n != 1) throw Error(ERR_SHAPE, "batch sizes differ");
    CtBatch out(&c, a.n, a.lv, a.scale);
    LimbMap qm = c.q_map(a.lv);
    for (int k = 0; k < 2; k++) {
        PolyBatch bb = b.comp(k);
        if (b.n == 1) bb.stride = 0;
        if (sub)
            k_sub(c, out.comp(k), a.comp(k), bb, qm);
        else
            k_add(c, out.comp(k), a.comp(k), bb, qm);
    }
    return out;
}

CtBatch ct_add(Context &c, const CtView &a, const CtView &b) { return add_sub(c, a, b, false); }
CtBatch ct_sub(Context &c, const CtView &a, const CtView &b) { return add_sub(c, a, b, true); }

void ct_add_inplace(Context &c, CtBatch &acc, const CtView &b)
{
    acc = ct_add(c, acc.view(), b);
}

CtBatch ct_mul_i(Context &c, const CtView &a)
{
    CtBatch out(&c, a.n, a.lv, a.scale);
    k_mul_i(c, out.polys(), a.polys(), c.q_map(a.lv));
    return out;
}

CtBatch ct_sum(Context &c, const CtView &a)
{
    if (a.n == 1) return ct_copy(c, a);
    CtBatch out(&c, 1, a.lv, a.scale);
    LimbMap qm = c.q_map(a.lv);
    for (int k = 0; k < 2; k++) k_sum_polys(c, out.comp(k), a.comp(k), 1, qm);
    return out;
}

static void rescale_polys(Context &c, PolyBatch out, PolyBatch in, int lv)
{
    const int N = c.p.N;
    const int cnt = in.count;
    DBuf top(&c, (size_t)cnt * N);
    PolyBatch tb{top.ptr, cnt, (size_t)N};
    ntt_inverse_oop(c, tb, PolyBatch{in.ptr + (size_t)lv * N, cnt, in.stride}, single_map(lv), identity_pos(1));
    DBuf spread(&c, (size_t)cnt * lv * N);
    PolyBatch sb{spread.ptr, cnt, (size_t)lv * N};
    k_rescale_spread(c, sb, tb, lv);
    ntt_forward(c, sb, c.q_map(lv - 1), identity_pos(lv));
    k_rescale_finish(c, out, in, sb, lv);
    c.cnt.rescale += cnt / 2;
}

CtBatch rescale(Context &c, const CtView &a)
{
    if (a.lv < 1) throw Error(ERR_LEVEL, "no level left to rescale");
    CtBatch out(&c, a.n, a.lv - 1, a.scale / (double)c.p.mod[a.lv]);
    rescale_polys(c, out.polys(), a.polys(), a.lv);
    return out;
}

CtBatch mul_plain_rescale(Context &c, const CtView &a, const Plain &pt, double out_scale)
{
    if (pt.lv < a.lv) throw Error(ERR_LEVEL, "plaintext below ciphertext level");
    if (a.lv < 1) throw Error(ERR_LEVEL, "no level left for a plaintext product");
    CtBatch tmp(&c, a.n, a.lv, a.scale * pt.scale);
    k_mul_plain(c, tmp.polys(), a.polys(), pt.mont, c.q_map(a.lv));
    CtBatch out = rescale(c, tmp.view());
    out.scale = out_scale;
    c.cnt.cmult += a.n;
    return out;
}

// sum_i a_i (.) pt_i, then one rescale by q_lv; every a_i at one level, block count and
// scale, every plaintext at that level or above; the result is given out_scale.
CtBatch mul_plain_sum_rescale(Context &c, const std::vector<CtView> &as, const std::vector<const Plain *> &pts,
                              double out_scale)
{
    if (as.empty() || as.size() != pts.size()) throw Error(ERR_INVALID_ARG, "plaintext-product sum: term counts");
    const CtView &a0 = as[0];
    if (a0.lv < 1) throw Error(ERR_LEVEL, "no level left for a plaintext product");
    std::vector<const u64 *> cp, pp;
    for (size_t i = 0; i < as.size(); i++) {
        if (as[i].lv != a0.lv || as[i].n != a0.n) throw Error(ERR_SHAPE, "plaintext-product sum: levels or shapes differ");
        if (std::fabs(as[i].scale / a0.scale - 1.0) > 1e-9) throw Error(ERR_SCALE, "plaintext-product sum: scales differ");
        if (pts[i]->lv < a0.lv) throw Error(ERR_LEVEL, "plaintext below ciphertext level");
        cp.push_back(as[i].data);
        pp.push_back(pts[i]->mont);
    }
    CtBatch tmp(&c, a0.n, a0.lv, a0.scale);
    k_mul_plain_sum(c, tmp.polys(), cp, (size_t)(a0.lv + 1) * c.p.N, pp, c.q_map(a0.lv));
    CtBatch out = rescale(c, tmp.view());
    out.scale = out_scale;
    c.cnt.cmult += (long long)a0.n * as.size();
    return out;
}

CtBatch mul_const_rescale(Context &c, const CtView &a, double value, double out_scale)
{
    if (a.lv < 1) throw Error(ERR_LEVEL, "no level left for a constant product");
    if (!(out_scale > 0) || !std::isfinite(value)) throw Error(ERR_INVALID_ARG, "constant product: value or scale");
    const double q = (double)c.p.mod[a.lv];
    const double v = value * out_scale * q / a.scale;
    if (!(std::fabs(v) < 9.0e18)) throw Error(ERR_INVALID_ARG, "constant product: the integer constant exceeds 63 bits");
    const long long m = (long long)std::round(v);   // half away from zero
    ScalarMap sm;
    std::memset(&sm, 0, sizeof(sm));
    for (int i = 0; i <= a.lv; i++) {
        const u64 qi = c.p.mod[i];
        const u64 r = m >= 0 ? (u64)m % qi : (qi - (u64)(-(m + 1)) % qi - 1) % qi;
        sm.v[i] = r;
        sm.vs[i] = host_shoup(r, qi);
    }
    CtBatch tmp(&c, a.n, a.lv, out_scale * q);
    k_mul_scalar(c, tmp.polys(), a.polys(), sm, c.q_map(a.lv));
    CtBatch out = rescale(c, tmp.view());
    out.scale = out_scale;
    c.cnt.cmult += a.n;
    return out;
}

// Every block times the integer t (no level, no rescale): the message is
// multiplied by t, the scale is unchanged.
CtBatch mul_int(Context &c, const CtView &a, long long t)
{
    if (t == 0 || t == LLONG_MIN) throw Error(ERR_INVALID_ARG, "integer product: t must be nonzero and above -2^63");
    ScalarMap sm;
    std::memset(&sm, 0, sizeof(sm));
    for (int i = 0; i <= a.lv; i++) {
        const u64 qi = c.p.mod[i];
        const u64 r = t > 0 ? (u64)t % qi : (qi - (u64)(-t) % qi) % qi;
        sm.v[i] = r;
        sm.vs[i] = host_shoup(r, qi);
    }
    CtBatch out(&c, a.n, a.lv, a.scale);
    k_mul_scalar(c, out.polys(), a.polys(), sm, c.q_map(a.lv));
    return out;
}

// Mult landing on the scale `target`: the first operand is first multiplied by
// the integer t = round(target * q_lv / (scale_a * scale_b)) (half away from
// zero), so that the rescale by q_lv leaves scale_a * t * scale_b / q_lv, within
// a factor 1 +- 1/(2t) of target.  Each product re-aims at target, so the scale
// does not drift along a chain of squarings.
CtBatch mult_scaled(Context &c, const EvalKeys &ek, const CtView &a0, const CtView &b0, double target)
{
    CtView a = a0, b = b0;
    CtBatch tmp;
    align(c, a, b, tmp);
    if (a.lv < 1) throw Error(ERR_LEVEL, "no level left for a product");
    if (!(target > 0) || !std::isfinite(target)) throw Error(ERR_INVALID_ARG, "scaled product: target scale");
    const double q = (double)c.p.mod[a.lv];
    const double v = target * q / (a.scale * b.scale);
    if (!(v >= 1.0 && v < 4.0e18))
        throw Error(ERR_INVALID_ARG, "scaled product: the integer factor must lie in [1, 2^62)");
    const long long t = (long long)std::round(v);
    CtBatch at = mul_int(c, a, t);
    at.scale = a.scale * (double)t;
    return mult(c, ek, at.view(), b);
}

// Bootstrapping's first step: a level-0 ciphertext (c0, c1) mod q_0 as one at level lv
// whose residues are the centred level-0 values reduced modulo q_0..q_lv.  It decrypts, over
// the integers, to t = Delta m + e + q_0 I; it is given the scale q_0.
CtBatch mod_raise(Context &c, const CtView &a, int lv)
{
    if (a.lv != 0) throw Error(ERR_LEVEL, "ModRaise takes a level-0 ciphertext");
    if (lv < 1 || lv >= c.p.L) throw Error(ERR_LEVEL, "ModRaise: target level out of range");
    const int N = c.p.N, cnt = 2 * a.n;
    DBuf coef(&c, (size_t)cnt * N);
    PolyBatch cb{coef.ptr, cnt, (size_t)N};
    k_copy(c, cb, PolyBatch{a.data, cnt, (size_t)N}, 1);
    ntt_inverse(c, cb, single_map(0), identity_pos(1));
    long long *v = (long long *)c.alloc_bytes(sizeof(long long) * cnt * N);
    k_center_i64(c, v, cb, c.p.mod[0]);
    CtBatch out(&c, a.n, lv, (double)c.p.mod[0]);
    k_reduce_i64(c, out.polys(), v, (size_t)N, c.q_map(lv));
    c.free_bytes(v);
    ntt_forward(c, out.polys(), c.q_map(lv), identity_pos(lv + 1));
    return out;
}

CtBatch add_plain(Context &c, const CtView &a, const Plain &pt)
{
    if (pt.lv < a.lv) throw Error(ERR_LEVEL, "plaintext below ciphertext level");
    CtBatch out = ct_copy(c, a);
    k_add(c, out.comp(0), out.comp(0), PolyBatch{pt.data, a.n, 0}, c.q_map(a.lv));
    return out;
}

// ---------------------------------------------------------------------------
// key switching
// ---------------------------------------------------------------------------
// ext: [dnum][B][lv+1+K][N] extended digits of d (NTT domain); the limbs a digit
// already has are not copied: the key inner product reads them from d.
static void modup_all(Context &c, PolyBatch d, int lv, u64 *ext)
{
    const Params &p = c.p;
    const int N = p.N, B = d.count, nl = lv + 1 + p.K, dnum = p.dnum(lv);
    DBuf coef(&c, (size_t)B * (lv + 1) * N);
    PolyBatch cb{coef.ptr, B, (size_t)(lv + 1) * N};
    // coefficients times (D_j/q_i)^{-1}: the conversion's first factor rides on the INTT's N^{-1}
    const Context::LimbScale &sc = c.modup_scale(lv);
    ntt_inverse_scaled(c, cb, d, c.q_map(lv), identity_pos(lv + 1), sc.sc, sc.sc_sh);
    for (int j = 0; j < dnum; j++) {
        PolyBatch ej{ext + (size_t)j * B * nl * N, B, (size_t)nl * N};
        const ModUpTables &t = c.modup_tables(lv, j);
        if (t.a <= MAX_FUSED_CONV) {   // the conversion rides on the transform's first pass
            ntt_forward_conv(c, ej, t.dst, t.dst_pos, ConvSrc{cb, t.src, t.hat_mont, t.a});
        } else {
            k_base_conv(c, "modup_conv", ej, cb, t.a, t.src, t.dst, t.dst_pos, t.hat_mont);
            ntt_forward(c, ej, t.dst, t.dst_pos);
        }
    }
    c.cnt.modup_digits += (long long)B * dnum;
}

// ModDown of 2B accumulators [acc_0 (B polys), acc_1 (B polys)] (lv+1+K limbs):
// out_c = (acc_c - conv_c) P^{-1} (+ add_c).
static void moddown(Context &c, u64 *acc, int B, int lv, PolyBatch out0, PolyBatch out1, PolyBatch add0,
                    PolyBatch add1)
{
    const Params &p = c.p;
    const int N = p.N, nl = lv + 1 + p.K;
    PolyBatch acc0{acc, B, (size_t)nl * N}, acc1{acc + (size_t)B * nl * N, B, (size_t)nl * N};
    PolyBatch accAll{acc, 2 * B, (size_t)nl * N};
    LimbMap spm, spos;
    spm.n = spos.n = p.K;
    for (int k = 0; k < p.K; k++) {
        spm.idx[k] = (unsigned char)(p.L + k);
        spos.idx[k] = (unsigned char)(lv + 1 + k);
    }
    // special limbs times (P/p_k)^{-1}, folded into the INTT's N^{-1}
    ntt_inverse_scaled(c, accAll, accAll, spm, spos, c.d_md_scale, c.d_md_scale_sh);
    DBuf conv(&c, (size_t)2 * B * (lv + 1) * N);
    PolyBatch convAll{conv.ptr, 2 * B, (size_t)(lv + 1) * N};
    ModDownTail tail{{out0, out1}, {acc0, acc1}, {add0, add1}, B};
    if (p.K <= MAX_FUSED_CONV) {   // the conversion rides on the transform's first pass
        ntt_forward_moddown_conv(c, convAll, lv, tail, ConvSrc{accAll, spos, c.d_phat_mont, p.K});
    } else {
        k_base_conv(c, "moddown_conv", convAll, accAll, p.K, spos, c.q_map(lv), identity_pos(lv + 1),
                    c.d_phat_mont);
        ntt_forward_moddown(c, convAll, lv, tail);
    }
}

static void ks_core(Context &c, const u64 *ext, PolyBatch d, int B, int lv, const SwitchKey &key, u64 g,
                    PolyBatch out0, PolyBatch out1, PolyBatch add0, PolyBatch add1)
{
    const Params &p = c.p;
    const int N = p.N, nl = lv + 1 + p.K, dnum = p.dnum(lv);
    DBuf acc(&c, (size_t)2 * B * nl * N);
    PolyBatch acc0{acc.ptr, B, (size_t)nl * N}, acc1{acc.ptr + (size_t)B * nl * N, B, (size_t)nl * N};
    k_kip(c, acc0, acc1, ext, (size_t)B * nl * N, dnum, key.data, lv, g, d);
    moddown(c, acc.ptr, B, lv, out0, out1, add0, add1);
    c.cnt.keyswitch += B;
}

void keyswitch(Context &c, PolyBatch d, const SwitchKey &key, int lv, PolyBatch out0, PolyBatch out1,
               PolyBatch addend0, PolyBatch addend1)
{
    const Params &p = c.p;
    const int B = d.count, nl = lv + 1 + p.K, dnum = p.dnum(lv);
    DBuf ext(&c, (size_t)dnum * B * nl * p.N);
    modup_all(c, d, lv, ext.ptr);
    ks_core(c, ext.ptr, d, B, lv, key, 1, out0, out1, addend0, addend1);
}

static const PolyBatch NOADD{nullptr, 0, 0};

static void tensor_into(Context &c, const CtView &a, const CtView &b, u64 *d, int lv)
{
    const int N = c.p.N, n = a.n;
    size_t ps = (size_t)(lv + 1) * N;
    PolyBatch d0{d, n, ps}, d1{d + (size_t)n * ps, n, ps}, d2{d + (size_t)2 * n * ps, n, ps};
    PolyBatch b0 = b.comp(0), b1 = b.comp(1);
    if (b.n == 1 && n > 1) b0.stride = b1.stride = 0;
    k_tensor(c, d0, d1, d2, a.comp(0), a.comp(1), b0, b1, lv);
}

CtBatch mult(Context &c, const EvalKeys &ek, const CtView &a0, const CtView &b0)
{
    if (!ek.has_relin) throw Error(ERR_MISSING_KEY, "no relinearisation key");
    CtView a = a0, b = b0;
    CtBatch tmp;
    align(c, a, b, tmp);
    if (a.lv < 1) throw Error(ERR_LEVEL, "no level left for a product");
    if (b.n != a.n && b.n != 1) throw Error(ERR_SHAPE, "batch sizes differ");
    const int lv = a.lv, n = a.n, N = c.p.N;
    size_t ps = (size_t)(lv + 1) * N;
    DBuf d(&c, 3 * (size_t)n * ps);
    tensor_into(c, a, b, d.ptr, lv);
    CtBatch r(&c, n, lv, a.scale * b.scale);
    PolyBatch d0{d.ptr, n, ps}, d1{d.ptr + (size_t)n * ps, n, ps}, d2{d.ptr + (size_t)2 * n * ps, n, ps};
    keyswitch(c, d2, ek.relin, lv, r.comp(0), r.comp(1), d0, d1);
    c.cnt.mult += n;
    return rescale(c, r.view());
}

CtBatch mult_sum(Context &c, const EvalKeys &ek, const CtView &a0, const CtView &b0)
{
    if (!ek.has_relin) throw Error(ERR_MISSING_KEY, "no relinearisation key");
    CtView a = a0, b = b0;
    CtBatch tmp;
    align(c, a, b, tmp);
    if (a.lv < 1) throw Error(ERR_LEVEL, "no level left for a product");
    if (b.n != a.n) throw Error(ERR_SHAPE, "batch sizes differ");
    const int lv = a.lv, n = a.n, N = c.p.N;
    size_t ps = (size_t)(lv + 1) * N;
    DBuf d(&c, 3 * (size_t)n * ps);
    tensor_into(c, a, b, d.ptr, lv);
    DBuf s(&c, 3 * ps);
    LimbMap qm = c.q_map(lv);
    for (int k = 0; k < 3; k++)
        k_sum_polys(c, PolyBatch{s.ptr + (size_t)k * ps, 1, ps}, PolyBatch{d.ptr + (size_t)k * n * ps, n, ps}, 1, qm);
    CtBatch r(&c, 1, lv, a.scale * b.scale);
    keyswitch(c, PolyBatch{s.ptr + 2 * ps, 1, ps}, ek.relin, lv, r.comp(0), r.comp(1), PolyBatch{s.ptr, 1, ps},
              PolyBatch{s.ptr + ps, 1, ps});
    c.cnt.mult += n;
    return rescale(c, r.view());
}

// Brings every group's operands to the lowest level among them; temporaries in `keep`.
static int grouped_operands(Context &c, const std::vector<CtView> &as, const std::vector<CtView> &bs,
                            std::vector<CtView> &A, std::vector<CtView> &B, std::vector<CtBatch> &keep)
{
    if (as.size() != bs.size() || as.empty()) throw Error(ERR_SHAPE, "group lists differ");
    int lv = 1 << 30;
    for (size_t g = 0; g < as.size(); g++) lv = std::min(lv, std::min(as[g].lv, bs[g].lv));
    if (lv < 1) throw Error(ERR_LEVEL, "no level left for a product");
    keep.reserve(2 * as.size());
    A.resize(as.size());
    B.resize(as.size());
    for (size_t g = 0; g < as.size(); g++) {
        A[g] = as[g];
        B[g] = bs[g];
        if (A[g].lv > lv) {
            keep.push_back(drop_level(c, A[g], lv));
            A[g] = keep.back().view();
        }
        if (B[g].lv > lv) {
            keep.push_back(drop_level(c, B[g], lv));
            B[g] = keep.back().view();
        }
        if (B[g].n != A[g].n && B[g].n != 1) throw Error(ERR_SHAPE, "batch sizes differ");
        check_scales(A[g].scale * B[g].scale, A[0].scale * B[0].scale);
    }
    return lv;
}

// Tensor products of every group into d = [3][total][lv+1][N]; returns total.
static int grouped_tensor(Context &c, const std::vector<CtView> &A, const std::vector<CtView> &B, int lv, DBuf &d)
{
    int total = 0;
    for (auto &a : A) total += a.n;
    const size_t ps = (size_t)(lv + 1) * c.p.N;
    d = DBuf(&c, 3 * (size_t)total * ps);
    bool uniform = true;
    for (auto &a : A) uniform = uniform && a.n == A[0].n;
    if (uniform && A.size() > 1) {   // every group in one launch (per 64 groups)
        std::vector<const u64 *> pa, pb;
        std::vector<int> bstep;
        for (size_t g = 0; g < A.size(); g++) {
            pa.push_back(A[g].data);
            pb.push_back(B[g].data);
            bstep.push_back(B[g].n == 1 && A[g].n > 1 ? 0 : 1);
        }
        k_tensor_groups(c, d.ptr, total, pa, pb, bstep, A[0].n, lv);
        return total;
    }
    int off = 0;
    for (size_t g = 0; g < A.size(); g++) {
        const int n = A[g].n;
        PolyBatch d0{d.ptr + (size_t)off * ps, n, ps}, d1{d.ptr + (size_t)(total + off) * ps, n, ps},
            d2{d.ptr + (size_t)(2 * total + off) * ps, n, ps};
        PolyBatch b0 = B[g].comp(0), b1 = B[g].comp(1);
        if (B[g].n == 1 && n > 1) b0.stride = b1.stride = 0;
        k_tensor(c, d0, d1, d2, A[g].comp(0), A[g].comp(1), b0, b1, lv);
        off += n;
    }
    return total;
}

CtBatch mult_grouped(Context &c, const EvalKeys &ek, const std::vector<CtView> &as, const std::vector<CtView> &bs)
{
    if (!ek.has_relin) throw Error(ERR_MISSING_KEY, "no relinearisation key");
    std::vector<CtView> A, B;
    std::vector<CtBatch> keep;
    const int lv = grouped_operands(c, as, bs, A, B, keep);
    DBuf d;
    const int total = grouped_tensor(c, A, B, lv, d);
    const size_t ps = (size_t)(lv + 1) * c.p.N;
    CtBatch r(&c, total, lv, A[0].scale * B[0].scale);
    keyswitch(c, PolyBatch{d.ptr + (size_t)2 * total * ps, total, ps}, ek.relin, lv, r.comp(0), r.comp(1),
              PolyBatch{d.ptr, total, ps}, PolyBatch{d.ptr + (size_t)total * ps, total, ps});
    c.cnt.mult += total;
    return rescale(c, r.view());
}

CtBatch mult_sum_grouped(Context &c, const EvalKeys &ek, const std::vector<CtView> &as,
                         const std::vector<CtView> &bs)
{
    if (!ek.has_relin) throw Error(ERR_MISSING_KEY, "no relinearisation key");
    std::vector<CtView> A, B;
    std::vector<CtBatch> keep;
    const int lv = grouped_operands(c, as, bs, A, B, keep);
    const int G = (int)A.size();
    int total = 0;
    for (int g = 0; g < G; g++) {
        if (B[g].n != A[g].n) throw Error(ERR_SHAPE, "the groups of a lazy product sum are pairs of equal batches");
        total += A[g].n;
    }
    const size_t ps = (size_t)(lv + 1) * c.p.N;
    // every group's tensor products summed in one pass (the sum of canonical residues, as
    // tensoring all pairs and adding them would give); groups may differ in size
    DBuf s(&c, 3 * (size_t)G * ps);
    {
        std::vector<const u64 *> pa, pb;
        std::vector<int> bstep, ns;
        for (int g = 0; g < G; g++) {
            pa.push_back(A[g].data);
            pb.push_back(B[g].data);
            bstep.push_back(1);
            ns.push_back(A[g].n);
        }
        k_tensor_sum_ragged(c, s.ptr, G, pa, pb, bstep, ns, lv);
    }
    CtBatch r(&c, G, lv, A[0].scale * B[0].scale);
    keyswitch(c, PolyBatch{s.ptr + (size_t)2 * G * ps, G, ps}, ek.relin, lv, r.comp(0), r.comp(1),
              PolyBatch{s.ptr, G, ps}, PolyBatch{s.ptr + (size_t)G * ps, G, ps});
    c.cnt.mult += total;
    return rescale(c, r.view());
}

CtBatch mul_plain2_rescale_grouped(Context &c, const CtView &a, const std::vector<const Plain *> &pa,
                                   const CtView &b, const std::vector<const Plain *> &pb, int n, double out_scale)
{
    const int G = (int)pa.size();
    if (a.lv < 1 || a.lv != b.lv) throw Error(ERR_LEVEL, "paired plaintext product: levels");
    if ((int)pb.size() != G || (a.n != n && a.n != G * n) || (b.n != n && b.n != G * n))
        throw Error(ERR_SHAPE, "paired plaintext product: batch sizes");
    check_scales(a.scale, b.scale);
    CtBatch tmp(&c, G * n, a.lv, out_scale);
    LimbMap qm = c.q_map(a.lv);
    for (int g = 0; g < G; g++) {
        if (pa[g]->lv < a.lv || pb[g]->lv < a.lv) throw Error(ERR_LEVEL, "plaintext below ciphertext level");
        CtView sa = a.n == n ? a : a.sub(g * n, n), sb = b.n == n ? b : b.sub(g * n, n);
        k_mul_plain2(c, tmp.view().sub(g * n, n).polys(), sa.polys(), pa[g]->mont, sb.polys(), pb[g]->mont, qm);
    }
    CtBatch out = rescale(c, tmp.view());
    out.scale = out_scale;
    c.cnt.cmult += (long long)2 * G * n;
    return out;
}

CtBatch mul_plain_rescale_grouped(Context &c, const CtView &a, const std::vector<const Plain *> &pts, int n,
                                  bool broadcast, double out_scale)
{
    const int G = (int)pts.size();
    if (a.lv < 1) throw Error(ERR_LEVEL, "no level left for a plaintext product");
    if (a.n != (broadcast ? n : G * n)) throw Error(ERR_SHAPE, "grouped plaintext product: batch size");
    CtBatch tmp(&c, G * n, a.lv, out_scale);
    LimbMap qm = c.q_map(a.lv);
    for (int g = 0; g < G; g++) {
        if (pts[g]->lv < a.lv) throw Error(ERR_LEVEL, "plaintext below ciphertext level");
        CtView src = broadcast ? a : a.sub(g * n, n);
        k_mul_plain(c, tmp.view().sub(g * n, n).polys(), src.polys(), pts[g]->mont, qm);
    }
    CtBatch out = rescale(c, tmp.view());
    out.scale = out_scale;
    c.cnt.cmult += (long long)G * n;
    return out;
}

// sigma_g(a) switched back to s, plus y (same level and batch size) if given:
// component 0 of y joins the automorphism's addend, component 1 the ModDown
// tail, so y + sigma_g(a) costs no separate addition pass.  Every step is exact
// modular arithmetic on canonical residues, so the bits equal those of ct_add.
static CtBatch automorph_ks(Context &c, const CtView &a, u64 g, const SwitchKey &key, const CtView *y = nullptr)
{
    CtBatch t(&c, a.n, a.lv, a.scale);
    if (y)
        k_automorphism_add0(c, t.polys(), a.polys(), y->comp(0), a.lv + 1, g);
    else
        k_automorphism(c, t.polys(), a.polys(), a.lv + 1, g);
    CtBatch out(&c, a.n, a.lv, a.scale);
    keyswitch(c, t.comp(1), key, a.lv, out.comp(0), out.comp(1), t.comp(0), y ? y->comp(1) : NOADD);
    return out;
}

// Amounts whose successive rotations add up to r, from the keys that exist:
// r itself if its key exists, else the non-adjacent form of r over +-2^u
// (right rotation by 2^u = left rotation by s - 2^u), else its binary digits.
static std::vector<int> rotation_path(const EvalKeys &ek, int r, int s)
{
    if (ek.rot.count(r)) return {r};
    std::vector<int> naf;
    bool ok = true;
    for (int v = r, u = 0; v; v >>= 1, u++) {
        if (!(v & 1)) continue;
        int d = (v & 3) == 3 ? -1 : 1;   // NAF digit at position u
        int amt = d > 0 ? (1 << u) : s - (1 << u);
        if (amt % s == 0) continue;
        if (!ek.rot.count(amt % s)) ok = false;
        naf.push_back(amt % s);
        v -= d;
    }
    if (ok && !naf.empty()) return naf;
    std::vector<int> bin;
    for (int u = 0; (1 << u) < s; u++)
        if (r & (1 << u)) {
            if (!ek.rot.count(1 << u)) throw Error(ERR_MISSING_KEY, "no rotation key for step " + std::to_string(r));
            bin.push_back(1 << u);
        }
    return bin;
}

CtBatch rotate(Context &c, const EvalKeys &ek, const CtView &a, int r0)
{
    const int s = c.p.slots();
    int r = ((r0 % s) + s) % s;
    if (r == 0) return ct_copy(c, a);
    std::vector<int> path = rotation_path(ek, r, s);
    c.cnt.rot += a.n;
    CtBatch x = automorph_ks(c, a, galois_rot(c.p, path[0]), rot_key(ek, path[0]));
    for (size_t i = 1; i < path.size(); i++) x = automorph_ks(c, x.view(), galois_rot(c.p, path[i]), rot_key(ek, path[i]));
    return x;
}

CtBatch conjugate(Context &c, const EvalKeys &ek, const CtView &a)
{
    if (!ek.has_conj) throw Error(ERR_MISSING_KEY, "no conjugation key");
    c.cnt.conj += a.n;
    return automorph_ks(c, a, galois_conj(c.p), ek.conj);
}

static bool fusable(const CtView &y, const CtView &x)
{
    if (y.lv != x.lv || y.n != x.n) return false;
    check_scales(y.scale, x.scale);
    return true;
}

CtBatch add_rotate(Context &c, const EvalKeys &ek, const CtView &y, const CtView &x, int r0)
{
    if (!fusable(y, x)) {
        CtBatch r = rotate(c, ek, x, r0);
        return ct_add(c, y, r.view());
    }
    const int s = c.p.slots();
    int r = ((r0 % s) + s) % s;
    if (r == 0) return ct_add(c, y, x);
    std::vector<int> path = rotation_path(ek, r, s);
    c.cnt.rot += x.n;
    CtBatch cur;
    CtView v = x;
    for (size_t i = 0; i + 1 < path.size(); i++) {
        cur = automorph_ks(c, v, galois_rot(c.p, path[i]), rot_key(ek, path[i]));
        v = cur.view();
    }
    return automorph_ks(c, v, galois_rot(c.p, path.back()), rot_key(ek, path.back()), &y);
}

CtBatch add_conjugate(Context &c, const EvalKeys &ek, const CtView &y, const CtView &x)
{
    if (!fusable(y, x)) {
        CtBatch cj = conjugate(c, ek, x);
        return ct_add(c, y, cj.view());
    }
    if (!ek.has_conj) throw Error(ERR_MISSING_KEY, "no conjugation key");
    c.cnt.conj += x.n;
    return automorph_ks(c, x, galois_conj(c.p), ek.conj, &y);
}

CtBatch rotate_sum(Context &c, const EvalKeys &ek, const CtView &a, const std::vector<int> &rs0)
{
    const Params &p = c.p;
    const int s = p.slots();
    std::vector<int> rs;
    bool keyed = true;
    for (int r0 : rs0) {
        const int r = ((r0 % s) + s) % s;
        if (!r) continue;
        rs.push_back(r);
        if (!ek.rot.count(r)) keyed = false;
    }
    if (rs.empty()) return ct_copy(c, a);
    if (!keyed || (int)rs.size() > MAX_KS_STEPS) {   // one rotation at a time
        CtBatch x = ct_copy(c, a);
        for (int r : rs) x = add_rotate(c, ek, x.view(), a, r);
        return x;
    }
    const int S = (int)rs.size(), B = a.n, lv = a.lv, N = p.N, nl = lv + 1 + p.K, dnum = p.dnum(lv);
    std::vector<const u64 *> keys;
    std::vector<u64> gs;
    for (int r : rs) {
        keys.push_back(rot_key(ek, r).data);
        gs.push_back(galois_rot(p, r));
    }
    HoistedSource hs = hoist_prepare(c, a);
    CtBatch out(&c, B, lv, a.scale);
    DBuf t0(&c, (size_t)B * (lv + 1) * N);
    PolyBatch t0b{t0.ptr, B, (size_t)(lv + 1) * N};
    k_automorphism_sum(c, t0b, a.comp(0), gs, lv + 1);   // a_0 + sum_s a_0(X^g_s)
    DBuf acc(&c, (size_t)2 * B * nl * N);
    PolyBatch acc0{acc.ptr, B, (size_t)nl * N}, acc1{acc.ptr + (size_t)B * nl * N, B, (size_t)nl * N};
    k_kip_sum(c, acc0, acc1, hs.ext.ptr, (size_t)B * nl * N, dnum, keys, gs, lv, a.comp(1));
    moddown(c, acc.ptr, B, lv, out.comp(0), out.comp(1), t0b, a.comp(1));
    c.cnt.keyswitch += B;
    c.cnt.rot += (long long)S * B;
    return out;
}

HoistedView hoisted_view(const Context &c, const HoistedSource &hs, int first, int count)
{
    if (first < 0 || count < 0 || first + count > hs.a.n) throw Error(ERR_INVALID_ARG, "hoisted view out of range");
    const size_t blk = (size_t)(hs.a.lv + 1 + c.p.K) * c.p.N;
    HoistedView v;
    v.a = hs.a.sub(first, count);
    v.ext = hs.ext.ptr + (size_t)first * blk;
    v.digit_stride = (size_t)hs.a.n * blk;
    return v;
}

HoistedSource hoist_prepare(Context &c, const CtView &a)
{
    const Params &p = c.p;
    HoistedSource hs;
    hs.a = a;
    const int nl = a.lv + 1 + p.K, dnum = p.dnum(a.lv);
    hs.ext = DBuf(&c, (size_t)dnum * a.n * nl * p.N);
    modup_all(c, a.comp(1), a.lv, hs.ext.ptr);
    return hs;
}

CtBatch hoist_rotate(Context &c, const EvalKeys &ek, const HoistedSource &hs, int r0)
{
    std::vector<CtBatch> r = hoist_rotate_many(c, ek, hs, std::vector<int>{r0});
    return std::move(r[0]);
}

// One batched key switch for S amounts with keys: automorphisms of component 0,
// key inner products and ModDown over all S x B ciphertexts at once; the result
// is [step][block].  Every step computes what hoist-rotating by it alone would.
static CtBatch hoist_rotate_keyed(Context &c, const EvalKeys &ek, const HoistedView &hs, const std::vector<int> &rs)
{
    const Params &p = c.p;
    const CtView &a = hs.a;
    const int S = (int)rs.size(), B = a.n, lv = a.lv, N = p.N, nl = lv + 1 + p.K, dnum = p.dnum(lv);
    std::vector<const u64 *> keys;
    std::vector<u64> gs;
    for (int r : rs) {
        keys.push_back(rot_key(ek, r).data);
        gs.push_back(galois_rot(p, r));
    }
    CtBatch out(&c, S * B, lv, a.scale);
    DBuf t0(&c, (size_t)S * B * (lv + 1) * N);
    PolyBatch t0b{t0.ptr, S * B, (size_t)(lv + 1) * N};
    k_automorphism_steps(c, t0b, a.comp(0), gs, lv + 1);
    DBuf acc(&c, (size_t)2 * S * B * nl * N);
    PolyBatch acc0{acc.ptr, S * B, (size_t)nl * N}, acc1{acc.ptr + (size_t)S * B * nl * N, S * B, (size_t)nl * N};
    k_kip_steps(c, acc0, acc1, hs.ext, hs.digit_stride, dnum, keys, gs, lv, a.comp(1));
    moddown(c, acc.ptr, S * B, lv, out.comp(0), out.comp(1), t0b, NOADD);
    c.cnt.keyswitch += (long long)S * B;
    c.cnt.rot += (long long)S * B;
    return out;
}

CtBatch hoist_rotate_batch(Context &c, const EvalKeys &ek, const HoistedSource &hs, const std::vector<int> &rs0)
{
    return hoist_rotate_batch(c, ek, hoisted_view(c, hs, 0, hs.a.n), rs0);
}

CtBatch hoist_rotate_batch(Context &c, const EvalKeys &ek, const HoistedView &hs, const std::vector<int> &rs0)
{
    const Params &p = c.p;
    const CtView &a = hs.a;
    const int s = p.slots(), S = (int)rs0.size(), B = a.n, lv = a.lv;
    std::vector<int> rs(S);
    bool all_keyed = true;
    for (int i = 0; i < S; i++) {
        rs[i] = ((rs0[i] % s) + s) % s;
        if (rs[i] == 0 || !ek.rot.count(rs[i])) all_keyed = false;
    }
    const size_t ctw = (size_t)2 * (lv + 1) * p.N;
    if (!all_keyed) {   // amounts 0 or without their own key: one at a time into the batch
        CtBatch out(&c, S * B, lv, a.scale);
        for (int i = 0; i < S; i++) {
            CtBatch r = rs[i] == 0 ? ct_copy(c, a) : ek.rot.count(rs[i]) ? hoist_rotate_keyed(c, ek, hs, {rs[i]})
                                                                          : rotate(c, ek, a, rs[i]);
            HETAL_CUDA_CHECK(cudaMemcpyAsync(out.data + (size_t)i * B * ctw, r.data, B * ctw * sizeof(u64),
                                             cudaMemcpyDeviceToDevice, c.stream));
        }
        return out;
    }
    // steps per pass so that the temporaries (component-0 automorphisms, accumulators,
    // ModDown conversions) of one pass stay within the context's batch budget
    const size_t per_step = (size_t)B * p.N * 8 * (3 * (lv + 1) + 2 * (lv + 1 + p.K));
    const int chunk = std::max<int>(1, (int)std::min<size_t>(S, c.batch_bytes / std::max<size_t>(per_step, 1)));
    if (chunk >= S) return hoist_rotate_keyed(c, ek, hs, rs);
    CtBatch out(&c, S * B, lv, a.scale);
    for (int i0 = 0; i0 < S; i0 += chunk) {
        std::vector<int> part(rs.begin() + i0, rs.begin() + std::min(S, i0 + chunk));
        CtBatch r = hoist_rotate_keyed(c, ek, hs, part);
        HETAL_CUDA_CHECK(cudaMemcpyAsync(out.data + (size_t)i0 * B * ctw, r.data, r.n * ctw * sizeof(u64),
                                         cudaMemcpyDeviceToDevice, c.stream));
    }
    return out;
}

std::vector<CtBatch> hoist_rotate_many(Context &c, const EvalKeys &ek, const HoistedSource &hs,
                                       const std::vector<int> &rs)
{
    return CtBatch::split(hoist_rotate_batch(c, ek, hs, rs), (int)rs.size());
}

std::vector<CtBatch> rotate_hoisted(Context &c, const EvalKeys &ek, const CtView &a, const std::vector<int> &rs)
{
    const Params &p = c.p;
    bool any = false;
    for (int r0 : rs) {
        int r = ((r0 % p.slots()) + p.slots()) % p.slots();
        if (r) {
            rotation_path(ek, r, p.slots());   // check that keys exist before any work
            if (ek.rot.count(r)) any = true;
        }
    }
    if (rs.empty()) return {};
    if (!any) {
        std::vector<CtBatch> outs;
        for (int r : rs) outs.push_back(rotate(c, ek, a, r));
        return outs;
    }
    HoistedSource hs = hoist_prepare(c, a);
    return hoist_rotate_many(c, ek, hs, rs);
}

}  // namespace hetal
