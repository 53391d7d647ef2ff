// ckks.h -- RNS-CKKS operations on the device (batched over ciphertexts).
//
// Ciphertexts live in the NTT domain; every operation acts on a batch of
// ciphertexts at one level.  The operations are those the paper builds its
// matrix products from (Sec. 2.2): Add, Mult (tensor, relinearisation,
// rescale), CMult (plaintext product and rescale), Lrot (automorphism
// X -> X^{5^r} and key switching), Conj (X -> X^{-1}), and multiplication by
// sqrt(-1) (X^{N/2}, no depth).
#pragma once
#include "context.h"

namespace hetal {

// Philox stream identifiers (key word 1); key word 0 is the caller's seed.
inline u64 stream_secret() { return (u64)0x01 << 56; }
inline u64 stream_key_a(u64 kid, u64 j) { return ((u64)0x02 << 56) | (kid << 8) | j; }
inline u64 stream_key_e(u64 kid, u64 j) { return ((u64)0x03 << 56) | (kid << 8) | j; }
inline u64 stream_enc_a(u64 nonce) { return ((u64)0x04 << 56) | (nonce & (((u64)1 << 56) - 1)); }
inline u64 stream_enc_e(u64 nonce) { return ((u64)0x05 << 56) | (nonce & (((u64)1 << 56) - 1)); }
constexpr u64 KID_RELIN = 0, KID_CONJ = 1;
inline u64 kid_rot(int r) { return 2 + (u64)r; }

u64 galois_rot(const Params &p, int r);      // 5^r mod 2N
u64 galois_conj(const Params &p);            // 2N - 1

// keys
SecretKey *keygen_secret(Context &c, u64 seed);
void free_secret(Context &c, SecretKey *sk);
SwitchKey gen_switch_key(Context &c, const SecretKey &sk, u64 seed, u64 kid, const u64 *s_from_ntt);
EvalKeys *keygen_eval(Context &c, const SecretKey &sk, u64 seed, const std::vector<int> &rots, bool conj,
                      bool relin);
void free_eval(Context &c, EvalKeys *ek);
const SwitchKey &rot_key(const EvalKeys &ek, int r);

// encryption: ciphertext i of the batch uses nonce nonce0 + i; m is device int64 [n][N]
CtBatch encrypt_int(Context &c, const SecretKey &sk, u64 seed, u64 nonce0, const long long *d_m, int n, int lv,
                    double scale);
// limb-0 message of each ciphertext as centred doubles (device [n][N])
void decrypt_to_double(Context &c, const SecretKey &sk, const CtView &a, double *d_out);

// import / export of coefficient-domain residues [n][2][lv+1][N] (device buffers)
CtBatch import_coeff(Context &c, const u64 *d_coeff, int n, int lv, double scale);
void export_coeff(Context &c, const CtView &a, u64 *d_coeff);

// plaintexts
Plain plain_from_int(Context &c, const long long *d_coeffs, int lv, double scale);
Plain plain_encode(Context &c, const double *d_re, const double *d_im, int lv, double scale);

// slot-wise operations
CtBatch ct_copy(Context &c, const CtView &a);
CtBatch drop_level(Context &c, const CtView &a, int lv);
CtBatch ct_add(Context &c, const CtView &a, const CtView &b);
CtBatch ct_sub(Context &c, const CtView &a, const CtView &b);
void ct_add_inplace(Context &c, CtBatch &acc, const CtView &b);   // acc += b (levels aligned first)
CtBatch ct_mul_i(Context &c, const CtView &a);
CtBatch ct_sum(Context &c, const CtView &a);                       // sum of the batch -> 1 ciphertext
CtBatch rescale(Context &c, const CtView &a);
// CMult: (a * pt) then rescale; out scale = a.scale * pt.scale / q_lv unless exact_scale > 0
CtBatch mul_plain_rescale(Context &c, const CtView &a, const Plain &pt, double out_scale);
CtBatch add_plain(Context &c, const CtView &a, const Plain &pt);
// CMult by the constant `value` landing on exactly out_scale: the product with the integer
// constant polynomial round(value * out_scale * q_lv / scale(a)) (half away from zero), then
// the rescale by q_lv.
CtBatch mul_const_rescale(Context &c, const CtView &a, double value, double out_scale);
CtBatch mul_plain_sum_rescale(Context &c, const std::vector<CtView> &as, const std::vector<const Plain *> &pts,
                              double out_scale);
// Mult: pairwise tensor, relinearisation, rescale (a.n == b.n, or b.n == 1 broadcast)
CtBatch mult(Context &c, const EvalKeys &ek, const CtView &a, const CtView &b);
CtBatch mul_int(Context &c, const CtView &a, long long t);
CtBatch mod_raise(Context &c, const CtView &a, int lv);
CtBatch mult_scaled(Context &c, const EvalKeys &ek, const CtView &a, const CtView &b, double target);
// lazy relinearisation: sum_i tensor(a_i, b_i), one relinearisation and rescale -> 1 ciphertext
CtBatch mult_sum(Context &c, const EvalKeys &ek, const CtView &a, const CtView &b);
// Grouped Mult: group g multiplies as[g] (n cts) with bs[g] (n cts, or 1 broadcast);
// all groups at one level; one relinearisation and one rescale for the whole batch.
// Output: the groups' products concatenated (sum of the groups' sizes).
CtBatch mult_grouped(Context &c, const EvalKeys &ek, const std::vector<CtView> &as, const std::vector<CtView> &bs);
// Grouped lazy Mult: group g -> sum_i tensor(as[g]_i, bs[g]_i), then one relinearisation
// and rescale over all groups.  Output: one ciphertext per group.
CtBatch mult_sum_grouped(Context &c, const EvalKeys &ek, const std::vector<CtView> &as,
                         const std::vector<CtView> &bs);
// Grouped CMult: a has G*n cts (or n cts when `broadcast`, then every group reads a);
// group g is multiplied by pts[g]; one rescale; the result carries out_scale.
// group g: a_g (.) pa[g] + b_g (.) pb[g], one rescale (a_g = a if a has n ciphertexts, else
// its g-th n; the same for b); out_scale as for one product
CtBatch mul_plain2_rescale_grouped(Context &c, const CtView &a, const std::vector<const Plain *> &pa,
                                   const CtView &b, const std::vector<const Plain *> &pb, int n, double out_scale);
CtBatch mul_plain_rescale_grouped(Context &c, const CtView &a, const std::vector<const Plain *> &pts, int n,
                                  bool broadcast, double out_scale);
// Lrot by r (plain key switching), Conj
CtBatch rotate(Context &c, const EvalKeys &ek, const CtView &a, int r);
CtBatch conjugate(Context &c, const EvalKeys &ek, const CtView &a);
// y + Lrot(x, r) and y + Conj(x), the addition folded into the key switch
// (same bits as ct_add of the separate results).
CtBatch add_rotate(Context &c, const EvalKeys &ek, const CtView &y, const CtView &x, int r);
CtBatch add_conjugate(Context &c, const EvalKeys &ek, const CtView &y, const CtView &x);
// a + sum_r Lrot(a, r): one ModUp of a, the amounts' key inner products summed in
// the extended basis, one ModDown (amounts without a key: composed one at a time)
CtBatch rotate_sum(Context &c, const EvalKeys &ek, const CtView &a, const std::vector<int> &rs);
// hoisted: one ModUp of a, then one key inner product / ModDown per amount
std::vector<CtBatch> rotate_hoisted(Context &c, const EvalKeys &ek, const CtView &a, const std::vector<int> &rs);
// the same in two steps: extend the digits of `a` once, then rotate by any amounts
struct HoistedSource {
    CtView a;
    DBuf ext;
};
// Blocks [first, first + count) of a hoisted source with their extended digits
// (ext points at the first block's digit 0; digit j of block b at ext + j * digit_stride
// + (b - first) * (lv + 1 + K) * N).
struct HoistedView {
    CtView a;
    const u64 *ext = nullptr;
    size_t digit_stride = 0;
};
HoistedView hoisted_view(const Context &c, const HoistedSource &hs, int first, int count);
HoistedSource hoist_prepare(Context &c, const CtView &a);
CtBatch hoist_rotate(Context &c, const EvalKeys &ek, const HoistedSource &hs, int r);
// all amounts at once: [step][block] (S x a.n ciphertexts); amounts with their own
// key share one batched key inner product and ModDown, others are composed
CtBatch hoist_rotate_batch(Context &c, const EvalKeys &ek, const HoistedSource &hs, const std::vector<int> &rs);
CtBatch hoist_rotate_batch(Context &c, const EvalKeys &ek, const HoistedView &hv, const std::vector<int> &rs);
// the same, split into one batch per amount (sharing the memory)
std::vector<CtBatch> hoist_rotate_many(Context &c, const EvalKeys &ek, const HoistedSource &hs,
                                       const std::vector<int> &rs);

// key switching of a batch of polynomials d (lv+1 limbs, NTT domain):
// out0 = addend0 + ks0(d), out1 = addend1 + ks1(d)
void keyswitch(Context &c, PolyBatch d, const SwitchKey &key, int lv, PolyBatch out0, PolyBatch out1,
               PolyBatch addend0, PolyBatch addend1);

}  // namespace hetal
