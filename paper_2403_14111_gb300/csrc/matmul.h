// matmul.h -- HETAL's encrypted matrix products on the device.
#pragma once
#include "ckks.h"

namespace hetal {

// Kinds of plaintext the algorithms multiply or add (also the keys of PtSet).
enum PtKind {
    PT_COLMASK = 1,   // column-0 selector inside SumCols
    PT_ABT_DIAG = 2,  // t * M_cplx^{(k,c)}
    PT_DMASK = 3,     // D_k: columns j < s1 - k
    PT_ATB_DIAG = 4,  // t * M_cplx^{(-k,c)}
    PT_SM_COEF = 5,   // c_i * valid   (softmax stand-in, term i)
    PT_SM_CONST = 6,  // c_{4j} * valid (softmax stand-in, constant of u_j)
    PT_DMASK_C = 7,   // 1 - D_k: columns j >= s1 - k
};

enum Flags {
    FLAG_HOIST = 1,       // rotations of one source by several amounts share one ModUp
    FLAG_LAZY_RELIN = 2,  // products summed before one relinearisation / rescale
    FLAG_RADIX_SUM = 4,   // SumCols / SumRows in radix steps, one ModUp and one ModDown per step
    FLAG_SHARED_ROT = 8,  // PRotUp with one RotUp(B, 1) for every k; RotLeft from two hoisted rotations of A
};

// A block-encoded encrypted matrix: m x n ciphertexts stored row-major in cts.
struct Mat {
    CtBatch cts;
    int m = 0, n = 0;
    int rows = 0, cols = 0;
    int s0 = 0, s1 = 0;
};

// Supplies the plaintexts an algorithm needs: from the caller's PtSet when it
// holds the key, else encoded on the device; cached for the call.
class PtProvider {
  public:
    PtProvider(Context &c, const PtSet *set) : c_(c), set_(set) {}
    const Plain &mask(int kind, int k, int lv, double scale, int cc, int s0, int s1, double t);
    const Plain &scaled_vec(int kind, int k, int lv, double scale, const double *d_vec, double coeff, u64 vec_hash);

  private:
    const Plain *lookup(int kind, int k, int lv, double scale);
    Context &c_;
    const PtSet *set_;
    std::map<std::tuple<int, int, int>, Plain> cache_;
};

Mat diag_abt(Context &c, const EvalKeys &ek, const Mat &A, const Mat &Bbar, int cc, double t, const PtSet *pts,
             int flags);
// Many instances of one block shape whose inputs share their levels and scales, run
// together: every primitive is one batched launch over all their ciphertexts (the
// instances still active at diagonal k -- k < c/2 -- in one batch), so that launches
// and the rotation keys' reads are shared.  Each ciphertext sees the operations it
// sees alone, so every result has the bits of the one-instance call.  Outputs are in
// the order of the jobs.
struct AbtJob {
    const Mat *A, *Bbar;
    int cc;
    double t;
};
std::vector<Mat> diag_abt_group(Context &c, const EvalKeys &ek, const std::vector<AbtJob> &jobs, const PtSet *pts,
                                int flags);
struct AtbJob {
    const Mat *Au, *B;
    int cc;
    double t;
};
// The same for DiagATB; the products of every instance must come out at one level (with
// RotLeft, c = 2 and larger c take them at different levels: separate groups).
std::vector<Mat> diag_atb_group(Context &c, const EvalKeys &ek, const std::vector<AtbJob> &jobs, const PtSet *pts,
                                int flags);
Mat diag_atb(Context &c, const EvalKeys &ek, const Mat &Au, const Mat &B, int cc, double t, const PtSet *pts,
             int flags);
// left-rotation amounts whose keys DiagABT / DiagATB use (ascending, in [1, s))
std::vector<int> rotation_amounts(int s0, int s1, int cc, int flags);
// sum_{i<16} coeffs[i] x^i (.) valid, depth 5, landing on target_scale
Mat softmax_poly(Context &c, const EvalKeys &ek, const Mat &X, const double *coeffs, const double *d_valid,
                 u64 valid_hash, double target_scale, const PtSet *pts);

}  // namespace hetal
