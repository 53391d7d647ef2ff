/*
 * hetal.h -- C ABI of the GB300 (sm_103a) implementation of HETAL's
 * encrypted matrix products (Lee et al., "HETAL: Efficient Privacy-preserving
 * Transfer Learning with Homomorphic Encryption", arXiv 2403.14111) and of the
 * RNS-CKKS operations beneath them.
 *
 * Conventions
 *  - Every function returns 0 (HETAL_OK) or a negative status; the message of
 *    the last failure on a context is returned by hetal_last_error().  No call
 *    aborts the process.
 *  - Handles are created and owned by the library; the caller releases them
 *    with the matching *_free / *_destroy call.  Freeing NULL is a no-op.
 *  - Pointers named host_* are host memory; pointers named dev_* are device
 *    memory on the context's GPU.  All device work is ordered on the context's
 *    stream; calls that return data to the host synchronise that stream.
 *  - A ciphertext at level lv has lv+1 RNS limbs (moduli q_0..q_lv).  Exported
 *    and imported ciphertexts are coefficient-domain residues, laid out
 *    [block][component 0/1][limb 0..lv][coefficient 0..N-1], uint64, each
 *    value in [0, q_limb).
 *  - A matrix is block-encoded (Sec. 4.2.1 and App. B.1): zero-padded and cut
 *    into s0 x s1 blocks (s0*s1 = N/2 slots), block (r, j) row-major in one
 *    ciphertext; entry (i, j) of a block is slot i*s1 + j.  Blocks of a matrix
 *    are stored row-major (m block rows, n block columns).
 */
#ifndef HETAL_H
#define HETAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define HETAL_OK 0
#define HETAL_ERR_INVALID_ARG (-1) /* a NULL handle, size or range error */
#define HETAL_ERR_SHAPE (-2)       /* c not a power of two, c > min(s0, s1), s0*s1 != N/2, block grids differ */
#define HETAL_ERR_LEVEL (-3)       /* not enough levels left for the requested operation */
#define HETAL_ERR_MISSING_KEY (-4) /* a rotation / conjugation / relinearisation key was not generated */
#define HETAL_ERR_OOM (-5)         /* device memory exhausted */
#define HETAL_ERR_CUDA (-6)        /* a CUDA runtime error */
#define HETAL_ERR_SCALE (-7)       /* operands of an addition carry different scales */
#define HETAL_ERR_TIMEOUT (-8)     /* a bounded device wait ran out */
#define HETAL_ERR_RECORDING (-9)   /* a call that cannot be recorded into a graph, or a void recording */
#define HETAL_ERR_CANCELLED (-10)  /* a queued serving request was withdrawn (hetal_server_cancel) */

/* Tiling of a block-encoded matrix (Sec. 4.2.2: B-bar, Sec. 4.2.3: A-underbar). */
#define HETAL_TILE_NONE 0
#define HETAL_TILE_VERT 1  /* c x b matrix, s0/c copies stacked vertically (one block row)     */
#define HETAL_TILE_HORIZ 2 /* a x c matrix, s1/c copies side by side (one block column)        */

/* Algorithm variants (same mathematics, different rounding, hence different bits). */
#define HETAL_FLAG_HOIST 1      /* rotations of one ciphertext by several amounts share one ModUp     */
#define HETAL_FLAG_LAZY_RELIN 2 /* ciphertext products summed before one relinearisation and rescale */
/* SumCols / SumRows as steps x <- x + sum_{0<j<2^b} Lrot(x, j t) of up to 8 terms, each with one
 * ModUp and one ModDown (the paper's log-depth rotate-and-add computes the same sums); needs the
 * keys of the amounts j t (hetal_rotation_amounts lists them) */
#define HETAL_FLAG_RADIX_SUM 4
/* PRotUp(B, k) as B (.) D_k + RotUp(B, 1) (.) (1 - D_k) with one RotUp(B, 1) for every k, and
 * RotLeft(A, k) as Lrot(A, k) (.) D_k + Lrot(A, k - s1) (.) (1 - D_k) with both rotations of A hoisted
 * (the algorithms' values, since 1 - D_k is unchanged by a rotation by whole rows); each pair of plaintext
 * products is summed before one rescale */
#define HETAL_FLAG_SHARED_ROT 8

/* Kinds of plaintext the algorithms use (keys of a plaintext set). */
#define HETAL_PT_COLMASK 1   /* column-0 selector inside SumCols                         */
#define HETAL_PT_ABT_DIAG 2  /* t * M_cplx^{(k,c)}  (Prop. ABT)                           */
#define HETAL_PT_DMASK 3     /* D_k: 1 in columns j < s1 - k (Algorithms RotLeft, PRotUp) */
#define HETAL_PT_ATB_DIAG 4  /* t * M_cplx^{(-k,c)} (Prop. ATB)                           */
#define HETAL_PT_SM_COEF 5   /* coeff_i * valid, degree-15 softmax stand-in                */
#define HETAL_PT_SM_CONST 6  /* coeff_{4j} * valid, constant term of the j-th giant step   */
#define HETAL_PT_DMASK_C 7   /* 1 - D_k: 1 in columns j >= s1 - k (HETAL_FLAG_SHARED_ROT)   */

typedef struct hetal_ctx hetal_ctx;     /* parameters, device tables, stream                    */
typedef struct hetal_sk hetal_sk;       /* client secret key (never needed by server calls)     */
typedef struct hetal_evk hetal_evk;     /* evaluation keys: relinearisation, conjugation, rotations */
typedef struct hetal_mat hetal_mat;     /* block-encoded encrypted matrix                       */
typedef struct hetal_ptset hetal_ptset; /* caller-supplied integer plaintexts                    */
typedef struct hetal_plain hetal_plain; /* one plaintext kept on the device                      */
typedef struct hetal_graph hetal_graph; /* a CUDA graph of recorded calls                       */

/*
 * CKKS parameters (Sec. 2.2, Sec. 5.1: the paper uses N = 2^16 and log q ~ 1555
 * inside a closed library and gives nothing else).  Ring degree N = 2^log_n;
 * ciphertext primes: q_0 = the largest prime below 2^q0_bits that is 1 mod 2N,
 * then the n_rescale largest such primes below 2^rescale_bits, then (n_upper > 0)
 * the n_upper largest below 2^upper_bits; then n_special special primes below
 * 2^special_bits (all distinct, skipping primes already taken, each list
 * descending).  alpha primes per key-switching digit (alpha and n_special at most
 * 7); secret Hamming weight h; default scale.  HETAL_ERR_INVALID_ARG when a
 * count or size is out of range or too few primes exist.
 */
/* Most moduli (ciphertext primes plus special primes) a context holds. */
#define HETAL_MAX_MODULI_ABI 128

typedef struct hetal_params {
    int log_n;        /* 10..16 */
    int q0_bits;      /* 20..61 */
    int n_rescale;    /* top level = n_rescale + n_upper; 1 + n_rescale + n_upper + n_special <= HETAL_MAX_MODULI */
    int rescale_bits; /* 20..61 */
    int n_special;    /* >= 1 */
    int special_bits; /* 20..61 */
    int alpha;        /* 1..7 */
    int hamming_weight;
    double scale;
    int n_upper;      /* more ciphertext primes above the n_rescale ones (0: none), e.g. 60-bit    */
    int upper_bits;   /* levels for bootstrapping over a chain of smaller training primes; 36..61  */
} hetal_params;

/* Shape and state of an encrypted matrix. */
typedef struct hetal_mat_desc {
    int m, n;         /* block rows, block columns */
    int rows, cols;   /* logical size of the stored layout */
    int s0, s1;       /* block shape */
    int level;        /* current level (limbs - 1) */
    double scale;     /* scale the message carries */
} hetal_mat_desc;

/* Paper-level operation counts and primitive work since the last reset. */
typedef struct hetal_counters {
    long long cmult, mult, rot, conj;  /* as counted in Table "tab:matnum_fixed" (Conj separate) */
    long long keyswitch, modup_digits, ntt_limbs, rescale;
    double modmul;                     /* modular multiplies issued by the kernels */
} hetal_counters;

/* ---- context ------------------------------------------------------------- */
/* Creates a context on `device`; cuda_stream may be NULL (a private stream is made). */
int hetal_ctx_create(const hetal_params *params, int device, void *cuda_stream, hetal_ctx **out);
void hetal_ctx_destroy(hetal_ctx *ctx);
const char *hetal_last_error(const hetal_ctx *ctx);
/* Writes the L+K moduli (q_0..q_{L-1}, p_0..p_{K-1}) to host_out[0..cap); returns L+K or a status. */
int hetal_ctx_moduli(const hetal_ctx *ctx, uint64_t *host_out, int cap);
/* N, L (ciphertext primes), K (special primes). */
int hetal_ctx_info(const hetal_ctx *ctx, int *n, int *l, int *k);
int hetal_ctx_sync(hetal_ctx *ctx);
/*
 * Budget (bytes, >= 1 MiB) for the temporaries of one batched step: the matrix
 * products take their c/2 diagonals, and hoisted rotations their amounts, in
 * chunks whose intermediates stay near it (default 8 GiB).  A smaller budget uses
 * less device memory and launches more kernels; results are the same bits (every
 * ciphertext sees the same operations in the same order).  Not recordable.
 */
int hetal_ctx_set_batch_bytes(hetal_ctx *ctx, size_t bytes);
/*
 * Polynomials a CTA of the NTT's row passes transforms (1..64): with 1, each CTA
 * transforms 16 rows of one polynomial and reads their twiddles from L2; with g > 1,
 * a CTA stages its rows' twiddles in shared memory once and transforms those rows of
 * up to g polynomials of the same limb (lowered per launch so that the grid still
 * fills the GPU).  Same results either way.  Not recordable.
 */
int hetal_ctx_set_row_group(hetal_ctx *ctx, int polys);
int hetal_counters_get(const hetal_ctx *ctx, hetal_counters *out);
int hetal_counters_reset(hetal_ctx *ctx);

/* ---- keys (Sec. 2.3: the client keeps sk; the server holds evaluation keys) --- */
/*
 * Secret key from `seed`: ternary, Hamming weight h, drawn by a partial
 * Fisher-Yates shuffle from Philox4x64-10 (key (seed, stream)).
 */
int hetal_keygen(hetal_ctx *ctx, uint64_t seed, hetal_sk **sk_out);
/* Copies the secret's N signed coefficients to host_out. */
int hetal_sk_export(const hetal_sk *sk, int64_t *host_out);
void hetal_sk_free(hetal_sk *sk);
/*
 * Evaluation keys: one hybrid switching key per left-rotation amount in
 * rot_steps (negative = right rotation), plus conjugation and relinearisation
 * keys when asked.  Each key is [dnum][2][L+K][N] residues.
 */
int hetal_evk_create(hetal_ctx *ctx, const hetal_sk *sk, uint64_t seed, const int32_t *rot_steps, size_t n_steps,
                     int with_conj, int with_relin, hetal_evk **out);
/* Copies a key in coefficient domain to host_out ([dnum][2][L+K][N]); kind 0 relin, 1 conj, 2 rotation by step. */
int hetal_evk_export(hetal_ctx *ctx, const hetal_evk *evk, int kind, int32_t step, uint64_t *host_out);
void hetal_evk_free(hetal_evk *evk);

/* ---- encrypted matrices --------------------------------------------------- */
/*
 * Encodes (FP64 canonical embedding, Sec. 2.2) and encrypts a row-major rows x
 * cols host matrix as blocks of s0 x s1 at `level` with `scale`.  tiling
 * HETAL_TILE_VERT stores s0/tile_c vertical copies of a (rows <= tile_c) x cols
 * matrix; HETAL_TILE_HORIZ s1/tile_c horizontal copies of a rows x (cols <=
 * tile_c) matrix.  Block b uses the Philox nonce nonce + b.
 */
int hetal_encrypt(hetal_ctx *ctx, const hetal_sk *sk, uint64_t seed, uint64_t nonce, const double *host_m, int rows,
                  int cols, int s0, int s1, int tiling, int tile_c, int level, double scale, hetal_mat **out);
/*
 * Encrypts already-encoded integer plaintexts host_pt[b][N] (b < m*n) as a
 * matrix with the given desc (level, scale and shape fields are used).
 */
int hetal_encrypt_int(hetal_ctx *ctx, const hetal_sk *sk, uint64_t seed, uint64_t nonce, const int64_t *host_pt,
                      const hetal_mat_desc *desc, hetal_mat **out);
/* Decrypts and decodes every block: host_out[(r*s0 + i) * (n*s1) + (j*s1 + jj)], (m*s0) x (n*s1) doubles. */
int hetal_decrypt(hetal_ctx *ctx, const hetal_sk *sk, const hetal_mat *mat, double *host_out);
/* FP64 encode of host slot vectors (real, imaginary; imaginary may be NULL) of `count` blocks: host_out[count][N]. */
int hetal_encode(hetal_ctx *ctx, const double *host_re, const double *host_im, int count, double scale,
                 int64_t *host_out);
int hetal_mat_desc_get(const hetal_mat *mat, hetal_mat_desc *out);
/* Coefficient-domain residues, [m*n][2][level+1][N] uint64.  Import checks on the device
 * that every residue is below its limb's modulus (HETAL_ERR_INVALID_ARG otherwise, nothing
 * is created) and waits for the answer; a recorded import (graph) copies without the check. */
int hetal_mat_export(hetal_ctx *ctx, const hetal_mat *mat, uint64_t *host_out);
int hetal_mat_import(hetal_ctx *ctx, const uint64_t *host_in, const hetal_mat_desc *desc, hetal_mat **out);
/* Same as export / import, but the residue buffer is device memory on the context's GPU. */
int hetal_mat_export_dev(hetal_ctx *ctx, const hetal_mat *mat, uint64_t *dev_out);
int hetal_mat_import_dev(hetal_ctx *ctx, const uint64_t *dev_in, const hetal_mat_desc *desc, hetal_mat **out);
/* Keeps only the limbs 0..level (same message and scale). */
int hetal_mat_drop(hetal_ctx *ctx, const hetal_mat *in, int level, hetal_mat **out);
/*
 * Block copies, for moving ciphertexts between matrices (the packed refresh of the training
 * loop gathers the blocks of W and V into few ciphertexts and scatters them back).
 * slice: blocks [first, first + count) of `in`, in row-major block order, as a new matrix of
 *   one block row (desc 1 x count, rows s0, cols count * s1), at in's level and scale.
 *   HETAL_ERR_SHAPE if the range leaves in's blocks.
 * stack: the blocks of mats[0..count) in order as one new matrix with desc's block grid and
 *   shape (desc->m * desc->n must equal the total number of blocks, desc->s0 and s1 those
 *   of the inputs); desc's level and scale are ignored: every input must be at one level
 *   and one scale (HETAL_ERR_LEVEL, HETAL_ERR_SCALE otherwise), which the result keeps.
 * The inputs are not changed; the caller frees the result.
 */
int hetal_mat_slice(hetal_ctx *ctx, const hetal_mat *in, int first, int count, hetal_mat **out);
int hetal_mat_stack(hetal_ctx *ctx, const hetal_mat *const *mats, int count, const hetal_mat_desc *desc,
                    hetal_mat **out);
/*
 * Releases a matrix (its device memory is returned in order on the context's
 * stream).  A handle passed to any call after it was freed is refused with
 * HETAL_ERR_INVALID_ARG (a freed handle's marker is cleared), and freeing it again
 * does nothing, as long as its host memory has not been reused meanwhile.
 */
void hetal_mat_free(hetal_mat *mat);

/* ---- caller-supplied plaintexts ------------------------------------------- */
/*
 * A plaintext set maps (kind, index, level) to N signed integer coefficients.
 * Algorithms that receive a set take a plaintext from it whenever it holds the
 * key, and encode their own (FP64, on the device) otherwise.
 */
int hetal_ptset_create(hetal_ptset **out);
int hetal_ptset_put(hetal_ptset *set, int kind, int index, int level, const int64_t *host_coeffs, int n);
void hetal_ptset_free(hetal_ptset *set);

/* ---- server-side operations ----------------------------------------------- */
/* Lrot by step (negative: Rrot) of every block (Sec. 2.2). */
int hetal_rotate(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *in, int32_t step, hetal_mat **out);
/* Lrot of every block by each of steps[0..n) sharing one ModUp (hoisting); outs[i] receives step i. */
int hetal_rotate_hoisted(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *in, const int32_t *steps, size_t n,
                         hetal_mat **outs);
/*
 * in + sum_i Lrot(in, steps[i]) for every block, with one ModUp of in, the
 * amounts' key inner products summed in the extended basis and one ModDown
 * (at most 64 amounts, each with its key; amounts without a key are composed and
 * added one at a time).  The building block of HETAL_FLAG_RADIX_SUM.
 */
int hetal_rotate_sum(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *in, const int32_t *steps, size_t n,
                     hetal_mat **out);
int hetal_conj(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *in, hetal_mat **out);
/* Blockwise Mult (tensor, relinearisation, rescale); b may have a single block (broadcast). */
int hetal_mult(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *a, const hetal_mat *b, hetal_mat **out);
/* Blockwise CMult by the FP64 slot vector host_slots (N/2 values, same for every block), rescaled. */
int hetal_cmult(hetal_ctx *ctx, const hetal_mat *a, const double *host_re, const double *host_im, hetal_mat **out);
/*
 * CMult by the constant `value` in every slot, landing on exactly out_scale: every block
 * times the integer constant round(value * out_scale * q_lv / scale(a)) (half away from
 * zero; q_lv the modulus of a's top limb), then rescaled by q_lv; one level.  With
 * out_scale = scale(a) it keeps the scale; with value 1 it moves a ciphertext to a given
 * scale (additions need equal scales).  HETAL_ERR_INVALID_ARG if the constant exceeds 63 bits.
 */
int hetal_mul_const(hetal_ctx *ctx, const hetal_mat *a, double value, double out_scale, hetal_mat **out);
/*
 * A copy of `a` read at `scale`: the residues are the same, the message becomes
 * scale(a) / scale times the old one.  Used to add two ciphertexts whose scales
 * differ by the rounding of hetal_mult_scaled's integer factor (the addition
 * itself allows a relative difference of 1e-9), and to read a bootstrapped
 * ciphertext at its message's scale.  HETAL_ERR_SCALE unless scale is positive
 * and finite.
 */
int hetal_mat_set_scale(hetal_ctx *ctx, const hetal_mat *a, double scale, hetal_mat **out);
/*
 * ModRaise (bootstrapping's first step, Sec. 2.2): a level-0 matrix as one at
 * `level` (1 <= level < L), every residue mod q_0 centred into (-q_0/2, q_0/2] and
 * reduced modulo q_0..q_level.  Each block then decrypts, over the integers, to
 * t = Delta m + e + q_0 I with a small integer polynomial I; the result carries the
 * scale q_0 (its slots are sigma(t) / q_0).  HETAL_ERR_LEVEL unless a is at level 0.
 */
int hetal_mod_raise(hetal_ctx *ctx, const hetal_mat *a, int level, hetal_mat **out);
/* Every block times sqrt(-1) in every slot (X^(N/2) in the ring, no level, no key). */
int hetal_mul_i(hetal_ctx *ctx, const hetal_mat *a, hetal_mat **out);
/*
 * Every block times the integer t (t != 0, t > -2^63): the message is multiplied
 * by t, the level and scale are unchanged (no rescale).
 */
int hetal_mul_int(hetal_ctx *ctx, const hetal_mat *a, int64_t t, hetal_mat **out);
/*
 * Mult (tensor, relinearisation, rescale by q_lv, one level) landing on a given
 * scale: a is first multiplied by the integer t = round(target_scale * q_lv /
 * (scale(a) * scale(b))) (half away from zero; q_lv the top modulus after the two
 * are brought to one level), and the result carries scale(a) * t * scale(b) / q_lv,
 * within a factor 1 +- 1/(2t) of target_scale.  Keeps the scale from drifting along
 * a deep circuit (Algorithm ASoftmax's squaring chains) when the primes are not
 * equal to the scale.  HETAL_ERR_INVALID_ARG unless 1 <= t < 2^62.
 */
int hetal_mult_scaled(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *a, const hetal_mat *b,
                      double target_scale, hetal_mat **out);
/*
 * CMult by the caller's integer plaintext host_pt[N] (the same for every block),
 * then the rescale by q_lv (one level).  The caller encoded it for the product to
 * carry out_scale, i.e. at scale out_scale * q_lv / scale(a); the result is given
 * that scale.  The plaintext is reduced modulo every prime of a's level.
 */
int hetal_cmult_int(hetal_ctx *ctx, const hetal_mat *a, const int64_t *host_pt, double out_scale, hetal_mat **out);
/*
 * A plaintext kept on the device: the caller's integer coefficients host_pt[N]
 * reduced modulo q_0..q_level and transformed once (NTT domain, normal and
 * Montgomery form), for products and additions that take no host copy and no
 * transform per use (and can be recorded into a graph).  `scale` is the scale it
 * was encoded at (bookkeeping).  Free with hetal_plain_free before the context.
 */
int hetal_plain_create(hetal_ctx *ctx, const int64_t *host_pt, int level, double scale, hetal_plain **out);
void hetal_plain_free(hetal_plain *pt);
/* hetal_cmult_int with a device plaintext (its level at least a's); the result carries out_scale. */
int hetal_cmult_plain(hetal_ctx *ctx, const hetal_mat *a, const hetal_plain *pt, double out_scale, hetal_mat **out);
/*
 * sum_i as[i] (.) pts[i], then one rescale by q_lv (one level): as[0..count) at one
 * level, block count and scale, each device plaintext encoded for the sum to carry
 * out_scale (at out_scale * q_lv / scale(as[0])).  The products are accumulated in
 * 128 bits and reduced before the single rescale, so the result differs in its
 * rounding from adding separately rescaled products.
 */
int hetal_cmult_plain_sum(hetal_ctx *ctx, const hetal_mat *const *as, const hetal_plain *const *pts, int count,
                          double out_scale, hetal_mat **out);
/* hetal_add_plain_int with a device plaintext (encoded at scale(a), its level at least a's). */
int hetal_add_plain(hetal_ctx *ctx, const hetal_mat *a, const hetal_plain *pt, hetal_mat **out);
/* Adds the caller's integer plaintext host_pt[N] (encoded at scale(a)) to every block; no level. */
int hetal_add_plain_int(hetal_ctx *ctx, const hetal_mat *a, const int64_t *host_pt, hetal_mat **out);
int hetal_add(hetal_ctx *ctx, const hetal_mat *a, const hetal_mat *b, hetal_mat **out);
int hetal_sub(hetal_ctx *ctx, const hetal_mat *a, const hetal_mat *b, hetal_mat **out);
int hetal_rescale(hetal_ctx *ctx, const hetal_mat *a, hetal_mat **out);

/*
 * DiagABT (Algorithm DiagABT, App. B.3; Prop. ABT, Sec. 4.2.2):
 * out = <t A Bbar^T>, A given as m x n blocks, Bbar (c x b, tiled vertically)
 * as 1 x n blocks; c a power of two with 2 <= c <= min(s0, s1).  Output: m
 * blocks holding t*A*B^T tiled s1/c times horizontally, three levels below
 * min(level(A), level(Bbar)).  Needs rotation keys for k*s1 (1 <= k <= c/2),
 * 2^u and -2^u (u < log2 s1), conjugation and relinearisation keys.
 */
int hetal_diag_abt(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *a, const hetal_mat *bbar, int c, double t,
                   const hetal_ptset *pts, int flags, hetal_mat **out);
/*
 * DiagATB (Algorithm DiagATB, App. B.3; Prop. ATB, Sec. 4.2.3):
 * out = <t A^T B>, A-underbar (a x c tiled horizontally) as m x 1 blocks, B as
 * m x n blocks.  Takes the PRotUp branch when level(A) < level(B), else the
 * RotLeft branch.  Output: n blocks holding t*A^T*B tiled s0/c times
 * vertically (the layout of Bbar).  Needs rotation keys for k (1 <= k <= c/2),
 * -s1, s1, 2^u * s1 (u < log2 s0), conjugation and relinearisation keys.
 */
int hetal_diag_atb(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *a_under, const hetal_mat *b, int c,
                   double t, const hetal_ptset *pts, int flags, hetal_mat **out);
/*
 * The left-rotation amounts (in [1, N/2), right rotations as N/2 - r) whose keys
 * DiagABT and DiagATB use for blocks s0 x s1, c classes and `flags` (RotUp,
 * SumCols, SumRows, RotLeft, PRotUp; with HETAL_FLAG_RADIX_SUM the radix steps'
 * amounts).  Writes at most cap amounts, ascending, to out (host memory) and
 * returns how many there are (so a call with cap 0 sizes the buffer), or
 * HETAL_ERR_SHAPE for an invalid shape (c a power of two, 2 <= c <= min(s0, s1)).
 */
int hetal_rotation_amounts(int s0, int s1, int c, int flags, int32_t *out, size_t cap);
/*
 * Softmax stand-in of the encrypted training step (not the paper's ASoftmax,
 * App. A): elementwise sum_{i<16} coeffs[i] x^i times the 0/1 slot mask
 * host_valid (N/2 values), baby-step giant-step, depth 5, result at
 * target_scale.
 */
int hetal_softmax_approx(hetal_ctx *ctx, const hetal_evk *evk, const hetal_mat *m, const double *coeffs16,
                         const double *host_valid, double target_scale, const hetal_ptset *pts, hetal_mat **out);

/* ---- many independent instances (batching) --------------------------------- */
/*
 * One DiagABT + DiagATB instance: out_abt = <t_abt x wbar^T> (hetal_diag_abt),
 * out_atb = <t_atb a_under^T b> (hetal_diag_atb), with the same c.
 */
typedef struct hetal_pair_job {
    const hetal_mat *x, *wbar, *a_under, *b;
    int c;
    double t_abt, t_atb;
    int flags;   /* HETAL_FLAG_* of this instance, or -1 for the call's flags */
} hetal_pair_job;
/*
 * Runs n independent instances.  workers == 1: one after another on the
 * context's stream.  workers > 1: on that many worker contexts of the same
 * device, each with its own CUDA stream, instances handed to whichever worker is
 * free, so that their kernels overlap on the GPU; the results are the same bits
 * as with workers == 1.  Returns when every result is complete.  Worker contexts
 * are kept by `ctx` until hetal_ctx_destroy.  The results belong to `ctx` (their
 * memory is released in order on its stream), whatever worker made them.
 * Evaluation keys must hold every rotation the instances' shapes need.
 */
int hetal_run_pairs(hetal_ctx *ctx, const hetal_evk *evk, const hetal_pair_job *jobs, size_t n, int workers,
                    int flags, hetal_mat **out_abt, hetal_mat **out_atb);
/*
 * The same instances run batched across instances: instances are grouped by block
 * shape, flags, the levels and scales of their inputs (and, for DiagATB's RotLeft
 * branch, c = 2 apart from larger c), groups are cut so that their temporaries stay
 * near the context's batch budget (hetal_ctx_set_batch_bytes), and every primitive of a group runs as one
 * launch over all its instances' ciphertexts (at diagonal k, those with k < c/2):
 * hoisted rotations, key inner products, ModDown, tensor products, SumCols and
 * SumRows, and work-list kernels for the per-instance masks and sums.  Each
 * ciphertext sees the operations it sees alone, so every result has the bits of
 * hetal_run_pairs / hetal_diag_abt / hetal_diag_atb.  Runs on the context's stream
 * without waiting for it, so a fixed batch can be recorded into a graph (after one
 * eager run, which encodes the masks).
 */
int hetal_run_pairs_batched(hetal_ctx *ctx, const hetal_evk *evk, const hetal_pair_job *jobs, size_t n, int flags,
                            hetal_mat **out_abt, hetal_mat **out_atb);
/*
 * Block shape for an instance with an a x b matrix and c classes: s0 (a power of
 * two, s1 = N/(2 s0), c <= min(s0, s1)) minimising a cost model of DiagABT +
 * DiagATB whose key-switching times per level are measured on the device by the
 * first call (it times rotations with the first rotation key of evk).
 */
int hetal_tile_choose(hetal_ctx *ctx, const hetal_evk *evk, int a, int b, int c, int *s0_out);
/*
 * Tile and variant for the same instance: s0 and the flags (HETAL_FLAG_HOIST |
 * HETAL_FLAG_LAZY_RELIN, with HETAL_FLAG_RADIX_SUM and / or HETAL_FLAG_SHARED_ROT
 * where the cost model says they pay) minimising the model, whose per-level costs of a
 * rotation and of one more summed amount are measured on the device by the first call
 * (rotations with the first rotation key of evk).  The keys the chosen variant needs
 * are hetal_rotation_amounts(s0, N/(2 s0), c, flags).
 */
int hetal_plan_choose(hetal_ctx *ctx, const hetal_evk *evk, int a, int b, int c, int *s0_out, int *flags_out);

/* ---- serving (continuous batching of encrypted-matmul requests) ------------ */
/*
 * A request loop on one device: `slots` worker threads, each with its own CUDA
 * stream, and a scheduler that admits requests in arrival order whenever a slot
 * is free and the request's estimated device footprint fits `budget_bytes`
 * beside the clients' resident keys and the requests in flight.  Requests that
 * arrive while others run are admitted as slots and memory free up, and run
 * concurrently with them.  Results do not depend on what else is running.
 * A request whose estimated footprint alone exceeds the budget left beside the
 * resident keys is refused at submission (HETAL_ERR_OOM).  A collected result
 * belongs to the server's context (released in order on its stream) and may
 * outlive the server.  Destroy the server before its context.
 */
typedef struct hetal_server hetal_server;
typedef struct hetal_request {
    int client;                  /* id from hetal_server_add_client */
    int kind;                    /* 0: DiagABT(a, b = B-bar), 1: DiagATB(a = A-underbar, b = B) */
    const hetal_mat *a, *b;      /* operands on the device; keep them until the result is collected */
    int c;
    double t;
    int flags;
} hetal_request;
int hetal_server_create(hetal_ctx *ctx, int slots, size_t budget_bytes, hetal_server **out);
void hetal_server_destroy(hetal_server *srv);
/* Registers a client's evaluation keys (kept by the caller, resident on the device; their bytes count
 * against the budget).  Rotations without their own key are composed from the +-2^u keys present. */
int hetal_server_add_client(hetal_server *srv, const hetal_evk *evk, int *client_id);
/* Queues a request; returns at once with a ticket (HETAL_ERR_OOM: it can never fit the budget). */
int hetal_server_submit(hetal_server *srv, const hetal_request *req, uint64_t *ticket);
/* Blocks until the ticket's result is ready; reports its time in the queue and running (ms).
 * A cancelled ticket returns HETAL_ERR_CANCELLED. */
int hetal_server_wait(hetal_server *srv, uint64_t ticket, hetal_mat **out, double *queue_ms, double *run_ms);
/* Withdraws a request that is still queued (not yet admitted to a slot): it will not run,
 * and hetal_server_wait on its ticket returns HETAL_ERR_CANCELLED.  HETAL_ERR_INVALID_ARG if
 * the ticket is unknown, already running, finished or collected. */
int hetal_server_cancel(hetal_server *srv, uint64_t ticket);
int hetal_server_stats(const hetal_server *srv, long long *completed, size_t *resident_bytes,
                       size_t *peak_inflight_bytes);

/* ---- raw primitives on device buffers (for measurement and tests) --------- */
/*
 * In-place forward (inverse) negacyclic NTT of dev_polys[p][limb][N] for p <
 * n_polys, limb < n_limbs, limb l using modulus l.  Forward output is in
 * bit-reversed order; the inverse expects that order.
 */
int hetal_ntt_forward(hetal_ctx *ctx, uint64_t *dev_polys, int n_polys, int n_limbs);
int hetal_ntt_inverse(hetal_ctx *ctx, uint64_t *dev_polys, int n_polys, int n_limbs);
/* Primitive 2N-th root of unity the NTT of modulus `limb` uses. */
int hetal_ntt_root(const hetal_ctx *ctx, int limb, uint64_t *out);

/* ---- 32-bit words, for the choice of the RNS word size (no counterpart in the paper) --- */
/*
 * The library computes on 64-bit words.  The alternative, 32-bit words with primes
 * below 2^30 (about twice the limbs for a modulus of the same size, each product far
 * cheaper), has its transform here so that the two can be measured side by side.
 * hetal_ntt32_moduli: the first n_limbs primes below 2^30 that are 1 mod 2N, descending,
 * to host_moduli, and their primitive 2N-th roots to host_roots (may be NULL); makes the
 * transform's tables for n_limbs (1..64) limbs.
 * hetal_ntt32_forward: in-place forward negacyclic NTT of dev_polys[p][limb][N] (uint32,
 * values below the limb's prime, limb l modulo prime l), output in bit-reversed order
 * (slot j holds a(psi^{2 brv(j) + 1})), the same transform as hetal_ntt_forward.
 * hetal_probe_butterfly32_rate: the rate of its lazy butterfly in a register-only loop
 * over every SM (iters >= 10).
 */
int hetal_ntt32_moduli(hetal_ctx *ctx, int n_limbs, uint32_t *host_moduli, uint32_t *host_roots);
int hetal_ntt32_forward(hetal_ctx *ctx, uint32_t *dev_polys, int n_polys, int n_limbs);
int hetal_probe_butterfly32_rate(hetal_ctx *ctx, int iters, double *butterflies_per_s);

/* ---- CUDA graphs of recorded calls (no counterpart in the paper) ---------- */
/*
 * A fixed sequence of calls (a training step, one request shape) can be recorded
 * once and replayed with one launch, which removes the host's per-kernel work.
 * hetal_graph_begin opens a recording on ctx's stream: the calls that follow are
 * captured instead of run.  Recordable: the server-side operations (rotate*,
 * conj, mult, add, sub, rescale, mat_drop, diag_abt, diag_atb, softmax_approx),
 * mat_import / mat_export from / to pinned host memory (the graph copies at every
 * launch), mat_import_dev / mat_export_dev, the raw NTTs, hetal_rescale_noalloc
 * and hetal_mat_free.
 * Every other call that touches the device returns HETAL_ERR_RECORDING before
 * any device work.  Plaintexts the library encodes itself (masks, softmax
 * coefficients) must already be cached, i.e. the same sequence ran once before;
 * calls given a caller's plaintext set (pts not NULL) cannot be recorded.
 * A call that fails while recording voids the recording.
 * hetal_graph_end closes the recording, instantiates the graph and launches it
 * once, so that the matrices created while recording hold their results as
 * without a graph; each hetal_graph_launch recomputes them in place (same device
 * memory) from the current contents of the inputs.  Matrices and keys used by the
 * graph must outlive it; releasing a handle made before the recording while it
 * is open is deferred until hetal_graph_free.  On a void recording, *out is NULL,
 * the matrices created meanwhile are empty and HETAL_ERR_RECORDING is returned.
 * Launches run asynchronously on ctx's stream (hetal_ctx_sync waits).  Free
 * every graph (hetal_graph_free) before its context.
 */
int hetal_graph_begin(hetal_ctx *ctx);
int hetal_graph_end(hetal_ctx *ctx, hetal_graph **out);
int hetal_graph_launch(hetal_ctx *ctx, hetal_graph *graph);
/* Kernels one launch of the graph runs (counted by hetal_launch_count too). */
int hetal_graph_kernels(const hetal_graph *graph, long long *out);
void hetal_graph_free(hetal_graph *graph);

/* ---- measurement hooks (no counterpart in the paper) ----------------------- */
/*
 * Times every later launch of the kernel named kernel_name (e.g. "ntt_fwd_rows",
 * "kip", "modup_conv") with CUDA events on the context's stream; NULL or ""
 * stops timing.  Clears earlier records.
 */
int hetal_profile_kernel(hetal_ctx *ctx, const char *kernel_name);
/* Launches timed so far, their summed device time (ms), and their algorithmic
 * modular multiplies and bytes (as the launch wrappers count them). */
int hetal_profile_read(hetal_ctx *ctx, long long *launches, double *total_ms, double *modmul, double *bytes);
/* With kernel_name "*" every launch is timed; this writes one line per kernel
 * name, "name<TAB>launches<TAB>ms<TAB>modmul<TAB>bytes", NUL-terminated, into buf. */
int hetal_profile_summary(hetal_ctx *ctx, char *buf, size_t cap);
/* Number of kernels the library has launched on this context. */
int hetal_launch_count(const hetal_ctx *ctx, long long *out);
/* Number of device allocations the library has made on this context. */
int hetal_alloc_count(const hetal_ctx *ctx, long long *out);
/* Rate of the NTT's lazy butterfly (one Shoup product, two additions) in a
 * register-only loop over every SM: the ALU ceiling of the NTT kernels. */
int hetal_probe_butterfly_rate(hetal_ctx *ctx, int iters, double *butterflies_per_s);
/* Rate of the 64 x 64 -> 128-bit multiply-accumulate that the key inner product
 * and the base conversion issue per modular product (REDC deferred), in the same
 * register-only form: with the butterfly's rate it weighs a kernel that issues
 * both kinds of product.  iters >= 10; HETAL_ERR_INVALID_ARG otherwise. */
int hetal_probe_mac_rate(hetal_ctx *ctx, int iters, double *products_per_s);

/* ---- rescale without device allocation (the paper has no counterpart) ------ */
/*
 * For callers that may not let the library allocate device memory once they
 * run (a server that fixes its device-memory budget at start-up, an
 * application that owns every device buffer and lends pointers): rescales
 * n_ct ciphertexts from `level` to level-1, the same result as hetal_rescale.
 * dev_in:  [n_ct][2][level+1][N] uint64, NTT domain (as hetal_ntt_forward leaves it);
 * dev_out: [n_ct][2][level][N] uint64, NTT domain; an output overlapping dev_in
 * returns HETAL_ERR_INVALID_ARG before any device work.
 * Intermediate limbs use one static device array of 2^21 words (16 MiB) that
 * every GPU loading the library holds until exit; 2*n_ct*N*(level+1) above 2^21
 * returns HETAL_ERR_INVALID_ARG before any device work.  No cudaMalloc, cudaFree
 * or other allocating call is made (with kernel timing off, the default;
 * hetal_alloc_count does not move).  The array's device address is looked up when
 * a context is created on the device (hetal_ctx_create), never inside a call.
 * All calls share the array and it keeps the last call's contents (nothing in it
 * needs to start at zero), so calls that overlap on the GPU race: issue them on
 * one stream or serialise them.
 */
int hetal_rescale_noalloc(hetal_ctx *ctx, const uint64_t *dev_in, uint64_t *dev_out, int n_ct, int level);

#ifdef __cplusplus
}
#endif

#endif /* HETAL_H */
