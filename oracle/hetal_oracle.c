/*
 * hetal_oracle.c -- plain, slow CPU reference for the RNS-CKKS ring arithmetic
 * underneath HETAL's encrypted matrix products (arXiv 2403.14111).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * Everything here works on polynomials in the COEFFICIENT domain, one residue
 * vector per RNS modulus, values in [0, m).  Products use the textbook
 * definition (u128 product, then %).  Polynomial products mod X^N+1 go through
 * a textbook radix-2 number-theoretic transform, which the test-suite pins
 * against schoolbook negacyclic convolution.
 *
 * The paper (Sec. 2.2, Sec. 5.1) runs CKKS inside a closed library and does
 * not spell out the RNS variant; the definitions below are the standard
 * RNS-CKKS ones with hybrid key switching, and every choice that fixes bits
 * (rounding of rescale, fast base conversion without correction, the order in
 * which a sampler consumes random words) is written out where it is made.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef uint64_t u64;
typedef unsigned __int128 u128;
typedef int64_t i64;

/* ------------------------------------------------------------------------ */
/* Work split over independent limbs.  A loop whose iterations touch disjoint */
/* outputs (one RNS limb each) runs its iterations on several POSIX threads: */
/* thread k takes iterations k, k+T, k+2T, ...  Each iteration computes       */
/* exactly what the sequential loop computes, so results do not depend on T. */
/* ------------------------------------------------------------------------ */
#define ORC_MAX_THREADS 256
static int g_threads = 0;   /* 0: the number of online processors */

/* Sets the number of threads (1 = sequential); returns the number in use. */
int orc_set_threads(int n)
{
    g_threads = n < 0 ? 0 : (n > ORC_MAX_THREADS ? ORC_MAX_THREADS : n);
    return g_threads;
}

int orc_get_threads(void)
{
    if (g_threads > 0) return g_threads;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c < 1 ? 1 : (c > ORC_MAX_THREADS ? ORC_MAX_THREADS : (int)c);
}

typedef void (*orc_body)(void *arg, int i);
typedef struct {
    orc_body fn;
    void *arg;
    int first, n, step;
} orc_share;

static void *orc_run_share(void *v)
{
    orc_share *s = (orc_share *)v;
    for (int i = s->first; i < s->n; i += s->step) s->fn(s->arg, i);
    return NULL;
}

static void orc_parallel_for(int n, orc_body fn, void *arg)
{
    int T = orc_get_threads();
    if (T > n) T = n;
    if (T <= 1) {
        for (int i = 0; i < n; i++) fn(arg, i);
        return;
    }
    pthread_t th[ORC_MAX_THREADS];
    int started[ORC_MAX_THREADS];
    orc_share sh[ORC_MAX_THREADS];
    for (int k = 0; k < T; k++) {
        sh[k].fn = fn;
        sh[k].arg = arg;
        sh[k].first = k;
        sh[k].n = n;
        sh[k].step = T;
    }
    for (int k = 1; k < T; k++) started[k] = pthread_create(&th[k], NULL, orc_run_share, &sh[k]) == 0;
    orc_run_share(&sh[0]);
    for (int k = 1; k < T; k++) {
        if (started[k]) pthread_join(th[k], NULL);
        else orc_run_share(&sh[k]);   /* no thread could be made: run its share here */
    }
}

/* ------------------------------------------------------------------------ */
/* Modular arithmetic, by definition.                                        */
/* ------------------------------------------------------------------------ */
static u64 mmul(u64 a, u64 b, u64 m) { return (u64)(((u128)a * b) % m); }
static u64 madd(u64 a, u64 b, u64 m) { u128 s = (u128)a + b; return (u64)(s % m); }
static u64 msub(u64 a, u64 b, u64 m) { return a >= b ? a - b : (u64)((u128)a + m - b); }
static u64 mpow(u64 a, u64 e, u64 m)
{
    u64 r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = mmul(r, a, m);
        a = mmul(a, a, m);
        e >>= 1;
    }
    return r;
}
/* Inverse modulo a prime by Fermat's little theorem. */
static u64 minv(u64 a, u64 m) { return mpow(a % m, m - 2, m); }
/* Residue of a signed integer. */
static u64 mred_signed(i64 v, u64 m)
{
    if (v >= 0) return (u64)v % m;
    u64 r = (u64)(-(v + 1)) % m;       /* -(v+1) >= 0, avoids overflow at INT64_MIN */
    r = (r + 1) % m;                    /* |v| mod m */
    return r == 0 ? 0 : m - r;
}

u64 orc_mulmod(u64 a, u64 b, u64 m) { return mmul(a, b, m); }
u64 orc_powmod(u64 a, u64 e, u64 m) { return mpow(a, e, m); }

/* Deterministic Miller-Rabin: the first twelve primes as bases decide every n < 2^64. */
int orc_is_prime(u64 n)
{
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; r++; }
    for (int i = 0; i < 12; i++) {
        u64 x = mpow(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int k = 1; k < r; k++) {
            x = mmul(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/*
 * The `count` largest primes p < 2^bits with p = 1 (mod step), in descending
 * order.  An NTT of length N needs step a multiple of 2N; the parameter sets
 * use step = 2^32 (see prime_chain in ckks.py).  The paper gives only N = 2^16
 * and log q ~ 1555 (Sec. 5.1).  Returns the number of primes written.
 */
int orc_gen_primes(u64 step, int bits, int count, u64 *out)
{
    u64 top = (bits >= 64) ? ~(u64)0 : (((u64)1 << bits) - 1);
    u64 p = top - ((top - 1) % step);  /* largest value <= top with p = 1 mod step */
    int found = 0;
    while (found < count && p > step) {
        if (orc_is_prime(p)) out[found++] = p;
        p -= step;
    }
    return found;
}

/* A primitive 2N-th root of unity mod q (psi^N = -1). */
u64 orc_find_psi(u64 q, u64 two_n)
{
    for (u64 x = 2; x < q; x++) {
        u64 psi = mpow(x, (q - 1) / two_n, q);
        if (mpow(psi, two_n / 2, q) == q - 1) return psi;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Textbook NTT: cyclic radix-2 Cooley-Tukey with an explicit bit-reversal    */
/* permutation, used through a psi-twist for negacyclic products.            */
/* ------------------------------------------------------------------------ */
static void bitrev_permute(u64 *a, int n)
{
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { u64 t = a[i]; a[i] = a[j]; a[j] = t; }
    }
}

/* In place: A_k = sum_i a_i w^{ik} for a primitive n-th root w. */
static void dft_cyclic(u64 *a, int n, u64 w, u64 q)
{
    bitrev_permute(a, n);
    for (int len = 2; len <= n; len <<= 1) {
        u64 wl = mpow(w, (u64)(n / len), q);
        for (int i = 0; i < n; i += len) {
            u64 x = 1;
            for (int j = 0; j < len / 2; j++) {
                u64 u = a[i + j];
                u64 v = mmul(a[i + j + len / 2], x, q);
                a[i + j] = madd(u, v, q);
                a[i + j + len / 2] = msub(u, v, q);
                x = mmul(x, wl, q);
            }
        }
    }
}

/* Forward negacyclic transform: twist by psi^i, then cyclic DFT with psi^2. */
void orc_ntt_fwd(u64 *a, int n, u64 q, u64 psi)
{
    u64 t = 1;
    for (int i = 0; i < n; i++) { a[i] = mmul(a[i], t, q); t = mmul(t, psi, q); }
    dft_cyclic(a, n, mmul(psi, psi, q), q);
}

/* Inverse of orc_ntt_fwd. */
void orc_ntt_inv(u64 *a, int n, u64 q, u64 psi)
{
    u64 psi_inv = minv(psi, q);
    dft_cyclic(a, n, mmul(psi_inv, psi_inv, q), q);
    u64 n_inv = minv((u64)n, q);
    u64 t = n_inv;
    for (int i = 0; i < n; i++) { a[i] = mmul(a[i], t, q); t = mmul(t, psi_inv, q); }
}

/* out = a * b mod (X^n + 1, q), by definition (O(n^2)); the pin for the NTT. */
void orc_polymul_schoolbook(const u64 *a, const u64 *b, u64 *out, int n, u64 q)
{
    memset(out, 0, sizeof(u64) * (size_t)n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            u64 p = mmul(a[i], b[j], q);
            int k = i + j;
            if (k < n) out[k] = madd(out[k], p, q);
            else out[k - n] = msub(out[k - n], p, q);
        }
}

/* out = a * b mod (X^n + 1, q) through the transform. */
void orc_polymul(const u64 *a, const u64 *b, u64 *out, int n, u64 q, u64 psi)
{
    u64 *ta = (u64 *)malloc(sizeof(u64) * (size_t)n);
    u64 *tb = (u64 *)malloc(sizeof(u64) * (size_t)n);
    memcpy(ta, a, sizeof(u64) * (size_t)n);
    memcpy(tb, b, sizeof(u64) * (size_t)n);
    orc_ntt_fwd(ta, n, q, psi);
    orc_ntt_fwd(tb, n, q, psi);
    for (int i = 0; i < n; i++) ta[i] = mmul(ta[i], tb[i], q);
    orc_ntt_inv(ta, n, q, psi);
    memcpy(out, ta, sizeof(u64) * (size_t)n);
    free(ta);
    free(tb);
}

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC 2011): ten rounds of the 4x64 Philox S-box with the    */
/* published multipliers and Weyl key increments.                            */
/* ------------------------------------------------------------------------ */
void orc_philox4x64(const u64 ctr[4], const u64 key[2], u64 out[4])
{
    const u64 M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const u64 W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    u64 c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    u64 k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        u128 p0 = (u128)M0 * c0, p1 = (u128)M1 * c2;
        u64 hi0 = (u64)(p0 >> 64), lo0 = (u64)p0;
        u64 hi1 = (u64)(p1 >> 64), lo1 = (u64)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Samplers.  Each draw has its own Philox counter so that the result of one  */
/* coefficient never depends on another's.  Key = (seed, stream).            */
/* ------------------------------------------------------------------------ */
static int bitlen(u64 x) { int b = 0; while (x) { b++; x >>= 1; } return b; }

/*
 * Uniform residue mod m for coefficient i of modulus index `limb`:
 * counters (i, limb, blk, 0) for blk = 0, 1, ...; the four words of each block
 * are masked to bitlen(m) bits and the first one below m is taken.
 */
static u64 sample_uniform_one(u64 seed, u64 stream, u64 i, u64 limb, u64 m)
{
    u64 key[2] = {seed, stream};
    u64 mask = (bitlen(m) >= 64) ? ~(u64)0 : (((u64)1 << bitlen(m)) - 1);
    for (u64 blk = 0;; blk++) {
        u64 ctr[4] = {i, limb, blk, 0}, w[4];
        orc_philox4x64(ctr, key, w);
        for (int r = 0; r < 4; r++) {
            u64 x = w[r] & mask;
            if (x < m) return x;
        }
    }
}

void orc_sample_uniform(u64 seed, u64 stream, int n, u64 limb, u64 m, u64 *out)
{
    for (int i = 0; i < n; i++) out[i] = sample_uniform_one(seed, stream, (u64)i, limb, m);
}

/*
 * Centred binomial error with eta = 21 (sigma ~ 3.24): one Philox word per
 * coefficient, counter (i, 0, 0, 1); e = popcount(w[0..20]) - popcount(w[21..41]).
 */
void orc_sample_cbd(u64 seed, u64 stream, int n, i64 *out)
{
    u64 key[2] = {seed, stream};
    const u64 m21 = ((u64)1 << 21) - 1;
    for (int i = 0; i < n; i++) {
        u64 ctr[4] = {(u64)i, 0, 0, 1}, w[4];
        orc_philox4x64(ctr, key, w);
        i64 a = __builtin_popcountll(w[0] & m21);
        i64 b = __builtin_popcountll((w[0] >> 21) & m21);
        out[i] = a - b;
    }
}

/*
 * Ternary secret of Hamming weight h (sparse secret, as the paper's SparseLWE
 * security estimate implies, Sec. 5.1): a partial Fisher-Yates shuffle of the
 * positions 0..N-1.  Draw t uses counter (t, 0, 0, 2): position
 * t + (w[0] mod (N - t)) is swapped into slot t and receives sign -1 if bit 0
 * of w[1] is set, +1 otherwise.
 */
void orc_sample_secret(u64 seed, u64 stream, int n, int h, i64 *out)
{
    u64 key[2] = {seed, stream};
    int *idx = (int *)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; i++) { idx[i] = i; out[i] = 0; }
    for (int t = 0; t < h; t++) {
        u64 ctr[4] = {(u64)t, 0, 0, 2}, w[4];
        orc_philox4x64(ctr, key, w);
        int r = t + (int)(w[0] % (u64)(n - t));
        int tmp = idx[t]; idx[t] = idx[r]; idx[r] = tmp;
        out[idx[t]] = (w[1] & 1) ? -1 : 1;
    }
    free(idx);
}

/* ------------------------------------------------------------------------ */
/* Parameters.  moduli[0..L) are q_0..q_{L-1}; moduli[L..L+K) are p_0..p_{K-1}.*/
/* ------------------------------------------------------------------------ */
#define ORC_MAXMOD 128
typedef struct {
    int n;                   /* ring degree N */
    int L;                   /* number of ciphertext primes (top level L-1) */
    int K;                   /* number of special primes */
    int alpha;               /* primes per key-switching digit */
    u64 mod[ORC_MAXMOD];
    u64 psi[ORC_MAXMOD];
} orc_params;

int orc_params_size(void) { return (int)sizeof(orc_params); }

/* moduli: L ciphertext primes followed by K special primes. */
void orc_params_init(orc_params *p, int n, int L, int K, int alpha, const u64 *moduli)
{
    memset(p, 0, sizeof(*p));
    p->n = n; p->L = L; p->K = K; p->alpha = alpha;
    for (int i = 0; i < L + K; i++) {
        p->mod[i] = moduli[i];
        p->psi[i] = orc_find_psi(moduli[i], 2 * (u64)n);
    }
}

#define LIMB(ptr, t, n) ((ptr) + (size_t)(t) * (size_t)(n))

/* Residues of a signed-integer polynomial on moduli idx[0..cnt). */
void orc_reduce_signed(const orc_params *p, const i64 *v, const int *idx, int cnt, u64 *out)
{
    for (int t = 0; t < cnt; t++)
        for (int i = 0; i < p->n; i++) LIMB(out, t, p->n)[i] = mred_signed(v[i], p->mod[idx[t]]);
}

/* ------------------------------------------------------------------------ */
/* Automorphism X -> X^g (g odd) on one residue vector: coefficient i goes to */
/* i*g mod 2N, negated when that lands in [N, 2N).                           */
/* ------------------------------------------------------------------------ */
void orc_automorphism(const u64 *in, u64 *out, int n, u64 g, u64 m)
{
    u64 two_n = 2 * (u64)n;
    for (int i = 0; i < n; i++) {
        u64 e = ((u64)i * g) % two_n;
        if (e < (u64)n) out[e] = in[i];
        else out[e - n] = (in[i] == 0) ? 0 : m - in[i];
    }
}

/* ------------------------------------------------------------------------ */
/* Hybrid key switching (RNS digit decomposition with K special primes).      */
/* ------------------------------------------------------------------------ */

/* Number of digits at a ciphertext with lv+1 limbs. */
int orc_dnum(const orc_params *p, int lv) { return (lv + 1 + p->alpha - 1) / p->alpha; }

/*
 * ModUp of digit j at level lv: the digit's limbs I = [j*alpha, min((j+1)*alpha, lv+1))
 * carry x mod D_j (D_j = prod_{i in I} q_i).  For every other modulus m of
 * {q_0..q_lv, p_0..p_{K-1}} the fast base conversion
 *     out_m = [ sum_{i in I} [x_i * (D_j/q_i)^{-1}]_{q_i} * (D_j/q_i) ]_m
 * is written (no correction of the u*D_j overflow); the digit's own limbs are
 * copied.  `out` has lv+1+K limbs ordered q_0..q_lv, p_0..p_{K-1}.
 */
typedef struct {
    const orc_params *p;
    int lv, lo, hi;
    const u64 *x, *y;
    u64 *out;
} modup_args;

/* Target limb t of a ModUp (see orc_modup). */
static void modup_limb(void *v, int t)
{
    const modup_args *A = (const modup_args *)v;
    const orc_params *p = A->p;
    int n = p->n, lv = A->lv, lo = A->lo, hi = A->hi, cnt = hi - lo;
    int gi = (t <= lv) ? t : (p->L + (t - lv - 1));  /* global modulus index */
    u64 m = p->mod[gi];
    if (t >= lo && t < hi) {
        memcpy(LIMB(A->out, t, n), LIMB(A->x, t, n), sizeof(u64) * (size_t)n);
        return;
    }
    u64 dhat_m[ORC_MAXMOD];
    for (int a = 0; a < cnt; a++) {
        u64 w = 1;
        for (int b = 0; b < cnt; b++) if (b != a) w = mmul(w, p->mod[lo + b] % m, m);
        dhat_m[a] = w;
    }
    for (int c = 0; c < n; c++) {
        u64 acc = 0;
        for (int a = 0; a < cnt; a++) acc = madd(acc, mmul(LIMB(A->y, a, n)[c] % m, dhat_m[a], m), m);
        LIMB(A->out, t, n)[c] = acc;
    }
}

void orc_modup(const orc_params *p, int lv, int j, const u64 *x, u64 *out)
{
    int n = p->n, K = p->K;
    int lo = j * p->alpha, hi = (j + 1) * p->alpha;
    if (hi > lv + 1) hi = lv + 1;
    int cnt = hi - lo;
    int nout = lv + 1 + K;
    u64 *y = (u64 *)malloc(sizeof(u64) * (size_t)cnt * (size_t)n);
    /* y_i = x_i * (D/q_i)^{-1} mod q_i */
    for (int a = 0; a < cnt; a++) {
        u64 qi = p->mod[lo + a];
        u64 dhat = 1;
        for (int b = 0; b < cnt; b++) if (b != a) dhat = mmul(dhat, p->mod[lo + b] % qi, qi);
        u64 dinv = minv(dhat, qi);
        for (int c = 0; c < n; c++) LIMB(y, a, n)[c] = mmul(LIMB(x, lo + a, n)[c], dinv, qi);
    }
    modup_args A = {p, lv, lo, hi, x, y, out};
    orc_parallel_for(nout, modup_limb, &A);
    free(y);
}

/*
 * ModDown at level lv: `in` has lv+1+K limbs (q_0..q_lv, p_0..p_{K-1}).
 *     y_k    = [in_{p_k} * (P/p_k)^{-1}]_{p_k}
 *     conv_i = [ sum_k y_k * (P/p_k) ]_{q_i}
 *     out_i  = [ (in_i - conv_i) * P^{-1} ]_{q_i}
 * (fast base conversion without correction, then exact division by P).
 */
typedef struct {
    const orc_params *p;
    int lv;
    const u64 *in, *y;
    u64 *out;
} moddown_args;

/* Output limb i of a ModDown (see orc_moddown). */
static void moddown_limb(void *v, int i)
{
    const moddown_args *A = (const moddown_args *)v;
    const orc_params *p = A->p;
    int n = p->n, K = p->K, L = p->L;
    u64 qi = p->mod[i];
    u64 phat_q[ORC_MAXMOD];
    u64 P_mod = 1;
    for (int k = 0; k < K; k++) {
        u64 w = 1;
        for (int b = 0; b < K; b++) if (b != k) w = mmul(w, p->mod[L + b] % qi, qi);
        phat_q[k] = w;
        P_mod = mmul(P_mod, p->mod[L + k] % qi, qi);
    }
    u64 P_inv = minv(P_mod, qi);
    for (int c = 0; c < n; c++) {
        u64 conv = 0;
        for (int k = 0; k < K; k++) conv = madd(conv, mmul(LIMB(A->y, k, n)[c] % qi, phat_q[k], qi), qi);
        LIMB(A->out, i, n)[c] = mmul(msub(LIMB(A->in, i, n)[c], conv, qi), P_inv, qi);
    }
}

void orc_moddown(const orc_params *p, int lv, const u64 *in, u64 *out)
{
    int n = p->n, K = p->K, L = p->L;
    u64 *y = (u64 *)malloc(sizeof(u64) * (size_t)K * (size_t)n);
    for (int k = 0; k < K; k++) {
        u64 pk = p->mod[L + k];
        u64 phat = 1;
        for (int b = 0; b < K; b++) if (b != k) phat = mmul(phat, p->mod[L + b] % pk, pk);
        u64 pinv = minv(phat, pk);
        for (int c = 0; c < n; c++) LIMB(y, k, n)[c] = mmul(LIMB(in, lv + 1 + k, n)[c], pinv, pk);
    }
    moddown_args A = {p, lv, in, y, out};
    orc_parallel_for(lv + 1, moddown_limb, &A);
    free(y);
}

/*
 * Key inner product at level lv.  `ext` holds dnum extended digits, each with
 * lv+1+K limbs (q_0..q_lv, p_0..p_{K-1}).  `key` is a switching key stored over
 * all L+K moduli: key[(j*2 + c)*(L+K) + t] is limb t of component c of digit j.
 * acc_c[t] = sum_j ext_j[t] * key_{j,c}[t]  (polynomial products mod X^N+1).
 */
typedef struct {
    const orc_params *p;
    int lv, dnum;
    const u64 *ext, *key;
    u64 *acc0, *acc1;
} kip_args;

/* Limb t of both accumulators of a key inner product (see orc_kip). */
static void kip_limb(void *v, int t)
{
    const kip_args *A = (const kip_args *)v;
    const orc_params *p = A->p;
    int n = p->n, K = p->K, L = p->L, lv = A->lv;
    int nl = lv + 1 + K;
    int gi = (t <= lv) ? t : (L + (t - lv - 1));
    u64 m = p->mod[gi], psi = p->psi[gi];
    u64 *tmp = (u64 *)malloc(sizeof(u64) * (size_t)n);
    u64 *a0 = LIMB(A->acc0, t, n), *a1 = LIMB(A->acc1, t, n);
    memset(a0, 0, sizeof(u64) * (size_t)n);
    memset(a1, 0, sizeof(u64) * (size_t)n);
    for (int j = 0; j < A->dnum; j++) {
        const u64 *e = A->ext + ((size_t)j * nl + t) * (size_t)n;
        const u64 *k0 = A->key + ((size_t)(j * 2 + 0) * (L + K) + gi) * (size_t)n;
        const u64 *k1 = A->key + ((size_t)(j * 2 + 1) * (L + K) + gi) * (size_t)n;
        orc_polymul(e, k0, tmp, n, m, psi);
        for (int c = 0; c < n; c++) a0[c] = madd(a0[c], tmp[c], m);
        orc_polymul(e, k1, tmp, n, m, psi);
        for (int c = 0; c < n; c++) a1[c] = madd(a1[c], tmp[c], m);
    }
    free(tmp);
}

void orc_kip(const orc_params *p, int lv, int dnum, const u64 *ext, const u64 *key, u64 *acc0, u64 *acc1)
{
    kip_args A = {p, lv, dnum, ext, key, acc0, acc1};
    orc_parallel_for(lv + 1 + p->K, kip_limb, &A);
}

/*
 * Key switching of one polynomial d (lv+1 limbs) with `key`:
 * ModUp every digit, key inner product, ModDown both accumulators.
 */
void orc_keyswitch(const orc_params *p, int lv, const u64 *d, const u64 *key, u64 *out0, u64 *out1)
{
    int n = p->n, K = p->K;
    int nl = lv + 1 + K;
    int dnum = orc_dnum(p, lv);
    u64 *ext = (u64 *)malloc(sizeof(u64) * (size_t)dnum * nl * (size_t)n);
    for (int j = 0; j < dnum; j++) orc_modup(p, lv, j, d, ext + (size_t)j * nl * n);
    u64 *a0 = (u64 *)malloc(sizeof(u64) * (size_t)nl * n);
    u64 *a1 = (u64 *)malloc(sizeof(u64) * (size_t)nl * n);
    orc_kip(p, lv, dnum, ext, key, a0, a1);
    orc_moddown(p, lv, a0, out0);
    orc_moddown(p, lv, a1, out1);
    free(ext); free(a0); free(a1);
}

/* ------------------------------------------------------------------------ */
/* Key generation.  Stream identifiers: see orc_stream_* below.              */
/* ------------------------------------------------------------------------ */
u64 orc_stream_secret(void) { return (u64)0x01 << 56; }
u64 orc_stream_key_a(u64 kid, u64 j) { return ((u64)0x02 << 56) | (kid << 8) | j; }
u64 orc_stream_key_e(u64 kid, u64 j) { return ((u64)0x03 << 56) | (kid << 8) | j; }
u64 orc_stream_enc_a(u64 nonce) { return ((u64)0x04 << 56) | (nonce & (((u64)1 << 56) - 1)); }
u64 orc_stream_enc_e(u64 nonce) { return ((u64)0x05 << 56) | (nonce & (((u64)1 << 56) - 1)); }

/*
 * Switching key from s' to s (both small signed polynomials), over all L+K
 * moduli, for key id `kid`.  For digit j (limbs [j*alpha, (j+1)*alpha) of the
 * full chain):
 *     a_j  uniform (stream key_a(kid, j), limb index = global modulus index)
 *     e_j  centred binomial (stream key_e(kid, j))
 *     b_j  = -a_j*s + e_j + [t in digit j] * (P mod m_t) * s'   (mod m_t)
 * The gadget factor P*Qhat_j*[Qhat_j^{-1}]_{D_j} reduces to P on the digit's own
 * limbs and to 0 on every other limb.  Layout: key[(j*2 + c)*(L+K) + t].
 */
typedef struct {
    const orc_params *p;
    u64 seed, kid;
    const i64 *s, *s_from, *e;   /* e: dnum error polynomials, [j][N] */
    u64 *key;
} swk_args;

/* Limb t of digit j of a switching key, item = j * (L + K) + t (see orc_gen_switch_key). */
static void swk_limb(void *v, int item)
{
    const swk_args *A = (const swk_args *)v;
    const orc_params *p = A->p;
    int n = p->n, L = p->L, K = p->K;
    int j = item / (L + K), t = item % (L + K);
    const i64 *e = A->e + (size_t)j * n;
    u64 m = p->mod[t];
    u64 *b = A->key + ((size_t)(j * 2 + 0) * (L + K) + t) * (size_t)n;
    u64 *a = A->key + ((size_t)(j * 2 + 1) * (L + K) + t) * (size_t)n;
    u64 *sr = (u64 *)malloc(sizeof(u64) * (size_t)n);
    u64 *tmp = (u64 *)malloc(sizeof(u64) * (size_t)n);
    orc_sample_uniform(A->seed, orc_stream_key_a(A->kid, (u64)j), n, (u64)t, m, a);
    for (int c = 0; c < n; c++) sr[c] = mred_signed(A->s[c], m);
    orc_polymul(a, sr, tmp, n, m, p->psi[t]);
    u64 gadget = 0;
    if (t < L && t >= j * p->alpha && t < (j + 1) * p->alpha) {
        gadget = 1;
        for (int k = 0; k < K; k++) gadget = mmul(gadget, p->mod[L + k] % m, m);
    }
    for (int c = 0; c < n; c++) {
        u64 w = msub(0, tmp[c], m);
        w = madd(w, mred_signed(e[c], m), m);
        if (gadget) w = madd(w, mmul(gadget, mred_signed(A->s_from[c], m), m), m);
        b[c] = w;
    }
    free(sr); free(tmp);
}

void orc_gen_switch_key(const orc_params *p, u64 seed, u64 kid, const i64 *s, const i64 *s_from, u64 *key)
{
    int n = p->n, L = p->L, K = p->K;
    int dnum = (L + p->alpha - 1) / p->alpha;
    i64 *e = (i64 *)malloc(sizeof(i64) * (size_t)dnum * (size_t)n);
    for (int j = 0; j < dnum; j++) orc_sample_cbd(seed, orc_stream_key_e(kid, (u64)j), n, e + (size_t)j * n);
    swk_args A = {p, seed, kid, s, s_from, e, key};
    orc_parallel_for(dnum * (L + K), swk_limb, &A);
    free(e);
}

/* s(X^g) for a small signed polynomial. */
void orc_automorphism_signed(const i64 *in, i64 *out, int n, u64 g)
{
    u64 two_n = 2 * (u64)n;
    for (int i = 0; i < n; i++) {
        u64 e = ((u64)i * g) % two_n;
        if (e < (u64)n) out[e] = in[i];
        else out[e - n] = -in[i];
    }
}

/* s^2 mod X^N+1 over the integers (schoolbook; |coefficients| stay small). */
void orc_square_signed(const i64 *s, i64 *out, int n)
{
    memset(out, 0, sizeof(i64) * (size_t)n);
    for (int i = 0; i < n; i++) {
        if (s[i] == 0) continue;
        for (int j = 0; j < n; j++) {
            if (s[j] == 0) continue;
            i64 v = s[i] * s[j];
            int k = i + j;
            if (k < n) out[k] += v; else out[k - n] -= v;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Ciphertext operations.  A ciphertext at level lv is 2*(lv+1) limbs:        */
/* ct[(c*(lv+1) + i)*N + x], c in {0,1}, i in [0, lv].                        */
/* ------------------------------------------------------------------------ */
#define CT(ptr, c, i, lv, n) ((ptr) + ((size_t)(c) * ((lv) + 1) + (i)) * (size_t)(n))

/*
 * Symmetric encryption at level lv of an integer plaintext m (signed coeffs):
 * a uniform (stream enc_a(nonce)), e centred binomial (stream enc_e(nonce)),
 * c0 = -a*s + e + m, c1 = a.
 */
typedef struct {
    const orc_params *p;
    u64 seed, nonce;
    const i64 *s, *m, *e;
    int lv;
    u64 *ct;
} enc_args;

/* Limb i of both components of an encryption (see orc_encrypt). */
static void enc_limb(void *v, int i)
{
    const enc_args *A = (const enc_args *)v;
    const orc_params *p = A->p;
    int n = p->n, lv = A->lv;
    u64 q = p->mod[i];
    u64 *c0 = CT(A->ct, 0, i, lv, n), *c1 = CT(A->ct, 1, i, lv, n);
    u64 *sr = (u64 *)malloc(sizeof(u64) * (size_t)n);
    u64 *tmp = (u64 *)malloc(sizeof(u64) * (size_t)n);
    orc_sample_uniform(A->seed, orc_stream_enc_a(A->nonce), n, (u64)i, q, c1);
    for (int c = 0; c < n; c++) sr[c] = mred_signed(A->s[c], q);
    orc_polymul(c1, sr, tmp, n, q, p->psi[i]);
    for (int c = 0; c < n; c++) {
        u64 w = msub(0, tmp[c], q);
        w = madd(w, mred_signed(A->e[c], q), q);
        w = madd(w, mred_signed(A->m[c], q), q);
        c0[c] = w;
    }
    free(sr); free(tmp);
}

void orc_encrypt(const orc_params *p, u64 seed, u64 nonce, const i64 *s, const i64 *m, int lv, u64 *ct)
{
    int n = p->n;
    i64 *e = (i64 *)malloc(sizeof(i64) * (size_t)n);
    orc_sample_cbd(seed, orc_stream_enc_e(nonce), n, e);
    enc_args A = {p, seed, nonce, s, m, e, lv, ct};
    orc_parallel_for(lv + 1, enc_limb, &A);
    free(e);
}

typedef struct {
    const orc_params *p;
    const i64 *s;
    const u64 *ct;
    int lv;
    u64 *out;
} dec_args;

static void dec_limb(void *v, int i)
{
    const dec_args *A = (const dec_args *)v;
    const orc_params *p = A->p;
    int n = p->n, lv = A->lv;
    u64 q = p->mod[i];
    u64 *sr = (u64 *)malloc(sizeof(u64) * (size_t)n);
    u64 *tmp = (u64 *)malloc(sizeof(u64) * (size_t)n);
    for (int c = 0; c < n; c++) sr[c] = mred_signed(A->s[c], q);
    orc_polymul(CT(A->ct, 1, i, lv, n), sr, tmp, n, q, p->psi[i]);
    for (int c = 0; c < n; c++) LIMB(A->out, i, n)[c] = madd(CT(A->ct, 0, i, lv, n)[c], tmp[c], q);
    free(sr); free(tmp);
}

/* out[i] = c0 + c1*s mod q_i for i in [0, lv]  (lv+1 limbs). */
void orc_decrypt(const orc_params *p, const i64 *s, const u64 *ct, int lv, u64 *out)
{
    dec_args A = {p, s, ct, lv, out};
    orc_parallel_for(lv + 1, dec_limb, &A);
}

/* Limb-wise sum / difference of two ciphertexts at the same level. */
void orc_ct_add(const orc_params *p, const u64 *a, const u64 *b, int lv, u64 *out)
{
    int n = p->n;
    for (int c = 0; c < 2; c++)
        for (int i = 0; i <= lv; i++)
            for (int x = 0; x < n; x++) CT(out, c, i, lv, n)[x] = madd(CT(a, c, i, lv, n)[x], CT(b, c, i, lv, n)[x], p->mod[i]);
}
void orc_ct_sub(const orc_params *p, const u64 *a, const u64 *b, int lv, u64 *out)
{
    int n = p->n;
    for (int c = 0; c < 2; c++)
        for (int i = 0; i <= lv; i++)
            for (int x = 0; x < n; x++) CT(out, c, i, lv, n)[x] = msub(CT(a, c, i, lv, n)[x], CT(b, c, i, lv, n)[x], p->mod[i]);
}

/* Plaintext addition: c0 += m (signed integer plaintext). */
void orc_ct_add_plain(const orc_params *p, const u64 *a, const i64 *m, int lv, u64 *out)
{
    int n = p->n;
    memcpy(out, a, sizeof(u64) * 2 * (size_t)(lv + 1) * n);
    for (int i = 0; i <= lv; i++)
        for (int x = 0; x < n; x++) CT(out, 0, i, lv, n)[x] = madd(CT(a, 0, i, lv, n)[x], mred_signed(m[x], p->mod[i]), p->mod[i]);
}

/* Drop limbs: a ciphertext at level lv read at level lv2 <= lv (same message, same scale). */
void orc_ct_drop(const orc_params *p, const u64 *a, int lv, int lv2, u64 *out)
{
    int n = p->n;
    for (int c = 0; c < 2; c++)
        for (int i = 0; i <= lv2; i++) memcpy(CT(out, c, i, lv2, n), CT(a, c, i, lv, n), sizeof(u64) * (size_t)n);
}

/* Multiply by X^{N/2} (which is sqrt(-1) in every slot): a negacyclic shift by N/2. */
void orc_ct_mul_i(const orc_params *p, const u64 *a, int lv, u64 *out)
{
    int n = p->n, h = n / 2;
    for (int c = 0; c < 2; c++)
        for (int i = 0; i <= lv; i++) {
            const u64 *src = CT(a, c, i, lv, n);
            u64 *dst = CT(out, c, i, lv, n);
            u64 q = p->mod[i];
            for (int x = 0; x < n; x++) {
                if (x + h < n) dst[x + h] = src[x];
                else dst[x + h - n] = (src[x] == 0) ? 0 : q - src[x];
            }
        }
}

/*
 * Rescale one ciphertext from level lv to lv-1 (divide by q_lv with rounding):
 * v = top limb, centred to (-q_lv/2, q_lv/2); out_i = (x_i - [v]_{q_i}) * q_lv^{-1} mod q_i.
 */
typedef struct {
    const orc_params *p;
    const u64 *a;
    int lv;
    u64 *out;
} rs_args;

/* Limb i of component c of a rescale, item = c * lv + i (see orc_rescale). */
static void rescale_limb(void *v, int item)
{
    const rs_args *A = (const rs_args *)v;
    const orc_params *p = A->p;
    int n = p->n, lv = A->lv;
    int c = item / lv, i = item % lv;
    u64 ql = p->mod[lv];
    const u64 *top = CT(A->a, c, lv, lv, n);
    u64 qi = p->mod[i];
    u64 qinv = minv(ql % qi, qi);
    const u64 *src = CT(A->a, c, i, lv, n);
    u64 *dst = CT(A->out, c, i, lv - 1, n);
    for (int x = 0; x < n; x++) {
        u64 w = top[x];
        u64 vr;
        if (w <= (ql - 1) / 2) vr = w % qi;
        else vr = msub(0, (ql - w) % qi, qi);   /* w - q_lv < 0 */
        dst[x] = mmul(msub(src[x], vr, qi), qinv, qi);
    }
}

void orc_rescale(const orc_params *p, const u64 *a, int lv, u64 *out)
{
    rs_args A = {p, a, lv, out};
    orc_parallel_for(2 * lv, rescale_limb, &A);
}

/* Plaintext product without rescale: (c0*m, c1*m), m a signed integer plaintext. */
typedef struct {
    const orc_params *p;
    const u64 *a, *b;
    const i64 *m;
    int lv;
    u64 *d0, *d1, *d2;
} limb_prod_args;

static void mul_plain_limb(void *v, int i)
{
    const limb_prod_args *A = (const limb_prod_args *)v;
    const orc_params *p = A->p;
    int n = p->n, lv = A->lv;
    u64 q = p->mod[i];
    u64 *mr = (u64 *)malloc(sizeof(u64) * (size_t)n);
    for (int x = 0; x < n; x++) mr[x] = mred_signed(A->m[x], q);
    for (int c = 0; c < 2; c++) orc_polymul(CT(A->a, c, i, lv, n), mr, CT(A->d0, c, i, lv, n), n, q, p->psi[i]);
    free(mr);
}

void orc_ct_mul_plain(const orc_params *p, const u64 *a, const i64 *m, int lv, u64 *out)
{
    limb_prod_args A = {p, a, NULL, m, lv, out, NULL, NULL};
    orc_parallel_for(lv + 1, mul_plain_limb, &A);
}

/* Tensor product of two ciphertexts at level lv: d0=a0b0, d1=a0b1+a1b0, d2=a1b1. */
static void tensor_limb(void *v, int i)
{
    const limb_prod_args *A = (const limb_prod_args *)v;
    const orc_params *p = A->p;
    int n = p->n, lv = A->lv;
    u64 q = p->mod[i], psi = p->psi[i];
    u64 *tmp = (u64 *)malloc(sizeof(u64) * (size_t)n);
    orc_polymul(CT(A->a, 0, i, lv, n), CT(A->b, 0, i, lv, n), LIMB(A->d0, i, n), n, q, psi);
    orc_polymul(CT(A->a, 0, i, lv, n), CT(A->b, 1, i, lv, n), LIMB(A->d1, i, n), n, q, psi);
    orc_polymul(CT(A->a, 1, i, lv, n), CT(A->b, 0, i, lv, n), tmp, n, q, psi);
    for (int x = 0; x < n; x++) LIMB(A->d1, i, n)[x] = madd(LIMB(A->d1, i, n)[x], tmp[x], q);
    orc_polymul(CT(A->a, 1, i, lv, n), CT(A->b, 1, i, lv, n), LIMB(A->d2, i, n), n, q, psi);
    free(tmp);
}

void orc_tensor(const orc_params *p, const u64 *a, const u64 *b, int lv, u64 *d0, u64 *d1, u64 *d2)
{
    limb_prod_args A = {p, a, b, NULL, lv, d0, d1, d2};
    orc_parallel_for(lv + 1, tensor_limb, &A);
}

/* Relinearisation: (d0 + ks0(d2), d1 + ks1(d2)) with the key for s^2. */
void orc_relin(const orc_params *p, const u64 *d0, const u64 *d1, const u64 *d2, const u64 *rlk, int lv, u64 *out)
{
    int n = p->n;
    size_t sz = sizeof(u64) * (size_t)(lv + 1) * n;
    u64 *k0 = (u64 *)malloc(sz), *k1 = (u64 *)malloc(sz);
    orc_keyswitch(p, lv, d2, rlk, k0, k1);
    for (int i = 0; i <= lv; i++)
        for (int x = 0; x < n; x++) {
            CT(out, 0, i, lv, n)[x] = madd(LIMB(d0, i, n)[x], LIMB(k0, i, n)[x], p->mod[i]);
            CT(out, 1, i, lv, n)[x] = madd(LIMB(d1, i, n)[x], LIMB(k1, i, n)[x], p->mod[i]);
        }
    free(k0); free(k1);
}

/*
 * Plain rotation / conjugation by the automorphism g with the key from s(X^g)
 * to s: c0' = c0(X^g), c1' = c1(X^g), (k0, k1) = KS(c1'), out = (c0' + k0, k1).
 */
void orc_automorph_ct(const orc_params *p, const u64 *a, int lv, u64 g, const u64 *key, u64 *out)
{
    int n = p->n;
    size_t sz = sizeof(u64) * (size_t)(lv + 1) * n;
    u64 *c0 = (u64 *)malloc(sz), *c1 = (u64 *)malloc(sz);
    u64 *k0 = (u64 *)malloc(sz), *k1 = (u64 *)malloc(sz);
    for (int i = 0; i <= lv; i++) {
        orc_automorphism(CT(a, 0, i, lv, n), LIMB(c0, i, n), n, g, p->mod[i]);
        orc_automorphism(CT(a, 1, i, lv, n), LIMB(c1, i, n), n, g, p->mod[i]);
    }
    orc_keyswitch(p, lv, c1, key, k0, k1);
    for (int i = 0; i <= lv; i++)
        for (int x = 0; x < n; x++) {
            CT(out, 0, i, lv, n)[x] = madd(LIMB(c0, i, n)[x], LIMB(k0, i, n)[x], p->mod[i]);
            CT(out, 1, i, lv, n)[x] = LIMB(k1, i, n)[x];
        }
    free(c0); free(c1); free(k0); free(k1);
}

/*
 * Hoisted rotations of one source ciphertext by several automorphisms:
 * the digits of c1 are extended once (ModUp); for every g the extended digits
 * are mapped by X -> X^g limb by limb, multiplied with that g's key and brought
 * down (ModDown); out_r = (c0(X^g) + k0, k1).  outs is n_g consecutive ciphertexts.
 */
void orc_automorph_hoisted(const orc_params *p, const u64 *a, int lv, int n_g, const u64 *gs,
                           const u64 *const *keys, u64 *outs)
{
    int n = p->n, K = p->K, L = p->L;
    int nl = lv + 1 + K;
    int dnum = orc_dnum(p, lv);
    size_t csz = (size_t)2 * (lv + 1) * n;
    u64 *ext = (u64 *)malloc(sizeof(u64) * (size_t)dnum * nl * n);
    u64 *extg = (u64 *)malloc(sizeof(u64) * (size_t)dnum * nl * n);
    for (int j = 0; j < dnum; j++) orc_modup(p, lv, j, CT(a, 1, 0, lv, n), ext + (size_t)j * nl * n);
    u64 *a0 = (u64 *)malloc(sizeof(u64) * (size_t)nl * n);
    u64 *a1 = (u64 *)malloc(sizeof(u64) * (size_t)nl * n);
    size_t lsz = sizeof(u64) * (size_t)(lv + 1) * n;
    u64 *k0 = (u64 *)malloc(lsz), *k1 = (u64 *)malloc(lsz);
    for (int r = 0; r < n_g; r++) {
        u64 g = gs[r];
        for (int j = 0; j < dnum; j++)
            for (int t = 0; t < nl; t++) {
                int gi = (t <= lv) ? t : (L + (t - lv - 1));
                orc_automorphism(ext + ((size_t)j * nl + t) * n, extg + ((size_t)j * nl + t) * n, n, g, p->mod[gi]);
            }
        orc_kip(p, lv, dnum, extg, keys[r], a0, a1);
        orc_moddown(p, lv, a0, k0);
        orc_moddown(p, lv, a1, k1);
        u64 *o = outs + (size_t)r * csz;
        for (int i = 0; i <= lv; i++) {
            orc_automorphism(CT(a, 0, i, lv, n), CT(o, 0, i, lv, n), n, g, p->mod[i]);
            for (int x = 0; x < n; x++) {
                CT(o, 0, i, lv, n)[x] = madd(CT(o, 0, i, lv, n)[x], LIMB(k0, i, n)[x], p->mod[i]);
                CT(o, 1, i, lv, n)[x] = LIMB(k1, i, n)[x];
            }
        }
    }
    free(ext); free(extg); free(a0); free(a1); free(k0); free(k1);
}

/*
 * Sum of a ciphertext and its rotations, a + sum_r sigma_{g_r}(a), with one
 * ModUp and one ModDown: the digits of c1 are extended once; for every g the
 * mapped digits' key inner product is added into one pair of extended-basis
 * accumulators, which are brought down once.  ModDown is linear, so this is the
 * sum of the rotations up to the rounding of one ModDown instead of several.
 *     out = (c0 + sum_r c0(X^g_r) + k0, c1 + k1)
 */
void orc_rot_sum(const orc_params *p, const u64 *a, int lv, int n_g, const u64 *gs, const u64 *const *keys,
                 u64 *out)
{
    int n = p->n, K = p->K, L = p->L;
    int nl = lv + 1 + K;
    int dnum = orc_dnum(p, lv);
    u64 *ext = (u64 *)malloc(sizeof(u64) * (size_t)dnum * nl * n);
    u64 *extg = (u64 *)malloc(sizeof(u64) * (size_t)dnum * nl * n);
    for (int j = 0; j < dnum; j++) orc_modup(p, lv, j, CT(a, 1, 0, lv, n), ext + (size_t)j * nl * n);
    u64 *a0 = (u64 *)malloc(sizeof(u64) * (size_t)nl * n);
    u64 *a1 = (u64 *)malloc(sizeof(u64) * (size_t)nl * n);
    u64 *s0 = (u64 *)calloc((size_t)nl * n, sizeof(u64));
    u64 *s1 = (u64 *)calloc((size_t)nl * n, sizeof(u64));
    size_t lsz = sizeof(u64) * (size_t)(lv + 1) * n;
    u64 *k0 = (u64 *)malloc(lsz), *k1 = (u64 *)malloc(lsz), *tmp = (u64 *)malloc(sizeof(u64) * (size_t)n);
    memcpy(out, a, sizeof(u64) * (size_t)2 * (lv + 1) * n);
    for (int r = 0; r < n_g; r++) {
        u64 g = gs[r];
        for (int j = 0; j < dnum; j++)
            for (int t = 0; t < nl; t++) {
                int gi = (t <= lv) ? t : (L + (t - lv - 1));
                orc_automorphism(ext + ((size_t)j * nl + t) * n, extg + ((size_t)j * nl + t) * n, n, g, p->mod[gi]);
            }
        orc_kip(p, lv, dnum, extg, keys[r], a0, a1);
        for (int t = 0; t < nl; t++) {
            int gi = (t <= lv) ? t : (L + (t - lv - 1));
            u64 m = p->mod[gi];
            for (int x = 0; x < n; x++) {
                LIMB(s0, t, n)[x] = madd(LIMB(s0, t, n)[x], LIMB(a0, t, n)[x], m);
                LIMB(s1, t, n)[x] = madd(LIMB(s1, t, n)[x], LIMB(a1, t, n)[x], m);
            }
        }
        for (int i = 0; i <= lv; i++) {
            orc_automorphism(CT(a, 0, i, lv, n), tmp, n, g, p->mod[i]);
            for (int x = 0; x < n; x++) CT(out, 0, i, lv, n)[x] = madd(CT(out, 0, i, lv, n)[x], tmp[x], p->mod[i]);
        }
    }
    orc_moddown(p, lv, s0, k0);
    orc_moddown(p, lv, s1, k1);
    for (int i = 0; i <= lv; i++)
        for (int x = 0; x < n; x++) {
            CT(out, 0, i, lv, n)[x] = madd(CT(out, 0, i, lv, n)[x], LIMB(k0, i, n)[x], p->mod[i]);
            CT(out, 1, i, lv, n)[x] = madd(CT(out, 1, i, lv, n)[x], LIMB(k1, i, n)[x], p->mod[i]);
        }
    free(ext); free(extg); free(a0); free(a1); free(s0); free(s1); free(k0); free(k1); free(tmp);
}
