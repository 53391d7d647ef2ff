"""CKKS bootstrapping (Sec. 2.2; the paper relies on it between training steps and reports its
time, 159 ms on an A40, in Sec. 5.1): the full-slot procedure of Cheon, Han, Kim, Kim and
Song, written from the mathematics.

TEST INFRASTRUCTURE ONLY.  Only the test-suite (and the CPU leg of the benchmark) may import
this module; the product path never does.  It shares no code with the CUDA library.

A ciphertext at level 0 decrypts, over the integers, to t = Delta m + e + q_0 I with a small
integer polynomial I (|I| below ~20 for the secrets used here, h = 192).  Then:

  ModRaise     the level-0 residues, centred, reduced modulo every prime of a high level:
               a ciphertext of t itself, read at scale q_0 (its slots are sigma(t) / q_0).
  CoeffToSlot  with z = sigma(t) / q_0 and U[j][k] = zeta^(5^j k) (j, k < n = N/2),
               z = U (t_lo + i t_hi) / q_0 and U^-1 = (2/N) U^H, so v = (1/N) U^H z holds
               (t_lo + i t_hi) / (2 q_0); with its conjugate, the real part is v + conj(v)
               and the imaginary part i (conj(v) - v): two ciphertexts whose slots are the
               coefficients t_k / q_0 = I_k + eps_k, eps_k = (Delta m + e)_k / q_0.
  EvalMod      eps = sin(2 pi x) / (2 pi) + O(eps^3), x = I + eps: cos(2 pi (x - 1/4)) by a
               Taylor polynomial of cos at theta = 2 pi (x - 1/4) / 2^r, then r double-angle
               steps c <- 2c^2 - 1; valid for |x| <= K.
  SlotToCoeff  U (eps_lo + i eps_hi) = sigma(Delta m + e) / q_0: the message at scale
               (working scale) * Delta / q_0.

Both linear transforms are dense n x n matrices, evaluated by the baby-step / giant-step
diagonal method: M z = sum_g Rot_{n1 g}( sum_i Rot_{-n1 g}(d_{i + n1 g}) (.) Rot_i(z) ), d_k
the k-th diagonal (d_k[j] = M[j][(j + k) mod n]), the n1 baby rotations hoisted.  Their
cost grows with n (n plaintext products per transform), which limits this oracle to small
rings; the plaintexts are logged under (name, diagonal, level) like every RnsOps product.
The factored form (factored, the default) groups the log2(n) butterfly stages of the special
FFT a few to a level instead.

Built on it, for training with bootstrapping: refresh_packed (W and V refreshed together,
their repeated rows packed into few ciphertexts), Refresher (the refresh points inside
Algorithm ASoftmax, softmax.ScaledOps.keep), nag_train_boot and train_step_asoftmax (NAG
iterations with the stand-in or with ASoftmax), and train_epochs with ValidationClient
(Protocol 1's epochs, validation logits and early stopping).
"""
import math
from dataclasses import dataclass

import numpy as np

from . import ckks


@dataclass
class BootParams:
    K: float = 24.5       # EvalMod covers |x| <= K (|I| <= 24)
    r: int = 5            # double-angle steps
    taylor: int = 14      # cos by its Taylor polynomial of degree 2 * taylor
    n1: int = 0           # baby steps of the dense transforms (0: the power of two nearest sqrt(n))
    fft: bool = True      # factored transforms (below) instead of the dense ones
    per_level: int = 3    # FFT stages merged into one level of the factored transforms


def encoding_matrix(N):
    """U[j][k] = zeta^(5^j k), zeta = exp(i pi / N): sigma of the first N/2 coefficients."""
    n = N // 2
    g = ckks.slot_exponents(N).astype(np.int64)
    k = np.arange(n, dtype=np.int64)
    return np.exp(1j * np.pi * ((g[:, None] * k[None, :]) % (2 * N)) / N)


def diagonal(M, k):
    n = M.shape[0]
    j = np.arange(n)
    return M[j, (j + k) % n]


def baby_steps(n, prm):
    if prm.n1:
        return prm.n1
    return 1 << int(round(math.log2(n) / 2))


def lintrans(ops, ct, M, name, out_scale, prm):
    """M z for a ciphertext of z (baby-step / giant-step diagonal method), each giant step's
    products summed before one rescale that lands on out_scale; one level."""
    n = M.shape[0]
    n1 = baby_steps(n, prm)
    n2 = n // n1
    baby = [ct] + ops.rot_many(ct, list(range(1, n1)))
    out = None
    for g in range(n2):
        # Rot_{-n1 g}(d_k) (.) Rot_i(ct) summed over the baby steps, one rescale
        inner = ops.cmult_scaled_sum([(baby[i], np.roll(diagonal(M, i + n1 * g), n1 * g), (name, i + n1 * g))
                                      for i in range(n1)], out_scale)
        part = ops.rot(inner, n1 * g) if g else inner
        out = part if out is None else ops.add(out, part)
    return out


# ---------------------------------------------------------------------------
# Factored transforms.  U = S_L ... S_1 P: P puts a vector in bit-reversed order and
# stage s (block length 2^s, half h = 2^(s-1)) replaces, in every block, the pair
# (v[p], v[p+h]) (p in the first half, j = p mod 2^s) by (v[p] + xi v[p+h], v[p] - xi v[p+h]),
# xi = zeta^((5^j mod 2^(s+2)) * 2N / 2^(s+2)).  Each stage is three diagonals (rotations by
# 0 and +-h).  CoeffToSlot applies S_L^-1 .. S_1^-1 and stops before P^-1, so its slots hold
# the coefficients in bit-reversed order; EvalMod works slot by slot, and SlotToCoeff
# applies S_1 .. S_L to that order, so P is never applied.  Groups of `per_level`
# consecutive stages are merged into one matrix of at most 2^(per_level+1) - 1 diagonals,
# one level each (the stages split as evenly as the level count allows).  A matrix is a
# dict {offset r: d_r}: x -> sum_r d_r (.) Lrot(x, r).
# ---------------------------------------------------------------------------
def _stage(N, s, inverse):
    n = N // 2
    L, h = 1 << s, 1 << (s - 1)
    g = ckks.slot_exponents(N).astype(np.int64)
    p = np.arange(n)
    j = p % L
    first = j < h
    jj = np.where(first, j, j - h)
    xi = np.exp(1j * np.pi * ((g[jj] % (4 * L)) * (2 * N // (4 * L))) / N)
    d = {}

    def put(r, v):
        r %= n
        d[r] = d.get(r, 0) + v
    if not inverse:
        put(0, np.where(first, 1.0, -xi))
        put(h, np.where(first, xi, 0.0))
        put(-h, np.where(first, 0.0, 1.0))
    else:
        put(0, np.where(first, 0.5, -0.5 / xi))
        put(h, np.where(first, 0.5, 0.0))
        put(-h, np.where(first, 0.0, 0.5 / xi))
    return d


def _compose(A, B, n):
    """The matrix A B (B applied first): offset a + b gets d^A_a (.) Lrot(d^B_b, a)."""
    out = {}
    for a, da in A.items():
        for b, db in B.items():
            r = (a + b) % n
            out[r] = out.get(r, 0) + da * np.roll(db, -a)
    return out


def factored(N, inverse, per_level):
    """The level matrices of U (S_1 first) or of (1/2) U^-1 without P^-1 (S_L^-1 first, the
    1/2 in the first level), in the order they are applied."""
    n = N // 2
    Ls = n.bit_length() - 1
    order = list(range(Ls, 0, -1)) if inverse else list(range(1, Ls + 1))
    nlev = -(-Ls // per_level)
    sizes = [Ls // nlev + (1 if i < Ls % nlev else 0) for i in range(nlev)]   # as even as can be
    starts = np.cumsum([0] + sizes)
    groups = [order[starts[i]:starts[i + 1]] for i in range(nlev)]
    mats = []
    for gi, grp in enumerate(groups):
        M = {0: np.ones(n, dtype=complex) * (0.5 if (inverse and gi == 0) else 1.0)}
        for s in grp:
            M = _compose(_stage(N, s, inverse), M, n)
        mats.append({r: v for r, v in M.items() if np.max(np.abs(v)) > 0})
    return mats


def apply_diagonals(ops, ct, M, name, out_scale):
    """sum_r d_r (.) Lrot(ct, r): every nonzero offset's rotation hoisted from one ModUp, the
    products summed before one rescale that lands on out_scale; one level."""
    rs = sorted(M)
    nz = [r for r in rs if r]
    rot = dict(zip(nz, ops.rot_many(ct, nz))) if nz else {}
    rot[0] = ct
    return ops.cmult_scaled_sum([(rot[r], M[r], (name, r)) for r in rs], out_scale)


def coeff_to_slot_fft(ops, ct, N, out_scale, prm):
    """(ct_lo, ct_hi) with the coefficients in bit-reversed order."""
    v = ct
    for li, M in enumerate(factored(N, True, prm.per_level)):
        v = apply_diagonals(ops, v, M, "cts%d" % li, out_scale)
    c = ops.conj(v)
    return ops.add(v, c), ops.mul_i(ops.sub(c, v))


def slot_to_coeff_fft(ops, lo, hi, N, out_scale, prm):
    u = ops.add(lo, ops.mul_i(hi))
    for li, M in enumerate(factored(N, False, prm.per_level)):
        u = apply_diagonals(ops, u, M, "stc%d" % li, out_scale)
    return u


def transform_levels(N, prm):
    if not prm.fft:
        return 1
    return -(-((N // 2).bit_length() - 1) // prm.per_level)


def fft_rotations(N, prm):
    """The rotation amounts of both factored transforms."""
    out = set()
    for inv in (True, False):
        for M in factored(N, inv, prm.per_level):
            out |= {r for r in M if r}
    return sorted(out)


def coeff_to_slot(ops, ct, N, out_scale, prm):
    """(ct_lo, ct_hi): slots t_k / q_0 and t_{k+N/2} / q_0 (k < N/2)."""
    U = encoding_matrix(N)
    v = lintrans(ops, ct, U.conj().T / N, "cts", out_scale, prm)
    c = ops.conj(v)
    lo = ops.add(v, c)
    hi = ops.mul_i(ops.sub(c, v))
    return lo, hi


def _lin(ops, pw, coef, name, base, target):
    """coef[0] + sum_{r=1..3} coef[r] pw[r], each product landing on exactly `target`
    (plaintext products at a chosen scale, one rescale for each: the powers sit at different
    levels; values above 4 first times an integer 2^k)."""
    one = np.ones(ops.s)
    acc = None
    for r in (1, 2, 3):
        a, v = pw[r], coef[r]
        if abs(v) > 4.0:
            k = int(math.ceil(math.log2(abs(v) / 4.0)))
            a, v = ops.mul_int(a, 1 << k), v / float(1 << k)
        term = ops.cmult_scaled(a, v * one, (name, base + r), target)
        acc = term if acc is None else ops.add(acc, term)
    return ops.add_plain(acc, coef[0] * one, (name, base))


def cos_poly(ops, w, coef, name, target):
    """sum_k coef[k] w^k (degree <= 15) by baby steps w, w^2, w^3 and giant steps w^4, w^8:
    (u0 + u1 w^4) + (u2 + u3 w^4) w^8.  Every addition meets two exactly equal scales
    (up to rounding of the last bit): each inner sum u_j is aimed at the scale of the
    product it is added to, or at the one that makes its own product land on the other
    half's scale."""
    c = list(coef) + [0.0] * (16 - len(coef))
    w2 = ops.mult_to(w, w, target)
    w3 = ops.mult_to(w2, w, target)
    w4 = ops.mult_to(w2, w2, target)
    w8 = ops.mult_to(w4, w4, target)
    pw = (None, w, w2, w3)
    u3 = _lin(ops, pw, c[12:16], name, 12, target)
    p3 = ops.mult_to(u3, w4, target)
    u2 = _lin(ops, pw, c[8:12], name, 8, p3.scale)
    high = ops.mult_to(ops.add(u2, p3), w8, target)
    # u1 (one level below w^3) at the scale whose product with w^4 lands on high's scale
    T1 = ops.operand_scale_for(w3.lv - 1, w4, high.scale, target)
    u1 = _lin(ops, pw, c[4:8], name, 4, T1)
    p1 = ops.mult_to(u1, w4, high.scale)
    u0 = _lin(ops, pw, c[0:4], name, 0, p1.scale)
    return ops.add(ops.add(u0, p1), high)


def eval_mod(ops, x, prm, target):
    """sin(2 pi x) / (2 pi) for |x| <= K: cos(theta), theta = 2 pi (x - 1/4) / 2^r, by its
    Taylor polynomial in w = theta^2 / W (W bounds theta^2, keeping every power of w
    below 1), then r double-angle steps c <- 2 c^2 - 1 (cos(2^r theta) = sin(2 pi x))."""
    one = np.ones(ops.s)
    theta_max = 2 * math.pi * (prm.K + 0.25) / 2 ** prm.r
    W = theta_max ** 2
    u = ops.add_plain(x, -0.25 * one, ("em_shift", 0))
    th = ops.cmult(u, 2 * math.pi / 2 ** prm.r / math.sqrt(W) * one, ("em_theta", 0))
    w = ops.mult_to(th, th, target)
    coef = [(-1) ** k * W ** k / math.factorial(2 * k) for k in range(prm.taylor + 1)]
    c = cos_poly(ops, w, coef, "em_cos", target)
    for j in range(prm.r):
        c = ops.add_plain(ops.mul_int(ops.mult_to(c, c, target), 2), -one, ("em_double", j))
    return ops.cmult(c, one / (2 * math.pi), ("em_out", 0))


def slot_to_coeff(ops, lo, hi, N, out_scale, prm):
    U = encoding_matrix(N)
    return lintrans(ops, ops.add(lo, ops.mul_i(hi)), U, "stc", out_scale, prm)


def bootstrap_raised(ops, ct, N, delta_w, prm):
    """CoeffToSlot, EvalMod on both halves, SlotToCoeff, on a raised ciphertext read at scale
    q_0; the products aim at delta_w.  The result's slots are (Delta m + e) / q_0 at scale
    delta_w (a caller reads it at delta_w * Delta / q_0 to get m back)."""
    cts, stc = (coeff_to_slot_fft, slot_to_coeff_fft) if prm.fft else (coeff_to_slot, slot_to_coeff)
    lo, hi = cts(ops, ct, N, delta_w, prm)
    lo = eval_mod(ops, lo, prm, delta_w)
    hi = eval_mod(ops, hi, prm, delta_w)
    return stc(ops, lo, hi, N, delta_w, prm)


def depth(prm, N=None):
    """Levels: CoeffToSlot, EvalMod (theta 1, w 1, the degree-14 polynomial 5, r doublings,
    the 1 / 2 pi product 1), SlotToCoeff; a transform takes 1 level dense and
    ceil(log2(N/2) / per_level) factored."""
    t = 1 if (not prm.fft or N is None) else transform_levels(N, prm)
    return t + (1 + 1 + 5 + prm.r + 1) + t


# ---------------------------------------------------------------------------
# The training loop of Protocol 1 (step 3, NAG of Sec. 2.1) for any number of iterations:
# after each update W and V are refreshed by bootstrapping, on a chain whose upper group of
# primes (levels above the training ones) holds exactly the bootstrapping, followed by one
# plaintext product that puts the refreshed ciphertext at the training scale, one level
# below the training primes' top.  refresh_packed gathers the distinct slots of many
# periodic ciphertexts into few before bootstrapping them (one window of all the slots
# refreshes a ciphertext that has no period).
# ---------------------------------------------------------------------------
class Refresher:
    """The refresh behind softmax.ScaledOps.keep, for circuits that run at sops.delta on the
    levels below a chain's bootstrapping primes.  A ciphertext a (level >= 1, |message|
    <= bound) becomes:
      1. a times the integer 2^k, read at exactly delta_in (2^k scale(a) is delta_in up to
         the rounding of a's scale, below 2^-16): the scale bootstrapping expects;
      2. times 1 / bound (one level), landing on delta_in: the message bootstrapped is
         m / bound, in [-1, 1];
      3. bootstrapped (bops) and read at its message's scale divided by bound (the message
         is m again);
      4. times 1 (one level), landing on exactly sops.delta.
    bound is rounded up to a power of two 2^e; the plaintexts are named ("refresh_in",
    e + 64) and ("refresh_out", e + 64) at their levels.

    pair() refreshes two values whose slots repeat every P slots within each aligned run of
    2P slots (a row of 2P or more slots tiled with period P; the values may differ from
    row to row) with one bootstrapping: value j in the windows {t : (t // P) mod 2 = j},
    each times its own 1 / bound in step 2 (one summed product); after bootstrapping,
    value j is read at its own bound, masked to its windows (step 4's product) and copied
    into the other window of its run: value 0 by one rotation right by P, value 1 left.  The plaintexts are named
    ("refresh_in_p<P>_w<j>", e + 64) and ("refresh_out_p<P>_w<j>", e + 64)."""

    def __init__(self, sops, bops, prm, delta_w, delta_in=2.0 ** 50):
        self.sops, self.bops, self.prm = sops, bops, prm
        self.delta_w, self.delta_in = float(delta_w), float(delta_in)
        self.calls = 0

    def _pre(self, a):
        """Step 1: times 2^k, read at exactly delta_in."""
        o = self.sops.o
        k = int(round(math.log2(self.delta_in / a.scale)))
        assert k >= 0 and a.lv >= 1
        if k:
            a = o.mul_int(a, 1 << k)
        assert abs(a.scale * 2.0 ** k / self.delta_in - 1.0) <= 2.0 ** -16
        return ckks.Ct(a.data, a.lv, self.delta_in)

    def _boot(self, x):
        """Step 3's bootstrapping of a ciphertext at delta_in, read at its message's scale."""
        o = self.sops.o
        ct0 = o.drop(x, 0)
        b = bootstrap_raised(self.bops, o.mod_raise(ct0, o.p.top), o.p.N, self.delta_w, self.prm)
        self.calls += 1
        return b, b.scale * ct0.scale / float(o.p.q[0])

    def __call__(self, a, bound):
        e = int(math.ceil(math.log2(bound)))
        bound, idx = 2.0 ** e, e + 64
        ones = np.ones(self.sops.o.p.slots)
        x = self.sops.cmult_scaled(self._pre(a), ones / bound, ("refresh_in", idx), self.delta_in)
        b, sc = self._boot(x)
        r = ckks.Ct(b.data, b.lv, sc / bound)
        return self.sops.cmult_scaled(r, ones, ("refresh_out", idx), self.sops.delta)

    def pair(self, a, bound_a, b, bound_b, P):
        o, sops = self.sops.o, self.sops
        t = np.arange(o.p.slots)
        win = [((t // P) % 2 == j).astype(np.float64) for j in (0, 1)]
        es = [int(math.ceil(math.log2(bd))) for bd in (bound_a, bound_b)]
        xs = [self._pre(a), self._pre(b)]
        lv = min(x.lv for x in xs)
        xs = [o.drop(x, lv) for x in xs]
        x = sops.cmult_scaled_sum([(xs[j], win[j] / 2.0 ** es[j], ("refresh_in_p%d_w%d" % (P, j), es[j] + 64))
                                   for j in (0, 1)], self.delta_in)
        boot, sc = self._boot(x)
        out = []
        for j in (0, 1):
            r = ckks.Ct(boot.data, boot.lv, sc / 2.0 ** es[j])
            v = sops.cmult_scaled(r, win[j], ("refresh_out_p%d_w%d" % (P, j), es[j] + 64), sops.delta)
            out.append(sops.add(v, sops.rot(v, -P if j == 0 else P)))
        return out


def window(k, P, slots):
    """The 0/1 slot vector of window k: slots [k P, (k + 1) P)."""
    v = np.zeros(slots)
    v[k * P:(k + 1) * P] = 1.0
    return v


def replicate_stages(w):
    """Rotate-and-sum stages that copy one window of P slots to all w windows (w a power of
    two): log2 w split into stages of at most 3 bits, each [(radix, stride in windows)]."""
    e, stride, out = int(round(math.log2(w))), 1, []
    assert 1 << e == w
    while e > 0:
        b = min(3, e)
        out.append((1 << b, stride))
        stride <<= b
        e -= b
    return out


def replicate_rotations(P, w):
    """The rotation amounts (right rotations, as negative Lrot amounts) of replicate_stages."""
    return sorted({-(j * stride * P) for radix, stride in replicate_stages(w) for j in range(1, radix)})


def refresh_packed(o, bops, blocks, P, w, target_scale, prm, delta_w, bound=1.0):
    """Bootstrapping of ciphertexts whose slots repeat with period P (w = slots / P periods; a
    vertically tiled W-bar has P = c s1, w = s0 / c), w of them per bootstrapping:
      pack:   ciphertext k holds window i - k w of block i for i in [k w, (k + 1) w), one
              plaintext-product sum of the window masks (one level), landing on target_scale;
      refresh: bootstrapped and read at its message's scale;
      unpack: block i keeps its window (a window-mask product landing on exactly target_scale,
              one level) and copies it to all w windows by rotate-and-sum stages
              (right rotations by multiples of P; replicate_stages).
    The blocks (at one level >= 1 and one scale) come back at bootstrapping's output level
    minus one, at exactly target_scale, holding the same periodic messages.  With bound (a
    power of two, |message| <= bound) the pack masks are 1 / bound, so that bootstrapping sees
    messages in [-1, 1], and the bootstrapped ciphertext is read at its scale / bound; the
    plaintexts of bound 2^e != 1 are named "pack_e<e>" and "unpack_e<e>"."""
    slots = o.p.slots
    e = int(math.ceil(math.log2(bound)))
    bound = 2.0 ** e
    names = ("pack", "unpack") if e == 0 else ("pack_e%d" % e, "unpack_e%d" % e)
    out = [None] * len(blocks)
    for k0 in range(0, len(blocks), w):
        idx = range(k0, min(len(blocks), k0 + w))
        packed = bops.cmult_scaled_sum([(blocks[i], window(i - k0, P, slots) / bound, (names[0], i - k0))
                                        for i in idx], target_scale)
        ct0 = o.drop(packed, 0)
        b = bootstrap_raised(bops, o.mod_raise(ct0, o.p.top), o.p.N, delta_w, prm)
        r = ckks.Ct(b.data, b.lv, b.scale * ct0.scale / float(o.p.q[0]) / bound)
        for i in idx:
            x = bops.cmult_scaled(r, window(i - k0, P, slots), (names[1], i - k0), target_scale)
            for radix, stride in replicate_stages(w):
                x = o.rot_sum(x, [-(j * stride * P) for j in range(1, radix)])
            out[i] = x
    return out


def train_step_asoftmax(ops, sops, X, Wbar, Y, c_real, c, valid, lr_over_n, target_scale, sm_prm):
    """Protocol 1, step 3(a) with the paper's softmax (Algorithm ASoftmax) in place of the
    degree-15 stand-in, on a chain whose softmax runs on refreshes (sops.refresh):
      logits = DiagABT(X, W-bar, t = 1), moved to the softmax's scale sops.delta (a constant
               product, one level);
      P      = ASoftmax(logits) over the c_real classes, refreshed if it has fewer than 6
               levels left, times the valid mask (rows and classes of the batch) landing on
               exactly sops.delta (one level);
      D      = P - Y (Y at sops.delta);
      G      = DiagATB(D, X at level(D) + 1, lr/N), then times the integer 2^k and read at
               2^k its scale, about target_scale (DiagATB leaves D's scale).
    Returns (G, logits, P, D)."""
    from . import matmul as mm
    from . import softmax as sm
    logits = mm.diag_abt(ops, X, Wbar, c, 1.0)
    P, D = [], []
    for r in range(logits.m):
        Ml = ops.mul_const(logits.blocks[r][0], 1.0, sops.delta)
        Pr = sops.keep(sm.asoftmax_block(sops, Ml, c_real, X.s0, X.s1, sm_prm), 5, 2.0)
        Pr = sops.cmult_scaled(Pr, valid, ("valid", 0), sops.delta)
        P.append([Pr])
        D.append([ops.sub(Pr, Y.blocks[r][0])])
    lv = ops.level(D[0][0]) + 1
    Xl = mm.EncMat([[ops.drop(b, lv) for b in row] for row in X.blocks], X.rows, X.cols, X.s0, X.s1)
    G = mm.diag_atb(ops, mm.EncMat(D, logits.rows, logits.cols, X.s0, X.s1), Xl, c, lr_over_n)
    k = int(round(math.log2(target_scale / G.blocks[0][0].scale)))
    G = mm.EncMat([[ckks.Ct(g.data, g.lv, g.scale * 2.0 ** k) for g in (ops.mul_int(b, 1 << k) for b in row)]
                   for row in G.blocks], G.rows, G.cols, G.s0, G.s1)
    return G, logits, P, D


def nag_train_boot(ops, bops, X, Wbar, Y, coeffs, valid, c, lr_over_n, target_scale, steps, Xval, prm,
                   delta_w, vops=None, grad=None):
    """`steps` NAG updates (Sec. 2.1) with W and V refreshed by bootstrapping after every update
    (ops: the training step's RnsOps; bops: ScaledOps for bootstrapping, on the same oracle),
    then the validation logits on vops (default ops).  Wbar is at target_scale.

    The update is matmul.nag_train's with V_{t+1} written as
        V_{t+1} = W_{t+1} + gamma (W_t - W_{t+1}) = (1 - gamma) V_t + gamma W_t - (1 - gamma) G,
    every term moved to target_scale by a constant product, so that W_{t+1} and V_{t+1} end
    at the same level (the gradient's minus one), one above 0; the blocks of both are then
    refreshed together by refresh_packed (W-bar's rows repeat every c rows: period c s1).
    A separate vops keeps the logits' plaintexts (t = 1) apart from the training step's
    DiagABT ones: after a refresh both products run at the same level, under the same
    plaintext names.  grad(V), if given, replaces the stand-in step (matmul.train_step) and
    returns the gradient at about target_scale (e.g. train_step_asoftmax).  Returns
    (W, V, logits)."""
    from . import matmul as mm
    S = target_scale
    assert Wbar.blocks[0][0].scale == S
    P, w = c * Wbar.s1, Wbar.s0 // c
    W = V = Wbar
    for gamma in mm.nag_gammas(steps):
        if grad is None:
            G = mm.train_step(ops, X, V, Y, coeffs, valid, c, lr_over_n, S)[0]
        else:
            G = grad(V)
        W, V = nag_update_refresh(ops, bops, W, V, G, gamma, S, prm, delta_w, P, w)
    logits = mm.diag_abt(vops or ops, Xval, W, c, 1.0)
    return W, V, logits


def nag_update_refresh(ops, bops, W, V, G, gamma, target_scale, prm, delta_w, P, w, bound=1.0):
    """One NAG update (Sec. 2.1) from the gradient G (at about target_scale), block by block:
        W_{t+1} = V_t - G,  V_{t+1} = (1 - gamma) V_t + gamma W_t - (1 - gamma) G,
    every term moved to target_scale by a constant product; then the blocks of W_{t+1} and
    V_{t+1} refreshed together (refresh_packed, with `bound` on their entries).  Returns
    (W_{t+1}, V_{t+1})."""
    from . import matmul as mm
    S, n = target_scale, len(W.blocks[0])
    Wn, Vn = [], []
    for w_t, v_t, g in zip(W.blocks[0], V.blocks[0], G.blocks[0]):
        Wn.append(ops.sub(v_t, ops.mul_const(g, 1.0, S)))
        a = ops.add(ops.mul_const(v_t, 1.0 - gamma, S), ops.mul_const(w_t, gamma, S))
        Vn.append(ops.sub(a, ops.mul_const(g, 1.0 - gamma, S)))
    fresh = refresh_packed(bops.o, bops, Wn + Vn, P, w, S, prm, delta_w, bound)
    return (mm.EncMat([fresh[:n]], W.rows, W.cols, W.s0, W.s1), mm.EncMat([fresh[n:]], W.rows, W.cols, W.s0, W.s1))


class ValidationClient:
    """The client of Protocol 1, step 3(c)-(d), on the oracle: decrypts the validation logits
    (row blocks of s0 rows), takes the cross-entropy of the softmax over the c_real classes
    against the labels, and answers (stop, improved): improved when the loss is below every
    earlier epoch's, stop once it has not improved for `patience` epochs in a row."""

    def __init__(self, o, labels, c_real, patience=3):
        self.o, self.labels, self.c_real, self.patience = o, np.asarray(labels), c_real, patience
        self.best, self.bad, self.losses = math.inf, 0, []

    def __call__(self, logits):
        rows = [self.o.decrypt_slots(row[0]).real.reshape(logits.s0, logits.s1) for row in logits.blocks]
        z = np.concatenate(rows)[:len(self.labels), :self.c_real]
        z = z - z.max(axis=1, keepdims=True)
        logp = z - np.log(np.sum(np.exp(z), axis=1, keepdims=True))
        loss = float(-np.mean(logp[np.arange(len(self.labels)), self.labels]))
        self.losses.append(loss)
        improved = loss < self.best
        if improved:
            self.best, self.bad = loss, 0
        else:
            self.bad += 1
        return self.bad >= self.patience, improved


def train_epochs(ops, bops, Wbar, grads, Xval, c, target_scale, max_epochs, client, prm, delta_w, vops=None,
                 w_bound=1.0):
    """Protocol 1, step 3 (reading P1): for each epoch, one NAG update per mini-batch in order
    (grads[b](V) gives batch b's gradient at about target_scale), gamma_t running on across
    batches and epochs; after each epoch the validation logits DiagABT(X_val, W, t = 1) (on
    vops, default ops) go to client(logits) -> (stop, improved); the W of an improved epoch is
    the best weight W*.  Stops after max_epochs or when the client says so.  w_bound bounds
    the entries of W and V for their refreshes.  Returns (W*, epochs run)."""
    from . import matmul as mm
    S = target_scale
    assert Wbar.blocks[0][0].scale == S
    P, w = c * Wbar.s1, Wbar.s0 // c
    gammas = mm.nag_gammas(max_epochs * len(grads))
    W = V = best = Wbar
    t = 0
    for epoch in range(max_epochs):
        for grad in grads:
            W, V = nag_update_refresh(ops, bops, W, V, grad(V), gammas[t], S, prm, delta_w, P, w, w_bound)
            t += 1
        stop, improved = client(mm.diag_abt(vops or ops, Xval, W, c, 1.0))
        if improved:
            best = W
        if stop:
            break
    return best, epoch + 1
