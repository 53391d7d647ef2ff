"""CKKS bootstrapping (Sec. 2.2) on the GPU, as a sequence of C-ABI calls: a level-0
matrix becomes one at a high level that decrypts to the same message.

Every homomorphic step runs in the library's kernels (ModRaise, rotations, conjugation,
plaintext and ciphertext products); this module orders them (through circuit.Circuit).
The procedure is the full-slot one of Cheon, Han, Kim, Kim and Song:

  ModRaise     residues mod q_0, centred, reduced modulo every prime of the top level:
               a ciphertext of t = Delta m + e + q_0 I (I small), read at scale q_0.
  CoeffToSlot  with U the canonical embedding of the first N/2 coefficients (U[j][k] =
               zeta^(5^j k)) and U^-1 = (2/N) U^H: v = (1/N) U^H z, then v + conj(v) and
               i (conj(v) - v) carry the coefficients t_k / q_0 = I_k + eps_k as slots.
  EvalMod      sin(2 pi x) / (2 pi) ~ eps: cos(2 pi (x - 1/4) / 2^r) by its Taylor
               polynomial (degree 28, in w = theta^2 / W), then r double-angle steps.
  SlotToCoeff  U (lo + i hi): sigma(Delta m + e) / q_0, read at working scale *
               Delta / q_0 to give m back.

Both transforms are products of log2(N/2) butterfly stages (the special FFT of the
canonical embedding), merged a few stages per level into matrices of at most 2^(k+1) - 1 diagonals
(k stages a level)
whose rotations share one ModUp; the bit-reversal permutation between them is never
applied, EvalMod being slot-wise.  A dense form (N/2 diagonals, baby-step / giant-step) is
kept as an option (fft=False).  The rotation keys needed are rotations(N).  Every addition inside EvalMod meets
two scales equal to the last bit or two (each polynomial part is aimed at the scale of the
term it joins), because the double-angle steps amplify any error 4^r times.
"""
import functools
import math
from dataclasses import dataclass

import numpy as np

from . import hetal as H
from .circuit import Circuit


@dataclass
class BootstrapParams:
    K: float = 24.5     # EvalMod's range: |I| <= 24 (about 6 standard deviations for h = 192)
    r: int = 5          # double-angle steps
    taylor: int = 14    # cos(theta) by its Taylor polynomial of degree 2 * taylor
    n1: int = 0         # baby steps of the dense transforms (0: the power of two nearest sqrt(N/2))
    fft: bool = True    # factored transforms (a few levels, 2^(per_level+1) - 1 diagonals each) instead of dense
    per_level: int = 3  # FFT stages merged into one level (3: the fastest of 2-5 measured at N = 2^16)


def transform_levels(N, prm=None):
    """Levels of one transform: 1 dense; ceil(log2(N/2) / per_level) factored."""
    prm = prm or BootstrapParams()
    if not prm.fft:
        return 1
    stages = (N // 2).bit_length() - 1
    return -(-stages // prm.per_level)


def levels(N, prm=None):
    """Levels consumed: CoeffToSlot; EvalMod: theta 1, w 1, the polynomial 5, r steps, the
    1 / 2 pi product 1; SlotToCoeff."""
    prm = prm or BootstrapParams()
    t = transform_levels(N, prm)
    return t + (1 + 1 + 5 + prm.r + 1) + t


def _baby(n, prm):
    return prm.n1 or 1 << int(round(math.log2(n) / 2))


def rotations(N, prm=None):
    """The slot rotations both transforms use (the keys bootstrap() needs besides Conj)."""
    prm = prm or BootstrapParams()
    n = N // 2
    if prm.fft:
        out = set()
        for inverse in (True, False):
            for M in _factored(N, inverse, prm.per_level):
                out |= {r for r in M if r}
        return sorted(out)
    n1 = _baby(n, prm)
    return sorted(set(range(1, n1)) | {n1 * g for g in range(1, n // n1)})


def _exponents(N):
    """5^j mod 2N for j < N/2: slot j of a plaintext is its value at zeta^(5^j)."""
    n = N // 2
    e = np.empty(n, dtype=np.int64)
    acc = 1
    for j in range(n):
        e[j] = acc
        acc = acc * 5 % (2 * N)
    return e


def embedding_diagonal(N, k, inverse):
    """Diagonal k (entries [j][j+k mod n]) of U, U[j][l] = zeta^(5^j l), zeta = exp(i pi / N);
    with inverse, of (1/N) U^H = U^-1 / 2, whose entry [j][l] is zeta^(-5^l j) / N.  Computed
    one diagonal at a time, so a transform never holds the n x n matrix."""
    n, N2 = N // 2, 2 * N
    e = _exponents(N)
    j = np.arange(n, dtype=np.int64)
    l = (j + k) % n
    if inverse:
        return np.exp(-1j * np.pi * ((e[l] * j) % N2) / N) / N
    return np.exp(1j * np.pi * ((e[j] * l) % N2) / N)


def _matvec(C, x, N, inverse, name, scale, prm):
    """M z for a ciphertext x of z, M = U or (1/N) U^H: the sum over giant steps g of
    Rot_{n1 g} of the sum over baby steps i of (d_{i + n1 g} rotated right by n1 g) (.)
    Rot_i(x), d_k the k-th diagonal; the n1 - 1 baby rotations share one ModUp, and each
    giant step's products are summed before one rescale."""
    n = N // 2
    n1 = _baby(n, prm)
    babies = [x] + C.rot_many(x, list(range(1, n1)))
    total = None
    for g in range(n // n1):
        part = C.cmult_scaled_sum([(babies[i], np.roll(embedding_diagonal(N, i + n1 * g, inverse), n1 * g), name,
                                    i + n1 * g) for i in range(n1)], scale)
        if g:
            part = C.rot(part, n1 * g)
        total = part if total is None else C.add(total, part)
    return total


# Factored transforms: U = S_L ... S_1 P, P the bit-reversal permutation and S_s (block
# 2^s, half h = 2^(s-1)) the butterfly (v[p], v[p+h]) -> (v[p] + xi v[p+h], v[p] - xi v[p+h])
# for p in each block's first half, j = p mod 2^s, xi = zeta^((5^j mod 2^(s+2)) N / 2^(s+1)).
# A stage is three diagonals (offsets 0, +h, -h).  CoeffToSlot applies S_L^-1 .. S_1^-1 (with
# the 1/2 of the real / imaginary split) and never P^-1, SlotToCoeff S_1 .. S_L: EvalMod is
# slot-wise, so the bit-reversed order in between needs no permutation.  Consecutive stages
# are merged per level; a matrix is {offset r: d_r}, x -> sum_r d_r (.) Lrot(x, r).
def _butterfly_stage(N, s, inverse):
    n = N // 2
    blk, h = 1 << s, 1 << (s - 1)
    e = _exponents(N)
    p = np.arange(n)
    j = p % blk
    lower = j < h
    jl = np.where(lower, j, j - h)
    xi = np.exp(1j * np.pi * ((e[jl] % (4 * blk)) * (N // (2 * blk))) / N)
    if inverse:
        parts = [(0, np.where(lower, 0.5, -0.5 / xi)), (h, np.where(lower, 0.5, 0)),
                 (n - h, np.where(lower, 0, 0.5 / xi))]
    else:
        parts = [(0, np.where(lower, 1.0, -xi)), (h, np.where(lower, xi, 0)), (n - h, np.where(lower, 0, 1.0))]
    M = {}
    for r, d in parts:
        M[r % n] = M.get(r % n, 0) + d
    return M


def _after(A, B, n):
    """A applied after B: offset a + b collects d^A_a (.) (d^B_b shifted left by a)."""
    out = {}
    for a, da in A.items():
        for b, db in B.items():
            r = (a + b) % n
            out[r] = out.get(r, 0) + da * np.roll(db, -a)
    return out


@functools.lru_cache(maxsize=16)
def _factored(N, inverse, per_level):
    """The level matrices (built once per ring degree; callers only read them)."""
    n = N // 2
    stages = n.bit_length() - 1
    seq = list(range(stages, 0, -1)) if inverse else list(range(1, stages + 1))
    nlev = -(-stages // per_level)
    mats, first = [], 0
    for li in range(nlev):
        count = stages // nlev + (1 if li < stages % nlev else 0)   # as even as can be
        M = {0: np.full(n, 0.5 if (inverse and li == 0) else 1.0, dtype=complex)}
        for s in seq[first:first + count]:
            M = _after(_butterfly_stage(N, s, inverse), M, n)
        first += count
        mats.append({r: d for r, d in M.items() if np.max(np.abs(d)) > 0})
    return mats


def _apply(C, x, M, name, scale):
    """sum_r d_r (.) Lrot(x, r), the rotations hoisted, the products summed before one
    rescale that lands on `scale`."""
    offs = sorted(M)
    moved = [r for r in offs if r]
    rot = dict(zip(moved, C.rot_many(x, moved))) if moved else {}
    rot[0] = x
    return C.cmult_scaled_sum([(rot[r], M[r], name, r) for r in offs], scale)


def _affine(C, pw, cf, name, base, scale):
    """cf[0] + cf[1] pw[1] + cf[2] pw[2] + cf[3] pw[3], each product landing on `scale`."""
    ones = np.ones(C.slots)
    acc = None
    for r in (1, 2, 3):
        term = C.cmult_scaled(pw[r], cf[r] * ones, name, base + r, scale)
        acc = term if acc is None else C.add(acc, term)
    return C.add_plain(acc, cf[0] * ones, name, base)


def _cos_series(C, w, cf, name, target):
    """sum_k cf[k] w^k, k <= 15, as (u0 + u1 w^4) + (u2 + u3 w^4) w^8 with matched scales."""
    cf = list(cf) + [0.0] * (16 - len(cf))
    w2 = C.mult_to(w, w, target)
    w3 = C.mult_to(w2, w, target)
    w4 = C.mult_to(w2, w2, target)
    w8 = C.mult_to(w4, w4, target)
    pw = (None, w, w2, w3)
    u3 = _affine(C, pw, cf[12:16], name, 12, target)
    p3 = C.mult_to(u3, w4, target)
    u2 = _affine(C, pw, cf[8:12], name, 8, p3.scale)
    high = C.mult_to(C.add(u2, p3), w8, target)
    s1 = C.operand_scale_for(w3.lv - 1, w4, high.scale, target)
    u1 = _affine(C, pw, cf[4:8], name, 4, s1)
    p1 = C.mult_to(u1, w4, high.scale)
    u0 = _affine(C, pw, cf[0:4], name, 0, p1.scale)
    return C.add(C.add(u0, p1), high)


def _eval_mod(C, x, prm, target):
    ones = np.ones(C.slots)
    W = (2 * math.pi * (prm.K + 0.25) / 2 ** prm.r) ** 2
    shifted = C.add_plain(x, -0.25 * ones, "em_shift", 0)
    theta = C.cmult(shifted, 2 * math.pi / 2 ** prm.r / math.sqrt(W) * ones, "em_theta", 0)
    w = C.mult_to(theta, theta, target)
    cos = _cos_series(C, w, [(-1) ** k * W ** k / math.factorial(2 * k) for k in range(prm.taylor + 1)],
                      "em_cos", target)
    for j in range(prm.r):
        cos = C.add_plain(C.mul_int(C.mult_to(cos, cos, target), 2), -ones, "em_double", j)
    return C.cmult(cos, ones / (2 * math.pi), "em_out", 0)


class Refresher:
    """The refresh behind circuit.Circuit.keep, for circuits that run at the circuit's scale
    on the levels below a chain's bootstrapping primes.  A ciphertext a (level >= 1,
    |message| <= bound) becomes:
      1. a times the integer 2^k, read at exactly delta_in (2^k scale(a) is delta_in up to
         the rounding of a's scale, below 2^-16): the scale bootstrapping expects;
      2. times 1 / bound (one level), landing on delta_in: the message bootstrapped is
         m / bound, in [-1, 1];
      3. bootstrapped (bootstrap) and read at its message's scale divided by bound (the
         message is m again);
      4. times 1 (one level), landing on exactly the circuit's scale.
    bound is rounded up to a power of two 2^e; the plaintexts are named ("refresh_in",
    e + 64) and ("refresh_out", e + 64) at their levels, in the circuit's plaintexts;
    pts / cache are bootstrapping's (bootstrap).

    pair() refreshes two values whose slots repeat every P slots within each aligned run of
    2P slots (a row of 2P or more slots tiled with period P; the values may differ from
    row to row) with one bootstrapping: value j in the windows {t : (t // P) mod 2 = j},
    each times its own 1 / bound in step 2 (one summed product); after bootstrapping,
    value j is read at its own bound, masked to its windows (step 4's product) and copied
    into the other window of its run: value 0 by one rotation right by P, value 1 left.
    The plaintexts are named ("refresh_in_p<P>_w<j>", e + 64) and
    ("refresh_out_p<P>_w<j>", e + 64)."""

    def __init__(self, prm=None, delta_w=2.0 ** 55, delta_in=2.0 ** 50, pts=None, cache=None):
        self.prm, self.delta_w, self.delta_in = prm, float(delta_w), float(delta_in)
        self.pts, self.cache = pts, cache
        self.calls = 0

    def _pre(self, C, a):
        """Step 1: times 2^k, read at exactly delta_in."""
        k = int(round(math.log2(self.delta_in / a.scale)))
        if k < 0 or a.lv < 1:
            raise ValueError("a refresh needs one level and a scale at most delta_in")
        if k:
            a = C.mul_int(a, 1 << k)
        if abs(a.scale * 2.0 ** k / self.delta_in - 1.0) > 2.0 ** -16:
            raise ValueError("the scale is not a power of two times delta_in, rounded")
        return C.read_at(a, self.delta_in)

    def _boot(self, C, x):
        """Step 3's bootstrapping of a ciphertext at delta_in (read at its message's scale)."""
        x0 = C.wrap(H.hetal_mat_drop(C.ctx, x.h, 0))
        self.calls += 1
        return C.wrap(bootstrap(C.ctx, C.evk, x0.h, x0.scale, self.delta_w, self.prm, pts=self.pts, cache=self.cache))

    def __call__(self, C, a, bound):
        e = int(math.ceil(math.log2(bound)))
        bound, idx = 2.0 ** e, e + 64
        ones = np.ones(C.slots)
        x = C.cmult_scaled(self._pre(C, a), ones / bound, "refresh_in", idx, self.delta_in)
        b = self._boot(C, x)
        r = C.read_at(b, b.scale / bound)
        return C.cmult_scaled(r, ones, "refresh_out", idx, C.delta)

    def pair(self, C, a, bound_a, b, bound_b, P):
        t = np.arange(C.slots)
        win = [((t // P) % 2 == j).astype(np.float64) for j in (0, 1)]
        es = [int(math.ceil(math.log2(bd))) for bd in (bound_a, bound_b)]
        xs = [self._pre(C, a), self._pre(C, b)]
        lv = min(x.lv for x in xs)
        xs = [x if x.lv == lv else C.wrap(H.hetal_mat_drop(C.ctx, x.h, lv)) for x in xs]
        x = C.cmult_scaled_sum([(xs[j], win[j] / 2.0 ** es[j], "refresh_in_p%d_w%d" % (P, j), es[j] + 64)
                                for j in (0, 1)], self.delta_in)
        boot = self._boot(C, x)
        out = []
        for j in (0, 1):
            r = C.read_at(boot, boot.scale / 2.0 ** es[j])
            v = C.cmult_scaled(r, win[j], "refresh_out_p%d_w%d" % (P, j), es[j] + 64, C.delta)
            out.append(C.add(v, C.rot(v, -P if j == 0 else P)))
        return out


def bootstrap(ctx, evk, a, delta_in, delta_w=2.0 ** 55, prm=None, pts=None, record=None, cache=None):
    """Refreshes a level-0 matrix `a` (every block at scale delta_in, messages of modulus
    below about q_0 / (2 delta_in)): returns a new handle at level top - levels(N, prm)
    holding the same messages at scale about delta_w * delta_in / q_0.  evk must hold the
    conjugation key and the rotations(N) keys; `a` is left as it is.  pts / record / cache:
    the plaintexts to use, a dict to keep the ones encoded, a dict of device plaintexts
    reused across calls (circuit.Circuit)."""
    prm = prm or BootstrapParams()
    N, L, _ = H.hetal_ctx_info(ctx)
    d = H.hetal_mat_desc_get(a)
    if d.level != 0:
        raise ValueError("bootstrapping takes a level-0 matrix")
    if L - 1 < levels(N, prm) + 1:
        raise ValueError("the chain needs more than %d levels" % levels(N, prm))
    C = Circuit(ctx, evk, delta_w, pts, record, cache)
    try:
        # the intermediates are locals of _run, released as it returns (before close)
        return _run(C, a, N, L, delta_in, delta_w, prm).detach()
    finally:
        C.close()


def _run(C, a, N, L, delta_in, delta_w, prm):
    q0 = float(C.q[0])
    raised = C.mod_raise(C.adopt(a), L - 1)
    if prm.fft:
        v = raised
        for li, M in enumerate(_factored(N, True, prm.per_level)):
            v = _apply(C, v, M, "cts%d" % li, delta_w)
    else:
        v = _matvec(C, raised, N, True, "cts", delta_w, prm)
    vc = C.conj(v)
    lo = _eval_mod(C, C.add(v, vc), prm, delta_w)
    hi = _eval_mod(C, C.mul_i(C.sub(vc, v)), prm, delta_w)
    u = C.add(lo, C.mul_i(hi))
    if prm.fft:
        for li, M in enumerate(_factored(N, False, prm.per_level)):
            u = _apply(C, u, M, "stc%d" % li, delta_w)
    else:
        u = _matvec(C, u, N, False, "stc", delta_w, prm)
    return C.read_at(u, u.scale * delta_in / q0)
