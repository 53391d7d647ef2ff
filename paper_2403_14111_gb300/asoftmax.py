"""Algorithm ASoftmax (App. A) on encrypted blocks, as a sequence of C-ABI calls.

Every homomorphic step runs in the library's kernels; this module only orders
the calls and frees what it no longer needs.  The approximation is the paper's:

  Norm   subtract an approximate row maximum.  The maximum is a tournament over
         the c' = 2^ceil(log2 c) columns with Acomp(a, b) = (f(g(g(a - b))) + 1) / 2
         (f, g the odd degree-7 polynomials printed in App. A) on inputs scaled by
         1 / (2 R_max) into [-1/2, 1/2]; the winner of column 0 is copied to every
         column of its row.
  D_n    the domain extension: n times x <- L^i B(x / L^i), B(x) = x - 4x^3 / (27 R^2),
         i = n-1 .. 0, then (optionally, `precise`) the degree-5 correction B_inv.
  p      AExp(x) = p_12(x / 8)^8 with p_12 the degree-12 least-squares fit of e^t on
         [-1, 1], the padded classes masked to 0, the row sum over the c' columns, its
         inverse by Goldschmidt's iteration AInv(y) = (1/R) prod_i (1 + e^(2^i)),
         e = 1 - y / R, and the product with the exponentials.

The readings where the printed listing is garbled (loop bounds, which range R is
meant where, the sign of B_inv's correction, the broadcast amounts) are the same
as the test oracle's and are listed beside the paper's parameters in the design
notes.  Two choices belong to running it on RNS-CKKS through ~100 levels:

  * every ciphertext product goes through hetal_mult_scaled and aims at one scale
    `delta`; two ciphertexts whose scales differ by that rounding (at most 1e-6
    with 60-bit primes and delta = 2^40) are added after hetal_mat_set_scale reads
    the second at the first one's scale;
  * a plaintext product keeps the scale (the plaintext is encoded at scale q_l);
    slot values above 4 in magnitude would not fit a 64-bit coefficient at
    q_l ~ 2^60, so the ciphertext is first multiplied by the integer 2^k
    (hetal_mul_int, no level) and then by the values / 2^k.

Plaintexts are named (name, index, level).  By default they are encoded with the
library's FP64 encoder (hetal_encode); a caller may supply integer plaintexts
under the same names instead (`pts`), e.g. to reproduce another implementation's
encodings bit for bit.
"""
import math
from dataclasses import dataclass

import numpy as np

from . import hetal as H
from .circuit import Circuit

# App. A: Acomp's odd polynomials, coefficients of x, x^3, x^5, x^7.
G_COEF = (4589.0 / 1024, -16577.0 / 1024, 25614.0 / 1024, -12860.0 / 1024)
F_COEF = (35.0 / 16, -35.0 / 16, 21.0 / 16, -5.0 / 16)


@dataclass
class ASoftmaxParams:
    R_orig: float = 4.0   # inputs covered without extension: [-R_orig, R_orig]^c
    L: float = 2.0        # domain extension ratio
    n: int = 5            # domain extension rounds
    precise: bool = False
    exp_B: int = 8        # AExp: p(x / B)^B
    exp_deg: int = 12
    inv_R: float = 100.0  # AInv: inputs in (0, 2R)
    inv_n: int = 16       # AInv: Goldschmidt iterations

    @property
    def cmp_bound(self):
        """R_max = ceil(R_orig L^n): the comparison's inputs are M / (2 R_max)."""
        return math.ceil(self.R_orig * self.L ** self.n)

    @property
    def dep_R(self):
        """R of the extension polynomial: twice R_orig (the normalised inputs span twice the range)."""
        return 2.0 * self.R_orig


def exp_fit(deg):
    """Power-basis coefficients of the least-squares polynomial of degree `deg` for e^t on
    [-1, 1]: the orthogonal projection onto the Legendre polynomials P_0..P_deg, each
    inner product by Gauss-Legendre quadrature (exact for the polynomial part)."""
    from numpy.polynomial import legendre as lg
    nodes, weights = lg.leggauss(deg + 40)
    fx = np.exp(nodes)
    coef = np.empty(deg + 1)
    for k in range(deg + 1):
        pk = lg.Legendre.basis(k)(nodes)
        coef[k] = (k + 0.5) * float(np.dot(weights, fx * pk))
    return lg.leg2poly(coef)


def rotations(c, s1):
    """Slot rotations the algorithm needs on one block: left by 2^j (j < log2 c') for the
    tournament and the row sum, right by 2^j (j < log2 s1) for the broadcasts; and left by
    c' when a row holds two copies or more (a paired refresh copies its second window)."""
    cp = padded_classes(c)
    return sorted({1 << j for j in range(cp.bit_length() - 1)} | ({cp} if 2 * cp <= s1 else set()) |
                  {-(1 << j) for j in range(int(math.log2(s1)))})


def padded_classes(c):
    return 1 << max(1, math.ceil(math.log2(c)))


def depth(c, prm):
    """Levels one block consumes: 1 (input scaling) + 15 per tournament round (three
    odd polynomials of 4 levels, the 1/2 scaling, the complement and the selecting
    products) + 3 (column-0 mask, rescaling, class mask) + 5 per extension round
    (+4 precise) + AExp (1 + 5 + log2 B) + 2 masks + AInv (2 + inv_n) + the final
    product."""
    rounds = padded_classes(c).bit_length() - 1
    exp_d = 1 + 5 + int(round(math.log2(prm.exp_B)))
    return 1 + 15 * rounds + 3 + 5 * prm.n + (4 if prm.precise else 0) + exp_d + 2 + (2 + prm.inv_n) + 1


def _odd7(E, x, coef, name):
    """x (c1 + c3 x^2 + x^4 (c5 + c7 x^2)): three levels for the powers, one for the product with x."""
    ones = np.ones(E.slots)
    x2 = E.mult(x, x)
    x4 = E.mult(x2, x2)
    lo = E.add_plain(E.cmult(x2, coef[1] * ones, name, 0), coef[0] * ones, name, 1)
    hi = E.add_plain(E.cmult(x2, coef[3] * ones, name, 2), coef[2] * ones, name, 3)
    return E.mult(x, E.add(lo, E.mult(x4, hi)))


def _compare(E, a, b):
    """Acomp(a, b): about 1 where a > b, 0 where a < b."""
    ones = np.ones(E.slots)
    y = E.sub(a, b)
    for coef, name in ((G_COEF, "g1"), (G_COEF, "g2"), (F_COEF, "f")):
        y = _odd7(E, E.keep(y, 4, 1.0), coef, name)   # |y| <= 1: g and f map [-1, 1] into itself
    y = E.keep(y, 1, 1.0)
    return E.add_plain(E.cmult(y, 0.5 * ones, "half", 0), 0.5 * ones, "half", 1)


def _poly15(E, x, coef, name):
    """sum_k coef[k] x^k for degree <= 15: x, x^2, x^3 and x^4, x^8, four inner cubics."""
    c = list(coef) + [0.0] * (16 - len(coef))
    ones = np.ones(E.slots)
    x2 = E.mult(x, x)
    x3 = E.mult(x2, x)
    x4 = E.mult(x2, x2)
    x8 = E.mult(x4, x4)
    pw = (None, x, x2, x3)
    inner = []
    for j in range(4):
        acc = None
        for r in (1, 2, 3):
            term = E.cmult(pw[r], c[4 * j + r] * ones, name, 4 * j + r)
            acc = term if acc is None else E.add(acc, term)
        inner.append(E.add_plain(acc, c[4 * j] * ones, name, 16 + j))
    high = E.add(inner[2], E.mult(inner[3], x4))
    return E.add(E.add(inner[0], E.mult(inner[1], x4)), E.mult(high, x8))


def _exp(E, x, prm):
    ones = np.ones(E.slots)
    y = E.cmult(E.keep(x, 1, prm.dep_R), ones / prm.exp_B, "exp_in", 0)
    y = _poly15(E, E.keep(y, 5, 1.0), exp_fit(prm.exp_deg), "exp")
    for _ in range(int(round(math.log2(prm.exp_B)))):
        y = E.keep(y, 1, 2.0)   # p(x / B) ~ e^(x / B) <= 1 for the normalised x <= 0
        y = E.mult(y, y)
    return y


# the Goldschmidt product tends to R / y <= R = 100 for row sums y >= 1
INV_ACC_BOUND = 128.0


def _inverse(E, y, prm, layout=(1, 1)):
    """layout: (period of the slots, slots per row) for keep2."""
    ones = np.ones(E.slots)
    e = E.add_plain(E.cmult(y, -ones / prm.inv_R, "inv_in", 0), ones, "inv_in", 1)
    acc = E.add_plain(e, ones, "inv_in", 2)
    for i in range(1, prm.inv_n):
        e, acc = E.keep2(e, 2, 1.0, acc, 1, INV_ACC_BOUND, *layout)   # e = 1 - y / R in (0, 1)
        e = E.mult(e, e)
        acc = E.mult(acc, E.add_plain(e, ones, "inv_step", i))
    acc = E.keep(acc, 1, INV_ACC_BOUND)
    return E.cmult(acc, ones / prm.inv_R, "inv_out", 0)


def _block_mask(s0, s1, keep):
    j = np.tile(np.arange(s1), s0)
    return keep(j).astype(np.float64)


def asoftmax(ctx, evk, M, c, s0, s1, delta, prm=None, pts=None, cache=None, refresh=None):
    """Row-wise ASoftmax of encrypted blocks M (handle): each s0 x s1 block holds s0 rows
    of c softmax inputs in columns 0..c-1, tiled s1 / c' times horizontally (c' = c
    rounded up to a power of two), at scale about `delta` and at least depth(c, prm)
    levels.  evk must hold the relinearisation key and the rotations(c, s1) keys.
    Returns a new handle in the same layout; M is left as it is.  pts: integer plaintexts
    to use by name; cache: a dict of device plaintexts reused across calls (circuit.Circuit).
    refresh: a bootstrap.Refresher, with which M needs one level only and the circuit
    bootstraps values whose levels run out (M at scale delta; evk then also holds
    bootstrapping's rotations and the conjugation key)."""
    prm = prm or ASoftmaxParams()
    d = H.hetal_mat_desc_get(M)
    if d.s0 != s0 or d.s1 != s1:
        raise ValueError("block shape differs from the matrix's")
    slots = s0 * s1
    if slots != H.hetal_ctx_info(ctx)[0] // 2:
        raise ValueError("s0 * s1 must equal the slot count")
    cp = padded_classes(c)
    if cp > s1:
        raise ValueError("c' must not exceed s1")
    need = depth(c, prm) if refresh is None else 1
    if d.level < need:
        raise ValueError("ASoftmax needs %d levels, the input has %d" % (need, d.level))
    E = Circuit(ctx, evk, delta, pts, cache=cache, refresh=refresh)
    try:
        return _run(E, M, c, s0, s1, prm, cp).detach()
    finally:
        E.close()


def _run(E, M_handle, c, s0, s1, prm, cp):
    ones = np.ones(E.slots)
    real = _block_mask(s0, s1, lambda j: (j % cp) < c)   # D_c: the real classes
    col0 = _block_mask(s0, s1, lambda j: j == 0)
    M = E.adopt(M_handle)
    # Refresh points (E.keep; nothing happens without a refresher): before each run of
    # products, a value with too few levels left is bootstrapped, with the bound of its
    # message.  Scale into the comparison's domain; padded classes at -1/2 never win.
    M = E.keep(M, 1, prm.cmp_bound)
    Ms = E.cmult(M, ones / (2 * prm.cmp_bound), "scale_in", 0)
    if c != cp:
        Ms = E.add_plain(Ms, -0.5 * (1.0 - real), "padmask", 0)
    # the tournament over the c' columns
    best = Ms
    for j in range(cp.bit_length() - 1):
        other = E.rot(best, 1 << j)
        win = E.keep(_compare(E, best, other), 2, 1.0)
        best, other = E.keep2(best, 1, 1.0, other, 1, 1.0, cp, s1)
        lose = E.add_plain(E.cmult(win, -ones, "neg", j), ones, "one", j)
        best = E.add(E.mult(best, win), E.mult(other, lose))
    # column 0's maximum, copied across its row, back to the inputs' range
    best = E.cmult(E.keep(best, 1, 1.0), col0, "firstcol", 0)
    for j in range(int(math.log2(s1))):
        best = E.add(best, E.rot(best, -(1 << j)))
    best = E.cmult(E.keep(best, 1, 1.0), 2 * prm.cmp_bound * ones, "scale_out", 0)
    M, best = E.keep2(M, 1, prm.cmp_bound, best, 1, prm.cmp_bound, cp, s1)
    x = E.cmult(E.sub(M, best), real, "dc", 0)
    # the domain extension, largest ratio first
    k_b = 4.0 / (27.0 * prm.dep_R ** 2)
    for i in reversed(range(prm.n)):
        Li = prm.L ** i
        x = E.keep(x, 5, prm.dep_R * prm.L ** (i + 1))   # |x| <= R L^(i+1) before round i
        y = E.cmult(x, ones / Li, "dep_in", i)
        y3 = E.mult(E.mult(y, y), y)
        x = E.cmult(E.sub(y, E.cmult(y3, k_b * ones, "dep_k", i)), Li * ones, "dep_out", i)
    if prm.precise:
        L2, L2n = prm.L ** 2, prm.L ** (2 * prm.n)
        kk = 4.0 / 27.0 * L2 * (L2n - 1) / (L2n * (L2 - 1))
        x = E.keep(x, 4, prm.dep_R)
        x2 = E.mult(x, x)
        x3 = E.mult(x2, x)
        x5 = E.mult(x3, x2)
        t3 = E.cmult(x3, kk / prm.dep_R ** 2 * ones, "binv", 3)
        t5 = E.cmult(x5, kk / prm.dep_R ** 4 * ones, "binv", 5)
        x = E.sub(E.add(x, t3), t5)
    # exponentials, padded classes to 0, row sums broadcast, times their inverse
    ex = E.cmult(E.keep(_exp(E, x, prm), 1, 2.0), real, "dc", 1)
    tot = ex
    for j in range(cp.bit_length() - 1):
        tot = E.add(tot, E.rot(tot, 1 << j))
    tot = E.cmult(E.keep(tot, 1, 2.0 * cp), col0, "firstcol", 1)
    for j in range(int(math.log2(s1))):
        tot = E.add(tot, E.rot(tot, -(1 << j)))
    inv = _inverse(E, E.keep(tot, 1, 2.0 * cp), prm, (cp, s1))
    ex, inv = E.keep2(ex, 1, 2.0, inv, 1, 2.0, cp, s1)
    return E.mult(ex, inv)
