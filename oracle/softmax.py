"""Algorithm ASoftmax (App. A): the paper's row-wise softmax approximation of a
block-encoded matrix tiled horizontally, on the oracle's slot operations.

TEST INFRASTRUCTURE ONLY.  Only the test-suite (and the CPU leg of the benchmark)
may import this module; the product path never does.  It shares no code with
the CUDA library.

ASoftmax = p o D_n o Norm (Sec. 4.1 and App. A):
  Norm   subtract an approximate row maximum Amax, computed by a tournament over
         the c' = 2^ceil(log2 c) columns with the comparison
         Acomp(a, b) = (f(g(g(a - b))) + 1) / 2 of Cheon et al. (f and g the odd
         degree-7 polynomials printed in App. A), on inputs scaled into [-1/2, 1/2];
  D_n    the domain-extension polynomial: n times x <- L^i B(x / L^i),
         B(x) = x - 4 x^3 / (27 R^2), for i = n-1 .. 0, mapping [-L^n R, L^n R]
         into [-R, R]; with `precise`, then B_inv (the printed degree-5 correction);
  p      exp then the normalisation by the row sum: AExp and AInv.

Readings of the printed algorithm, where it is garbled or silent (each one a
choice, stated where it is made below):
  A1  M_max starts as M' (the listing uses it before it is set).
  A2  Loop bounds "0 to log2 x" are exclusive (j < log2 x).
  A3  The maximum's broadcast adds Rrot(M_max, 2^j) for j < log2 s1 (within a row:
      the column-0 maximum is copied to every column, as SumCols does); the
      printed amount 2^i * s1 would move whole rows.
  A4  RS(M_exp) is the row sum over the c' columns: left rotate-and-add by 2^j
      (j < log2 c') puts it in column 0 of each row, which is kept (D_firstcol)
      and broadcast like A3; then M_sm = M_exp (.) AInv(expsum) (the listing's
      M_expsum (.) M_Z is the sum times its own inverse) is already tiled
      horizontally, so the final re-tiling loop is an identity and is left out.
  A5  Two ranges named R in the listing: R_orig = 4, the inputs the softmax covers
      without extension ([-4, 4]^c, App. A.3), gives R_max = ceil(R_orig L^n) = 128
      (L = 2, n = 5) and M' = M / (2 R_max) in [-1/2, 1/2], the comparison's domain;
      the normalised inputs span twice that, so the DEP's B(x) = x - 4x^3/(27 R^2)
      and B_inv take R = 2 R_orig = 8, AExp's domain [-8, 8], and D_n maps
      [-256, 256] into [-8, 8].  With these two readings Table tab:softmaxerr's
      errors are reproduced (tests/test_oracle_softmax.py); taking R = 8 in line 1
      as well doubles them for c >= 5.
  A6  AExp and AInv follow the cited work, which is not in the paper; taken as
      AExp(x) = p_12(x / B)^B with B = 8 (three squarings), p_12 the degree-12
      least-squares (Legendre) approximation of e^t on [-1, 1]; and
      AInv(y) = (1/R) prod_{i<n} (1 + e^(2^i)), e = 1 - y / R (Goldschmidt) with
      R = 100, n = 16 (App. A.3's parameters).
  A7  D_c keeps the columns whose class (column mod c') is below c; padded
      classes start at -1/2 after scaling (line 6), so they never win the max.
  A8  B_inv adds the correction: D_n(x) = x - k x^3 + O(x^5) with the printed
      k = (4/27) L^2 (L^2n - 1) / (L^2n (L^2 - 1)) / R^2, whose inverse is x + k x^3 + ...;
      the printed leading minus would double the distortion instead of undoing it
      (and make the "precise" errors of Table tab:softmaxerr larger, not smaller).
      Taken as B_inv(x) = x + k' (x^3 / R^2 - x^5 / R^4), k' = k R^2.

On RNS-CKKS ciphertexts (ScaledOps below), two more choices the paper leaves open:
  A10 Scale through ~100 levels: the paper rescales after every product and says no
      more.  With primes that are not equal to the scale, a chain of squarings (AInv's
      e^(2^i), AExp's p^8) would multiply the scale's deviation at every step.  Taken:
      every ciphertext product aims at one scale delta, its first operand multiplied
      beforehand by the integer t = round(delta q_l / (s_a s_b)) (Oracle.mult_scaled;
      no level), so every ciphertext carries delta (1 + e), |e| <= 1 / (2t).  With
      60-bit primes and delta = 2^40, t ~ 2^20 and |e| <= 4.8e-7; an addition of two
      such ciphertexts reads the second at the first one's scale, a relative error
      of at most 1e-6 in that operand (far below the algorithm's own 1e-3).
  A11 A plaintext product keeps the scale (the plaintext is encoded at scale q_l);
      slot values above 4 in magnitude would not fit a signed 64-bit coefficient at
      q_l ~ 2^60, so such a product first multiplies the ciphertext by the integer
      2^k (no level) and then by the values / 2^k.
"""
import math
from dataclasses import dataclass

import numpy as np
from numpy.polynomial import legendre as Leg

from . import ckks

# Acomp's polynomials (App. A), power-basis coefficients of x, x^3, x^5, x^7.
F_ODD = (35.0 / 16, -35.0 / 16, 21.0 / 16, -5.0 / 16)
G_ODD = (4589.0 / 1024, -16577.0 / 1024, 25614.0 / 1024, -12860.0 / 1024)


@dataclass
class Params:
    R_orig: float = 4.0     # inputs covered without extension: [-R_orig, R_orig]^c
    L: float = 2.0          # domain extension ratio
    n: int = 5              # domain extension index
    precise: bool = False   # apply B_inv after the extension
    exp_B: int = 8          # AExp: p(x / B)^B
    exp_deg: int = 12       # AExp: degree of p
    inv_R: float = 100.0    # AInv: inputs in (0, 2 R)
    inv_n: int = 16         # AInv: Goldschmidt iterations
    # for tests that plant a mistake: the printed sign of B_inv's correction (-1), the
    # comparison's input scale 1 / (2 R_max) with R_max computed from 2 R_orig (2)
    binv_sign: float = 1.0
    cmp_range: float = 1.0

    @property
    def R_max(self):
        return math.ceil(self.cmp_range * self.R_orig * self.L ** self.n)

    @property
    def R_dep(self):
        """The DEP's R: AExp's domain, twice the inputs' (normalisation doubles the range)."""
        return 2.0 * self.R_orig


def exp_poly(deg):
    """Power-basis coefficients of the degree-`deg` least-squares approximation of e^t on
    [-1, 1]: the Legendre projection, its coefficients by 64-point Gauss-Legendre quadrature."""
    t, w = Leg.leggauss(64)
    c = [(2 * k + 1) / 2.0 * np.sum(w * np.exp(t) * Leg.legval(t, [0] * k + [1])) for k in range(deg + 1)]
    return Leg.leg2poly(np.array(c))


def _ones(ops):
    return np.ones(ops.s)


def _odd7(ops, x, coef, key):
    """c1 x + c3 x^3 + c5 x^5 + c7 x^7 = x (lo + x^4 hi), lo = c1 + c3 x^2, hi = c5 + c7 x^2."""
    one = _ones(ops)
    x2 = ops.mult(x, x)
    x4 = ops.mult(x2, x2)
    lo = ops.add_plain(ops.cmult(x2, coef[1] * one, (key, 0)), coef[0] * one, (key, 1))
    hi = ops.add_plain(ops.cmult(x2, coef[3] * one, (key, 2)), coef[2] * one, (key, 3))
    u = ops.add(lo, ops.mult(x4, hi))
    return ops.mult(x, u)


def acomp(ops, a, b):
    """Acomp(a, b) = (f(g(g(a - b))) + 1) / 2, a, b in [-1/2, 1/2] (App. A)."""
    y = ops.sub(a, b)
    for coef, key in ((G_ODD, "g1"), (G_ODD, "g2"), (F_ODD, "f")):
        y = _odd7(ops, ops.keep(y, 4, 1.0), coef, key)   # |y| <= 1: g and f map [-1, 1] into itself
    one = _ones(ops)
    y = ops.keep(y, 1, 1.0)
    return ops.add_plain(ops.cmult(y, 0.5 * one, ("half", 0)), 0.5 * one, ("half", 1))


def _poly_bsgs(ops, x, coeffs, key):
    """sum_i coeffs[i] x^i (degree <= 15): baby steps x, x^2, x^3, giant steps x^4, x^8."""
    c = list(coeffs) + [0.0] * (16 - len(coeffs))
    one = _ones(ops)
    x2 = ops.mult(x, x)
    x3 = ops.mult(x2, x)
    x4 = ops.mult(x2, x2)
    x8 = ops.mult(x4, x4)
    xs = {1: x, 2: x2, 3: x3}
    u = []
    for j in range(4):
        acc = None
        for r in range(1, 4):
            t = ops.cmult(xs[r], c[4 * j + r] * one, (key, 4 * j + r))
            acc = t if acc is None else ops.add(acc, t)
        u.append(ops.add_plain(acc, c[4 * j] * one, (key, 16 + j)))
    inner = ops.add(u[2], ops.mult(u[3], x4))
    return ops.add(ops.add(u[0], ops.mult(u[1], x4)), ops.mult(inner, x8))


def aexp(ops, x, prm):
    """AExp(x) = p(x / B)^B (reading A6)."""
    one = _ones(ops)
    y = ops.cmult(ops.keep(x, 1, prm.R_dep), one / prm.exp_B, ("exp_in", 0))
    y = _poly_bsgs(ops, ops.keep(y, 5, 1.0), exp_poly(prm.exp_deg), "exp")
    for _ in range(int(round(math.log2(prm.exp_B)))):
        y = ops.keep(y, 1, 2.0)   # p(x / B) ~ e^(x / B) <= 1 for the normalised x <= 0
        y = ops.mult(y, y)
    return y


# the Goldschmidt product tends to R / y <= R = 100 for row sums y >= 1
INV_ACC_BOUND = 128.0


def ainv(ops, y, prm, layout=(1, 1)):
    """AInv(y) = (1/R) prod_{i<n} (1 + e^(2^i)), e = 1 - y/R (Goldschmidt, reading A6).
    layout: (period of the slots, slots per row) for keep2."""
    one = _ones(ops)
    e = ops.add_plain(ops.cmult(y, -one / prm.inv_R, ("inv_in", 0)), one, ("inv_in", 1))
    a = ops.add_plain(e, one, ("inv_in", 2))
    for i in range(1, prm.inv_n):
        e, a = ops.keep2(e, 2, 1.0, a, 1, INV_ACC_BOUND, *layout)   # e = 1 - y / R in (0, 1)
        e = ops.mult(e, e)
        a = ops.mult(a, ops.add_plain(e, one, ("inv_step", i)))
    a = ops.keep(a, 1, INV_ACC_BOUND)
    return ops.cmult(a, one / prm.inv_R, ("inv_out", 0))


def _mask(s0, s1, fn):
    i = np.arange(s0)[:, None]
    j = np.arange(s1)[None, :]
    return np.broadcast_to(fn(i, j), (s0, s1)).astype(np.float64).reshape(-1)


def asoftmax_block(ops, M, c, s0, s1, prm):
    """ASoftmax of one block (Algorithm ASoftmax): M holds an s0 x c matrix tiled s1/c'
    times horizontally; returns its row-wise softmax approximation in the same layout."""
    cp = 1 << max(1, math.ceil(math.log2(c)))
    one = np.ones(s0 * s1)
    Dc = _mask(s0, s1, lambda i, j: (j % cp) < c)
    first = _mask(s0, s1, lambda i, j: j == 0)
    # Refresh points (ops.keep; nothing happens without a refresher): before each run of
    # products, a value with too few levels left is bootstrapped, with the bound of its
    # message.  lines 1-7: scale into [-1/2, 1/2]; padded classes at -1/2 (reading A7)
    M = ops.keep(M, 1, prm.R_max)
    Mp = ops.cmult(M, one / (2 * prm.R_max), ("scale_in", 0))
    if c != cp:
        Mp = ops.add_plain(Mp, -0.5 * (1.0 - Dc), ("padmask", 0))
    # lines 8-13: tournament maximum over the c' columns (readings A1, A2)
    mx = Mp
    for j in range(int(math.log2(cp))):
        rot = ops.rot(mx, 1 << j)
        cmp = ops.keep(acomp(ops, mx, rot), 2, 1.0)
        mx, rot = ops.keep2(mx, 1, 1.0, rot, 1, 1.0, cp, s1)
        notc = ops.add_plain(ops.cmult(cmp, -one, ("neg", j)), one, ("one", j))
        mx = ops.add(ops.mult(mx, cmp), ops.mult(rot, notc))
    # lines 14-17: keep column 0 and copy it to every column of its row (reading A3)
    mx = ops.cmult(ops.keep(mx, 1, 1.0), first, ("firstcol", 0))
    for j in range(int(math.log2(s1))):
        mx = ops.add(mx, ops.rot(mx, -(1 << j)))
    mx = ops.cmult(ops.keep(mx, 1, 1.0), 2 * prm.R_max * one, ("scale_out", 0))
    # line 18: normalise, padded classes to 0
    M, mx = ops.keep2(M, 1, prm.R_max, mx, 1, prm.R_max, cp, s1)
    x = ops.cmult(ops.sub(M, mx), Dc, ("dc", 0))
    # lines 19-22: domain extension, i = n-1 .. 0
    kB = 4.0 / (27.0 * prm.R_dep ** 2)
    for i in range(prm.n - 1, -1, -1):
        Li = prm.L ** i
        x = ops.keep(x, 5, prm.R_dep * prm.L ** (i + 1))        # |x| <= R L^(i+1) before round i
        y = ops.cmult(x, one / Li, ("dep_in", i))                 # x / L^i
        y3 = ops.mult(ops.mult(y, y), y)
        b = ops.sub(y, ops.cmult(y3, kB * one, ("dep_k", i)))     # B(x / L^i)
        x = ops.cmult(b, Li * one, ("dep_out", i))                 # L^i B(.)
    # lines 23-26: precise inverse of the extension
    if prm.precise:
        L2, L2n = prm.L ** 2, prm.L ** (2 * prm.n)
        kk = 4.0 / 27.0 * L2 * (L2n - 1) / (L2n * (L2 - 1))
        x = ops.keep(x, 4, prm.R_dep)
        x2 = ops.mult(x, x)
        x3 = ops.mult(x2, x)
        x5 = ops.mult(x3, x2)
        t3 = ops.cmult(x3, prm.binv_sign * kk / prm.R_dep ** 2 * one, ("binv", 3))
        t5 = ops.cmult(x5, prm.binv_sign * kk / prm.R_dep ** 4 * one, ("binv", 5))
        x = ops.sub(ops.add(x, t3), t5)   # reading A8: the correction adds k x^3
    # lines 27-31: exp, padded classes to 0, row sums, inverse (reading A4)
    e = ops.cmult(ops.keep(aexp(ops, x, prm), 1, 2.0), Dc, ("dc", 1))
    sm = e
    for j in range(int(math.log2(cp))):
        sm = ops.add(sm, ops.rot(sm, 1 << j))
    sm = ops.cmult(ops.keep(sm, 1, 2.0 * cp), first, ("firstcol", 1))
    for j in range(int(math.log2(s1))):
        sm = ops.add(sm, ops.rot(sm, -(1 << j)))
    inv = ainv(ops, ops.keep(sm, 1, 2.0 * cp), prm, (cp, s1))
    e, inv = ops.keep2(e, 1, 2.0, inv, 1, 2.0, cp, s1)
    return ops.mult(e, inv)


class ScaledOps:
    """The oracle's RNS-CKKS operations (oracle/matmul.py's RnsOps) with the scale held
    at delta (readings A10, A11): ciphertext products through Oracle.mult_scaled,
    plaintext products with values above 4 split into an integer power of two and the
    rest.  Encoded plaintexts are logged in self.pts under (name, index, level) like
    RnsOps's."""

    CMULT_MAX = 4.0
    RELABEL_MAX = 2.0 ** -16

    def __init__(self, oracle, delta, hoist=False):
        from . import matmul as mm
        self.rns = mm.RnsOps(oracle, hoist=hoist)
        self.o = oracle
        self.s = oracle.p.slots
        self.delta = float(delta)
        self.pts = self.rns.pts
        self.counts = {"Mult": 0, "CMult": 0, "Rot": 0}
        self.refresh = None   # (ciphertext, bound) -> its bootstrapped copy (bootstrap.Refresher)

    def keep(self, a, need, bound):
        """A refresh point: a itself while it holds more than `need` levels (the products
        before the value's next refresh point), else, with a refresher, its bootstrapped
        copy; bound is a power of two with |message| <= bound."""
        if a.lv > need or self.refresh is None:
            return a
        return self.refresh(a, bound)

    def keep2(self, a, need_a, bound_a, b, need_b, bound_b, period, slots_per_row):
        """keep() of two values; when both need a refresh and their slots repeat every
        `period` slots with room for two windows in a row, one bootstrapping serves both
        (Refresher.pair)."""
        if (a.lv <= need_a and b.lv <= need_b and self.refresh is not None
                and slots_per_row >= 2 * period and hasattr(self.refresh, "pair")):
            return tuple(self.refresh.pair(a, bound_a, b, bound_b, period))
        return self.keep(a, need_a, bound_a), self.keep(b, need_b, bound_b)

    def level(self, a):
        return a.lv

    def _match(self, a, b):
        """b read at a's scale when the two differ by more than the additions allow
        (reading A10: at most the rounding of the products' integer factors)."""
        if abs(a.scale / b.scale - 1.0) > 1e-9:
            if abs(a.scale / b.scale - 1.0) > self.RELABEL_MAX:
                raise ValueError("scales %r and %r are not the same scale rounded" % (a.scale, b.scale))
            b = ckks.Ct(b.data, b.lv, a.scale)
        return b

    def add(self, a, b):
        return self.o.add(a, self._match(a, b))

    def sub(self, a, b):
        return self.o.sub(a, self._match(a, b))

    def mult(self, a, b):
        self.counts["Mult"] += 1
        return self.o.mult_scaled(a, b, self.delta)

    def cmult(self, a, vals, key):
        self.counts["CMult"] += 1
        big = float(np.max(np.abs(vals)))
        if big > self.CMULT_MAX:
            k = int(math.ceil(math.log2(big / self.CMULT_MAX)))
            a = self.o.mul_int(a, 1 << k)
            vals = np.asarray(vals) / float(1 << k)
        return self.rns.cmult(a, vals, key)

    def add_plain(self, a, vals, key):
        return self.rns.add_plain(a, vals, key)

    def rot(self, a, r):
        if r % self.s:
            self.counts["Rot"] += 1
        return self.rns.rot(a, r)

    # the rest of RnsOps's operations, as they are (bootstrapping's linear transforms)
    def rot_many(self, a, rs):
        self.counts["Rot"] += sum(1 for r in rs if r % self.s)
        return self.rns.rot_many(a, rs)

    def conj(self, a):
        return self.rns.conj(a)

    def mul_i(self, a):
        return self.o.mul_i(a)

    def mul_int(self, a, t):
        return self.o.mul_int(a, t)

    def mult_to(self, a, b, target):
        """A product aimed at `target` (Oracle.mult_scaled)."""
        self.counts["Mult"] += 1
        return self.o.mult_scaled(a, b, target)

    def operand_scale_for(self, lv_a, b, product_scale, target):
        """The scale s_a that makes mult_to(a, b, product_scale), a at level lv_a, land on
        product_scale to the last bit or two: s_a = product_scale q / (t s_b), t =
        round(product_scale q / (target s_b)) (so s_a is near target), q the prime of the
        level the product is rescaled at."""
        q = float(self.o.p.q[min(lv_a, b.lv)])
        t = float(ckks.round_half_away(product_scale * q / (target * b.scale)))
        return product_scale * q / (t * b.scale)

    def cmult_scaled(self, a, vals, key, target_scale):
        self.counts["CMult"] += 1
        return self.rns.cmult_scaled(a, vals, key, target_scale)

    def cmult_scaled_sum(self, terms, target_scale):
        """sum of plaintext products [(ciphertext, values, key)], all at one level and scale,
        with one rescale (Oracle.mul_plain_sum), landing on target_scale; values above 4
        first times an integer 2^k (reading A11)."""
        cts, ms = [], []
        for a, vals, key in terms:
            vals = np.asarray(vals)
            big = float(np.max(np.abs(vals)))
            if big > self.CMULT_MAX:
                k = int(math.ceil(math.log2(big / self.CMULT_MAX)))
                a = self.o.mul_int(a, 1 << k)
                vals = vals / float(1 << k)
            pt_scale = target_scale * float(self.o.p.q[a.lv]) / a.scale
            cts.append(a)
            ms.append(self.rns._encode(vals, pt_scale, key, a.lv))
        self.counts["CMult"] += len(terms)
        return self.o.mul_plain_sum(cts, ms, target_scale)


def rotation_amounts(c, s1):
    """The slot rotations Algorithm ASoftmax uses on one block (readings A2-A4), and left by
    c' where a row holds two copies (the second window of a paired refresh)."""
    cp = 1 << max(1, math.ceil(math.log2(c)))
    lefts = [1 << j for j in range(int(math.log2(cp)))] + ([cp] if 2 * cp <= s1 else [])
    rights = [-(1 << j) for j in range(int(math.log2(s1)))]
    return sorted(set(lefts + rights))


def asoftmax_rows(X, c, prm, s1=16, s0=256):
    """ASoftmax of the rows of X (rows x c, entries the softmax inputs) on the FP64 slot
    simulator: rows are packed s0 to a block, each tiled s1/c' times horizontally.
    Returns (rows x c) and the depth (levels) the algorithm consumed."""
    from . import matmul as mm
    cp = 1 << max(1, math.ceil(math.log2(c)))
    assert cp <= s1
    ops = mm.SlotOps(s0 * s1)
    out = []
    depth = None
    for r0 in range(0, X.shape[0], s0):
        blk = np.zeros((s0, cp))
        part = X[r0:r0 + s0]
        blk[:len(part), :c] = part
        z = np.tile(blk, (1, s1 // cp)).reshape(-1).astype(np.complex128)
        top = 1000
        res = asoftmax_block(ops, mm.SV(z, top), c, s0, s1, prm)
        depth = top - res.lv
        out.append(res.z.real.reshape(s0, s1)[:len(part), :c])
    return np.concatenate(out), depth


def softmax(X):
    """The exact row-wise softmax."""
    Z = X - X.max(axis=1, keepdims=True)
    E = np.exp(Z)
    return E / E.sum(axis=1, keepdims=True)
