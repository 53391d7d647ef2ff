"""HETAL's encrypted matrix products, step by step as the paper states them,
over an abstract set of CKKS operations.

TEST INFRASTRUCTURE ONLY (see oracle/ckks.py).

Two back-ends run the same algorithm code:
  * SlotOps -- FP64 slot simulator: every ciphertext is its complex slot
    vector, Lrot is a cyclic shift.  Pinned against the FP64 matrix product
    (Props. ABT / ATB, Sec. 4.2.2-4.2.3 and App. B.2) and against the paper's
    corrected operation counts (Table "tab:matnum_fixed", App. D).
  * RnsOps  -- the plain RNS-CKKS oracle (oracle/ckks.py); produces the
    reference ciphertexts and records every plaintext it encodes, keyed by
    (kind, index, level), so that the same plaintexts can be handed to the
    CUDA library for a bit-exact comparison.

Matrix layout (Sec. 4.2.1, App. B.1): a matrix is zero-padded and cut into
s0 x s1 blocks, each stored row-major in the s = s0*s1 slots of one
ciphertext; entry (i, j) of a block is slot i*s1 + j.
"""
import math

import numpy as np

from . import ckks


# --------------------------------------------------------------------------
# Block encoding and tiling (Sec. 4.2.1, App. B.1; tilings Sec. 4.2.2, 4.2.3)
# --------------------------------------------------------------------------
def block_split(M, s0, s1):
    """Zero-pad M to multiples of (s0, s1) and cut it into row-major block slot
    vectors: blocks[r][j] is a length-s0*s1 float vector."""
    M = np.asarray(M)
    rows, cols = M.shape
    m, n = -(-rows // s0), -(-cols // s1)
    pad = np.zeros((m * s0, n * s1), dtype=M.dtype)
    pad[:rows, :cols] = M
    return [[pad[r * s0:(r + 1) * s0, j * s1:(j + 1) * s1].reshape(-1) for j in range(n)]
            for r in range(m)]


def block_join(blocks, s0, s1, rows, cols):
    m, n = len(blocks), len(blocks[0])
    out = np.zeros((m * s0, n * s1), dtype=np.asarray(blocks[0][0]).dtype)
    for r in range(m):
        for j in range(n):
            out[r * s0:(r + 1) * s0, j * s1:(j + 1) * s1] = np.asarray(blocks[r][j]).reshape(s0, s1)
    return out[:rows, :cols]


def tile_vertical(B, c, s0):
    """B-bar: s0/c copies of the c x b matrix B stacked vertically (Sec. 4.2.2).
    B is zero-padded to c rows first."""
    B = np.asarray(B)
    Bp = np.zeros((c, B.shape[1]), dtype=B.dtype)
    Bp[:B.shape[0]] = B
    return np.tile(Bp, (s0 // c, 1))


def tile_horizontal(A, c, s1):
    """A-underbar: s1/c copies of the a x c matrix A side by side (Sec. 4.2.3).
    A is zero-padded to c columns first."""
    A = np.asarray(A)
    Ap = np.zeros((A.shape[0], c), dtype=A.dtype)
    Ap[:, :A.shape[1]] = A
    return np.tile(Ap, (1, s1 // c))


def pad_pow2(x, lo=2):
    v = lo
    while v < x:
        v *= 2
    return v


# --------------------------------------------------------------------------
# Masks, as slot vectors of one s0 x s1 block
# --------------------------------------------------------------------------
def _grid(s0, s1):
    i = np.arange(s0)[:, None]
    j = np.arange(s1)[None, :]
    return i, j


def mask_offdiag(k, c, s0, s1):
    """M^{(k,c)}: 1 where j = i + k (mod c) (Prop. ABT, Sec. 4.2.2)."""
    i, j = _grid(s0, s1)
    return ((j - i - k) % c == 0).astype(np.float64).reshape(-1)


def mask_cplx(k, c, s0, s1):
    """M_cplx^{(k,c)} = 1/2 M^{(k,c)} - (sqrt(-1)/2) M^{(k+c/2,c)} (Sec. 4.2.2)."""
    return 0.5 * mask_offdiag(k, c, s0, s1) - 0.5j * mask_offdiag(k + c // 2, c, s0, s1)


def mask_col0(s0, s1):
    """Column-0 selector used inside SumCols."""
    _, j = _grid(s0, s1)
    return np.broadcast_to(j == 0, (s0, s1)).astype(np.float64).reshape(-1)


def mask_d(k, s0, s1):
    """D_k: 1 in columns j < s1 - k (Algorithms RotLeft and PRotUp, App. B.3)."""
    _, j = _grid(s0, s1)
    return np.broadcast_to(j < s1 - k, (s0, s1)).astype(np.float64).reshape(-1)


def mask_dc(k, s0, s1):
    """1 - D_k: 1 in columns j >= s1 - k.  It depends on the column only, so a
    rotation by a whole row (s1 slots) leaves it unchanged."""
    return 1.0 - mask_d(k, s0, s1)


# --------------------------------------------------------------------------
# Encrypted (or simulated) matrix: a grid of ciphertexts
# --------------------------------------------------------------------------
class EncMat:
    def __init__(self, blocks, rows, cols, s0, s1):
        self.blocks = blocks
        self.rows, self.cols = rows, cols
        self.s0, self.s1 = s0, s1

    @property
    def m(self):
        return len(self.blocks)

    @property
    def n(self):
        return len(self.blocks[0])


# --------------------------------------------------------------------------
# Back-ends
# --------------------------------------------------------------------------
class _Counted:
    def __init__(self):
        self.counts = {"CMult": 0, "Mult": 0, "Rot": 0, "Conj": 0}

    def _c(self, k, v=1):
        self.counts[k] = self.counts.get(k, 0) + v


class SV:
    """Simulated ciphertext: slot vector, level, scale."""
    __slots__ = ("z", "lv", "scale")

    def __init__(self, z, lv, scale=1.0):
        self.z, self.lv, self.scale = z, lv, scale


class SlotOps(_Counted):
    """FP64 slot simulator with the level bookkeeping of CKKS.

    by_level counts the ciphertext operations by (kind, level, group size):
    'rot', 'hoist' (one hoisted group of `size` rotations), 'mult' (`size`
    products summed before one relinearisation when lazy), 'cmult', 'conj'."""

    def __init__(self, slots, hoist=False, lazy_relin=False, radix_sum=False, shared_rot=False):
        super().__init__()
        self.s = slots
        self.hoist = hoist
        self.lazy_relin = lazy_relin
        self.radix_sum = radix_sum
        self.shared_rot = shared_rot
        self.by_level = {}

    def _rec(self, kind, lv, size=1):
        k = (kind, lv, size)
        self.by_level[k] = self.by_level.get(k, 0) + 1

    def level(self, a):
        return a.lv

    def scale(self, a):
        return a.scale

    def drop(self, a, lv):
        assert lv <= a.lv
        return SV(a.z, lv, a.scale)

    def keep(self, a, need, bound):
        """A bootstrapping refresh point (softmax.ScaledOps.keep): the simulator's levels
        never run out, so the value itself."""
        return a

    def keep2(self, a, need_a, bound_a, b, need_b, bound_b, period, slots_per_row):
        return a, b

    def add(self, a, b):
        return SV(a.z + b.z, min(a.lv, b.lv))

    def sub(self, a, b):
        return SV(a.z - b.z, min(a.lv, b.lv))

    def mul_i(self, a):
        return SV(1j * a.z, a.lv)

    def mul_int(self, a, t):
        """The message times the integer t (no level)."""
        return SV(int(t) * a.z, a.lv, a.scale)

    def cmult_scaled_sum(self, terms, target_scale):
        out = None
        for a, vals, key in terms:
            t = self.cmult_scaled(a, vals, key, target_scale)
            out = t if out is None else self.add(out, t)
        return out

    def mult_to(self, a, b, target):
        """A product that lands on `target` (scales are bookkeeping here)."""
        r = self.mult(a, b)
        return SV(r.z, r.lv, target)

    def operand_scale_for(self, lv_a, b, product_scale, target):
        return target

    def mult(self, a, b):
        self._c("Mult")
        lv = min(a.lv, b.lv)
        self._rec("mult", lv)
        return SV(a.z * b.z, lv - 1)

    def mult_sum(self, pairs):
        lv = min(min(a.lv, b.lv) for a, b in pairs)
        if not self.lazy_relin:
            out = None
            for a, b in pairs:
                r = self.mult(a, b)
                out = r if out is None else self.add(out, r)
            return out
        self._c("Mult", len(pairs))
        self._rec("mult", lv, len(pairs))
        z = sum(a.z * b.z for a, b in pairs)
        return SV(z, lv - 1)

    def cmult(self, a, vals, key):
        self._c("CMult")
        self._rec("cmult", a.lv)
        return SV(a.z * vals, a.lv - 1)

    def cmult_scaled(self, a, vals, key, target_scale):
        return self.cmult(a, vals, key)

    def cmult2(self, a, va, b, vb, keys):
        """a (.) va + b (.) vb with one rescale (a and b at one level)."""
        assert a.lv == b.lv
        self._c("CMult", 2)
        self._rec("cmult", a.lv)
        return SV(a.z * va + b.z * vb, a.lv - 1)

    def add_plain(self, a, vals, key):
        return SV(a.z + vals, a.lv)

    def mul_const(self, a, value, out_scale):
        self._c("CMult")
        self._rec("cmult", a.lv)
        return SV(a.z * value, a.lv - 1)

    def rot(self, a, r):
        r %= self.s
        if r == 0:
            return a
        self._c("Rot")
        self._rec("rot", a.lv)
        return SV(np.roll(a.z, -r), a.lv)

    def rot_many(self, a, rs):
        nz = [r for r in rs if r % self.s]
        if not self.hoist or not nz:
            return [self.rot(a, r) for r in rs]
        self._c("Rot", len(nz))
        self._rec("hoist", a.lv, len(nz))
        return [SV(np.roll(a.z, -(r % self.s)), a.lv) for r in rs]

    def rot_sum(self, a, rs):
        """a + sum_r Lrot(a, r) (rs nonzero mod s), one ModUp and one ModDown in the RNS form."""
        self._c("Rot", len(rs))
        self._rec("rotsum", a.lv, len(rs))
        z = a.z.copy()
        for r in rs:
            z = z + np.roll(a.z, -(r % self.s))
        return SV(z, a.lv, a.scale)

    def conj(self, a):
        self._c("Conj")
        self._rec("conj", a.lv)
        return SV(np.conj(a.z), a.lv)


class RnsOps(_Counted):
    """The plain RNS-CKKS oracle behind the same interface.

    Every plaintext product encodes its slot vector at the ciphertext's level;
    CMult uses scale q_lv (the prime the following rescale divides by) so that
    the ciphertext keeps its scale; cmult_scaled picks the plaintext scale that
    lands on a requested scale.  Encoded plaintexts are logged in self.pts under
    (kind, index, level).

    lazy_relin: mult_sum() adds the tensor products of several pairs and
    relinearises / rescales once.  hoist: rot_many() shares one ModUp."""

    def __init__(self, oracle, hoist=False, lazy_relin=False, radix_sum=False, shared_rot=False):
        super().__init__()
        self.o = oracle
        self.s = oracle.p.slots
        self.hoist = hoist
        self.lazy_relin = lazy_relin
        self.radix_sum = radix_sum
        self.shared_rot = shared_rot
        self.pts = {}

    def level(self, a):
        return a.lv

    def scale(self, a):
        return a.scale

    def drop(self, a, lv):
        return self.o.drop(a, lv)

    def add(self, a, b):
        return self.o.add(a, b)

    def sub(self, a, b):
        return self.o.sub(a, b)

    def mul_i(self, a):
        return self.o.mul_i(a)

    def mul_int(self, a, t):
        return self.o.mul_int(a, t)

    def mult(self, a, b):
        self._c("Mult")
        d, lv, sc = self.o.tensor(a, b)
        ct = self.o.relin(d, lv, sc)
        return self.o.rescale(ct)

    def mult_sum(self, pairs):
        if not self.lazy_relin:
            out = None
            for a, b in pairs:
                r = self.mult(a, b)
                out = r if out is None else self.add(out, r)
            return out
        self._c("Mult", len(pairs))
        lv = min(min(a.lv, b.lv) for a, b in pairs)
        acc, sc = None, None
        for a, b in pairs:
            d, _, s = self.o.tensor(self.drop(a, lv), self.drop(b, lv))
            if acc is None:
                acc, sc = d, s
            else:
                if abs(s / sc - 1) > 1e-9:
                    raise ValueError("scale mismatch in lazy sum")
                q = np.array(self.o.p.q[:lv + 1], dtype=np.uint64)[:, None]
                acc = [(x + y) % q for x, y in zip(acc, d)]
        ct = self.o.relin(acc, lv, sc)
        return self.o.rescale(ct)

    def _encode(self, vals, scale, key, lv):
        m = ckks.encode(vals, scale, self.o.p.N)
        self.pts[key + (lv,)] = m
        return m

    def cmult(self, a, vals, key):
        self._c("CMult")
        q = float(self.o.p.q[a.lv])
        m = self._encode(vals, q, key, a.lv)
        r = self.o.mul_plain_int(a, m, q)
        r.scale = a.scale
        return r

    def cmult2(self, a, va, b, vb, keys):
        self._c("CMult", 2)
        q = float(self.o.p.q[a.lv])
        ma = self._encode(va, q, keys[0], a.lv)
        mb = self._encode(vb, q, keys[1], b.lv)
        r = self.o.mul_plain2_int(a, ma, b, mb, q)
        r.scale = a.scale
        return r

    def cmult_scaled(self, a, vals, key, target_scale):
        self._c("CMult")
        pt_scale = target_scale * float(self.o.p.q[a.lv]) / a.scale
        m = self._encode(vals, pt_scale, key, a.lv)
        r = self.o.mul_plain_int(a, m, pt_scale)
        r.scale = target_scale
        return r

    def add_plain(self, a, vals, key):
        m = self._encode(vals, a.scale, key, a.lv)
        return self.o.add_plain_int(a, m)

    def mul_const(self, a, value, out_scale):
        self._c("CMult")
        return self.o.mul_const(a, value, out_scale)

    def rot(self, a, r):
        r %= self.s
        if r == 0:
            return a
        self._c("Rot")
        return self.o.rot_raw(a, r)

    def rot_many(self, a, rs):
        rs = [r % self.s for r in rs]
        if not self.hoist:
            return [self.rot(a, r) for r in rs]
        nz = [r for r in rs if r != 0]
        self._c("Rot", len(nz))
        gs = [self.o.p.galois_rot(r) for r in nz]
        outs = iter(self.o.automorph_hoisted(a, gs, [ckks.kid_rot(r) for r in nz]))
        return [a if r == 0 else next(outs) for r in rs]

    def rot_sum(self, a, rs):
        self._c("Rot", len(rs))
        return self.o.rot_sum(a, rs)

    def conj(self, a):
        self._c("Conj")
        return self.o.conj_raw(a)


# --------------------------------------------------------------------------
# Matrix helpers (Sec. 4.2.2-4.2.3, App. B.1 and B.3)
# --------------------------------------------------------------------------
def log2i(x):
    v = int(round(math.log2(x)))
    assert (1 << v) == x, x
    return v


def radix_plan(bits):
    """Split a rotate-and-sum over 2^bits positions into steps of at most 3 bits
    (radix <= 8), as evenly as possible, larger steps first: 10 -> [3, 3, 2, 2]."""
    if bits <= 0:
        return []
    steps = -(-bits // 3)
    base, extra = divmod(bits, steps)
    return [base + 1] * extra + [base] * (steps - extra)


def rot_sum_steps(ops, x, bits, unit, s, sign):
    """x summed over its rotations by sign * u * unit, u < 2^bits, in radix steps:
    x <- x + sum_{0 < j < 2^b} Lrot(x, sign * j * t * unit), t the product of the
    earlier radices.  Equal to the log-depth rotate-and-add (same sum)."""
    t = 1
    for b in radix_plan(bits):
        rs = [(sign * j * t * unit) % s for j in range(1, 1 << b)]
        x = ops.rot_sum(x, rs)
        t <<= b
    return x


def sum_cols(ops, x, s0, s1):
    """SumCols on one block: every column := the row sum.  Rotate-and-add
    by 2^u (u < log s1), keep column 0, rotate-and-add rightwards by 2^u
    (2 log s1 rotations, one CMult; Sec. 4.2.2).  With ops.radix_sum the two
    rotate-and-add chains run as radix steps (rot_sum_steps)."""
    s = s0 * s1
    if getattr(ops, "radix_sum", False):
        x = rot_sum_steps(ops, x, log2i(s1), 1, s, 1)
        x = ops.cmult(x, mask_col0(s0, s1), ("colmask", 0))
        return rot_sum_steps(ops, x, log2i(s1), 1, s, -1)
    for u in range(log2i(s1)):
        x = ops.add(x, ops.rot(x, 1 << u))
    x = ops.cmult(x, mask_col0(s0, s1), ("colmask", 0))
    for u in range(log2i(s1)):
        x = ops.add(x, ops.rot(x, s - (1 << u)))
    return x


def sum_rows(ops, x, s0, s1):
    """SumRows on one block: every row := the column sum; rotate-and-add by
    2^u * s1 for u < log s0 (log s0 rotations, no depth; Sec. 4.2.3).  With
    ops.radix_sum it runs as radix steps (rot_sum_steps)."""
    if getattr(ops, "radix_sum", False):
        return rot_sum_steps(ops, x, log2i(s0), s1, s0 * s1, 1)
    for u in range(log2i(s0)):
        x = ops.add(x, ops.rot(x, (1 << u) * s1))
    return x


def rot_left(ops, a, k, s0, s1, a1=None):
    """RotLeft(A, k) (Algorithm RotLeft): A1 = Lrot(A, k); A2 = A1 (.) D_k;
    result A2 + Rrot(A1 - A2, s1).  a1 may be passed in pre-rotated."""
    s = s0 * s1
    if a1 is None:
        a1 = ops.rot(a, k)
    a2 = ops.cmult(a1, mask_d(k, s0, s1), ("dmask", k))
    return ops.add(a2, ops.rot(ops.sub(a1, a2), s - s1))


def rot_left_shared(ops, a1, a1p, k, s0, s1):
    """RotLeft(A, k) from A1 = Lrot(A, k) and A1' = Lrot(A, k - s1) = Rrot(A1, s1):
    A1 (.) D_k + A1' (.) (1 - D_k).  Rrot(A1 - A1 (.) D_k, s1) = Rrot(A1, s1) (.)
    Rrot(1 - D_k, s1) and the complement mask is row-invariant, so this is the
    algorithm's value; both rotations are of A (one hoisted ModUp)."""
    return ops.cmult2(a1, mask_d(k, s0, s1), a1p, mask_dc(k, s0, s1), (("dmask", k), ("dmask_c", k)))


def prot_up_shared(ops, b, bu, k, s0, s1):
    """PRotUp(B, k) from B and RotUp(B, 1) = Lrot(B, s1), shared by every k:
    B (.) D_k + RotUp(B, 1) (.) (1 - D_k), the value of Algorithm PRotUp since
    RotUp(B (.) (1 - D_k), 1) = RotUp(B, 1) (.) (1 - D_k)."""
    return ops.cmult2(b, mask_d(k, s0, s1), bu, mask_dc(k, s0, s1), (("dmask", k), ("dmask_c", k)))


def prot_up(ops, b, k, s0, s1):
    """PRotUp(B, k) (Algorithm PRotUp): B' = B (.) D_k; result B' + RotUp(B - B', 1)
    with RotUp(., 1) = Lrot(., s1)."""
    b2 = ops.cmult(b, mask_d(k, s0, s1), ("dmask", k))
    return ops.add(b2, ops.rot(ops.sub(b, b2), s1))


def diag_abt(ops, A, Bbar, c, t):
    """DiagABT (Algorithm DiagABT, App. B.3): <t A Bbar^T> from <A> (m x n blocks)
    and <Bbar> (1 x n blocks).  Output: m blocks, t*A*B^T tiled s1/c times
    horizontally.  Multi-block lifting as in App. B.1: RotUp per block,
    products per block, SumCols after adding the n column blocks of a row."""
    s0, s1 = A.s0, A.s1
    h = c // 2
    if c < 2 or (c & (c - 1)) or c > s0 or c > s1:
        raise ValueError("c must be a power of two with 2 <= c <= min(s0, s1)")
    if Bbar.m != 1 or Bbar.n != A.n:
        raise ValueError("B-bar must be one block row with A's column blocks")
    m, n = A.m, A.n
    # B_cplx = Bbar + sqrt(-1) RotUp(Bbar, c/2)
    Bc = [ops.add(b, ops.mul_i(ops.rot(b, h * s1))) for b in Bbar.blocks[0]]
    BR = [ops.rot_many(b, [k * s1 for k in range(1, h)]) for b in Bc] if h > 1 else None
    X = [None] * m
    for k in range(h):
        Bk = Bc if k == 0 else [BR[j][k - 1] for j in range(n)]
        for r in range(m):
            S = ops.mult_sum([(A.blocks[r][j], Bk[j]) for j in range(n)])
            x = sum_cols(ops, S, s0, s1)
            x = ops.cmult(x, t * mask_cplx(k, c, s0, s1), ("abt_diag", k))
            X[r] = x if X[r] is None else ops.add(X[r], x)
    out = [[ops.add(x, ops.conj(x))] for x in X]
    return EncMat(out, A.rows, s1, s0, s1)


def diag_atb(ops, Au, B, c, t):
    """DiagATB (Algorithm DiagATB, App. B.3): <t A^T B> from <A-underbar>
    (m x 1 blocks, A tiled s1/c times horizontally) and <B> (m x n blocks).
    Output: n blocks, t*A^T*B tiled s0/c times vertically (the layout of
    B-bar in DiagABT).  The PRotUp branch is taken when level(A) < level(B)."""
    s0, s1 = B.s0, B.s1
    s = s0 * s1
    h = c // 2
    if c < 2 or (c & (c - 1)) or c > s0 or c > s1:
        raise ValueError("c must be a power of two with 2 <= c <= min(s0, s1)")
    if Au.n != 1 or Au.m != B.m:
        raise ValueError("A-underbar must be one block column with B's row blocks")
    m, n = B.m, B.n
    pru = ops.level(Au.blocks[0][0]) < ops.level(B.blocks[0][0])
    shared = getattr(ops, "shared_rot", False)
    # A_cplx = A + sqrt(-1) RotLeft(A, c/2)
    if shared:
        Ac = []
        for a in Au.blocks:
            a1, a1p = ops.rot_many(a[0], [h, (h - s1) % s])
            Ac.append(ops.add(a[0], ops.mul_i(rot_left_shared(ops, a1, a1p, h, s0, s1))))
    else:
        Ac = [ops.add(a[0], ops.mul_i(rot_left(ops, a[0], h, s0, s1))) for a in Au.blocks]
    extra = [(k - s1) % s for k in range(1, h)] if (shared and not pru) else []
    AR = [ops.rot_many(a, list(range(1, h)) + extra) for a in Ac] if h > 1 else None
    BU = [[ops.rot(b, s1) for b in row] for row in B.blocks] if (shared and pru and h > 1) else None
    if not pru and h > 1:
        # RotLeft(A_cplx, k >= 1) sits one level below A_cplx; bring the k = 0
        # term down too so that all c/2 products share one rescale prime.
        Ac0 = [ops.drop(a, ops.level(a) - 1) for a in Ac]
    else:
        Ac0 = Ac
    X = [None] * n
    for k in range(h):
        if pru:
            Ak = Ac if k == 0 else [AR[r][k - 1] for r in range(m)]
            if k == 0:
                Bk = B.blocks
            elif shared:
                Bk = [[prot_up_shared(ops, b, bu, k, s0, s1) for b, bu in zip(row, urow)]
                      for row, urow in zip(B.blocks, BU)]
            else:
                Bk = [[prot_up(ops, b, k, s0, s1) for b in row] for row in B.blocks]
        else:
            if k == 0:
                Ak = Ac0
            elif shared:
                Ak = [rot_left_shared(ops, AR[r][k - 1], AR[r][h - 1 + k - 1], k, s0, s1) for r in range(m)]
            else:
                Ak = [rot_left(ops, Ac[r], k, s0, s1, a1=AR[r][k - 1]) for r in range(m)]
            Bk = B.blocks
        for j in range(n):
            S = ops.mult_sum([(Ak[r], Bk[r][j]) for r in range(m)])
            x = sum_rows(ops, S, s0, s1)
            x = ops.cmult(x, t * mask_cplx(-k, c, s0, s1), ("atb_diag", k))
            X[j] = x if X[j] is None else ops.add(X[j], x)
    out = [[ops.add(x, ops.conj(x)) for x in X]]
    return EncMat(out, s0, B.cols, s0, s1)


# --------------------------------------------------------------------------
# Softmax stand-in for the training-step workload: an elementwise degree-15
# polynomial (power basis, coefficients given) times a 0/1 validity mask,
# evaluated baby-step / giant-step with depth 5 and exact scale bookkeeping.
# (The paper's ASoftmax, Algorithm ASoftmax in App. A, is not this.)
# --------------------------------------------------------------------------
def poly15_masked(ops, x, coeffs, valid, target_scale):
    """p(x) (.) v with p(x) = sum_{i<16} coeffs[i] x^i:
      x2 = x*x, x3 = x2*x, x4 = x2*x2, x8 = x4*x4,
      u_j = c_{4j} v + sum_{r=1..3} c_{4j+r} v (.) x^r          (j = 0..3)
      p   = u_0 + u_1*x4 + (u_2 + u_3*x4) * x8.
    Plaintext scales are chosen so that every term lands on target_scale."""
    assert len(coeffs) == 16
    x2 = ops.mult(x, x)
    x3 = ops.mult(x2, x)
    x4 = ops.mult(x2, x2)
    x8 = ops.mult(x4, x4)
    xs = {1: x, 2: x2, 3: x3}
    lu = ops.level(x) - 3                    # level of every u_j
    p = getattr(ops, "o", None)
    if p is not None:
        qs = p.p.q
        s4, s8 = ops.scale(x4), ops.scale(x8)
        S0 = target_scale
        S1 = target_scale * qs[lu] / s4
        S2 = target_scale * qs[lu - 1] / s8
        S3 = S2 * qs[lu] / s4
    else:
        S0 = S1 = S2 = S3 = 1.0
    S = [S0, S1, S2, S3]
    u = []
    for j in range(4):
        acc = None
        for r in range(1, 4):
            term = ops.cmult_scaled(xs[r], coeffs[4 * j + r] * valid, ("sm_coef", 4 * j + r), S[j])
            term = ops.drop(term, lu)
            acc = term if acc is None else ops.add(acc, term)
        acc = ops.add_plain(acc, coeffs[4 * j] * valid, ("sm_const", j))
        u.append(acc)
    inner = ops.add(u[2], ops.mult(u[3], x4))
    outer = ops.mult(inner, x8)
    low = ops.add(u[0], ops.mult(u[1], x4))
    return ops.add(low, outer)


def train_step(ops, X, Wbar, Y, coeffs, valid, c, lr_over_n, target_scale):
    """One encrypted softmax-regression step (Protocol 1, step 3(a), without the
    NAG update): logits/8 = DiagABT(X, Wbar, 1/8); P = p15(logits/8) (.) valid;
    D = P - Y; G = DiagATB(D, X brought to level(D)+1, lr/N) (PRotUp branch)."""
    logits = diag_abt(ops, X, Wbar, c, 1.0 / 8.0)
    P = [[poly15_masked(ops, logits.blocks[r][0], coeffs, valid, target_scale)] for r in range(logits.m)]
    D = [[ops.sub(P[r][0], Y.blocks[r][0])] for r in range(logits.m)]
    lv = ops.level(D[0][0]) + 1
    Xl = EncMat([[ops.drop(b, lv) for b in row] for row in X.blocks], X.rows, X.cols, X.s0, X.s1)
    G = diag_atb(ops, EncMat(D, logits.rows, logits.cols, X.s0, X.s1), Xl, c, lr_over_n)
    return G, logits, P, D


# --------------------------------------------------------------------------
# The training loop (Protocol 1, step 3, Sec. 3) with NAG (Sec. 2.1):
#   W_{t+1} = V_t - (alpha/N) (P - Y)^T X,   P = softmax(X V_t^T)
#   V_{t+1} = (1 - gamma_t) W_{t+1} + gamma_t W_t = W_{t+1} + gamma_t (W_t - W_{t+1})
# gamma_t = (1 - lambda_t) / lambda_{t+1}, lambda_0 = 0, lambda_{t+1} = (1 + sqrt(1 + 4 lambda_t^2)) / 2,
# V_1 = W_1; then the validation logits X_val W^T with the last W (step 3(b)).
# The gradient comes out of DiagATB at the scale its products leave; it is moved to V's
# scale with a constant product by 1 so that the subtraction sees equal scales.
# --------------------------------------------------------------------------
def nag_gammas(steps):
    """gamma_1 .. gamma_steps."""
    lam, out = [0.0], []
    for t in range(steps + 1):
        lam.append((1.0 + (1.0 + 4.0 * lam[-1] ** 2) ** 0.5) / 2.0)
    for t in range(1, steps + 1):
        out.append((1.0 - lam[t]) / lam[t + 1])
    return out


def nag_train(ops, X, Wbar, Y, coeffs, valid, c, lr_over_n, target_scale, steps, Xval):
    """`steps` NAG updates of W-bar (c x b, tiled vertically) from (X, Y), then the validation
    logits DiagABT(X_val, W-bar); returns (W-bar, V-bar, logits)."""
    W = V = Wbar
    for gamma in nag_gammas(steps):
        G = train_step(ops, X, V, Y, coeffs, valid, c, lr_over_n, target_scale)[0]
        Wn_blocks = []
        for v, g in zip(V.blocks[0], G.blocks[0]):
            Wn_blocks.append(ops.sub(v, ops.mul_const(g, 1.0, ops.scale(v))))
        Vn_blocks = []
        for w_old, w_new in zip(W.blocks[0], Wn_blocks):
            d = ops.sub(w_old, w_new)
            Vn_blocks.append(ops.add(w_new, ops.mul_const(d, gamma, ops.scale(w_new))))
        W = EncMat([Wn_blocks], Wbar.rows, Wbar.cols, Wbar.s0, Wbar.s1)
        V = EncMat([Vn_blocks], Wbar.rows, Wbar.cols, Wbar.s0, Wbar.s1)
    logits = diag_abt(ops, Xval, W, c, 1.0)
    return W, V, logits
