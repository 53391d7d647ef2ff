"""Algorithmic work of HETAL's matrix products, for the step-level roofline.

The work of an instance is the paper's operation counts (Table
"tab:matnum_fixed", App. D; the formulas that reproduce its 30 values) at the
levels where the algorithms run them (Algorithms DiagABT, DiagATB, RotLeft and
PRotUp, App. B.3), times the modular multiplications of one RNS-CKKS primitive
(Sec. 2.2) with hybrid key switching:

  NTT of one limb            N/2 log2 N butterflies
  key switch at l limbs      INTT of c1 (l NTTs); ModUp of each digit (its first
                             factor, the conversion to the other l+K-a moduli,
                             their NTTs); key inner product 2 dnum (l+K) N;
                             ModDown 2K NTTs + 2(K + K l) N + 2l NTTs + 2l N
  hoisted extra rotation     the key inner product and ModDown only
  rescale at l limbs         2l NTTs + 2(l-1) N
  Mult                       tensor 4 l N + key switch + rescale
  CMult                      2 l N + rescale

With flags = HOIST (the default), rotations of one source by several amounts
(RotUp(B_cplx, k), Lrot(A_cplx, k)) are hoisted, as the paper's method rotates
one ciphertext by many steps, and nothing else changes: the paper's method's
work.  The library's other variants can be counted the same way, from their own
operation sequences: LAZY (the tensor products of a sum relinearised and rescaled
once), RADIX (SumCols / SumRows as radix steps: one full key switch per step plus
one key inner product per further amount), SHARED (PRotUp from one RotUp(B, 1)
per block, RotLeft from two hoisted rotations of A; pairs of plaintext products
rescaled once).
Butterflies and the other modular products (multiply-accumulates) are kept
apart, so that a roofline can weigh each at its own measured rate.  Nothing here
reads a kernel counter.
"""
import math
from dataclasses import dataclass, field

# Variants (the values of the library's HETAL_FLAG_*).  The paper's method is HOIST.
HOIST, LAZY, RADIX, SHARED = 1, 2, 4, 8


@dataclass
class Work:
    bfly: float = 0.0      # NTT butterflies
    mac: float = 0.0       # other modular products (conversions, key inner products, pointwise products)
    nbytes: float = 0.0    # ciphertexts, plaintexts read and written, and each distinct key once
    counts: dict = field(default_factory=lambda: {"cmult": 0, "mult": 0, "rot": 0, "conj": 0})
    keys: set = field(default_factory=set)

    def add(self, o):
        self.bfly += o.bfly
        self.mac += o.mac
        self.nbytes += o.nbytes
        for k, v in o.counts.items():
            self.counts[k] = self.counts.get(k, 0) + v
        self.keys |= o.keys
        return self

    def equivalents(self, mac_weight):
        """Butterfly-equivalents: butterflies plus products weighed by mac_weight."""
        return self.bfly + mac_weight * self.mac


class Costs:
    """Primitive costs of one parameter set: ring degree N, K special primes, alpha
    primes per key-switching digit.  Levels are 0-based (level l has l+1 limbs)."""

    def __init__(self, N, K, alpha):
        self.N, self.K, self.alpha = N, K, alpha
        self.ntt = N // 2 * int(math.log2(N))

    def digits(self, lv):
        l = lv + 1
        sizes = []
        while l > 0:
            sizes.append(min(self.alpha, l))
            l -= self.alpha
        return sizes

    def ct_bytes(self, lv):
        return 2.0 * (lv + 1) * self.N * 8

    def key_bytes(self, lv):
        return 2.0 * len(self.digits(lv)) * (lv + 1 + self.K) * self.N * 8

    def _kip_moddown(self, lv):
        l, K, N = lv + 1, self.K, self.N
        dnum = len(self.digits(lv))
        bf = 2 * K * self.ntt + 2 * l * self.ntt
        mac = 2 * dnum * (l + K) * N + 2 * (K + K * l) * N + 2 * l * N
        return bf, mac

    def keyswitch(self, lv, key, hoisted_extra=False):
        """One key switch of one polynomial at level lv with key `key`."""
        if lv < 0:
            raise ValueError("a key switch below level 0")
        l, K, N = lv + 1, self.K, self.N
        bf, mac = self._kip_moddown(lv)
        if not hoisted_extra:
            bf += l * self.ntt
            for a in self.digits(lv):
                mac += a * N + a * (l + K - a) * N
                bf += (l + K - a) * self.ntt
        w = Work(bf, mac, 2 * self.ct_bytes(lv))
        w.keys.add((key, lv))
        return w

    def kip_only(self, lv, key):
        """One more amount of a rotation sum: its key inner product (the ModUp and the
        ModDown are shared with the sum's first amount)."""
        l, K, N = lv + 1, self.K, self.N
        w = Work(0.0, 2.0 * len(self.digits(lv)) * (l + K) * N, 0.0)
        w.keys.add((key, lv))
        return w

    def tensor(self, lv):
        return Work(0.0, 4.0 * (lv + 1) * self.N, 1.5 * self.ct_bytes(lv))

    def cmult2(self, lv):
        """a (.) p + b (.) q with one rescale."""
        w = Work(0.0, 4.0 * (lv + 1) * self.N, 3.0 * self.ct_bytes(lv) + self.ct_bytes(lv - 1))
        w.add(self.rescale(lv))
        w.counts["cmult"] = 2
        return w

    def rescale(self, lv):
        if lv < 1:
            raise ValueError("no level left to rescale")
        l = lv + 1
        return Work(2 * l * self.ntt, 2 * (l - 1) * self.N, 0.0)

    def rot(self, lv, amount, hoisted_extra=False):
        w = self.keyswitch(lv, ("rot", amount), hoisted_extra)
        w.counts["rot"] = 1
        return w

    def conj(self, lv):
        w = self.keyswitch(lv, ("conj",))
        w.counts["conj"] = 1
        return w

    def mult(self, lv):
        w = Work(0.0, 4.0 * (lv + 1) * self.N, self.ct_bytes(lv))
        w.add(self.keyswitch(lv, ("relin",)))
        w.add(self.rescale(lv))
        w.counts["mult"] = 1
        return w

    def cmult(self, lv):
        w = Work(0.0, 2.0 * (lv + 1) * self.N, 1.5 * self.ct_bytes(lv) + self.ct_bytes(lv - 1))
        w.add(self.rescale(lv))
        w.counts["cmult"] = 1
        return w


def _times(w, k):
    out = Work()
    out.bfly, out.mac, out.nbytes = w.bfly * k, w.mac * k, w.nbytes * k
    out.counts = {key: v * k for key, v in w.counts.items()}
    out.keys = set(w.keys) if k else set()
    return out


def _blocks(a, b, s0, s1):
    return -(-a // s0), -(-b // s1)


def _hoisted(costs, lv, amounts, sources, hoist=True):
    """`sources` ciphertexts each rotated by every amount, one ModUp per source (hoist)."""
    w = Work()
    for i, r in enumerate(amounts):
        w.add(_times(costs.rot(lv, r, hoisted_extra=hoist and i > 0), sources))
    return w


def _radix_plan(bits):
    if bits <= 0:
        return []
    steps = -(-bits // 3)
    base, extra = divmod(bits, steps)
    return [base + 1] * extra + [base] * (steps - extra)


def _rot_chain(costs, lv, bits, unit, sign, flags):
    """x + Lrot(x, sign * u * unit) summed over u < 2^bits: log-depth rotate-and-add,
    or with RADIX steps of one key switch plus a key inner product per further amount."""
    w = Work()
    if flags & RADIX:
        t = 1
        for b in _radix_plan(bits):
            amts = [sign * j * t * unit for j in range(1, 1 << b)]
            w.add(costs.rot(lv, amts[0]))
            for r in amts[1:]:
                kw = costs.kip_only(lv, ("rot", r))
                kw.counts["rot"] = 1
                w.add(kw)
            t <<= b
    else:
        for u in range(bits):
            w.add(costs.rot(lv, sign * (1 << u) * unit))
    return w


def _products(costs, lv, groups, size, flags):
    """`groups` sums of `size` ciphertext products each."""
    if flags & LAZY:
        one = _times(costs.tensor(lv), size)
        one.add(costs.keyswitch(lv, ("relin",)))
        one.add(costs.rescale(lv))
        one.counts["mult"] = size
        return _times(one, groups)
    return _times(costs.mult(lv), groups * size)


def diag_abt(costs, a, b, c, s0, s1, lv, flags=HOIST):
    """DiagABT of an a x b matrix by (c x b)^T (blocks s0 x s1) with both inputs at level lv."""
    m, n = _blocks(a, b, s0, s1)
    h, lg1 = c // 2, int(math.log2(s1))
    w = Work()
    w.add(_times(costs.rot(lv, h * s1), n))                           # RotUp(B-bar, c/2)
    if h > 1:                                                         # RotUp(B_cplx, k)
        w.add(_hoisted(costs, lv, [k * s1 for k in range(1, h)], n, bool(flags & HOIST)))
    w.add(_products(costs, lv, h * m, n, flags))
    sc = _rot_chain(costs, lv - 1, lg1, 1, 1, flags)                  # SumCols
    sc.add(costs.cmult(lv - 1))
    sc.add(_rot_chain(costs, lv - 2, lg1, 1, -1, flags))
    w.add(_times(sc, h * m))
    w.add(_times(costs.cmult(lv - 2), h * m))                         # t M_cplx^{(k,c)}
    w.add(_times(costs.conj(lv - 3), m))
    return w


def diag_atb(costs, a, b, c, s0, s1, lv_a, lv_b, flags=HOIST):
    """DiagATB of A (a x c, tiled horizontally) and B (a x b), A at level lv_a, B at
    lv_b; the PRotUp branch when lv_a < lv_b, else the RotLeft branch."""
    m, n = _blocks(a, b, s0, s1)
    h, lg0 = c // 2, int(math.log2(s0))
    pru = lv_a < lv_b
    hoist, shared = bool(flags & HOIST), bool(flags & SHARED)
    w = Work()
    # A_cplx = A + i RotLeft(A, c/2) (per row block)
    if shared:
        w.add(_hoisted(costs, lv_a, [h, h - s1], m, hoist))
        w.add(_times(costs.cmult2(lv_a), m))
    else:
        w.add(_times(costs.rot(lv_a, h), m))
        w.add(_times(costs.cmult(lv_a), m))
        w.add(_times(costs.rot(lv_a - 1, -s1), m))
    lac = lv_a - 1
    if pru:
        lvp = min(lac, lv_b - 1 if h > 1 else lv_b)
        if h > 1:
            w.add(_hoisted(costs, lac, list(range(1, h)), m, hoist))  # Lrot(A_cplx, k)
            if shared:                                                # PRotUp from RotUp(B, 1)
                w.add(_times(costs.rot(lv_b, s1), m * n))
                w.add(_times(costs.cmult2(lv_b), (h - 1) * m * n))
            else:                                                     # PRotUp: B (.) D_k, RotUp(., 1)
                w.add(_times(costs.cmult(lv_b), (h - 1) * m * n))
                w.add(_times(costs.rot(lv_b - 1, s1), (h - 1) * m * n))
    else:
        lvp = min(lac - 1 if h > 1 else lac, lv_b)
        if h > 1:
            if shared:                                                # Lrot(A_cplx, k), Lrot(A_cplx, k - s1)
                w.add(_hoisted(costs, lac, list(range(1, h)) + [k - s1 for k in range(1, h)], m, hoist))
                w.add(_times(costs.cmult2(lac), (h - 1) * m))
            else:                                                     # RotLeft(A_cplx, k): Lrot, D_k, Rrot
                w.add(_hoisted(costs, lac, list(range(1, h)), m, hoist))
                w.add(_times(costs.cmult(lac), (h - 1) * m))
                w.add(_times(costs.rot(lac - 1, -s1), (h - 1) * m))
    w.add(_products(costs, lvp, h * n, m, flags))
    w.add(_times(_rot_chain(costs, lvp - 1, lg0, s1, 1, flags), h * n))   # SumRows
    w.add(_times(costs.cmult(lvp - 1), h * n))                        # t M_cplx^{(-k,c)}
    w.add(_times(costs.conj(lvp - 2), n))
    return w


def softmax_standin(costs, lv, blocks):
    """The degree-15 stand-in p(x) (.) valid on `blocks` ciphertexts at level lv:
    x^2, x^3, x^4, x^8, the 12 scaled plaintext products of the baby steps and the
    3 products of the giant steps (result at level lv - 5)."""
    one = Work()
    for l in (lv, lv - 1, lv - 1, lv - 2):            # x2, x3, x4, x8
        one.add(costs.mult(l))
    for l in (lv, lv - 1, lv - 2):                    # c_{4j+r} v (.) x^r, four j each
        one.add(_times(costs.cmult(l), 4))
    for l in (lv - 3, lv - 4, lv - 3):                # u3 x4, (u2 + u3 x4) x8, u1 x4
        one.add(costs.mult(l))
    return _times(one, blocks)


def training_step(costs, a, b, c, s0, s1, top, flags=HOIST):
    """DiagABT (logits) -> softmax stand-in -> -Y -> DiagATB at level(P - Y) and X
    one level above it (PRotUp branch), as the training step runs them."""
    w = Work()
    w.add(diag_abt(costs, a, b, c, s0, s1, top, flags))
    m, _ = _blocks(a, b, s0, s1)
    w.add(softmax_standin(costs, top - 3, m))
    lv_d = top - 8
    w.add(diag_atb(costs, a, b, c, s0, s1, lv_d, lv_d + 1, flags))
    return w


def instance_pair(costs, a, b, c, s0, s1, top, flags=HOIST):
    """One DiagABT + DiagATB instance of the batched workload: DiagABT with both inputs
    at the top level, DiagATB from A three levels below it and B two levels below."""
    w = Work()
    w.add(diag_abt(costs, a, b, c, s0, s1, top, flags))
    w.add(diag_atb(costs, a, b, c, s0, s1, top - 3, top - 2, flags))
    return w


def finish(w, costs):
    """Adds the bytes of each distinct key (read once) to w and returns it."""
    w.nbytes += sum(costs.key_bytes(lv) for _, lv in w.keys)
    w.keys = set()
    return w
