"""A fake of the C ABI for host-logic tests of the circuits built on it (asoftmax.py,
bootstrap.py): it tracks every handle, level and scale the way the library does (products
aimed at a scale through an integer factor, plaintext products at a given scale, additions
that need equal scales) and checks use after free, double frees and missing keys.  No GPU."""
from types import SimpleNamespace

import numpy as np


class FakeABI:
    def __init__(self, N, moduli, rotations):
        self.N, self.q, self.rot_ok = N, moduli, set(rotations)
        self.live, self.next = {}, 1
        self.calls = {}
        self.relabels = 0
        self.max_coeff = 0.0
        self.plains = {}
        self.nb = {}   # block count of a handle made by a block-aware call (else 1)

    def _new(self, lv, scale, nb=1):
        h = self.next
        self.next += 1
        self.live[h] = (lv, scale)
        if nb != 1:
            self.nb[h] = nb
        return h

    def _blocks(self, h):
        self._get(h)
        return self.nb.get(h, 1)

    def _get(self, h):
        assert h in self.live, "handle %r used after it was freed" % h
        return self.live[h]

    def _count(self, name):
        self.calls[name] = self.calls.get(name, 0) + 1

    # -- the calls the circuits make -----------------------------------------
    def hetal_ctx_info(self, ctx):
        return self.N, len(self.q) - 4, 4

    def hetal_rotations_ok(self, rs):
        self.rot_ok = set(rs)

    def hetal_ctx_moduli(self, ctx):
        return list(self.q)

    def hetal_mat_desc_get(self, h):
        lv, sc = self._get(h)
        return SimpleNamespace(level=lv, scale=sc, s0=1024, s1=32, m=1, n=self._blocks(h), rows=1024,
                               cols=32 * self._blocks(h))

    @staticmethod
    def make_desc(m, n, rows, cols, s0, s1, level, scale):
        return SimpleNamespace(m=m, n=n, rows=rows, cols=cols, s0=s0, s1=s1, level=level, scale=scale)

    def hetal_mat_drop(self, ctx, a, lv):
        la, sa = self._get(a)
        assert 0 <= lv <= la
        return self._new(lv, sa, self._blocks(a))

    def hetal_mat_slice(self, ctx, a, first, count):
        self._count("slice")
        assert 0 <= first and count >= 1 and first + count <= self._blocks(a), "slice outside the matrix"
        return self._new(*self._get(a), count)

    def hetal_mat_stack(self, ctx, mats, desc):
        self._count("stack")
        got = [self._get(a) for a in mats]
        assert all(g == got[0] for g in got), "stacked blocks at different levels or scales"
        total = sum(self._blocks(a) for a in mats)
        assert desc.m * desc.n == total
        return self._new(*got[0], total)

    def hetal_mul_const(self, ctx, a, value, out_scale):
        la, sa = self._get(a)
        assert la >= 1
        return self._new(la - 1, out_scale, self._blocks(a))

    def hetal_diag_abt(self, ctx, evk, a, b, c, t, pts=None, flags=0):
        """DiagABT's three levels (Algorithm DiagABT: Mult, the column-0 mask, the class mask)."""
        self._count("diag_abt")
        (la, sa), (lb, sb) = self._get(a), self._get(b)
        lv = min(la, lb) - 3
        assert lv >= 0
        return self._new(lv, sa)

    def hetal_rotate_sum(self, ctx, evk, a, steps):
        self._count("rot_sum")
        for r in steps:
            assert r in self.rot_ok, "rotation %d has no key" % r
        return self._new(*self._get(a), self._blocks(a))

    def hetal_mat_free(self, h):
        assert h in self.live, "handle %r freed twice" % h
        del self.live[h]

    def hetal_mult_scaled(self, ctx, evk, a, b, delta):
        self._count("mult")
        (la, sa), (lb, sb) = self._get(a), self._get(b)
        lv = min(la, lb)
        assert lv >= 1
        t = round(delta * self.q[lv] / (sa * sb))
        assert 1 <= t < 2 ** 62
        return self._new(lv - 1, sa * t * sb / self.q[lv])

    def _addsub(self, a, b):
        (la, sa), (lb, sb) = self._get(a), self._get(b)
        assert abs(sa / sb - 1) <= 1e-9, "addition of unequal scales"
        assert self._blocks(a) == self._blocks(b), "addition of matrices with different block counts"
        return self._new(min(la, lb), sa, self._blocks(a))

    def hetal_add(self, ctx, a, b):
        return self._addsub(a, b)

    def hetal_sub(self, ctx, a, b):
        return self._addsub(a, b)

    def hetal_mat_set_scale(self, ctx, a, scale):
        la, sa = self._get(a)
        if abs(scale / sa - 1) <= 2.0 ** -16:   # a rounding difference, before an addition
            self.relabels += 1
        return self._new(la, scale)

    def hetal_mul_int(self, ctx, a, t):
        assert t != 0
        return self._new(*self._get(a))

    def hetal_cmult_int(self, ctx, a, pt, out_scale):
        self._count("cmult")
        la, sa = self._get(a)
        assert la >= 1 and np.asarray(pt).shape == (self.N,)
        return self._new(la - 1, out_scale)

    def hetal_add_plain_int(self, ctx, a, pt):
        assert np.asarray(pt).shape == (self.N,)
        return self._new(*self._get(a))

    def hetal_rotate(self, ctx, evk, a, r):
        self._count("rot")
        assert r in self.rot_ok, "rotation %d has no key" % r
        return self._new(*self._get(a))

    def hetal_mod_raise(self, ctx, a, lv):
        self._count("mod_raise")
        la, sa = self._get(a)
        assert la == 0 and 0 < lv < len(self.q) - 4
        return self._new(lv, float(self.q[0]))

    def hetal_mul_i(self, ctx, a):
        return self._new(*self._get(a))

    def hetal_conj(self, ctx, evk, a):
        self._count("conj")
        return self._new(*self._get(a))

    def hetal_rotate_hoisted(self, ctx, evk, a, steps):
        self._count("rot")
        for r in steps:
            assert r in self.rot_ok, "rotation %d has no key" % r
        return [self._new(*self._get(a)) for _ in steps]

    def hetal_plain_create(self, ctx, pt, lv, scale):
        self._count("upload")
        h = ("pt", self.next)
        self.next += 1
        self.plains[h] = lv
        return h

    def hetal_plain_free(self, h):
        assert h in self.plains, "plaintext %r freed twice" % (h,)
        del self.plains[h]

    def hetal_cmult_plain(self, ctx, a, pt, out_scale):
        self._count("cmult")
        la, sa = self._get(a)
        assert pt in self.plains and self.plains[pt] >= la >= 1
        return self._new(la - 1, out_scale)

    def hetal_cmult_plain_sum(self, ctx, mats, plains, out_scale):
        self._count("cmult")
        self.calls["cmult_terms"] = self.calls.get("cmult_terms", 0) + len(mats)
        got = [self._get(a) for a in mats]
        lv, sc = got[0]
        assert all(g[0] == lv and abs(g[1] / sc - 1) <= 1e-9 for g in got), "sum terms at different levels/scales"
        assert lv >= 1 and all(p in self.plains and self.plains[p] >= lv for p in plains)
        return self._new(lv - 1, out_scale)

    def hetal_add_plain(self, ctx, a, pt):
        la, sa = self._get(a)
        assert pt in self.plains and self.plains[pt] >= la
        return self._new(la, sa)

    def hetal_encode(self, ctx, re, im, scale):
        self._count("encode")
        re = np.atleast_2d(re)
        assert re.shape == (1, self.N // 2)
        mag = np.abs(re) if im is None else np.abs(re + 1j * np.atleast_2d(im))
        self.max_coeff = max(self.max_coeff, float(np.max(mag)) * scale)
        return np.zeros((1, self.N), dtype=np.int64)


def chain(levels):
    # 60-bit primes of slightly different sizes, as a real chain has (values only; the
    # fake needs their magnitudes), then 4 special primes
    q = [2 ** 60 - (1 + 37 * i) * 2 ** 32 + 1 for i in range(levels + 1)]
    return q + [2 ** 61 - (1 + 5 * i) * 2 ** 32 + 1 for i in range(4)]


