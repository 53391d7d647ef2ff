"""Deep CKKS circuits as sequences of C-ABI calls: ciphertext handles that free themselves,
products aimed at a given scale, plaintexts encoded on demand or supplied by the caller.

Every homomorphic step runs in the library's kernels; a Circuit only orders the calls,
keeps the scale bookkeeping the algorithms need and releases intermediate handles.

Scales.  A ciphertext product goes through hetal_mult_scaled, which multiplies its first
operand by an integer t so that the rescaled product lands within 1/(2t) of a target
scale.  A plaintext product is encoded for the scale it should produce (cmult_scaled), or
at q_l so that it keeps the ciphertext's scale (cmult).  Two ciphertexts whose scales
differ only by the integer factor's rounding are added after hetal_mat_set_scale reads the
second at the first one's scale; algorithms that cannot afford that error aim each
operand at its partner's exact scale instead (operand_scale_for).

With a refresher (`refresh`), keep(a, need, bound) bootstraps a value that has too few
levels left for the products before its next refresh point, so that circuits deeper than
the chain run on the levels below bootstrapping's primes.

Plaintexts are named (name, index, level).  By default they are encoded with the library's
FP64 encoder (hetal_encode), and kept in `record` when one is given; a caller may supply
integer plaintexts under the same names (`pts`): encodings made once and reused, or
another implementation's, to reproduce its results bit for bit.  With a `cache` dict each
plaintext is uploaded once as a device plaintext (hetal_plain_create) and reused by later
runs of the circuit without a host copy or a transform; the caller frees them
(free_plains) before the context.
"""
import math

import numpy as np

from . import hetal as H


class Ct:
    """One owned matrix handle; freed when the last reference goes.  A handle is only
    passed to the library while its Ct is bound to a name (never from a temporary)."""
    __slots__ = ("h", "lv", "scale", "_circ")

    def __init__(self, circ, h):
        d = H.hetal_mat_desc_get(h)
        self.h, self.lv, self.scale, self._circ = h, d.level, d.scale, circ

    def detach(self):
        h, self.h = self.h, None
        return h

    def __del__(self):
        if self.h is not None and self._circ.alive:
            H.hetal_mat_free(self.h)


class Circuit:
    RELABEL = 1e-9          # scale differences the library's additions accept
    RELABEL_MAX = 2.0 ** -16   # larger ones are an algorithm's mistake, not rounding
    CMULT_MAX = 4.0         # plaintext values above this are split (64-bit coefficients)

    def __init__(self, ctx, evk, delta, pts=None, record=None, cache=None, refresh=None):
        self.ctx, self.evk, self.delta = ctx, evk, float(delta)
        self.refresh = refresh   # (circuit, Ct, bound) -> its bootstrapped copy (bootstrap.Refresher)
        self.slots = H.hetal_ctx_info(ctx)[0] // 2
        self.s = self.slots
        self.q = H.hetal_ctx_moduli(ctx)
        self.pts = pts
        self.record = record   # a dict that keeps the plaintexts this circuit encodes
        self.cache = cache     # a dict of device plaintexts (hetal_plain) the caller owns
        self.alive = True

    def close(self):
        self.alive = False

    def wrap(self, h):
        return Ct(self, h)

    def adopt(self, h):
        """A caller's handle, used but never freed by the circuit."""
        d = H.hetal_mat_desc_get(h)
        return _Borrowed(h, d.level, d.scale)

    # -- plaintexts ---------------------------------------------------------
    def plain(self, vals, scale, name, index, lv):
        if self.pts is not None:
            got = self.pts.get((name, index, lv))
            if got is None:
                raise KeyError("no plaintext supplied for %r" % ((name, index, lv),))
            return got
        vals = np.asarray(vals)
        im = vals.imag if np.iscomplexobj(vals) else None
        pt = H.hetal_encode(self.ctx, np.ascontiguousarray(vals.real, dtype=np.float64), im, scale)[0]
        if self.record is not None:
            self.record[(name, index, lv)] = pt
        return pt

    def _device_or_host(self, vals, scale, name, index, lv):
        """The plaintext for (name, index, lv): from the device cache when there is one
        (uploaded on first use), else host coefficients."""
        key = (name, index, lv)
        if self.cache is not None and key in self.cache:
            return self.cache[key]
        pt = self.plain(vals, scale, name, index, lv)
        if self.cache is None:
            return pt
        h = H.hetal_plain_create(self.ctx, pt, lv, scale)
        self.cache[key] = h
        return h

    def _times_plain(self, a, pt, out_scale):
        if isinstance(pt, np.ndarray):
            return self.wrap(H.hetal_cmult_int(self.ctx, a.h, pt, out_scale))
        return self.wrap(H.hetal_cmult_plain(self.ctx, a.h, pt, out_scale))

    def _split(self, a, vals):
        top = float(np.max(np.abs(vals)))
        if top > self.CMULT_MAX:
            k = int(math.ceil(math.log2(top / self.CMULT_MAX)))
            a = self.wrap(H.hetal_mul_int(self.ctx, a.h, 1 << k))
            vals = vals / float(1 << k)
        return a, vals

    # -- operations ---------------------------------------------------------
    def mult(self, a, b):
        return self.mult_to(a, b, self.delta)

    def mult_to(self, a, b, target):
        return self.wrap(H.hetal_mult_scaled(self.ctx, self.evk, a.h, b.h, target))

    def operand_scale_for(self, lv_a, b, product_scale, target):
        """The scale s_a that makes mult_to(a, b, product_scale), a at level lv_a, land on
        product_scale to the last bit or two: s_a = product_scale q / (t s_b) with
        t = round(product_scale q / (target s_b)), q the prime the product is rescaled by."""
        q = float(self.q[min(lv_a, b.lv)])
        t = float(math.floor(product_scale * q / (target * b.scale) + 0.5))
        return product_scale * q / (t * b.scale)

    def _binary(self, fn, a, b):
        if abs(a.scale / b.scale - 1.0) > self.RELABEL:
            if abs(a.scale / b.scale - 1.0) > self.RELABEL_MAX:
                raise ValueError("scales %r and %r are not one scale rounded" % (a.scale, b.scale))
            # a local name keeps the relabelled copy (and its handle) alive through the call
            b = self.wrap(H.hetal_mat_set_scale(self.ctx, b.h, a.scale))
        return self.wrap(fn(self.ctx, a.h, b.h))

    def add(self, a, b):
        return self._binary(H.hetal_add, a, b)

    def sub(self, a, b):
        return self._binary(H.hetal_sub, a, b)

    def cmult(self, a, vals, name, index):
        """Plaintext product keeping a's scale (the plaintext encoded at q_lv)."""
        a, vals = self._split(a, np.asarray(vals))
        pt = self._device_or_host(vals, float(self.q[a.lv]), name, index, a.lv)
        return self._times_plain(a, pt, a.scale)

    def cmult_scaled(self, a, vals, name, index, target):
        """Plaintext product landing on exactly `target` (the plaintext encoded at
        target * q_lv / scale(a))."""
        a, vals = self._split(a, np.asarray(vals))
        pt = self._device_or_host(vals, target * float(self.q[a.lv]) / a.scale, name, index, a.lv)
        return self._times_plain(a, pt, target)

    def cmult_scaled_sum(self, terms, target):
        """sum of plaintext products [(a, vals, name, index)], every a at one level and scale,
        accumulated before one rescale that lands on `target` (hetal_cmult_plain_sum).  The
        plaintexts go to the device: kept in the cache when there is one, else for this call."""
        mats, plains, temps, keep = [], [], [], []
        try:
            for a, vals, name, index in terms:
                a, vals = self._split(a, np.asarray(vals))
                keep.append(a)   # a split term's handle stays alive through the call
                pt = self._device_or_host(vals, target * float(self.q[a.lv]) / a.scale, name, index, a.lv)
                if isinstance(pt, np.ndarray):
                    pt = H.hetal_plain_create(self.ctx, pt, a.lv, target * float(self.q[a.lv]) / a.scale)
                    temps.append(pt)
                mats.append(a.h)
                plains.append(pt)
            return self.wrap(H.hetal_cmult_plain_sum(self.ctx, mats, plains, target))
        finally:
            for pt in temps:
                H.hetal_plain_free(pt)

    def add_plain(self, a, vals, name, index):
        pt = self._device_or_host(vals, a.scale, name, index, a.lv)
        if isinstance(pt, np.ndarray):
            return self.wrap(H.hetal_add_plain_int(self.ctx, a.h, pt))
        return self.wrap(H.hetal_add_plain(self.ctx, a.h, pt))

    def rot(self, a, r):
        if r % self.slots == 0:
            return a
        return self.wrap(H.hetal_rotate(self.ctx, self.evk, a.h, int(r)))

    def rot_many(self, a, rs):
        """Rotations of a by every amount of rs sharing one ModUp (hoisted)."""
        return [self.wrap(h) for h in H.hetal_rotate_hoisted(self.ctx, self.evk, a.h, [int(r) for r in rs])]

    def conj(self, a):
        return self.wrap(H.hetal_conj(self.ctx, self.evk, a.h))

    def mul_i(self, a):
        return self.wrap(H.hetal_mul_i(self.ctx, a.h))

    def mul_int(self, a, t):
        return self.wrap(H.hetal_mul_int(self.ctx, a.h, int(t)))

    def mod_raise(self, a, lv):
        return self.wrap(H.hetal_mod_raise(self.ctx, a.h, lv))

    def read_at(self, a, scale):
        return self.wrap(H.hetal_mat_set_scale(self.ctx, a.h, scale))

    def keep(self, a, need, bound):
        """A refresh point: a itself while it holds more than `need` levels (the products
        before the value's next refresh point), else, with a refresher, its bootstrapped
        copy; bound is a power of two with |message| <= bound."""
        if a.lv > need or self.refresh is None:
            return a
        return self.refresh(self, a, bound)

    def keep2(self, a, need_a, bound_a, b, need_b, bound_b, period, slots_per_row):
        """keep() of two values; when both need a refresh and their slots repeat every
        `period` slots with room for two windows in a row, one bootstrapping serves both
        (the refresher's pair)."""
        if (a.lv <= need_a and b.lv <= need_b and self.refresh is not None
                and slots_per_row >= 2 * period and hasattr(self.refresh, "pair")):
            return tuple(self.refresh.pair(self, a, bound_a, b, bound_b, period))
        return self.keep(a, need_a, bound_a), self.keep(b, need_b, bound_b)


class _Borrowed:
    """A caller's handle inside a circuit: it behaves as a Ct but is never freed here."""
    __slots__ = ("h", "lv", "scale")

    def __init__(self, h, lv, scale):
        self.h, self.lv, self.scale = h, lv, scale


def free_plains(cache):
    """Releases the device plaintexts of a Circuit cache."""
    for h in cache.values():
        H.hetal_plain_free(h)
    cache.clear()
