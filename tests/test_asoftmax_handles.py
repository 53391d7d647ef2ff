"""Host logic of the ASoftmax composition (paper_2403_14111_gb300/asoftmax.py) against a
fake of the C ABI that tracks every handle, level and scale: no handle is used after it
is freed or freed twice, nothing leaks, the levels add up to depth(), additions see
equal scales (reading A10's relabel), every plaintext product's coefficients fit 64 bits
(reading A11's split) and only the listed rotations are asked for.  No GPU."""
import math
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2403_14111_gb300 import asoftmax as A


class FakeABI:
    def __init__(self, N, moduli, rotations):
        self.N, self.q, self.rot_ok = N, moduli, set(rotations)
        self.live, self.next = {}, 1
        self.calls = {}
        self.relabels = 0
        self.max_coeff = 0.0

    def _new(self, lv, scale):
        h = self.next
        self.next += 1
        self.live[h] = (lv, scale)
        return h

    def _get(self, h):
        assert h in self.live, "handle %r used after it was freed" % h
        return self.live[h]

    def _count(self, name):
        self.calls[name] = self.calls.get(name, 0) + 1

    # -- the calls asoftmax.py makes ---------------------------------------
    def hetal_ctx_info(self, ctx):
        return self.N, len(self.q) - 4, 4

    def hetal_ctx_moduli(self, ctx):
        return list(self.q)

    def hetal_mat_desc_get(self, h):
        lv, sc = self._get(h)
        return SimpleNamespace(level=lv, scale=sc, s0=1024, s1=32, m=1, n=1)

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
        return self._new(min(la, lb), sa)

    def hetal_add(self, ctx, a, b):
        return self._addsub(a, b)

    def hetal_sub(self, ctx, a, b):
        return self._addsub(a, b)

    def hetal_mat_set_scale(self, ctx, a, scale):
        self.relabels += 1
        la, sa = self._get(a)
        assert abs(scale / sa - 1) <= 2.0 ** -16
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

    def hetal_encode(self, ctx, re, im, scale):
        re = np.atleast_2d(re)
        assert re.shape == (1, self.N // 2)
        self.max_coeff = max(self.max_coeff, float(np.max(np.abs(re))) * scale)
        return np.zeros((1, self.N), dtype=np.int64)


def _moduli(levels):
    # 60-bit primes of slightly different sizes, as a real chain has (values only; the
    # fake needs their magnitudes), then 4 special primes
    q = [2 ** 60 - (1 + 37 * i) * 2 ** 32 + 1 for i in range(levels + 1)]
    return q + [2 ** 61 - (1 + 5 * i) * 2 ** 32 + 1 for i in range(4)]


@pytest.mark.parametrize("c", [2, 3, 10])
@pytest.mark.parametrize("precise", [False, True])
def test_composition_handles_levels_and_scales(monkeypatch, c, precise):
    prm = A.ASoftmaxParams(precise=precise)
    depth = A.depth(c, prm)
    fake = FakeABI(2 ** 16, _moduli(depth), A.rotations(c, 32))
    monkeypatch.setattr(A, "H", fake)
    delta = 2.0 ** 40
    M = fake._new(depth, delta)
    out = A.asoftmax(None, None, M, c, 1024, 32, delta, prm)
    lv, sc = fake._get(out)
    assert lv == 0
    assert abs(sc / delta - 1) < 1e-6
    assert fake.relabels > 0                      # the relabel path ran
    assert fake.max_coeff < 2.0 ** 63             # every encoded plaintext fits int64
    cp = A.padded_classes(c)
    assert fake.calls["rot"] == 2 * (int(math.log2(cp)) + 5)
    fake.hetal_mat_free(out)
    fake.hetal_mat_free(M)
    assert not fake.live, "%d handles leaked" % len(fake.live)


def test_refuses_too_few_levels_and_wrong_shapes(monkeypatch):
    prm = A.ASoftmaxParams()
    fake = FakeABI(2 ** 16, _moduli(130), A.rotations(10, 32))
    monkeypatch.setattr(A, "H", fake)
    M = fake._new(A.depth(10, prm) - 1, 2.0 ** 40)
    with pytest.raises(ValueError):
        A.asoftmax(None, None, M, 10, 1024, 32, 2.0 ** 40, prm)
    with pytest.raises(ValueError):
        A.asoftmax(None, None, M, 64, 1024, 32, 2.0 ** 40, prm)   # c' above s1
    assert list(fake.live) == [M]


def test_supplied_plaintexts_are_looked_up_by_name_and_level(monkeypatch):
    prm = A.ASoftmaxParams()
    depth = A.depth(2, prm)
    fake = FakeABI(2 ** 16, _moduli(depth), A.rotations(2, 32))
    monkeypatch.setattr(A, "H", fake)
    asked = []

    class Pts(dict):
        def get(self, key, default=None):
            asked.append(key)
            return np.zeros(2 ** 16, dtype=np.int64)

    M = fake._new(depth, 2.0 ** 40)
    out = A.asoftmax(None, None, M, 2, 1024, 32, 2.0 ** 40, prm, pts=Pts())
    assert fake.max_coeff == 0.0                  # nothing encoded by the library
    names = {k[0] for k in asked}
    assert {"scale_in", "g1", "g2", "f", "half", "neg", "one", "firstcol", "scale_out", "dc", "dep_in", "dep_k",
            "dep_out", "exp_in", "exp", "inv_in", "inv_step", "inv_out"} <= names
    assert all(0 <= k[2] <= depth for k in asked)
    fake.hetal_mat_free(out)
    fake.hetal_mat_free(M)
    assert not fake.live
