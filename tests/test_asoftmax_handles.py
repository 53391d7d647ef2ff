"""Host logic of the ASoftmax composition (paper_2403_14111_gb300/asoftmax.py) against a
fake of the C ABI that tracks every handle, level and scale: no handle is used after it
is freed or freed twice, nothing leaks, the levels add up to depth(), additions see
equal scales (reading A10's relabel), every plaintext product's coefficients fit 64 bits
(reading A11's split) and only the listed rotations are asked for.  No GPU."""
import math

import numpy as np
import pytest

from paper_2403_14111_gb300 import asoftmax as A
from paper_2403_14111_gb300 import circuit

from fake_abi import FakeABI, chain as _moduli


@pytest.mark.parametrize("c", [2, 3, 10])
@pytest.mark.parametrize("precise", [False, True])
def test_composition_handles_levels_and_scales(monkeypatch, c, precise):
    prm = A.ASoftmaxParams(precise=precise)
    depth = A.depth(c, prm)
    fake = FakeABI(2 ** 16, _moduli(depth), A.rotations(c, 32))
    monkeypatch.setattr(A, "H", fake)
    monkeypatch.setattr(circuit, "H", fake)
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
    monkeypatch.setattr(circuit, "H", fake)
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
    monkeypatch.setattr(circuit, "H", fake)
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


@pytest.mark.parametrize("precise", [False, True])
def test_composition_with_refreshes_on_a_short_chain(monkeypatch, precise):
    """ASoftmax on 14 levels below bootstrapping's (a training chain): every refresh point
    sees a value with a level left for its pre-scaling product, the output keeps a level,
    and every handle (bootstrapping's too) is released."""
    from paper_2403_14111_gb300 import bootstrap as B
    prm = A.ASoftmaxParams(precise=precise)
    N, c, s1 = 2 ** 16, 10, 32
    top = 14 + B.levels(N)
    fake = FakeABI(N, _moduli(top), sorted(set(A.rotations(c, s1)) | set(B.rotations(N))))
    for mod in (A, B, circuit):
        monkeypatch.setattr(mod, "H", fake)
    delta = 2.0 ** 32
    M = fake._new(13, delta)
    refresher = B.Refresher()
    out = A.asoftmax(None, None, M, c, 1024, s1, delta, prm, refresh=refresher)
    lv, sc = fake._get(out)
    assert lv >= 1 and abs(sc / delta - 1) < 1e-5
    assert refresher.calls == fake.calls["mod_raise"]
    # about one refresh per 12 levels of the straight-line depth, plus the values kept alive
    assert A.depth(c, prm) // 13 <= refresher.calls <= A.depth(c, prm) // 3
    fake.hetal_mat_free(out)
    fake.hetal_mat_free(M)
    assert not fake.live, "%d handles leaked" % len(fake.live)
    with pytest.raises(ValueError):   # without a refresher the 13 levels are refused
        A.asoftmax(None, None, fake._new(13, delta), c, 1024, s1, delta, prm)
