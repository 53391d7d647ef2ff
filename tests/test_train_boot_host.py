"""Host logic of the packed refresh of the bootstrapped training loop
(paper_2403_14111_gb300/step.py refresh_packed) against the fake C ABI: one bootstrapping
per w blocks, every handle released, the refreshed blocks at the training top level and
exactly the target scale, every rotation keyed, device plaintexts uploaded once and reused;
and the replication stages reaching every window exactly once.  No GPU."""
import itertools

import pytest

from paper_2403_14111_gb300 import bootstrap as B
from paper_2403_14111_gb300 import circuit, step
from oracle import bootstrap as bt

from fake_abi import FakeABI, chain


@pytest.mark.parametrize("w", [1, 2, 8, 16, 64, 512])
def test_replication_reaches_every_window_once(w):
    offsets = [0]
    for radix, stride in step.replicate_stages(w):
        offsets = [o + j * stride for o in offsets for j in range(radix)]
    assert sorted(offsets) == list(range(w))
    assert all(radix <= 8 for radix, _ in step.replicate_stages(w))
    # the oracle's stages, written separately, use the same rotations
    assert step.replicate_rotations(512, w) == bt.replicate_rotations(512, w)
    with pytest.raises(ValueError):
        step.replicate_stages(w * 3)


@pytest.mark.parametrize("n_blocks,s0,c", [(24, 1024, 16), (3, 16, 4), (5, 8, 4)])
def test_packed_refresh(monkeypatch, n_blocks, s0, c):
    s1 = 32
    N = 2 * s0 * s1
    prm = B.BootstrapParams()
    n_train = 14
    top = n_train + B.levels(N, prm)
    fake = FakeABI(N, chain(top), step.train_boot_rotations(s0, s1, c, 0, prm))
    for mod in (B, circuit, step):
        monkeypatch.setattr(mod, "H", fake)
    delta = 2.0 ** 50
    mats = [fake._new(1, delta, n_blocks), fake._new(1, delta, n_blocks)]
    P, w = c * s1, s0 // c
    cache = {}
    outs = step.refresh_packed(None, None, mats, P, w, delta, prm, boot_cache=cache)
    boots = -(-2 * n_blocks // w)
    assert fake.calls["mod_raise"] == boots
    assert fake.calls["slice"] == 2 * n_blocks and fake.calls["stack"] == 2
    assert fake.calls["rot_sum"] == 2 * len(step.replicate_stages(w))
    for h in outs:
        lv, sc = fake._get(h)
        assert lv == n_train - 1 and sc == delta
        assert fake._blocks(h) == n_blocks
    uploads = fake.calls["upload"]
    again = step.refresh_packed(None, None, mats, P, w, delta, prm, boot_cache=cache)
    assert fake.calls["upload"] == uploads            # every plaintext came from the device cache
    for h in outs + again + mats:
        fake.hetal_mat_free(h)
    circuit.free_plains(cache)
    assert not fake.live, "%d handles leaked" % len(fake.live)
    assert not fake.plains


def test_packed_refresh_releases_its_handles_on_error(monkeypatch):
    N, s0, s1, c = 1 << 12, 64, 32, 4
    prm = B.BootstrapParams()
    top = 14 + B.levels(N, prm)
    rots = [r for r in step.train_boot_rotations(s0, s1, c, 0, prm) if r not in step.replicate_rotations(c * s1,
                                                                                                        s0 // c)]
    fake = FakeABI(N, chain(top), rots)          # the replication's keys are missing
    for mod in (B, circuit, step):
        monkeypatch.setattr(mod, "H", fake)
    mats = [fake._new(1, 2.0 ** 50, 3)]
    with pytest.raises(AssertionError, match="has no key"):
        step.refresh_packed(None, None, mats, c * s1, s0 // c, 2.0 ** 50, prm)
    assert list(fake.live) == mats


def test_window_masks_partition_the_slots():
    for P, w in itertools.product((32, 512), (2, 64)):
        total = sum(step._window(k, P, P * w) for k in range(w))
        assert (total == 1).all()
