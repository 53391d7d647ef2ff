"""Algorithm ASoftmax (App. A) on RNS ciphertexts with bootstrapping between its stages
(oracle/softmax.py refresh points, oracle/bootstrap.py Refresher), on a chain of 14 training
levels (50-bit primes) under bootstrapping's 60-bit primes: pinned against the same
algorithm on the FP64 slot simulator (itself pinned against Table tab:softmaxerr), with a
planted mistake in the refresh caught."""
import numpy as np
import pytest

from oracle import bootstrap as bt
from oracle import ckks, softmax as sm


def _run(c, plant=None):
    log_n, top = 10, 13
    N = 1 << log_n
    prm = bt.BootParams()
    p = ckks.Params(log_n, 60, top + 1, 50, 2, 61, 2, log_delta=50, n_upper=bt.depth(prm, N), upper_bits=60)
    o = ckks.Oracle(p, seed=6)
    if plant is not None:
        plant(o)
    s1 = 16
    s0 = p.slots // s1
    cp = 1 << max(1, int(np.ceil(np.log2(c))))
    d_sm = 2.0 ** 32
    X = np.random.default_rng(5).uniform(-4, 4, (s0, c))
    blk = np.zeros((s0, cp))
    blk[:, :c] = X
    M = o.encrypt_int(ckks.encode(np.tile(blk, (1, s1 // cp)).reshape(-1), d_sm, p.N), top, d_sm, 31)
    sops = sm.ScaledOps(o, d_sm)
    bops = sm.ScaledOps(o, 2.0 ** 55, hoist=True)
    refresher = bt.Refresher(sops, bops, prm, 2.0 ** 55)
    sops.refresh = refresher
    out = sm.asoftmax_block(sops, M, c, s0, s1, sm.Params())
    got = o.decrypt_slots(out).real.reshape(s0, s1)[:, :c]
    ref, depth = sm.asoftmax_rows(X, c, sm.Params(), s1=s1, s0=s0)
    return out, got, ref, depth, refresher.calls, X


def test_asoftmax_with_refreshes_follows_the_slot_simulator():
    out, got, ref, depth, calls, X = _run(3)   # padded classes (c' = 4)
    assert depth > 13 and calls >= depth // 13
    assert out.lv >= 1 and abs(out.scale / 2.0 ** 32 - 1) < 1e-5
    assert np.max(np.abs(got - ref)) < 2e-3
    # and, as the simulator, close to the exact softmax
    assert np.max(np.abs(got - sm.softmax(X))) <= np.max(np.abs(ref - sm.softmax(X))) + 2e-3


def test_planted_mistake_in_the_refresh_is_caught():
    """The refresh's integer product 2^k (2^k scale(a) = delta_in) forgotten: the value is
    read at delta_in all the same, so every refreshed message comes back divided by 2^k."""
    def plant(o):
        mul_int = o.mul_int
        o.mul_int = lambda a, t: a if t == 1 << 18 else mul_int(a, t)   # 2^32 * 2^18 = delta_in
    _, got, ref, _, _, _ = _run(2, plant)
    assert np.max(np.abs(got - ref)) > 5e-2
