"""Algorithm ASoftmax (App. A) on RNS ciphertexts with bootstrapping between its stages
(oracle/softmax.py refresh points, oracle/bootstrap.py Refresher), on a chain of 14 training
levels (50-bit primes) under bootstrapping's 60-bit primes: pinned against the same
algorithm on the FP64 slot simulator (itself pinned against Table tab:softmaxerr), with a
planted mistake in the refresh caught."""
import numpy as np

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


def test_paired_refresh_keeps_every_row():
    """Refresher.pair on values tiled with period P = 4 inside rows of 16 slots but different
    from row to row (ASoftmax's row sums and products): both come back within bootstrapping's
    error of their bounds; with the second window copied rightwards (into the next row's
    first window) the row boundaries break."""
    log_n, top = 10, 13
    N = 1 << log_n
    prm = bt.BootParams()
    p = ckks.Params(log_n, 60, top + 1, 50, 2, 61, 2, log_delta=50, n_upper=bt.depth(prm, N), upper_bits=60)
    o = ckks.Oracle(p, seed=6)
    s1, P, d = 16, 4, 2.0 ** 32
    rows = p.slots // s1
    rng = np.random.default_rng(1)
    va = np.repeat(rng.uniform(-0.5, 0.5, rows), s1)                       # one value per row
    vb = np.tile(rng.uniform(-60, 60, (rows, P)), (1, s1 // P)).reshape(-1)   # period P in each row
    A = o.encrypt_int(ckks.encode(va, d, p.N), 3, d, 1)
    B = o.encrypt_int(ckks.encode(vb, d, p.N), 2, d, 2)

    def run(sops):
        R = bt.Refresher(sops, sm.ScaledOps(o, 2.0 ** 55, hoist=True), prm, 2.0 ** 55)
        ra, rb = R.pair(A, 1.0, B, 64.0, P)
        assert R.calls == 1 and ra.lv == rb.lv == top and ra.scale == rb.scale == d
        return (np.max(np.abs(o.decrypt_slots(ra).real - va)), np.max(np.abs(o.decrypt_slots(rb).real - vb)))
    ea, eb = run(sm.ScaledOps(o, d))
    assert ea < 1e-4 and eb < 64 * 1e-4
    wrong = sm.ScaledOps(o, d)
    rot = wrong.rot
    wrong.rot = lambda a, r: rot(a, -abs(r)) if abs(r) == P else rot(a, r)
    assert max(run(wrong)) > 1.0
