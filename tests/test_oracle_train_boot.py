"""The training loop (Protocol 1, step 3: NAG of Sec. 2.1) for several iterations with W and V
refreshed by bootstrapping after every update (oracle/bootstrap.py nag_train_boot), on a
chain of 50-bit training primes with 60-bit primes above them for the refresh: pinned
against the same loop on FP64 matrices with the same polynomial."""
import numpy as np

from oracle import bootstrap as bt
from oracle import ckks, matmul as mm, softmax as sm
from paper_2403_14111_gb300 import workloads as wl


def _run():
    log_n, steps, top = 10, 2, 13   # training primes up to level 14; a refresh lands at 13
    N = 1 << log_n
    prm = bt.BootParams()
    p = ckks.Params(log_n, 60, top + 1, 50, 2, 61, 2, log_delta=50, n_upper=bt.depth(prm, N), upper_bits=60)
    o = ckks.Oracle(p, seed=6)
    s1 = 32
    s0, c, b = p.slots // s1, 4, 64
    a = s0
    rng = np.random.default_rng(3)
    X = rng.standard_normal((a, b)) / np.sqrt(b)
    Xval = rng.standard_normal((a, b)) / np.sqrt(b)
    Y = wl.one_hot(rng.integers(0, c, a), c)
    W1 = rng.standard_normal((c, b)) * 0.1
    coeffs, valid, lr = wl.sigmoid_cheb15(), wl.valid_mask(a, c, c, s0, s1), 0.5 / a

    def enc(M, lv, nonce):
        return mm.EncMat([[o.encrypt_int(ckks.encode(bl, p.delta, p.N), lv, p.delta, nonce + 64 * r + j)
                           for j, bl in enumerate(row)] for r, row in enumerate(mm.block_split(M, s0, s1))],
                         M.shape[0], M.shape[1], s0, s1)
    EX, EXv = enc(X, top, 100), enc(Xval, top, 300)
    EW, EY = enc(mm.tile_vertical(W1, c, s0), top, 500), enc(mm.tile_horizontal(Y, c, s1), top - 8, 700)
    ops = mm.RnsOps(o, hoist=True, lazy_relin=True)
    bops = sm.ScaledOps(o, 2.0 ** 55, hoist=True)
    W, V, L = bt.nag_train_boot(ops, bops, EX, EW, EY, coeffs, valid, c, lr, p.delta, steps, EXv, prm, 2.0 ** 55)
    # every refresh lands back where W started, at exactly the training scale
    for ct in W.blocks[0] + V.blocks[0]:
        assert ct.lv == top and ct.scale == p.delta
    Wm, Vm = W1.copy(), W1.copy()
    for gamma in mm.nag_gammas(steps):
        Pm = np.polynomial.polynomial.polyval(X @ Vm.T / 8.0, coeffs)
        Wn = Vm - lr * (Pm - Y).T @ X
        Vm, Wm = Wn + gamma * (Wm - Wn), Wn
    # every row of every block: the refresh restores W-bar's s0 / c vertical copies
    got = np.concatenate([o.decrypt_slots(ct).real.reshape(s0, s1) for ct in W.blocks[0]], axis=1)[:, :b]
    gv = np.concatenate([o.decrypt_slots(ct).real.reshape(s0, s1) for ct in V.blocks[0]], axis=1)[:, :b]
    logits = o.decrypt_slots(L.blocks[0][0]).real.reshape(s0, s1)[:a, :c]
    return (np.max(np.abs(got - mm.tile_vertical(Wm, c, s0))), np.max(np.abs(gv - mm.tile_vertical(Vm, c, s0))),
            np.max(np.abs(logits - Xval @ Wm.T)))


def test_nag_loop_with_bootstrapping_follows_the_fp64_loop():
    errs = _run()
    assert max(errs) < 1e-5, errs


def test_planted_mistake_in_the_replication_is_caught(monkeypatch):
    """The unpack's last rotate-and-sum stage dropped: most windows keep zeros."""
    stages = bt.replicate_stages
    monkeypatch.setattr(bt, "replicate_stages", lambda w: stages(w)[:-1])
    assert max(_run()) > 1e-2


def test_packed_refresh_with_a_bound():
    """Entries near 3 (the worst case: a nearly constant vector puts its whole size into one
    coefficient, where bootstrapping's sine stands in for the modular reduction): with bound 4
    the packed refresh scales them into [-1, 1] for bootstrapping and reads them back, within
    5e-5; without it (bound 1) the sine bends them by more than 1e-4."""
    log_n, top = 10, 13
    N = 1 << log_n
    prm = bt.BootParams()
    p = ckks.Params(log_n, 60, top + 1, 50, 2, 61, 2, log_delta=50, n_upper=bt.depth(prm, N), upper_bits=60)
    o = ckks.Oracle(p, seed=6)
    m = 3.0 + np.random.default_rng(2).uniform(-0.05, 0.05, p.slots)
    ct = o.encrypt_int(ckks.encode(m, p.delta, p.N), 1, p.delta, 5)
    errs = {}
    for bound in (1.0, 4.0):
        out = bt.refresh_packed(o, sm.ScaledOps(o, 2.0 ** 55, hoist=True), [ct], p.slots, 1, p.delta, prm,
                                2.0 ** 55, bound)[0]
        assert out.lv == top and out.scale == p.delta
        errs[bound] = np.max(np.abs(o.decrypt_slots(out).real - m))
    assert errs[4.0] < 5e-5 and errs[1.0] > 1e-4, errs
