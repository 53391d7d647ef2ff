"""Protocol 1, step 3 on the oracle (oracle/bootstrap.py train_epochs, ValidationClient): epochs
of NAG updates over two mini-batches with W and V refreshed after every update, validation
logits after each epoch, the client's cross-entropy loss and early stopping, the best weight
kept.  Pinned against the same protocol on FP64 matrices with the same polynomial, and the
best-weight bookkeeping against a scripted client."""
import numpy as np

from oracle import bootstrap as bt
from oracle import ckks, matmul as mm, softmax as sm
from paper_2403_14111_gb300 import workloads as wl


def _setup():
    log_n, top = 10, 13
    N = 1 << log_n
    prm = bt.BootParams()
    p = ckks.Params(log_n, 60, top + 1, 50, 2, 61, 2, log_delta=50, n_upper=bt.depth(prm, N), upper_bits=60)
    o = ckks.Oracle(p, seed=6)
    s1 = 32
    s0, c, b = p.slots // s1, 4, 64
    rng = np.random.default_rng(8)
    Xs = [rng.standard_normal((s0, b)) / np.sqrt(b) * 3 for _ in range(2)]
    Ys = [wl.one_hot(rng.integers(0, c, s0), c) for _ in range(2)]
    Xval = rng.standard_normal((s0, b)) / np.sqrt(b) * 3
    yval = rng.integers(0, c, s0)
    W1 = rng.standard_normal((c, b)) * 0.1

    def enc(M, lv, nonce):
        return mm.EncMat([[o.encrypt_int(ckks.encode(bl, p.delta, p.N), lv, p.delta, nonce + 64 * r + j)
                           for j, bl in enumerate(row)] for r, row in enumerate(mm.block_split(M, s0, s1))],
                         M.shape[0], M.shape[1], s0, s1)
    EXs = [enc(X, top, 100 + 200 * i) for i, X in enumerate(Xs)]
    EYs = [enc(mm.tile_horizontal(Y, c, s1), top - 8, 900 + 200 * i) for i, Y in enumerate(Ys)]
    EXv, EW = enc(Xval, top, 1500), enc(mm.tile_vertical(W1, c, s0), top, 1700)
    ops = mm.RnsOps(o, hoist=True, lazy_relin=True)
    vops = mm.RnsOps(o, hoist=True, lazy_relin=True)   # the validation logits' plaintexts (t = 1)
    bops = sm.ScaledOps(o, 2.0 ** 55, hoist=True)
    coeffs, valid, lr = wl.sigmoid_cheb15(), wl.valid_mask(s0, c, c, s0, s1), 1.0 / s0
    grads = [(lambda V, EX=EX, EY=EY: mm.train_step(ops, EX, V, EY, coeffs, valid, c, lr, p.delta)[0])
             for EX, EY in zip(EXs, EYs)]
    return locals()


def _fp64_epochs(e, epochs):
    """The same epochs on FP64 matrices: W after each epoch and the validation losses."""
    W, V = e["W1"].copy(), e["W1"].copy()
    gammas = mm.nag_gammas(epochs * 2)
    Ws, losses, t = [], [], 0
    for _ in range(epochs):
        for X, Y in zip(e["Xs"], e["Ys"]):
            P = np.polynomial.polynomial.polyval(X @ V.T / 8.0, e["coeffs"])
            Wn = V - e["lr"] * (P - Y).T @ X
            V, W = Wn + gammas[t] * (W - Wn), Wn
            t += 1
        z = e["Xval"] @ W.T
        z = z - z.max(axis=1, keepdims=True)
        logp = z - np.log(np.exp(z).sum(axis=1, keepdims=True))
        losses.append(-logp[np.arange(len(e["yval"])), e["yval"]].mean())
        Ws.append(W)
    return Ws, losses


def _decrypt_w(e, Wenc):
    return np.concatenate([e["o"].decrypt_slots(ct).real.reshape(e["s0"], e["s1"]) for ct in Wenc.blocks[0]],
                          axis=1)[:, :e["b"]]


def test_epochs_follow_the_fp64_protocol():
    e = _setup()
    client = bt.ValidationClient(e["o"], e["yval"], e["c"], patience=3)
    best, epochs = bt.train_epochs(e["ops"], e["bops"], e["EW"], e["grads"], e["EXv"], e["c"], e["p"].delta, 2,
                                   client, e["prm"], 2.0 ** 55)
    Ws, losses = _fp64_epochs(e, 2)
    assert epochs == 2
    assert np.max(np.abs(np.array(client.losses) - losses)) < 1e-5
    want = Ws[int(np.argmin(losses))]
    assert np.max(np.abs(_decrypt_w(e, best) - mm.tile_vertical(want, e["c"], e["s0"]))) < 1e-5


def test_best_weight_and_stop():
    """A client that reports an improvement after epoch 1 and none after epoch 2 (and stop):
    training stops after epoch 2 and W* is epoch 1's W, which differs from epoch 2's by more
    than the tolerance, so keeping the last W instead would fail the comparison."""
    e = _setup()
    answers = iter([(False, True), (True, False)])
    seen = []

    def client(logits):
        seen.append(logits)
        return next(answers)
    best, epochs = bt.train_epochs(e["ops"], e["bops"], e["EW"], e["grads"], e["EXv"], e["c"], e["p"].delta, 5,
                                   client, e["prm"], 2.0 ** 55)
    Ws, _ = _fp64_epochs(e, 2)
    assert epochs == 2 and len(seen) == 2
    got = _decrypt_w(e, best)
    assert np.max(np.abs(got - mm.tile_vertical(Ws[0], e["c"], e["s0"]))) < 1e-5
    assert np.max(np.abs(got - mm.tile_vertical(Ws[1], e["c"], e["s0"]))) > 1e-3
