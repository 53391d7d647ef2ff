"""Pins for the oracle's training loop (Protocol 1, step 3, with NAG as Sec. 2.1 defines it):
the gamma sequence from its recurrence, and the loop on the FP64 slot simulator in the block
layout against the same updates written directly on matrices."""
import math

import numpy as np

from oracle import matmul as mm
from paper_2403_14111_gb300 import workloads as wl


def test_gammas():
    g = mm.nag_gammas(4)
    lam = [0.0, 1.0, (1 + math.sqrt(5)) / 2]
    lam.append((1 + math.sqrt(1 + 4 * lam[2] ** 2)) / 2)
    lam.append((1 + math.sqrt(1 + 4 * lam[3] ** 2)) / 2)
    lam.append((1 + math.sqrt(1 + 4 * lam[4] ** 2)) / 2)
    assert g[0] == 0.0   # V_2 = W_2
    for t in range(1, 5):
        assert abs(g[t - 1] - (1 - lam[t]) / lam[t + 1]) < 1e-15
    assert all(x <= 0 for x in g)


def fp64_nag(X, Y, W1, coeffs, c, s1, lr, steps, Xval):
    """The same NAG on plain matrices: logits/8 = X V^T / 8, P = p(logits/8) on the real
    classes (padded columns 0), G = lr (P - Y)^T X."""
    W = V = W1.copy()
    cls = np.arange(c) < c   # all c columns of the c-padded layout are classes here
    for gamma in mm.nag_gammas(steps):
        P = np.polynomial.polynomial.polyval(X @ V.T / 8.0, coeffs) * cls
        G = lr * (P - Y).T @ X
        Wn = V - G
        V = Wn + gamma * (W - Wn)
        W = Wn
    return W, V, Xval @ W.T


def test_loop_on_slots_matches_matrices():
    s0, s1, c, a, b = 128, 32, 4, 100, 64
    rng = np.random.default_rng(3)
    X = rng.standard_normal((a, b)) / np.sqrt(b)
    Xval = rng.standard_normal((a, b)) / np.sqrt(b)
    Y = wl.one_hot(rng.integers(0, c, a), c)
    W1 = rng.standard_normal((c, b)) * 0.1
    coeffs = wl.sigmoid_cheb15()
    valid = wl.valid_mask(a, c, c, s0, s1)
    lr = 0.5 / a
    ops = mm.SlotOps(s0 * s1)

    def enc(M):
        blocks = mm.block_split(M, s0, s1)
        return mm.EncMat([[mm.SV(b_.reshape(-1).astype(complex), 60) for b_ in row] for row in blocks],
                         M.shape[0], M.shape[1], s0, s1)

    EX, EXv = enc(X), enc(Xval)
    EY = enc(mm.tile_horizontal(Y, c, s1))
    EW = enc(mm.tile_vertical(W1, c, s0))
    W, V, logits = mm.nag_train(ops, EX, EW, EY, coeffs, valid, c, lr, 1.0, 2, EXv)
    Wm, Vm, Lm = fp64_nag(X, Y, W1, coeffs, c, s1, lr, 2, Xval)
    got_W = np.concatenate([blk.z.real.reshape(s0, s1) for blk in W.blocks[0]], axis=1)[:c, :b]
    got_V = np.concatenate([blk.z.real.reshape(s0, s1) for blk in V.blocks[0]], axis=1)[:c, :b]
    got_L = logits.blocks[0][0].z.real.reshape(s0, s1)[:a, :c]
    assert np.max(np.abs(got_W - Wm)) < 1e-9
    assert np.max(np.abs(got_V - Vm)) < 1e-9
    assert np.max(np.abs(got_L - Lm)) < 1e-9
    # the gradient step moved W
    assert np.max(np.abs(Wm - W1)) > 1e-3
