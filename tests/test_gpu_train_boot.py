"""The training loop for several iterations with W and V refreshed by bootstrapping after every
NAG update (paper_2403_14111_gb300/step.py nag_train_boot) through the C ABI, bit for bit
against the oracle's loop on the same ciphertexts (oracle/bootstrap.py nag_train_boot), and its
decryption against the loop on FP64 matrices."""
import numpy as np
import pytest

import paper_2403_14111_gb300.hetal as H
from paper_2403_14111_gb300 import bootstrap as B
from paper_2403_14111_gb300 import workloads as wl
from paper_2403_14111_gb300.step import nag_train_boot, train_boot_rotations
from oracle import bootstrap as bt
from oracle import ckks, matmul as mm, softmax as sm

pytestmark = pytest.mark.gpu

KINDS = {"colmask": H.PT_COLMASK, "abt_diag": H.PT_ABT_DIAG, "dmask": H.PT_DMASK, "atb_diag": H.PT_ATB_DIAG,
         "sm_coef": H.PT_SM_COEF, "sm_const": H.PT_SM_CONST, "dmask_c": H.PT_DMASK_C}


def test_nag_loop_with_bootstrapping_bit_exact():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")
    log_n, steps, top = 10, 2, 13   # training primes up to level 14; a refresh lands at 13
    N = 1 << log_n
    prm, bprm = bt.BootParams(), B.BootstrapParams()
    n_upper = bt.depth(prm, N)
    assert n_upper == B.levels(N, bprm)
    p = ckks.Params(log_n, 60, top + 1, 50, 2, 61, 2, log_delta=50, n_upper=n_upper, upper_bits=60)
    o = ckks.Oracle(p, seed=6)
    s1 = 32
    s0, c, b = p.slots // s1, 4, 64
    a = s0
    flags = H.FLAG_HOIST | H.FLAG_LAZY_RELIN
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
    vops = mm.RnsOps(o, hoist=True, lazy_relin=True)   # the validation logits' plaintexts, kept apart
    bops = sm.ScaledOps(o, 2.0 ** 55, hoist=True)
    oW, oV, oL = bt.nag_train_boot(ops, bops, EX, EW, EY, coeffs, valid, c, lr, p.delta, steps, EXv, prm,
                                   2.0 ** 55, vops=vops)

    ctx = H.hetal_ctx_create(log_n, 60, top + 1, 50, 2, 61, 2, scale=p.delta, n_upper=n_upper, upper_bits=60)
    handles = []
    try:
        sk = H.hetal_keygen(ctx, 6)
        rots = train_boot_rotations(s0, s1, c, flags, bprm)
        evk = H.hetal_evk_create(ctx, sk, 6, rots)
        pts, vpts = H.hetal_ptset_create(), H.hetal_ptset_create()
        for src, dst in ((ops.pts, pts), (vops.pts, vpts)):
            for (kind, k, lv), cf in src.items():
                H.hetal_ptset_put(dst, KINDS[kind], k, lv, cf)

        def up(E):
            cts = [bl for row in E.blocks for bl in row]
            d = H.make_desc(E.m, E.n, E.rows, E.cols, s0, s1, cts[0].lv, cts[0].scale)
            h = H.hetal_mat_import(ctx, np.stack([ct.data for ct in cts]), d)
            handles.append(h)
            return h
        hX, hXv, hW, hY = up(EX), up(EXv), up(EW), up(EY)
        W, V, L = nag_train_boot(ctx, evk, hX, hW, hY, coeffs, valid, c, lr, p.delta, steps, hXv, flags,
                                 pts=(pts, pts, pts, vpts), boot_prm=bprm, delta_w=2.0 ** 55, boot_pts=bops.pts)
        handles += [W, V, L]
        for h, E in ((W, oW), (V, oV), (L, oL)):
            d = H.hetal_mat_desc_get(h)
            cts = [bl for row in E.blocks for bl in row]
            assert d.level == cts[0].lv and d.scale == cts[0].scale
            assert np.array_equal(H.hetal_mat_export(ctx, h), np.stack([ct.data for ct in cts]))
        Wm, Vm = W1.copy(), W1.copy()
        for gamma in mm.nag_gammas(steps):
            Pm = np.polynomial.polynomial.polyval(X @ Vm.T / 8.0, coeffs)
            Wn = Vm - lr * (Pm - Y).T @ X
            Vm, Wm = Wn + gamma * (Wm - Wn), Wn
        assert np.max(np.abs(H.hetal_decrypt(ctx, sk, W)[:c, :b] - Wm)) < 1e-5
        assert np.max(np.abs(H.hetal_decrypt(ctx, sk, L)[:a, :c] - Xval @ Wm.T)) < 1e-5
        H.hetal_ptset_free(pts)
        H.hetal_ptset_free(vpts)
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
    finally:
        for h in handles:
            H.hetal_mat_free(h)
        H.hetal_ctx_destroy(ctx)


def test_training_iteration_with_asoftmax_bit_exact():
    """One NAG iteration whose gradient comes from the paper's softmax (Algorithm ASoftmax,
    refreshed between its stages; step.train_step_asoftmax), W and V refreshed after the
    update, then the validation logits: bit for bit against the oracle's, and within 10^-4
    of the loop on FP64 matrices with the slot simulator's ASoftmax."""
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")
    from paper_2403_14111_gb300 import asoftmax as A
    from paper_2403_14111_gb300.step import train_step_asoftmax
    log_n, top, c_real, c = 10, 13, 3, 4
    N = 1 << log_n
    prm, bprm = bt.BootParams(), B.BootstrapParams()
    n_upper = bt.depth(prm, N)
    p = ckks.Params(log_n, 60, top + 1, 50, 2, 61, 2, log_delta=50, n_upper=n_upper, upper_bits=60)
    o = ckks.Oracle(p, seed=6)
    s1 = 32
    s0, b = p.slots // s1, 64
    a = s0
    d_sm = 2.0 ** 32
    flags = H.FLAG_HOIST | H.FLAG_LAZY_RELIN
    rng = np.random.default_rng(3)
    X = rng.standard_normal((a, b)) / np.sqrt(b) * 4
    Xval = rng.standard_normal((a, b)) / np.sqrt(b)
    Y = wl.one_hot(rng.integers(0, c_real, a), c)
    W1 = rng.standard_normal((c, b)) * 0.5
    W1[c_real:] = 0
    valid, lr = wl.valid_mask(a, c_real, c, s0, s1), 0.5 / a

    def enc(M, lv, nonce, sc=p.delta):
        return mm.EncMat([[o.encrypt_int(ckks.encode(bl, sc, p.N), lv, sc, nonce + 64 * r + j)
                           for j, bl in enumerate(row)] for r, row in enumerate(mm.block_split(M, s0, s1))],
                         M.shape[0], M.shape[1], s0, s1)
    EX, EXv = enc(X, top, 100), enc(Xval, top, 300)
    EW, EY = enc(mm.tile_vertical(W1, c, s0), top, 500), enc(mm.tile_horizontal(Y, c, s1), top - 8, 700, d_sm)
    ops = mm.RnsOps(o, hoist=True, lazy_relin=True)
    vops = mm.RnsOps(o, hoist=True, lazy_relin=True)
    bops = sm.ScaledOps(o, 2.0 ** 55, hoist=True)
    sops = sm.ScaledOps(o, d_sm)
    sops.refresh = bt.Refresher(sops, bops, prm, 2.0 ** 55)
    oW, oV, oL = bt.nag_train_boot(
        ops, bops, EX, EW, EY, None, valid, c, lr, p.delta, 1, EXv, prm, 2.0 ** 55, vops=vops,
        grad=lambda V: bt.train_step_asoftmax(ops, sops, EX, V, EY, c_real, c, valid, lr, p.delta, sm.Params())[0])

    ctx = H.hetal_ctx_create(log_n, 60, top + 1, 50, 2, 61, 2, scale=p.delta, n_upper=n_upper, upper_bits=60)
    handles = []
    try:
        sk = H.hetal_keygen(ctx, 6)
        rots = sorted(set(train_boot_rotations(s0, s1, c, flags, bprm)) | set(A.rotations(c_real, s1)))
        evk = H.hetal_evk_create(ctx, sk, 6, rots)
        pts, vpts = H.hetal_ptset_create(), H.hetal_ptset_create()
        for src, dst in ((ops.pts, pts), (vops.pts, vpts)):
            for (kind, k, lv), cf in src.items():
                H.hetal_ptset_put(dst, KINDS[kind], k, lv, cf)

        def up(E):
            cts = [bl for row in E.blocks for bl in row]
            d = H.make_desc(E.m, E.n, E.rows, E.cols, s0, s1, cts[0].lv, cts[0].scale)
            h = H.hetal_mat_import(ctx, np.stack([ct.data for ct in cts]), d)
            handles.append(h)
            return h
        hX, hXv, hW, hY = up(EX), up(EXv), up(EW), up(EY)
        refresher = B.Refresher(bprm, 2.0 ** 55, pts=bops.pts)

        def grad(V):
            return train_step_asoftmax(ctx, evk, hX, V, hY, c_real, c, valid, lr, p.delta, d_sm, flags,
                                       (pts, pts, pts), A.ASoftmaxParams(), sops.pts, refresher)
        W, V, L = nag_train_boot(ctx, evk, hX, hW, hY, None, valid, c, lr, p.delta, 1, hXv, flags,
                                 pts=(pts, pts, pts, vpts), boot_prm=bprm, delta_w=2.0 ** 55, boot_pts=bops.pts,
                                 grad=grad)
        handles += [W, V, L]
        assert refresher.calls == sops.refresh.calls > 0
        for h, E in ((W, oW), (V, oV), (L, oL)):
            d = H.hetal_mat_desc_get(h)
            cts = [bl for row in E.blocks for bl in row]
            assert d.level == cts[0].lv and d.scale == cts[0].scale
            assert np.array_equal(H.hetal_mat_export(ctx, h), np.stack([ct.data for ct in cts]))
        Wm, Vm = W1.copy(), W1.copy()
        for gamma in mm.nag_gammas(1):
            Pm, _ = sm.asoftmax_rows((X @ Vm.T)[:, :c_real], c_real, sm.Params(), s1=s1, s0=s0)
            Pf = np.zeros((a, c))
            Pf[:, :c_real] = Pm
            Wn = Vm - lr * (Pf - Y).T @ X
            Vm, Wm = Wn + gamma * (Wm - Wn), Wn
        assert np.max(np.abs(H.hetal_decrypt(ctx, sk, W)[:c, :b] - Wm)) < 1e-4
        assert np.max(np.abs(H.hetal_decrypt(ctx, sk, L)[:a, :c] - Xval @ Wm.T)) < 1e-4
        H.hetal_ptset_free(pts)
        H.hetal_ptset_free(vpts)
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
    finally:
        for h in handles:
            H.hetal_mat_free(h)
        H.hetal_ctx_destroy(ctx)


def test_block_copies_and_one_window_refresh():
    """hetal_mat_slice / hetal_mat_stack move blocks unchanged and refuse bad ranges, mixed levels
    and scales and wrong grids; refresh_packed with one window of all the slots (a matrix
    without period) is bit for bit the oracle's, one bootstrapping per block, with and
    without a bound on the entries."""
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")
    from paper_2403_14111_gb300.step import refresh_packed
    log_n, top = 10, 13
    N = 1 << log_n
    prm, bprm = bt.BootParams(), B.BootstrapParams()
    n_upper = bt.depth(prm, N)
    p = ckks.Params(log_n, 60, top + 1, 50, 2, 61, 2, log_delta=50, n_upper=n_upper, upper_bits=60)
    o = ckks.Oracle(p, seed=6)
    s1 = 32
    s0 = p.slots // s1
    rng = np.random.default_rng(4)
    cts = [o.encrypt_int(ckks.encode(rng.uniform(-1, 1, p.slots), p.delta, p.N), 1, p.delta, 40 + i)
           for i in range(3)]
    bops = sm.ScaledOps(o, 2.0 ** 55, hoist=True)
    want = bt.refresh_packed(o, bops, cts, p.slots, 1, p.delta, prm, 2.0 ** 55)
    want4 = bt.refresh_packed(o, bops, cts, p.slots, 1, p.delta, prm, 2.0 ** 55, 4.0)   # with a bound

    ctx = H.hetal_ctx_create(log_n, 60, top + 1, 50, 2, 61, 2, scale=p.delta, n_upper=n_upper, upper_bits=60)
    handles = []
    try:
        sk = H.hetal_keygen(ctx, 6)
        evk = H.hetal_evk_create(ctx, sk, 6, B.rotations(N, bprm))
        M = H.hetal_mat_import(ctx, np.stack([ct.data for ct in cts]),
                               H.make_desc(1, 3, s0, 3 * s1, s0, s1, 1, p.delta))
        handles.append(M)
        # slice and stack: the same residues, in order
        parts = [H.hetal_mat_slice(ctx, M, j, 1) for j in range(3)]
        handles += parts
        again = H.hetal_mat_stack(ctx, parts[::-1], H.make_desc(3, 1, 3 * s0, s1, s0, s1, 0, 0.0))
        handles.append(again)
        d = H.hetal_mat_desc_get(again)
        assert (d.m, d.n, d.rows, d.cols, d.level, d.scale) == (3, 1, 3 * s0, s1, 1, p.delta)
        assert np.array_equal(H.hetal_mat_export(ctx, again), np.stack([ct.data for ct in cts[::-1]]))
        two = H.hetal_mat_slice(ctx, M, 1, 2)
        handles.append(two)
        assert np.array_equal(H.hetal_mat_export(ctx, two), np.stack([ct.data for ct in cts[1:]]))
        for first, count in ((-1, 1), (2, 2), (0, 0), (3, 1)):
            with pytest.raises(H.HetalError):
                H.hetal_mat_slice(ctx, M, first, count)
        low = H.hetal_mat_drop(ctx, parts[0], 0)
        other = H.hetal_mat_set_scale(ctx, parts[1], 2.0 * p.delta)
        handles += [low, other]
        for mats, desc in (([parts[0], low], H.make_desc(1, 2, s0, 2 * s1, s0, s1, 0, 0.0)),
                           ([parts[0], other], H.make_desc(1, 2, s0, 2 * s1, s0, s1, 0, 0.0)),
                           ([parts[0], parts[1]], H.make_desc(1, 3, s0, 3 * s1, s0, s1, 0, 0.0))):
            with pytest.raises(H.HetalError):
                H.hetal_mat_stack(ctx, mats, desc)
        # the refresh with one window of all the slots
        out = refresh_packed(ctx, evk, [M], p.slots, 1, p.delta, bprm, boot_pts=bops.pts)[0]
        handles.append(out)
        d = H.hetal_mat_desc_get(out)
        assert d.level == want[0].lv and d.scale == want[0].scale == p.delta
        assert np.array_equal(H.hetal_mat_export(ctx, out), np.stack([ct.data for ct in want]))
        out4 = refresh_packed(ctx, evk, [M], p.slots, 1, p.delta, bprm, boot_pts=bops.pts, bound=4.0)[0]
        handles.append(out4)
        assert H.hetal_mat_desc_get(out4).scale == want4[0].scale
        assert np.array_equal(H.hetal_mat_export(ctx, out4), np.stack([ct.data for ct in want4]))
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
    finally:
        for h in handles:
            H.hetal_mat_free(h)
        H.hetal_ctx_destroy(ctx)
