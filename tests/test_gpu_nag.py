"""The encrypted training loop (Protocol 1, step 3: two NAG iterations, Sec. 2.1, then the
validation logits) through the C ABI on a 28-level chain at N = 2^13, bit-exact with the
oracle's loop at every output, and its decryption against the same loop on FP64 matrices."""
import numpy as np
import pytest

import paper_2403_14111_gb300.hetal as H
from paper_2403_14111_gb300 import workloads as wl
from paper_2403_14111_gb300.step import nag_train, step_rotations
from oracle import ckks, matmul as mm

pytestmark = pytest.mark.gpu

KINDS = {"colmask": H.PT_COLMASK, "abt_diag": H.PT_ABT_DIAG, "dmask": H.PT_DMASK, "atb_diag": H.PT_ATB_DIAG,
         "sm_coef": H.PT_SM_COEF, "sm_const": H.PT_SM_CONST, "dmask_c": H.PT_DMASK_C}


@pytest.mark.parametrize("flags", [H.FLAG_HOIST | H.FLAG_LAZY_RELIN,
                                   H.FLAG_HOIST | H.FLAG_LAZY_RELIN | H.FLAG_RADIX_SUM | H.FLAG_SHARED_ROT],
                         ids=["hoist+lazy", "all"])
def test_nag_two_steps_and_validation_bit_exact(flags):
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")
    P = wl.PARAMS_N13_NAG
    op = ckks.Params(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                     P["special_bits"], P["alpha"], log_delta=P["log_scale"])
    o = ckks.Oracle(op, seed=6)
    p = o.p
    s0, s1, c, a, b = 128, 32, 4, 100, 64
    rng = np.random.default_rng(3)
    X = rng.standard_normal((a, b)) / np.sqrt(b)
    Xval = rng.standard_normal((a, b)) / np.sqrt(b)
    Y = wl.one_hot(rng.integers(0, c, a), c)
    W1 = rng.standard_normal((c, b)) * 0.1
    coeffs = wl.sigmoid_cheb15()
    valid = wl.valid_mask(a, c, c, s0, s1)
    lr = 0.5 / a
    top = p.top
    lvY = top - 8   # where the step's softmax lands

    def enc(M, lv, nonce):
        return mm.EncMat([[o.encrypt_int(ckks.encode(bl, p.delta, p.N), lv, p.delta, nonce + 64 * r + j)
                           for j, bl in enumerate(row)] for r, row in enumerate(mm.block_split(M, s0, s1))],
                         M.shape[0], M.shape[1], s0, s1)

    EX, EXv = enc(X, top, 100), enc(Xval, top, 300)
    EW = enc(mm.tile_vertical(W1, c, s0), top, 500)
    EY = enc(mm.tile_horizontal(Y, c, s1), lvY, 700)
    ops = mm.RnsOps(o, hoist=bool(flags & H.FLAG_HOIST), lazy_relin=bool(flags & H.FLAG_LAZY_RELIN),
                    radix_sum=bool(flags & H.FLAG_RADIX_SUM), shared_rot=bool(flags & H.FLAG_SHARED_ROT))
    oW, oV, oL = mm.nag_train(ops, EX, EW, EY, coeffs, valid, c, lr, p.delta, 2, EXv)

    ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                             P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"])
    handles = []
    try:
        sk = H.hetal_keygen(ctx, 6)
        evk = H.hetal_evk_create(ctx, sk, 6, step_rotations(s0, s1, c, flags))
        pts = H.hetal_ptset_create()
        for (kind, k, lv), cf in ops.pts.items():
            H.hetal_ptset_put(pts, KINDS[kind], k, lv, cf)

        def up(E):
            cts = [bl for row in E.blocks for bl in row]
            d = H.make_desc(E.m, E.n, E.rows, E.cols, s0, s1, cts[0].lv, cts[0].scale)
            h = H.hetal_mat_import(ctx, np.stack([ct.data for ct in cts]), d)
            handles.append(h)
            return h

        hX, hXv, hW, hY = up(EX), up(EXv), up(EW), up(EY)
        W, V, L = nag_train(ctx, evk, hX, hW, hY, coeffs, valid, c, lr, p.delta, 2, hXv, flags,
                            pts=(pts, pts, pts, pts))
        handles += [W, V, L]
        for h, E in ((W, oW), (V, oV), (L, oL)):
            d = H.hetal_mat_desc_get(h)
            cts = [bl for row in E.blocks for bl in row]
            assert d.level == cts[0].lv and d.scale == cts[0].scale
            assert np.array_equal(H.hetal_mat_export(ctx, h), np.stack([ct.data for ct in cts]))
        assert H.hetal_mat_desc_get(L).level >= 0
        # the loop on FP64 matrices
        Wm, Vm = W1.copy(), W1.copy()
        for gamma in mm.nag_gammas(2):
            Pm = np.polynomial.polynomial.polyval(X @ Vm.T / 8.0, coeffs)
            Wn = Vm - lr * (Pm - Y).T @ X
            Vm, Wm = Wn + gamma * (Wm - Wn), Wn
        got = H.hetal_decrypt(ctx, sk, W)[:c, :b]
        assert np.max(np.abs(got - Wm)) <= 1e-4
        got = H.hetal_decrypt(ctx, sk, L)[:a, :c]
        assert np.max(np.abs(got - Xval @ Wm.T)) <= 1e-4
        H.hetal_ptset_free(pts)
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
    finally:
        for h in handles:
            H.hetal_mat_free(h)
        H.hetal_ctx_destroy(ctx)
