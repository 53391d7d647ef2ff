"""Protocol 1, step 3 on the GPU (paper_2403_14111_gb300/step.py train_epochs): epochs of NAG
updates over two mini-batches with W and V refreshed after every update, validation logits
after each epoch sent to a client, the best weight kept -- bit for bit against the oracle's
run of the same protocol (oracle/bootstrap.py train_epochs).  The GPU run's client decrypts
the logits through the oracle so that both runs take the same early-stopping decisions."""
import numpy as np
import pytest

import paper_2403_14111_gb300.hetal as H
from paper_2403_14111_gb300 import bootstrap as B
from paper_2403_14111_gb300.step import train_boot_rotations, train_epochs, train_step
from oracle import bootstrap as bt
from oracle import ckks, matmul as mm

from test_oracle_protocol import _setup

pytestmark = pytest.mark.gpu

KINDS = {"colmask": H.PT_COLMASK, "abt_diag": H.PT_ABT_DIAG, "dmask": H.PT_DMASK, "atb_diag": H.PT_ATB_DIAG,
         "sm_coef": H.PT_SM_COEF, "sm_const": H.PT_SM_CONST, "dmask_c": H.PT_DMASK_C}


def test_protocol_epochs_bit_exact():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")
    e = _setup()
    o, p, s0, s1, c = e["o"], e["p"], e["s0"], e["s1"], e["c"]
    oclient = bt.ValidationClient(o, e["yval"], c, patience=1)
    obest, oepochs = bt.train_epochs(e["ops"], e["bops"], e["EW"], e["grads"], e["EXv"], c, p.delta, 3, oclient,
                                     e["prm"], 2.0 ** 55, vops=e["vops"])
    flags = H.FLAG_HOIST | H.FLAG_LAZY_RELIN
    bprm = B.BootstrapParams()
    ctx = H.hetal_ctx_create(10, 60, 14, 50, 2, 61, 2, scale=p.delta, n_upper=p.L - 15, upper_bits=60)
    handles = []
    try:
        assert H.hetal_ctx_moduli(ctx) == p.moduli
        sk = H.hetal_keygen(ctx, 6)
        evk = H.hetal_evk_create(ctx, sk, 6, train_boot_rotations(s0, s1, c, flags, bprm))
        pts, vpts = H.hetal_ptset_create(), H.hetal_ptset_create()
        for src, dst in ((e["ops"].pts, pts), (e["vops"].pts, vpts)):
            for (kind, k, lv), cf in src.items():
                H.hetal_ptset_put(dst, KINDS[kind], k, lv, cf)

        def up(E):
            cts = [bl for row in E.blocks for bl in row]
            d = H.make_desc(E.m, E.n, E.rows, E.cols, s0, s1, cts[0].lv, cts[0].scale)
            h = H.hetal_mat_import(ctx, np.stack([ct.data for ct in cts]), d)
            handles.append(h)
            return h
        hXs, hYs = [up(E) for E in e["EXs"]], [up(E) for E in e["EYs"]]
        hXv, hW = up(e["EXv"]), up(e["EW"])
        grads = [(lambda V, hX=hX, hY=hY: train_step(ctx, evk, hX, V, hY, e["coeffs"], e["valid"], c, e["lr"],
                                                       p.delta, flags, (pts, pts, pts)))
                 for hX, hY in zip(hXs, hYs)]
        gclient = bt.ValidationClient(o, e["yval"], c, patience=1)

        def client(h):   # the same decryption as the oracle's run: through the oracle
            d = H.hetal_mat_desc_get(h)
            data = H.hetal_mat_export(ctx, h)
            rows = [[ckks.Ct(data[r * d.n + j], d.level, d.scale) for j in range(d.n)] for r in range(d.m)]
            return gclient(mm.EncMat(rows, d.rows, d.cols, s0, s1))
        best, epochs = train_epochs(ctx, evk, hW, grads, hXv, c, p.delta, 3, client, flags, vpts, bprm, 2.0 ** 55,
                                    boot_pts=e["bops"].pts)
        handles.append(best)
        assert epochs == oepochs and gclient.losses == oclient.losses
        d = H.hetal_mat_desc_get(best)
        cts = obest.blocks[0]
        assert d.level == cts[0].lv and d.scale == cts[0].scale
        assert np.array_equal(H.hetal_mat_export(ctx, best), np.stack([ct.data for ct in cts]))
        H.hetal_ptset_free(pts)
        H.hetal_ptset_free(vpts)
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
    finally:
        for h in handles:
            H.hetal_mat_free(h)
        H.hetal_ctx_destroy(ctx)
