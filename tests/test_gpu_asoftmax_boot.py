"""Algorithm ASoftmax (App. A) with bootstrapping between its stages on the GPU through the
C ABI (paper_2403_14111_gb300/asoftmax.py refresh points, bootstrap.Refresher), bit for bit
against the oracle's run on the same ciphertexts (oracle/softmax.py, oracle/bootstrap.py
Refresher), on 14 training levels under bootstrapping's primes."""
import numpy as np
import pytest

import paper_2403_14111_gb300.hetal as H
from paper_2403_14111_gb300 import asoftmax as A
from paper_2403_14111_gb300 import bootstrap as B
from oracle import bootstrap as bt
from oracle import ckks, softmax as sm

pytestmark = pytest.mark.gpu


def test_asoftmax_with_refreshes_matches_oracle_bit_for_bit():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")
    log_n, top, c = 10, 13, 3
    N = 1 << log_n
    prm, bprm = bt.BootParams(), B.BootstrapParams()
    n_upper = bt.depth(prm, N)
    p = ckks.Params(log_n, 60, top + 1, 50, 2, 61, 2, log_delta=50, n_upper=n_upper, upper_bits=60)
    o = ckks.Oracle(p, seed=6)
    s1 = 16
    s0 = p.slots // s1
    cp = A.padded_classes(c)
    d_sm = 2.0 ** 32
    X = np.random.default_rng(5).uniform(-4, 4, (s0, c))
    blk = np.zeros((s0, cp))
    blk[:, :c] = X
    M = o.encrypt_int(ckks.encode(np.tile(blk, (1, s1 // cp)).reshape(-1), d_sm, p.N), top, d_sm, 31)
    sops = sm.ScaledOps(o, d_sm)
    bops = sm.ScaledOps(o, 2.0 ** 55, hoist=True)
    sops.refresh = bt.Refresher(sops, bops, prm, 2.0 ** 55)
    want = sm.asoftmax_block(sops, M, c, s0, s1, sm.Params())

    ctx = H.hetal_ctx_create(log_n, 60, top + 1, 50, 2, 61, 2, scale=p.delta, n_upper=n_upper, upper_bits=60)
    handles = []
    try:
        sk = H.hetal_keygen(ctx, 6)
        evk = H.hetal_evk_create(ctx, sk, 6, sorted(set(A.rotations(c, s1)) | set(B.rotations(N, bprm))))
        hM = H.hetal_mat_import(ctx, M.data[None], H.make_desc(1, 1, s0, s1, s0, s1, M.lv, M.scale))
        handles.append(hM)
        refresher = B.Refresher(bprm, 2.0 ** 55, pts=bops.pts)
        out = A.asoftmax(ctx, evk, hM, c, s0, s1, d_sm, A.ASoftmaxParams(), pts=sops.pts, refresh=refresher)
        handles.append(out)
        assert refresher.calls == sops.refresh.calls > 0
        d = H.hetal_mat_desc_get(out)
        assert d.level == want.lv and d.scale == want.scale
        got = H.hetal_mat_export(ctx, out)[0]
        bad = np.argwhere(got != want.data)
        assert bad.size == 0, "first mismatch at %s of %d" % (bad[0], len(bad))
        ref, _ = sm.asoftmax_rows(X, c, sm.Params(), s1=s1, s0=s0)
        assert np.max(np.abs(H.hetal_decrypt(ctx, sk, out)[:, :c] - ref)) < 2e-3
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
    finally:
        for h in handles:
            H.hetal_mat_free(h)
        H.hetal_ctx_destroy(ctx)
