"""CKKS bootstrapping (Sec. 2.2) on the GPU through the C ABI (paper_2403_14111_gb300/
bootstrap.py), bit for bit against the oracle's run on the same ciphertext
(oracle/bootstrap.py), and ModRaise and x sqrt(-1) on their own."""
import numpy as np
import pytest

import paper_2403_14111_gb300.hetal as H
from paper_2403_14111_gb300 import bootstrap as B
from oracle import bootstrap as bt
from oracle import ckks, softmax as sm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")


def _pair(log_n, n_rescale, seed, steps):
    P = dict(log_n=log_n, q0_bits=60, n_rescale=n_rescale, rescale_bits=60, n_special=2, special_bits=61, alpha=2)
    ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                             P["special_bits"], P["alpha"], scale=2.0 ** 40)
    o = ckks.Oracle(ckks.Params(log_n, 60, n_rescale, 60, 2, 61, 2, log_delta=40), seed=seed)
    sk = H.hetal_keygen(ctx, seed)
    evk = H.hetal_evk_create(ctx, sk, seed, steps)
    return ctx, o, sk, evk


def _up(ctx, ct, s0, s1):
    return H.hetal_mat_import(ctx, ct.data[None], H.make_desc(1, 1, s0, s1, s0, s1, ct.lv, ct.scale))


def _same(ctx, h, ct):
    d = H.hetal_mat_desc_get(h)
    assert d.level == ct.lv and d.scale == ct.scale, (d.level, ct.lv, d.scale, ct.scale)
    got = H.hetal_mat_export(ctx, h)[0]
    bad = np.argwhere(got != ct.data)
    assert bad.size == 0, "first mismatch at %s of %d" % (bad[0], len(bad))


def test_mod_raise_and_mul_i_match_oracle():
    ctx, o, sk, evk = _pair(12, 6, 3, [1])
    hs = []
    try:
        p = o.p
        z = np.random.default_rng(2).uniform(-1, 1, p.slots)
        ct = o.encrypt_int(ckks.encode(z, 2.0 ** 50, p.N), 0, 2.0 ** 50, 8)
        h = _up(ctx, ct, 128, 16)
        hs.append(h)
        r = H.hetal_mod_raise(ctx, h, p.top)
        hs.append(r)
        _same(ctx, r, o.mod_raise(ct, p.top))
        hi = H.hetal_mul_i(ctx, r)
        hs.append(hi)
        _same(ctx, hi, o.mul_i(o.mod_raise(ct, p.top)))
        with pytest.raises(H.HetalError):
            H.hetal_mod_raise(ctx, r, p.top)   # not a level-0 matrix
    finally:
        for x in hs:
            H.hetal_mat_free(x)
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
        H.hetal_ctx_destroy(ctx)


@pytest.mark.parametrize("log_n,fft", [(10, True), (11, True), (10, False)],
                         ids=["N10 factored", "N11 factored", "N10 dense"])
def test_bootstrap_matches_oracle_bit_for_bit(log_n, fft):
    prm = bt.BootParams(fft=fft)
    bprm = B.BootstrapParams(fft=fft)
    N = 1 << log_n
    n_rescale = bt.depth(prm, N) + 3
    ctx, o, sk, evk = _pair(log_n, n_rescale, 4, B.rotations(N, bprm))
    hs = []
    try:
        p = o.p
        assert B.levels(N, bprm) == bt.depth(prm, N)
        m = np.random.default_rng(1).uniform(-1, 1, p.slots)
        d_in, d_w = 2.0 ** 50, 2.0 ** 50
        ct = o.encrypt_int(ckks.encode(m, d_in, N), 0, d_in, 9)
        ops = sm.ScaledOps(o, d_w, hoist=True)
        want = bt.bootstrap_raised(ops, o.mod_raise(ct, p.top), N, d_w, prm)
        want = ckks.Ct(want.data, want.lv, want.scale * d_in / float(p.q[0]))
        s1 = 16
        h = _up(ctx, ct, p.slots // s1, s1)
        hs.append(h)
        out = B.bootstrap(ctx, evk, h, d_in, d_w, bprm, pts=ops.pts)
        hs.append(out)
        _same(ctx, out, want)
        got = H.hetal_decrypt(ctx, sk, out).reshape(-1)
        assert np.max(np.abs(got - m)) < 5e-5
        # the library's own plaintext encodings: the same refresh to CKKS noise
        # device plaintexts uploaded once and reused: the same bits, first run and second
        from paper_2403_14111_gb300 import circuit
        cache = {}
        try:
            for _ in range(2):
                again = B.bootstrap(ctx, evk, h, d_in, d_w, bprm, pts=ops.pts, cache=cache)
                hs.append(again)
                _same(ctx, again, want)
        finally:
            circuit.free_plains(cache)
        own = B.bootstrap(ctx, evk, h, d_in, d_w, bprm)
        hs.append(own)
        assert np.max(np.abs(H.hetal_decrypt(ctx, sk, own).reshape(-1) - m)) < 5e-5
        assert H.hetal_mat_desc_get(own).level == p.top - B.levels(N, bprm)
    finally:
        for x in hs:
            H.hetal_mat_free(x)
        H.hetal_evk_free(evk)
        H.hetal_sk_free(sk)
        H.hetal_ctx_destroy(ctx)
