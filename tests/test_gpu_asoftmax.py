"""Algorithm ASoftmax (App. A) on the GPU through the C ABI, bit for bit against the
oracle's run on the same ciphertexts (oracle/softmax.py ScaledOps), and the
primitives its deep parameter sets use for the first time: digits of 3, 4 and 6 primes
with as many special primes (base conversions of ModUp and ModDown fused into the
forward transform's column pass),
more than 8 digits (key inner products in groups of 8), the scaled product, the
integer product, integer plaintexts and the scale relabel."""
import numpy as np
import pytest

import paper_2403_14111_gb300.hetal as H
from paper_2403_14111_gb300 import asoftmax as A
from paper_2403_14111_gb300 import workloads as wl
from oracle import ckks, softmax as sm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")


class Pair:
    """A library context and an oracle with the same parameters and key seed."""

    def __init__(self, P, seed, steps):
        self.ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                                      P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"])
        self.o = ckks.Oracle(ckks.Params(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"],
                                         P["n_special"], P["special_bits"], P["alpha"], log_delta=P["log_scale"]),
                             seed=seed)
        self.p = self.o.p
        self.sk = H.hetal_keygen(self.ctx, seed)
        self.evk = H.hetal_evk_create(self.ctx, self.sk, seed, list(steps))
        self.handles = []

    def up(self, ct, s0, s1):
        h = H.hetal_mat_import(self.ctx, ct.data[None], H.make_desc(1, 1, s0, s1, s0, s1, ct.lv, ct.scale))
        self.handles.append(h)
        return h

    def keep(self, h):
        self.handles.append(h)
        return h

    def same(self, h, ct):
        d = H.hetal_mat_desc_get(h)
        assert d.level == ct.lv and d.scale == ct.scale, (d.level, ct.lv, d.scale, ct.scale)
        got = H.hetal_mat_export(self.ctx, h)[0]
        bad = np.argwhere(got != ct.data)
        assert bad.size == 0, "first mismatch at %s of %d" % (bad[0], len(bad))

    def close(self):
        for h in self.handles:
            H.hetal_mat_free(h)
        H.hetal_evk_free(self.evk)
        H.hetal_sk_free(self.sk)
        H.hetal_ctx_destroy(self.ctx)


WIDE = dict(log_n=12, q0_bits=60, n_rescale=9, rescale_bits=60, n_special=4, special_bits=61, alpha=4, log_scale=40)
WIDE3 = dict(log_n=12, q0_bits=60, n_rescale=9, rescale_bits=60, n_special=3, special_bits=61, alpha=3, log_scale=40)
WIDE6 = dict(log_n=12, q0_bits=60, n_rescale=11, rescale_bits=60, n_special=6, special_bits=61, alpha=6, log_scale=40)
MANY = dict(log_n=12, q0_bits=60, n_rescale=9, rescale_bits=60, n_special=1, special_bits=61, alpha=1, log_scale=40)


@pytest.mark.parametrize("P", [WIDE, WIDE3, WIDE6, MANY], ids=["4-prime digits, 4 special", "3-prime digits, 3 special",
                                                             "6-prime digits, 6 special", "10 digits"])
def test_deep_parameter_primitives_match_oracle(P):
    e = Pair(P, 9, [1, 2, 4, -1, -8])
    try:
        o, p = e.o, e.p
        delta = 2.0 ** 40
        s1 = 16
        s0 = p.slots // s1
        nm = p.L + p.K
        assert np.array_equal(H.hetal_evk_export(e.ctx, e.evk, 0, 0, p.dnum_full(), nm), o.key(ckks.KID_RELIN))
        assert np.array_equal(H.hetal_evk_export(e.ctx, e.evk, 2, -8, p.dnum_full(), nm),
                              o.key(ckks.kid_rot(p.slots - 8)))
        rng = np.random.default_rng(3)
        za, zb = rng.uniform(-1, 1, p.slots), rng.uniform(-1, 1, p.slots)
        a = o.encrypt_int(ckks.encode(za, delta, p.N), p.top, delta, 5)
        b = o.encrypt_int(ckks.encode(zb, delta, p.N), p.top - 2, delta, 6)
        ha, hb = e.up(a, s0, s1), e.up(b, s0, s1)
        for r in (1, -1, -8):
            e.same(e.keep(H.hetal_rotate(e.ctx, e.evk, ha, r)), o.rot_raw(a, r % p.slots))
        e.same(e.keep(H.hetal_rotate_sum(e.ctx, e.evk, ha, [1, 2, 4])), o.rot_sum(a, [1, 2, 4]))
        e.same(e.keep(H.hetal_mult_scaled(e.ctx, e.evk, ha, hb, delta)), o.mult_scaled(a, b, delta))
        e.same(e.keep(H.hetal_mul_int(e.ctx, ha, -37)), o.mul_int(a, -37))
        ops = sm.ScaledOps(o, delta)
        vals = rng.uniform(-12, 12, p.slots)   # above 4: split into 2^k and vals / 2^k
        k = int(np.ceil(np.log2(np.max(np.abs(vals)) / 4)))
        want = ops.cmult(a, vals, ("t", 0))
        pt = ops.pts[("t", 0, p.top)]
        got = e.keep(H.hetal_cmult_int(e.ctx, e.keep(H.hetal_mul_int(e.ctx, ha, 1 << k)), pt, a.scale))
        e.same(got, want)
        want = ops.add_plain(a, vals / 16, ("u", 0))
        e.same(e.keep(H.hetal_add_plain_int(e.ctx, ha, ops.pts[("u", 0, p.top)])), want)
        relabel = e.keep(H.hetal_mat_set_scale(e.ctx, ha, delta * (1 + 2e-7)))
        assert H.hetal_mat_desc_get(relabel).scale == delta * (1 + 2e-7)
        with pytest.raises(H.HetalError):
            H.hetal_mat_set_scale(e.ctx, ha, -delta)
    finally:
        e.close()


@pytest.mark.parametrize("P,c,s1", [(wl.PARAMS_N13_SMX2, 2, 16), (wl.PARAMS_N12_SMX4, 3, 16)],
                         ids=["N13 c=2", "N12 c=3 padded"])
def test_asoftmax_matches_oracle_bit_for_bit(P, c, s1):
    prm = A.ASoftmaxParams()
    e = Pair(P, 8, A.rotations(c, s1))
    try:
        o, p = e.o, e.p
        delta = 2.0 ** P["log_scale"]
        s0 = p.slots // s1
        assert A.depth(c, prm) == p.top
        rng = np.random.default_rng(10 + c)
        X = rng.uniform(-4, 4, (s0, c))
        cp = A.padded_classes(c)
        blk = np.zeros((s0, cp))
        blk[:, :c] = X
        M = o.encrypt_int(ckks.encode(np.tile(blk, (1, s1 // cp)).reshape(-1), delta, p.N), p.top, delta, 31)
        ops = sm.ScaledOps(o, delta)
        want = sm.asoftmax_block(ops, M, c, s0, s1, sm.Params())
        hM = e.up(M, s0, s1)
        out = e.keep(A.asoftmax(e.ctx, e.evk, hM, c, s0, s1, delta, prm, pts=ops.pts))
        e.same(out, want)
        got = H.hetal_decrypt(e.ctx, e.sk, out)[:, :c]
        ref, _ = sm.asoftmax_rows(X, c, sm.Params(), s1=s1, s0=s0)
        assert np.max(np.abs(got - ref)) < 5e-5
        exact = sm.softmax(X)
        assert np.max(np.abs(got - exact)) <= np.max(np.abs(ref - exact)) + 1e-4
        # the library's own plaintext encodings: the same function to CKKS noise
        own = e.keep(A.asoftmax(e.ctx, e.evk, hM, c, s0, s1, delta, prm))
        assert np.max(np.abs(H.hetal_decrypt(e.ctx, e.sk, own)[:, :c] - ref)) < 5e-5
    finally:
        e.close()
