"""Algorithm ASoftmax (App. A) on the oracle's RNS-CKKS ciphertexts: the scale held by
integer-factor products (Oracle.mult_scaled, reading A10) and the plaintext split
(reading A11), pinned by decryption against the slot simulator (itself pinned to
Table tab:softmaxerr and the worked example) and against closed forms."""
import numpy as np
import pytest

from oracle import ckks, softmax as sm


def _oracle(log_n, n_rescale, n_special=4, alpha=4, seed=5):
    p = ckks.Params(log_n, 60, n_rescale, 60, n_special, 61, alpha, log_delta=40)
    return ckks.Oracle(p, seed=seed)


def test_scaled_products_hold_the_scale_through_a_squaring_chain():
    o = _oracle(10, 13, n_special=2, alpha=2)
    p, delta = o.p, 2.0 ** 40
    rng = np.random.default_rng(4)
    z = rng.uniform(0.9999, 1.0001, p.slots)
    x = o.encrypt_int(ckks.encode(z, delta, p.N), p.top, delta, 11)
    for i in range(12):
        x = o.mult_scaled(x, x, delta)
        t = round(delta * float(p.q[x.lv + 1]) / (delta * delta))   # ~2^20 with 60-bit primes
        assert abs(x.scale / delta - 1) <= 1.5 / t
    assert x.lv == p.top - 12
    got = o.decrypt_slots(x).real
    assert np.max(np.abs(got / z ** 4096 - 1)) < 1e-5
    # the plain product divides by q_l ~ 2^60 and, at scale 2^40, leaves 2^20: the
    # chain's scale collapses, which is why the deep path needs the integer factor
    y = o.encrypt_int(ckks.encode(z, delta, p.N), p.top, delta, 12)
    d, lv, sc = o.tensor(y, y)
    assert o.rescale(o.relin(d, lv, sc)).scale < 2.0 ** 21


def test_integer_product_and_scale_relabel():
    o = _oracle(10, 3, n_special=2, alpha=2)
    p, delta = o.p, 2.0 ** 40
    z = np.random.default_rng(5).uniform(-1, 1, p.slots)
    x = o.encrypt_int(ckks.encode(z, delta, p.N), p.top, delta, 13)
    y = o.mul_int(x, -12)
    assert y.lv == x.lv and y.scale == x.scale
    assert np.max(np.abs(o.decrypt_slots(y).real + 12 * z)) < 1e-8
    ops = sm.ScaledOps(o, delta)
    a = o.encrypt_int(ckks.encode(z, delta, p.N), p.top, delta, 14)
    b = ckks.Ct(a.data.copy(), a.lv, delta * (1 + 3e-7))   # a scale off by a product's rounding
    s = ops.add(a, b)
    assert s.scale == a.scale
    assert np.max(np.abs(o.decrypt_slots(s).real - 2 * z)) < 1e-5
    with pytest.raises(ValueError):
        ops.add(a, ckks.Ct(a.data, a.lv, delta * 1.001))   # not a rounding: refused


@pytest.mark.parametrize("log_n,c,n_rescale", [(11, 2, 74), (10, 3, 89)], ids=["c2", "c3-padded"])
def test_asoftmax_on_ciphertexts_matches_the_slot_simulator(log_n, c, n_rescale):
    o = _oracle(log_n, n_rescale)
    p, delta = o.p, 2.0 ** 40
    s1 = 16
    s0 = p.slots // s1
    prm = sm.Params()
    rng = np.random.default_rng(c)
    X = rng.uniform(-4, 4, (s0, c))
    ref, depth = sm.asoftmax_rows(X, c, prm, s1=s1, s0=s0)
    assert depth == n_rescale
    cp = 1 << max(1, int(np.ceil(np.log2(c))))
    blk = np.zeros((s0, cp))
    blk[:, :c] = X
    M = o.encrypt_int(ckks.encode(np.tile(blk, (1, s1 // cp)).reshape(-1), delta, p.N), p.top, delta, 21)
    ops = sm.ScaledOps(o, delta)
    out = sm.asoftmax_block(ops, M, c, s0, s1, prm)
    assert out.lv == 0
    assert abs(out.scale / delta - 1) < 1e-6
    got = o.decrypt_slots(out).real.reshape(s0, s1)
    # CKKS noise at scale 2^40 through ~80 products: a few 1e-5 at most, against the
    # approximation's own 1e-3
    assert np.max(np.abs(got[:, :c] - ref)) < 5e-5
    # every tile of the row holds the same softmax; padded classes are 0
    for k in range(s1 // cp):
        assert np.max(np.abs(got[:, k * cp:k * cp + c] - got[:, :c])) < 5e-5
        if c < cp:
            assert np.max(np.abs(got[:, k * cp + c:(k + 1) * cp])) < 5e-5
    exact = sm.softmax(X)
    assert np.max(np.abs(got[:, :c] - exact)) <= np.max(np.abs(ref - exact)) + 1e-4
    assert set(k[0] for k in ops.pts) >= {"g1", "g2", "f", "exp", "inv_step", "dep_k"}
