"""Pins for the oracle's CKKS layer: encoding against its O(N^2) definition and
closed forms, exact encryption/decryption (the decrypted polynomial is the
message plus the sampled error, exactly), and the slot identities of Lrot,
Conj, multiplication by sqrt(-1), Mult and CMult (Sec. 2.2)."""
import numpy as np
import pytest

from oracle import ckks, matmul as mm

L = ckks.lib


@pytest.fixture(scope="module")
def o13():
    return ckks.Oracle(ckks.params_n13(), seed=1)


def test_encode_matches_definition():
    N = 64
    rng = np.random.default_rng(0)
    z = rng.uniform(-1, 1, N // 2) + 1j * rng.uniform(-1, 1, N // 2)
    assert np.array_equal(ckks.encode(z, 2.0 ** 30, N), ckks.encode_direct(z, 2.0 ** 30, N))


def test_encode_constant_is_constant_polynomial():
    N = 1 << 10
    m = ckks.encode(np.full(N // 2, 0.75), 2.0 ** 40, N)
    assert m[0] == int(0.75 * 2 ** 40) and np.all(m[1:] == 0)


def test_decode_inverts_encode():
    N = 1 << 13
    rng = np.random.default_rng(1)
    z = rng.uniform(-1, 1, N // 2) + 1j * rng.uniform(-1, 1, N // 2)
    m = ckks.encode(z, 2.0 ** 40, N)
    assert np.max(np.abs(ckks.decode_real_coeffs(m, 2.0 ** 40, N) - z)) < 1e-9


def test_slot_order_rotation_and_conjugation_on_plaintexts():
    """X -> X^{5^r} rotates slots left by r; X -> X^{-1} conjugates (slot j at zeta^{5^j})."""
    N = 1 << 10
    q = ckks.gen_primes(2 * N, 60, 1)[0]
    rng = np.random.default_rng(2)
    z = rng.uniform(-1, 1, N // 2) + 1j * rng.uniform(-1, 1, N // 2)
    m = ckks.encode(z, 2.0 ** 30, N)
    mr = ckks.u64([int(v) % q for v in m])
    for g, want in [(pow(5, 7, 2 * N), np.roll(z, -7)), (2 * N - 1, np.conj(z))]:
        out = np.zeros(N, dtype=np.uint64)
        L().orc_automorphism(ckks.P(mr), ckks.P(out), N, g, q)
        cen = np.array([int(v) if int(v) < q // 2 else int(v) - q for v in out], dtype=np.float64)
        assert np.max(np.abs(ckks.decode_real_coeffs(cen, 2.0 ** 30, N) - want)) < 1e-6


def test_encrypt_decrypt_exact(o13):
    p = o13.p
    rng = np.random.default_rng(3)
    m = rng.integers(-2 ** 40, 2 ** 40, p.N).astype(np.int64)
    for lv in (0, p.top):
        ct = o13.encrypt_int(m, lv, p.delta, nonce=5)
        e = np.zeros(p.N, dtype=np.int64)
        L().orc_sample_cbd(o13.seed, L().orc_stream_enc_e(5), p.N, ckks.P(e))
        assert np.array_equal(o13.decrypt_int(ct), (m + e).astype(np.float64))


def _enc(o, z, lv=None, nonce=1):
    p = o.p
    lv = p.top if lv is None else lv
    return o.encrypt_int(ckks.encode(z, p.delta, p.N), lv, p.delta, nonce)


def test_rotation_conjugation_and_i(o13):
    p = o13.p
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, p.slots) + 1j * rng.uniform(-1, 1, p.slots)
    ct = _enc(o13, z)
    for r in (1, 5, 64, p.slots - 1):
        assert np.max(np.abs(o13.decrypt_slots(o13.rot_raw(ct, r)) - np.roll(z, -r))) < 1e-5
    assert np.max(np.abs(o13.decrypt_slots(o13.conj_raw(ct)) - np.conj(z))) < 1e-5
    assert np.max(np.abs(o13.decrypt_slots(o13.mul_i(ct)) - 1j * z)) < 1e-8
    # group law on ciphertexts: Lrot(Lrot(ct, 3), 5) decrypts like Lrot(ct, 8)
    r35 = o13.rot_raw(o13.rot_raw(ct, 3), 5)
    assert np.max(np.abs(o13.decrypt_slots(r35) - np.roll(z, -8))) < 1e-5


def test_hoisted_equals_plain_after_decryption(o13):
    p = o13.p
    rng = np.random.default_rng(5)
    z = rng.uniform(-1, 1, p.slots)
    ct = _enc(o13, z)
    rs = [3, 32, 100]
    hs = o13.automorph_hoisted(ct, [p.galois_rot(r) for r in rs], [ckks.kid_rot(r) for r in rs])
    for r, h in zip(rs, hs):
        a = o13.decrypt_slots(h)
        b = o13.decrypt_slots(o13.rot_raw(ct, r))
        assert np.max(np.abs(a - b)) < 1e-5
        assert np.max(np.abs(a - np.roll(z, -r))) < 1e-5


def test_rot_sum_is_sum_of_rotations(o13):
    """rot_sum shares one ModUp and one ModDown: with one amount it is exactly
    a + (hoisted rotation); with several it decrypts to the sum of the rotated
    slot vectors, and its residues differ from the sum of separately switched
    rotations only by the rounding of ModDown (at most K + 1 per coefficient)."""
    p = o13.p
    rng = np.random.default_rng(8)
    z = rng.uniform(-1, 1, p.slots)
    ct = _enc(o13, z)
    one = o13.rot_sum(ct, [5])
    h = o13.automorph_hoisted(ct, [p.galois_rot(5)], [ckks.kid_rot(5)])[0]
    assert np.array_equal(one.data, o13.add(ct, h).data)
    rs = [3, 32, 100, p.slots - 7]
    many = o13.rot_sum(ct, rs)
    want = z + sum(np.roll(z, -r) for r in rs)
    assert np.max(np.abs(o13.decrypt_slots(many) - want)) < 1e-5
    sep = ct
    for r in rs:
        sep = o13.add(sep, o13.automorph_hoisted(ct, [p.galois_rot(r)], [ckks.kid_rot(r)])[0])
    q = np.array(p.q[:ct.lv + 1], dtype=object)[:, None]
    d = (many.data.astype(object) - sep.data.astype(object)) % q[None]
    d = np.where(d > q[None] // 2, d - q[None], d)
    assert np.abs(d).max() <= (p.K + 1) * len(rs)


def test_mult_cmult_rescale(o13):
    p = o13.p
    rng = np.random.default_rng(6)
    za = rng.uniform(-1, 1, p.slots)
    zb = rng.uniform(-1, 1, p.slots) + 1j * rng.uniform(-1, 1, p.slots)
    a, b = _enc(o13, za, nonce=1), _enc(o13, zb, nonce=2)
    ops = mm.RnsOps(o13)
    ab = ops.mult(a, b)
    assert ab.lv == p.top - 1
    assert np.max(np.abs(o13.decrypt_slots(ab) - za * zb)) < 1e-6
    mask = rng.uniform(-1, 1, p.slots)
    cm = ops.cmult(a, mask, ("t", 0))
    assert cm.lv == p.top - 1 and cm.scale == a.scale
    assert np.max(np.abs(o13.decrypt_slots(cm) - za * mask)) < 1e-6
    tgt = 3.0 * 2 ** 38
    cs = ops.cmult_scaled(ab, mask, ("t", 1), tgt)
    assert cs.scale == tgt
    assert np.max(np.abs(o13.decrypt_slots(cs) - za * zb * mask)) < 1e-5
    ap = ops.add_plain(a, mask, ("t", 2))
    assert np.max(np.abs(o13.decrypt_slots(ap) - (za + mask))) < 1e-8


def test_lazy_relin_sum_matches_sum_of_products(o13):
    p = o13.p
    rng = np.random.default_rng(7)
    zs = [rng.uniform(-1, 1, p.slots) for _ in range(4)]
    cts = [_enc(o13, z, nonce=10 + i) for i, z in enumerate(zs)]
    lazy = mm.RnsOps(o13, lazy_relin=True)
    eager = mm.RnsOps(o13)
    pairs = [(cts[0], cts[1]), (cts[2], cts[3])]
    want = zs[0] * zs[1] + zs[2] * zs[3]
    for ops in (lazy, eager):
        assert np.max(np.abs(o13.decrypt_slots(ops.mult_sum(pairs)) - want)) < 1e-6


def test_thread_count_does_not_change_results():
    """Each limb of the ring arithmetic is computed by one thread, the same way as in
    the sequential loop: keys, encryption, rotation, hoisted rotations, the rotation
    sum, Mult, rescale and decryption give the same residues with 1 and with 4 threads."""
    def run():
        o = ckks.Oracle(ckks.params_n13(), seed=7)
        p = o.p
        rng = np.random.default_rng(4)
        a = o.encrypt_int(ckks.encode(rng.uniform(-1, 1, p.slots), p.delta, p.N), p.top, p.delta, 3)
        b = o.encrypt_int(ckks.encode(rng.uniform(-1, 1, p.slots), p.delta, p.N), p.top, p.delta, 4)
        ops = mm.RnsOps(o)
        outs = [a.data, o.rot_raw(a, 5).data, o.conj_raw(a).data, ops.mult(a, b).data, o.rescale(a).data,
                o.rot_sum(a, [1, 2, 3]).data, o.mul_plain_int(a, np.arange(p.N, dtype=np.int64) % 7 - 3, 1.0).data]
        outs += [h.data for h in o.automorph_hoisted(a, [p.galois_rot(3), p.galois_rot(9)],
                                                     [ckks.kid_rot(3), ckks.kid_rot(9)])]
        dec = np.zeros((p.top + 1, p.N), dtype=np.uint64)
        L().orc_decrypt(p.c, ckks.P(o.sk), ckks.P(a.data), p.top, ckks.P(dec))
        return outs + [dec, o.key(ckks.KID_RELIN)]

    try:
        ckks.set_threads(1)
        seq = run()
        ckks.set_threads(4)
        par = run()
    finally:
        ckks.set_threads(0)
    for x, y in zip(seq, par):
        assert np.array_equal(x, y)
