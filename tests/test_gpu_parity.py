"""GPU parity: the CUDA library against the oracle, through the C ABI.

Ciphertexts are compared bit for bit in the coefficient domain (every
residue of every limb), starting from the same seeded randomness and the same
integer plaintexts; decrypted results are compared with the FP64 products
within 1e-4 (scale 2^40, U(-1,1) inputs).  The oracle runs on the host cores.
"""
import numpy as np
import pytest

import paper_2403_14111_gb300.hetal as H
from paper_2403_14111_gb300 import workloads as wl
from paper_2403_14111_gb300.step import step_rotations, train_step
from oracle import ckks, matmul as mm

pytestmark = pytest.mark.gpu

KINDS = {"colmask": H.PT_COLMASK, "abt_diag": H.PT_ABT_DIAG, "dmask": H.PT_DMASK, "atb_diag": H.PT_ATB_DIAG,
         "sm_coef": H.PT_SM_COEF, "sm_const": H.PT_SM_CONST, "dmask_c": H.PT_DMASK_C}
ALL = H.FLAG_HOIST | H.FLAG_LAZY_RELIN | H.FLAG_RADIX_SUM | H.FLAG_SHARED_ROT


def rns_ops(o, flags):
    return mm.RnsOps(o, hoist=bool(flags & H.FLAG_HOIST), lazy_relin=bool(flags & H.FLAG_LAZY_RELIN),
                     radix_sum=bool(flags & H.FLAG_RADIX_SUM), shared_rot=bool(flags & H.FLAG_SHARED_ROT))


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")


class Env:
    """A library context and an oracle with the same parameters and seed."""

    def __init__(self, P, oracle_params, seed, steps=(), lib_params=None):
        self.ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                                      P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"])
        self.o = ckks.Oracle(oracle_params, seed=seed)
        self.p = self.o.p
        self.seed = seed
        self.sk = H.hetal_keygen(self.ctx, seed)
        self.evk = H.hetal_evk_create(self.ctx, self.sk, seed, list(steps))
        self.handles = []

    def keep(self, h):
        self.handles.append(h)
        return h

    def close(self):
        for h in self.handles:
            H.hetal_mat_free(h)
        H.hetal_evk_free(self.evk)
        H.hetal_sk_free(self.sk)
        H.hetal_ctx_destroy(self.ctx)

    def desc(self, ct_list, m, n, rows, cols, s0, s1):
        return H.make_desc(m, n, rows, cols, s0, s1, ct_list[0].lv, ct_list[0].scale)

    def upload(self, E):
        """Oracle EncMat -> library matrix (import of the coefficient residues)."""
        cts = [b for row in E.blocks for b in row]
        res = np.stack([ct.data for ct in cts])
        return self.keep(H.hetal_mat_import(self.ctx, res, self.desc(cts, E.m, E.n, E.rows, E.cols, E.s0, E.s1)))

    def upload_ct(self, ct, s0, s1):
        d = H.make_desc(1, 1, s0, s1, s0, s1, ct.lv, ct.scale)
        return self.keep(H.hetal_mat_import(self.ctx, ct.data[None], d))

    def export(self, h):
        return H.hetal_mat_export(self.ctx, h)

    def ptset(self, ops):
        s = H.hetal_ptset_create()
        for (kind, k, lv), coeffs in ops.pts.items():
            H.hetal_ptset_put(s, KINDS[kind], k, lv, coeffs)
        return s


def enc_mat(o, M, s0, s1, lv, nonce):
    p = o.p
    blocks = mm.block_split(M, s0, s1)
    return mm.EncMat([[o.encrypt_int(ckks.encode(b, p.delta, p.N), lv, p.delta, nonce + 64 * r + j)
                       for j, b in enumerate(row)] for r, row in enumerate(blocks)],
                     M.shape[0], M.shape[1], s0, s1)


def same(env, h, cts):
    got = env.export(h)
    want = np.stack([c.data for c in cts])
    assert got.shape == want.shape
    bad = np.argwhere(got != want)
    assert bad.size == 0, "first mismatch at %s of %d" % (bad[0], len(bad))


# ---------------------------------------------------------------------------
def test_moduli_match_oracle():
    for P, op in [(wl.PARAMS_N13, ckks.params_n13()), (wl.PARAMS_N16, ckks.params_n16())]:
        ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                                 P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"])
        try:
            assert H.hetal_ctx_moduli(ctx) == op.moduli
        finally:
            H.hetal_ctx_destroy(ctx)
    # a chain with a group of 60-bit primes above 50-bit ones (bootstrapping over training levels)
    ctx = H.hetal_ctx_create(11, 60, 14, 50, 2, 61, 2, scale=2.0 ** 50, n_upper=19, upper_bits=60)
    try:
        op = ckks.Params(11, 60, 14, 50, 2, 61, 2, n_upper=19, upper_bits=60)
        assert H.hetal_ctx_moduli(ctx) == op.moduli
        assert H.hetal_ctx_info(ctx)[1] == 34
    finally:
        H.hetal_ctx_destroy(ctx)


@pytest.mark.parametrize("log_n", [10, 11, 12, 14, 15, 16])
def test_ntt_is_evaluation_and_inverts(log_n):
    """The forward transform at N = 2^10 .. 2^12 (the column pass's small shapes), 2^14,
    2^15 (the primitive sweep's sizes) and 2^16 evaluates each limb at psi^(2 brv(j) + 1), checked with Python integers, and the
    inverse gives the input back."""
    import torch
    P = dict(wl.PARAMS_N16, log_n=log_n)
    ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                             P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"])
    try:
        N, L, K = H.hetal_ctx_info(ctx)
        mods = H.hetal_ctx_moduli(ctx)
        nl = L + K
        rng = np.random.default_rng(5)
        a = np.stack([np.stack([rng.integers(0, q, N, dtype=np.uint64) for q in mods]) for _ in range(3)])
        t = torch.from_numpy(a.view(np.int64).copy()).cuda()
        H.hetal_ntt_forward(ctx, t.data_ptr(), 3, nl)
        H.hetal_ctx_sync(ctx)
        f = t.cpu().numpy().view(np.uint64)
        logn = N.bit_length() - 1
        for p in (0, 2):
            for l in (0, 5, nl - 1):
                q, psi = mods[l], H.hetal_ntt_root(ctx, l)
                assert pow(psi, N, q) == q - 1
                coeffs = [int(v) for v in a[p, l]]
                for j in (0, 1, 777, N - 1):
                    brv = int(format(j, "0%db" % logn)[::-1], 2)
                    x = pow(psi, 2 * brv + 1, q)
                    acc = 0
                    for cf in reversed(coeffs):
                        acc = (acc * x + cf) % q
                    assert int(f[p, l, j]) == acc
        H.hetal_ntt_inverse(ctx, t.data_ptr(), 3, nl)
        H.hetal_ctx_sync(ctx)
        assert np.array_equal(t.cpu().numpy().view(np.uint64), a)
    finally:
        H.hetal_ctx_destroy(ctx)


@pytest.fixture(scope="module")
def env13():
    e = Env(wl.PARAMS_N13, ckks.params_n13(), seed=3,
            steps=[1, 3, 5, 64, -7] + step_rotations(128, 32, 16, H.FLAG_RADIX_SUM))
    yield e
    e.close()


def test_keys_match_oracle(env13):
    e = env13
    assert np.array_equal(H.hetal_sk_export(e.ctx, e.sk), e.o.sk)
    nm = e.p.L + e.p.K
    for kind, step, kid in [(0, 0, ckks.KID_RELIN), (1, 0, ckks.KID_CONJ), (2, 3, ckks.kid_rot(3)),
                            (2, -7, ckks.kid_rot(e.p.slots - 7))]:
        got = H.hetal_evk_export(e.ctx, e.evk, kind, step, e.p.dnum_full(), nm)
        assert np.array_equal(got, e.o.key(kid)), (kind, step)


def test_encrypt_matches_oracle(env13):
    e = env13
    rng = np.random.default_rng(1)
    m = rng.integers(-2 ** 45, 2 ** 45, (2, e.p.N)).astype(np.int64)
    for lv in (0, e.p.top):
        d = H.make_desc(2, 1, 128, 32, 128, 32, lv, e.p.delta)
        h = e.keep(H.hetal_encrypt_int(e.ctx, e.sk, e.seed, 40, m, d))
        same(e, h, [e.o.encrypt_int(m[i], lv, e.p.delta, 40 + i) for i in range(2)])


def test_primitives_match_oracle(env13):
    e = env13
    o = e.o
    rng = np.random.default_rng(2)
    za, zb = rng.uniform(-1, 1, e.p.slots), rng.uniform(-1, 1, e.p.slots)
    a = o.encrypt_int(ckks.encode(za, e.p.delta, e.p.N), e.p.top, e.p.delta, 7)
    b = o.encrypt_int(ckks.encode(zb, e.p.delta, e.p.N), e.p.top, e.p.delta, 8)
    ha, hb = e.upload_ct(a, 128, 32), e.upload_ct(b, 128, 32)
    same(e, ha, [a])
    for r in (1, 5, 64):
        same(e, e.keep(H.hetal_rotate(e.ctx, e.evk, ha, r)), [o.rot_raw(a, r)])
    same(e, e.keep(H.hetal_rotate(e.ctx, e.evk, ha, -7)), [o.rot_raw(a, e.p.slots - 7)])
    same(e, e.keep(H.hetal_conj(e.ctx, e.evk, ha)), [o.conj_raw(a)])
    ops = mm.RnsOps(o)
    same(e, e.keep(H.hetal_mult(e.ctx, e.evk, ha, hb)), [ops.mult(a, b)])
    same(e, e.keep(H.hetal_rescale(e.ctx, ha)), [o.rescale(a)])
    same(e, e.keep(H.hetal_add(e.ctx, ha, hb)), [o.add(a, b)])
    same(e, e.keep(H.hetal_sub(e.ctx, ha, hb)), [o.sub(a, b)])
    outs = H.hetal_rotate_hoisted(e.ctx, e.evk, ha, [3, 64])
    for h in outs:
        e.keep(h)
    hs = o.automorph_hoisted(a, [e.p.galois_rot(3), e.p.galois_rot(64)], [ckks.kid_rot(3), ckks.kid_rot(64)])
    same(e, outs[0], [hs[0]])
    same(e, outs[1], [hs[1]])


@pytest.mark.parametrize("flags", [0, H.FLAG_HOIST | H.FLAG_LAZY_RELIN, H.FLAG_HOIST | H.FLAG_LAZY_RELIN | H.FLAG_RADIX_SUM],
                         ids=["plain", "hoist+lazy", "hoist+lazy+radix"])
def test_diag_abt_matches_oracle_n13(env13, flags):
    """X 128x32 times (16x32)^T at N=2^13: bit-exact with the oracle, |err| <= 1e-4."""
    e = env13
    s0, s1, c = 128, 32, 16
    X = wl.uniform_matrix(128, 32, 1)
    W = wl.uniform_matrix(16, 32, 2)
    EX = enc_mat(e.o, X, s0, s1, e.p.top, 100)
    EW = enc_mat(e.o, mm.tile_vertical(W, c, s0), s0, s1, e.p.top, 200)
    ops = mm.RnsOps(e.o, hoist=bool(flags & H.FLAG_HOIST), lazy_relin=bool(flags & H.FLAG_LAZY_RELIN),
                    radix_sum=bool(flags & H.FLAG_RADIX_SUM))
    ref = mm.diag_abt(ops, EX, EW, c, 1.0)
    pts = e.ptset(ops)
    H.hetal_counters_reset(e.ctx)
    out = e.keep(H.hetal_diag_abt(e.ctx, e.evk, e.upload(EX), e.upload(EW), c, 1.0, pts, flags))
    cnt = H.hetal_counters_get(e.ctx)
    H.hetal_ptset_free(pts)
    same(e, out, [ref.blocks[0][0]])
    rots = 168 if flags & H.FLAG_RADIX_SUM else 88
    assert (cnt["cmult"], cnt["mult"], cnt["rot"], cnt["conj"]) == (16, 8, rots, 1)
    dec = H.hetal_decrypt(e.ctx, e.sk, out)
    assert np.max(np.abs(dec[:128, :s1] - np.tile(X @ W.T, (1, s1 // c)))) <= 1e-4


def test_diag_abt_own_masks_within_tolerance(env13):
    e = env13
    s0, s1, c = 128, 32, 16
    X = wl.uniform_matrix(128, 32, 3)
    W = wl.uniform_matrix(10, 32, 4)
    hX = e.keep(H.hetal_encrypt(e.ctx, e.sk, e.seed, 300, X, s0, s1, H.TILE_NONE, 0, e.p.top, e.p.delta))
    hW = e.keep(H.hetal_encrypt(e.ctx, e.sk, e.seed, 400, W, s0, s1, H.TILE_VERT, c, e.p.top, e.p.delta))
    out = e.keep(H.hetal_diag_abt(e.ctx, e.evk, hX, hW, c, 1.0, None, H.FLAG_HOIST | H.FLAG_LAZY_RELIN))
    dec = H.hetal_decrypt(e.ctx, e.sk, out)
    Wp = np.zeros((c, 32))
    Wp[:10] = W
    assert np.max(np.abs(dec[:128, :s1] - np.tile(X @ Wp.T, (1, s1 // c)))) <= 1e-4


def test_encode_close_to_oracle(env13):
    e = env13
    rng = np.random.default_rng(9)
    re, im = rng.uniform(-1, 1, e.p.slots), rng.uniform(-1, 1, e.p.slots)
    got = H.hetal_encode(e.ctx, re, im, e.p.delta)[0]
    want = ckks.encode(re + 1j * im, e.p.delta, e.p.N)
    assert np.max(np.abs(got - want)) <= 2


def test_ragged_multiblock_abt(env13):
    """300 x 100 by (8 x 100)^T in 128 x 32 blocks: 3 x 4 ragged blocks, c = 8."""
    e = env13
    s0, s1, c = 128, 32, 8
    X = wl.uniform_matrix(300, 100, 5)
    W = wl.uniform_matrix(8, 100, 6)
    EX = enc_mat(e.o, X, s0, s1, e.p.top, 500)
    EW = enc_mat(e.o, mm.tile_vertical(W, c, s0), s0, s1, e.p.top, 600)
    ops = mm.RnsOps(e.o, hoist=True, lazy_relin=True)
    ref = mm.diag_abt(ops, EX, EW, c, 0.5)
    pts = e.ptset(ops)
    out = e.keep(H.hetal_diag_abt(e.ctx, e.evk, e.upload(EX), e.upload(EW), c, 0.5, pts,
                                  H.FLAG_HOIST | H.FLAG_LAZY_RELIN))
    H.hetal_ptset_free(pts)
    same(e, out, [ref.blocks[r][0] for r in range(3)])
    dec = H.hetal_decrypt(e.ctx, e.sk, out)
    assert np.max(np.abs(dec[:300, :s1] - np.tile(0.5 * X @ W.T, (1, s1 // c)))) <= 1e-4


def test_status_codes(env13):
    e = env13
    X = wl.uniform_matrix(128, 32, 7)
    h = e.keep(H.hetal_encrypt(e.ctx, e.sk, e.seed, 700, X, 128, 32, H.TILE_NONE, 0, e.p.top, e.p.delta))
    nokeys = H.hetal_evk_create(e.ctx, e.sk, e.seed, [], with_conj=False, with_relin=True)
    with pytest.raises(H.HetalError) as ei:
        H.hetal_rotate(e.ctx, nokeys, h, 11)
    assert ei.value.code == H.ERR_MISSING_KEY
    H.hetal_evk_free(nokeys)
    # without a key for 11, the rotation is composed from the +-2^u keys: same slots
    X2 = H.hetal_decrypt(e.ctx, e.sk, e.keep(H.hetal_rotate(e.ctx, e.evk, h, 11))).reshape(-1)
    assert np.max(np.abs(X2 - np.roll(X.reshape(-1), -11))) <= 1e-4
    with pytest.raises(H.HetalError) as ei:
        H.hetal_diag_abt(e.ctx, e.evk, h, h, 3, 1.0)
    assert ei.value.code == H.ERR_SHAPE
    low = e.keep(H.hetal_mat_drop(e.ctx, h, 1))
    with pytest.raises(H.HetalError) as ei:
        H.hetal_diag_abt(e.ctx, e.evk, low, low, 2, 1.0)
    assert ei.value.code == H.ERR_LEVEL
    other = e.keep(H.hetal_encrypt(e.ctx, e.sk, e.seed, 701, X, 128, 32, H.TILE_NONE, 0, e.p.top, 3.0 * e.p.delta))
    with pytest.raises(H.HetalError) as ei:
        H.hetal_add(e.ctx, h, other)
    assert ei.value.code == H.ERR_SCALE
    with pytest.raises(H.HetalError) as ei:
        H.hetal_encrypt(e.ctx, e.sk, e.seed, 702, X, 100, 32, H.TILE_NONE, 0, e.p.top, e.p.delta)
    assert ei.value.code == H.ERR_SHAPE
    # the context stays usable after every error
    ok = e.keep(H.hetal_rotate(e.ctx, e.evk, h, 1))
    assert H.hetal_mat_desc_get(ok).level == e.p.top


# ---------------------------------------------------------------------------
# DiagATB (both branches) and the softmax stand-in need more levels.
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def env13d():
    P = wl.PARAMS_N13_DEEP
    op = ckks.Params(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                     P["special_bits"], P["alpha"], log_delta=P["log_scale"])
    # keys for every variant the tests run: the shared-rotation variant needs no Rrot(., s1)
    steps = sorted(set(step_rotations(128, 32, 8, H.FLAG_RADIX_SUM) +
                       step_rotations(128, 32, 8, H.FLAG_RADIX_SUM | H.FLAG_SHARED_ROT)))
    e = Env(P, op, seed=4, steps=steps)
    yield e
    e.close()


@pytest.mark.parametrize("lvA", [6, 5], ids=["rotleft", "protup"])
@pytest.mark.parametrize("flags", [0, H.FLAG_HOIST | H.FLAG_LAZY_RELIN, H.FLAG_HOIST | H.FLAG_LAZY_RELIN | H.FLAG_RADIX_SUM,
                                   H.FLAG_SHARED_ROT, ALL],
                         ids=["plain", "hoist+lazy", "hoist+lazy+radix", "shared", "all"])
def test_diag_atb_matches_oracle(env13d, lvA, flags):
    e = env13d
    s0, s1, c = 128, 32, 8
    A = wl.uniform_matrix(128, 5, 10 + lvA)
    B = wl.uniform_matrix(128, 40, 20 + lvA)
    EA = enc_mat(e.o, mm.tile_horizontal(A, c, s1), s0, s1, lvA, 800)
    EB = enc_mat(e.o, B, s0, s1, 6, 900)
    ops = rns_ops(e.o, flags)
    t = 1.0 / 64
    ref = mm.diag_atb(ops, EA, EB, c, t)
    pts = e.ptset(ops)
    out = e.keep(H.hetal_diag_atb(e.ctx, e.evk, e.upload(EA), e.upload(EB), c, t, pts, flags))
    H.hetal_ptset_free(pts)
    same(e, out, ref.blocks[0])
    dec = H.hetal_decrypt(e.ctx, e.sk, out)
    Ap = np.zeros((128, c))
    Ap[:, :5] = A
    assert np.max(np.abs(dec[:s0, :40] - np.tile(t * Ap.T @ B, (s0 // c, 1)))) <= 1e-4


@pytest.mark.parametrize("lvA", [6, 5], ids=["rotleft", "protup"])
@pytest.mark.parametrize("flags", [H.FLAG_HOIST | H.FLAG_LAZY_RELIN, ALL], ids=["hoist+lazy", "all"])
def test_diag_atb_two_row_blocks(env13d, lvA, flags):
    """A 200 x 3 and B 200 x 40 in 128 x 32 blocks: two row blocks summed per column block (App. B.1)."""
    e = env13d
    s0, s1, c = 128, 32, 4
    A = wl.uniform_matrix(200, 3, 30 + lvA)
    B = wl.uniform_matrix(200, 40, 40 + lvA)
    EA = enc_mat(e.o, mm.tile_horizontal(A, c, s1), s0, s1, lvA, 1100)
    EB = enc_mat(e.o, B, s0, s1, 6, 1200)
    ops = rns_ops(e.o, flags)
    t = 1.0 / 256
    ref = mm.diag_atb(ops, EA, EB, c, t)
    pts = e.ptset(ops)
    out = e.keep(H.hetal_diag_atb(e.ctx, e.evk, e.upload(EA), e.upload(EB), c, t, pts, flags))
    H.hetal_ptset_free(pts)
    same(e, out, ref.blocks[0])
    dec = H.hetal_decrypt(e.ctx, e.sk, out)
    Ap = np.zeros((200, c))
    Ap[:, :3] = A
    assert np.max(np.abs(dec[:s0, :40] - np.tile(t * Ap.T @ B, (s0 // c, 1)))) <= 1e-4


def test_softmax_poly_matches_oracle(env13d):
    e = env13d
    p = e.p
    rng = np.random.default_rng(12)
    x = rng.uniform(-1, 1, p.slots)
    coeffs = wl.sigmoid_cheb15()
    valid = wl.valid_mask(100, 5, 8, 128, 32)
    ct = e.o.encrypt_int(ckks.encode(x, p.delta, p.N), p.top, p.delta, 77)
    ops = mm.RnsOps(e.o)
    ref = mm.poly15_masked(ops, ct, coeffs, valid, p.delta)
    pts = e.ptset(ops)
    out = e.keep(H.hetal_softmax_approx(e.ctx, e.evk, e.upload_ct(ct, 128, 32), coeffs, valid, p.delta, pts))
    H.hetal_ptset_free(pts)
    same(e, out, [ref])
    dec = H.hetal_decrypt(e.ctx, e.sk, out).reshape(-1)
    want = np.polynomial.polynomial.polyval(x, coeffs) * valid
    assert np.max(np.abs(dec - want)) <= 1e-4


# ---------------------------------------------------------------------------
# N = 2^16, the training-step parameters
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def env16():
    e = Env(wl.PARAMS_N16, ckks.params_n16(), seed=5,
            steps=sorted(set(step_rotations(1024, 32, 16) + step_rotations(1024, 32, 16, ALL) + [7])))
    yield e
    e.close()


def test_n16_primitives_match_oracle(env16):
    """Rotation, conjugation, Mult at the top level (12 limbs, 6 digits) bit-exact at N = 2^16."""
    e = env16
    o = e.o
    rng = np.random.default_rng(3)
    za, zb = rng.uniform(-1, 1, e.p.slots), rng.uniform(-1, 1, e.p.slots)
    a = o.encrypt_int(ckks.encode(za, e.p.delta, e.p.N), e.p.top, e.p.delta, 1)
    b = o.encrypt_int(ckks.encode(zb, e.p.delta, e.p.N), e.p.top, e.p.delta, 2)
    ha, hb = e.upload_ct(a, 1024, 32), e.upload_ct(b, 1024, 32)
    same(e, e.keep(H.hetal_rotate(e.ctx, e.evk, ha, 7)), [o.rot_raw(a, 7)])
    same(e, e.keep(H.hetal_mult(e.ctx, e.evk, ha, hb)), [mm.RnsOps(o).mult(a, b)])
    outs = H.hetal_rotate_hoisted(e.ctx, e.evk, ha, [32, 64])
    for h in outs:
        e.keep(h)
    hs = o.automorph_hoisted(a, [e.p.galois_rot(32), e.p.galois_rot(64)], [ckks.kid_rot(32), ckks.kid_rot(64)])
    same(e, outs[0], [hs[0]])
    same(e, outs[1], [hs[1]])
    # sum of seven rotations with one ModUp / ModDown (the first radix-8 SumRows step, keys j * s1)
    rs = [j * 32 for j in range(1, 8)]
    same(e, e.keep(H.hetal_rotate_sum(e.ctx, e.evk, ha, rs)), [o.rot_sum(a, rs)])


@pytest.mark.parametrize("flags", [H.FLAG_HOIST | H.FLAG_LAZY_RELIN, ALL], ids=["hoist+lazy", "all"])
def test_training_step_n16_full_size(env16, flags):
    """The benchmark workload (X 1024x768, 10 classes, c = 16, N = 2^16) through the
    C ABI with the library's own masks: each stage decrypts to its FP64 mirror."""
    e = env16
    X, Y, W, c = wl.training_step()
    s0, s1 = 1024, 32
    delta = e.p.delta
    coeffs = wl.sigmoid_cheb15()
    valid = wl.valid_mask(1024, 10, c, s0, s1)
    hX = e.keep(H.hetal_encrypt(e.ctx, e.sk, e.seed, 1000, X, s0, s1, H.TILE_NONE, 0, e.p.top, delta))
    hW = e.keep(H.hetal_encrypt(e.ctx, e.sk, e.seed, 2000, W, s0, s1, H.TILE_VERT, c, e.p.top, delta))
    lvP = e.p.top - 3 - 5
    hY = e.keep(H.hetal_encrypt(e.ctx, e.sk, e.seed, 3000, Y, s0, s1, H.TILE_HORIZ, c, lvP, delta))
    lr_n = 1.0 / 1024
    G, inter = train_step(e.ctx, e.evk, hX, hW, hY, coeffs, valid, c, lr_n, delta, flags)
    e.keep(G)
    for h in inter:
        e.keep(h)
    logits8 = np.tile(X @ W.T / 8.0, (1, s1 // c))
    got = H.hetal_decrypt(e.ctx, e.sk, inter[0])
    assert np.max(np.abs(got - logits8)) <= 1e-6
    Pm = np.polynomial.polynomial.polyval(logits8, coeffs) * valid.reshape(s0, s1)
    got = H.hetal_decrypt(e.ctx, e.sk, inter[1])
    assert np.max(np.abs(got - Pm)) <= 1e-6
    Dm = Pm - np.tile(Y, (1, s1 // c))
    Gm = lr_n * Dm[:, :c].T @ X
    got = H.hetal_decrypt(e.ctx, e.sk, G)
    assert got.shape == (1024, 768)
    assert np.max(np.abs(got - np.tile(Gm, (s0 // c, 1)))) <= 1e-6


@pytest.mark.parametrize("flags,dim", [(H.FLAG_HOIST | H.FLAG_LAZY_RELIN, 64), (ALL, 96)],
                         ids=["hoist+lazy-n2", "all-n3"])
def test_training_step_n16_bit_exact(env16, flags, dim):
    """The benchmarked configuration (N = 2^16, 12 + 2 primes, dnum 6, 1024 x 32 blocks,
    c = 16) with the feature count reduced to 2-3 column blocks: DiagABT (Algorithm
    DiagABT), the softmax stand-in, -Y and DiagATB (Algorithm DiagATB, PRotUp branch)
    bit-exact with the oracle at every stage.  The context's batch budget is lowered so
    that the c/2 diagonals and the hoisted amounts run in several chunks."""
    e = env16
    o, p = e.o, e.p
    s0, s1 = 1024, 32
    X, Y, W, c = wl.training_step(rows=1024, dim=dim)
    coeffs = wl.sigmoid_cheb15()
    valid = wl.valid_mask(1024, 10, c, s0, s1)
    lr_n = 1.0 / 1024
    EX = enc_mat(o, X, s0, s1, p.top, 5000)
    EW = enc_mat(o, mm.tile_vertical(W, c, s0), s0, s1, p.top, 5100)
    EY = enc_mat(o, mm.tile_horizontal(Y, c, s1), s0, s1, p.top - 8, 5200)
    ops = rns_ops(o, flags)
    G, logits, P, D = mm.train_step(ops, EX, EW, EY, coeffs, valid, c, lr_n, p.delta)
    pts = e.ptset(ops)
    hX, hW, hY = e.upload(EX), e.upload(EW), e.upload(EY)
    H.hetal_ctx_set_batch_bytes(e.ctx, 200 << 20)
    try:
        Gh, inter = train_step(e.ctx, e.evk, hX, hW, hY, coeffs, valid, c, lr_n, p.delta, flags,
                               pts=(pts, pts, pts))
    finally:
        H.hetal_ctx_set_batch_bytes(e.ctx, 8 << 30)
        H.hetal_ptset_free(pts)
    e.keep(Gh)
    for h in inter:
        e.keep(h)
    same(e, inter[0], [logits.blocks[0][0]])
    same(e, inter[1], [P[0][0]])
    same(e, inter[2], [D[0][0]])
    same(e, Gh, G.blocks[0])
    assert len(G.blocks[0]) == dim // s1
    Pm = np.polynomial.polynomial.polyval(np.tile(X @ W.T / 8.0, (1, s1 // c)), coeffs) * valid.reshape(s0, s1)
    Gm = lr_n * (Pm - np.tile(Y, (1, s1 // c)))[:, :c].T @ X
    got = H.hetal_decrypt(e.ctx, e.sk, Gh)
    assert np.max(np.abs(got[:, :dim] - np.tile(Gm, (s0 // c, 1)))) <= 1e-6


def pinned_u64(shape):
    """A uint64 array in pinned (page-locked) host memory, and the tensor that owns it."""
    import torch
    t = torch.empty(int(np.prod(shape)), dtype=torch.int64, pin_memory=True)
    return t.numpy().view(np.uint64).reshape(shape), t


def test_graph_replay_matches_eager(env13):
    """Import -> DiagABT -> export recorded into one CUDA graph: the launch that ends the
    recording and every later launch give the eager calls' bits, new pinned inputs are
    picked up at each launch, and a call that cannot be recorded voids the recording."""
    e = env13
    s0, s1, c = 128, 32, 16
    flags = H.FLAG_HOIST | H.FLAG_LAZY_RELIN | H.FLAG_RADIX_SUM
    W = wl.uniform_matrix(16, 32, 12)
    EW = enc_mat(e.o, mm.tile_vertical(W, c, s0), s0, s1, e.p.top, 700)
    cts_w = [b for row in EW.blocks for b in row]
    EXs = [enc_mat(e.o, wl.uniform_matrix(128, 32, 10 + i), s0, s1, e.p.top, 800 + 100 * i) for i in range(2)]
    res = [np.stack([b.data for row in EX.blocks for b in row]) for EX in EXs]
    dX = e.desc([EXs[0].blocks[0][0]], 1, 1, 128, 32, s0, s1)
    dW = e.desc(cts_w, EW.m, EW.n, EW.rows, EW.cols, s0, s1)
    in_x, tx = pinned_u64(res[0].shape)
    in_w, tw = pinned_u64(res[0].shape)
    in_w[...] = np.stack([b.data for b in cts_w])

    def calls():
        hx = H.hetal_mat_import(e.ctx, in_x, dX)
        hw = H.hetal_mat_import(e.ctx, in_w, dW)
        out = H.hetal_diag_abt(e.ctx, e.evk, hx, hw, c, 1.0, None, flags)
        H.hetal_mat_free(hx)
        H.hetal_mat_free(hw)
        return out

    want = []
    for i in range(2):   # eager: also caches the masks the recording needs
        in_x[...] = res[i]
        h = calls()
        want.append(H.hetal_mat_export(e.ctx, h))
        H.hetal_mat_free(h)
    assert not np.array_equal(want[0], want[1])
    out_host, to = pinned_u64(want[0].shape)
    in_x[...] = res[0]
    launches0 = H.hetal_launch_count(e.ctx)
    H.hetal_graph_begin(e.ctx)
    out = calls()
    H.hetal_mat_export(e.ctx, out, out_host)
    g = H.hetal_graph_end(e.ctx)   # launches once
    try:
        kernels = H.hetal_graph_kernels(g)
        assert kernels > 50 and H.hetal_launch_count(e.ctx) - launches0 == 2 * kernels
        H.hetal_ctx_sync(e.ctx)
        assert np.array_equal(out_host, want[0])
        assert np.array_equal(H.hetal_mat_export(e.ctx, out), want[0])
        for i in (1, 0, 1):
            in_x[...] = res[i]
            out_host[...] = 0
            H.hetal_graph_launch(e.ctx, g)
            H.hetal_ctx_sync(e.ctx)
            assert np.array_equal(out_host, want[i]), i
            assert np.array_equal(H.hetal_mat_export(e.ctx, out), want[i]), i
    finally:
        H.hetal_graph_free(g)
        H.hetal_mat_free(out)
    # a call that waits for the device is refused and voids the recording
    hx = e.keep(H.hetal_mat_import(e.ctx, res[0], dX))
    H.hetal_graph_begin(e.ctx)
    r = H.hetal_rotate(e.ctx, e.evk, hx, 1)
    with pytest.raises(H.HetalError) as ex:
        H.hetal_decrypt(e.ctx, e.sk, hx)
    assert ex.value.code == H.ERR_RECORDING
    with pytest.raises(H.HetalError) as ex:
        H.hetal_graph_end(e.ctx)
    assert ex.value.code == H.ERR_RECORDING
    assert H.hetal_mat_desc_get(r).m == 1
    H.hetal_mat_free(r)   # emptied: nothing to free
    # the context works normally afterwards
    same(e, e.keep(H.hetal_rotate(e.ctx, e.evk, hx, 1)), [e.o.rot_raw(EXs[0].blocks[0][0], 1)])
    del tx, tw, to


def test_ntt32_is_evaluation():
    """The 32-bit-word transform (primes below 2^30) at N = 2^16 evaluates each limb at
    psi^(2 brv(j) + 1), checked with Python integers, like the 64-bit one."""
    import torch
    P = wl.PARAMS_N16
    ctx = H.hetal_ctx_create(P["log_n"], P["q0_bits"], P["n_rescale"], P["rescale_bits"], P["n_special"],
                             P["special_bits"], P["alpha"], scale=2.0 ** P["log_scale"])
    try:
        N = H.hetal_ctx_info(ctx)[0]
        limbs = 21
        mods, roots = H.hetal_ntt32_moduli(ctx, limbs)
        assert all(q < 2 ** 30 and q % (2 * N) == 1 for q in mods) and len(set(mods)) == limbs
        assert mods == sorted(mods, reverse=True)
        rng = np.random.default_rng(7)
        a = np.stack([np.stack([rng.integers(0, q, N, dtype=np.uint32) for q in mods]) for _ in range(2)])
        t = torch.from_numpy(a.view(np.int32).copy()).cuda()
        H.hetal_ntt32_forward(ctx, t.data_ptr(), 2, limbs)
        H.hetal_ctx_sync(ctx)
        f = t.cpu().numpy().view(np.uint32)
        logn = N.bit_length() - 1
        for p in (0, 1):
            for l in (0, 9, limbs - 1):
                q, psi = mods[l], roots[l]
                assert pow(psi, N, q) == q - 1
                coeffs = [int(v) for v in a[p, l]]
                for j in (0, 1, 4097, N - 1):
                    brv = int(format(j, "0%db" % logn)[::-1], 2)
                    x = pow(psi, 2 * brv + 1, q)
                    acc = 0
                    for cf in reversed(coeffs):
                        acc = (acc * x + cf) % q
                    assert int(f[p, l, j]) == acc
        assert H.hetal_probe_butterfly32_rate(ctx, 2000) > 0
    finally:
        H.hetal_ctx_destroy(ctx)


def test_grouped_row_passes_same_bits(env16):
    """The NTT row passes with the rows' twiddles staged in shared memory for groups of
    polynomials give the bits of the one-polynomial-per-CTA passes: raw forward and
    inverse transforms, and a rotation and a Mult (ModDown tail, INTT of ModUp)."""
    import torch
    e = env16
    N, L, K = H.hetal_ctx_info(e.ctx)
    mods = H.hetal_ctx_moduli(e.ctx)
    rng = np.random.default_rng(8)
    a = np.stack([np.stack([rng.integers(0, q, N, dtype=np.uint64) for q in mods]) for _ in range(8)])
    outs = {}
    za = rng.uniform(-1, 1, e.p.slots)
    ct = e.o.encrypt_int(ckks.encode(za, e.p.delta, e.p.N), e.p.top, e.p.delta, 9)
    hc = e.upload_ct(ct, 1024, 32)
    try:
        for g in (1, 4):
            H.hetal_ctx_set_row_group(e.ctx, g)
            t = torch.from_numpy(a.view(np.int64).copy()).cuda()
            H.hetal_ntt_forward(e.ctx, t.data_ptr(), 8, L + K)
            H.hetal_ctx_sync(e.ctx)
            f = t.cpu().numpy().view(np.uint64).copy()
            H.hetal_ntt_inverse(e.ctx, t.data_ptr(), 8, L + K)
            H.hetal_ctx_sync(e.ctx)
            assert np.array_equal(t.cpu().numpy().view(np.uint64), a)
            r = H.hetal_rotate(e.ctx, e.evk, hc, 32)
            m = H.hetal_mult(e.ctx, e.evk, hc, hc)
            outs[g] = (f, H.hetal_mat_export(e.ctx, r), H.hetal_mat_export(e.ctx, m))
            H.hetal_mat_free(r)
            H.hetal_mat_free(m)
    finally:
        H.hetal_ctx_set_row_group(e.ctx, 1)
    for x, y in zip(outs[1], outs[4]):
        assert np.array_equal(x, y)
    assert np.array_equal(outs[1][1][0], e.o.rot_raw(ct, 32).data)
