"""Pins for the oracle's matrix layer: the block-encoding worked example
(App. B.1), the FP64 slot simulator against the FP64 matrix product
(Props. ABT / ATB) and against the paper's corrected operation counts
(Table "tab:matnum_fixed"), and the encrypted oracle against FP64 within the
1e-4 bound at scale 2^40.  The last tests plant mistakes in the oracle's
algorithm layer and check that a pin catches each one."""
import os

import numpy as np
import pytest

from oracle import ckks, matmul as mm

GOLD = os.path.join(os.path.dirname(__file__), "golden")
SLOTS = 32768


def load_counts():
    rows = []
    with open(os.path.join(GOLD, "tab_matnum_fixed.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    return rows


def test_block_encoding_worked_example():
    with open(os.path.join(GOLD, "encoding_3x3_in_4x4.txt")) as f:
        toks = [ln for ln in f if not ln.startswith("#")][0].split()
    A = np.array([[10 * i + j + 100 for j in range(3)] for i in range(3)], dtype=np.float64)
    got = mm.block_split(A, 4, 4)[0][0]
    want = [0.0 if t == "0" else A[int(t[0]), int(t[1])] for t in toks]
    assert got.tolist() == want


def _sim_mat(M, s0, s1, lv):
    return mm.EncMat([[mm.SV(b.astype(np.complex128), lv) for b in row] for row in mm.block_split(M, s0, s1)],
                     M.shape[0], M.shape[1], s0, s1)


def _sim_join(E, rows, cols):
    return mm.block_join([[x.z for x in row] for row in E.blocks], E.s0, E.s1, rows, cols)


def run_abt_sim(a, b, c, s0, t=1.0, seed=0, radix=False):
    s1 = SLOTS // s0
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, (a, b))
    B = rng.uniform(-1, 1, (c, b))
    ops = mm.SlotOps(SLOTS, radix_sum=radix)
    out = mm.diag_abt(ops, _sim_mat(A, s0, s1, 12), _sim_mat(mm.tile_vertical(B, c, s0), s0, s1, 12), c, t)
    res = _sim_join(out, a, s1)
    return ops, np.max(np.abs(res - np.tile(t * A @ B.T, (1, s1 // c))))


def run_atb_sim(a, b, c, s0, lvA, t=1.0, seed=0, radix=False, shared=False):
    s1 = SLOTS // s0
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, (a, c))
    B = rng.uniform(-1, 1, (a, b))
    ops = mm.SlotOps(SLOTS, radix_sum=radix, shared_rot=shared)
    out = mm.diag_atb(ops, _sim_mat(mm.tile_horizontal(A, c, s1), s0, s1, lvA), _sim_mat(B, s0, s1, 12), c, t)
    res = _sim_join(out, s0, b)
    return ops, np.max(np.abs(res - np.tile(t * A.T @ B, (s0 // c, 1))))


def _cmr(ops):
    return [ops.counts["CMult"], ops.counts["Mult"], ops.counts["Rot"]]


@pytest.mark.parametrize("row", load_counts(), ids=lambda r: "%d-%d-%d" % tuple(r[:3]))
def test_counts_and_values_match_paper(row):
    a, b, c = row[:3]
    ops, err = run_abt_sim(a, b, c, s0=a, t=0.5)
    assert _cmr(ops) == row[3:6] and err < 1e-12
    ops, err = run_atb_sim(a, b, c, s0=a, lvA=12, t=0.25)      # level(A) >= level(B): RotLeft
    assert _cmr(ops) == row[6:9] and err < 1e-12
    ops, err = run_atb_sim(a, b, c, s0=a, lvA=11, t=0.25)      # level(A) < level(B): PRotUp
    assert _cmr(ops) == row[9:12] and err < 1e-12


@pytest.mark.parametrize("a,b,c,s0", [(300, 100, 8, 128), (64, 200, 2, 64), (1024, 768, 16, 1024)])
def test_multiblock_values(a, b, c, s0):
    ops, err = run_abt_sim(a, b, c, s0, t=0.3, seed=1)
    assert err < 1e-12
    s1 = SLOTS // s0
    m, n = -(-a // s0), -(-b // s1)
    h = c // 2
    lg1 = s1.bit_length() - 1
    assert _cmr(ops) == [c * m, h * m * n, h * (n + 2 * m * lg1)]
    for lvA in (12, 11):
        ops, err = run_atb_sim(a, b, c, s0, lvA, t=0.7, seed=2)
        assert err < 1e-12


def test_radix_plan():
    for bits in range(0, 16):
        plan = mm.radix_plan(bits)
        assert sum(plan) == bits and all(1 <= b <= 3 for b in plan)
        assert plan == sorted(plan, reverse=True) and (not plan or plan[0] - plan[-1] <= 1)
        assert len(plan) == -(-bits // 3)


@pytest.mark.parametrize("a,b,c,s0", [(300, 100, 8, 128), (1024, 768, 16, 1024), (64, 64, 4, 64)])
def test_radix_sums_same_values(a, b, c, s0):
    """Radix rotate-and-sum steps give the paper's SumCols / SumRows values."""
    s1 = SLOTS // s0
    ops, err = run_abt_sim(a, b, c, s0, t=0.3, seed=1, radix=True)
    assert err < 1e-12
    m, n = -(-a // s0), -(-b // s1)
    lg1 = s1.bit_length() - 1
    # RotUp rotations plus 2 sums over s1 positions per (block row, k): sum(2^b - 1) per radix plan
    per_sum = sum((1 << bb) - 1 for bb in mm.radix_plan(lg1))
    assert ops.counts["Rot"] == (c // 2) * (n + 2 * m * per_sum)
    for lvA in (12, 11):
        ops, err = run_atb_sim(a, b, c, s0, lvA, t=0.7, seed=2, radix=True)
        assert err < 1e-12


@pytest.mark.parametrize("a,b,c,s0", [(300, 100, 8, 128), (1024, 768, 16, 1024), (200, 64, 4, 128)])
def test_shared_rotation_forms_same_values(a, b, c, s0):
    """PRotUp with one RotUp(B, 1) for every k, and RotLeft from Lrot(A, k) and
    Lrot(A, k - s1), give Algorithm DiagATB's values (both branches)."""
    s1 = SLOTS // s0
    m, n, h = -(-a // s0), -(-b // s1), c // 2
    for lvA in (12, 11):
        ops, err = run_atb_sim(a, b, c, s0, lvA, t=0.7, seed=2, shared=True)
        assert err < 1e-12
        ref, _ = run_atb_sim(a, b, c, s0, lvA, t=0.7, seed=2)
        if lvA == 11:   # PRotUp: m*n shared RotUp(B, 1) instead of (c/2 - 1) per block
            assert ref.counts["Rot"] - ops.counts["Rot"] == (h - 1) * m * n - m * n
        else:           # RotLeft: as many rotations, but the Rrot(., s1) become hoisted rotations of A_cplx
            assert ops.counts["Rot"] == ref.counts["Rot"]
    ops, err = run_atb_sim(a, b, c, s0, 11, t=0.7, seed=2, radix=True, shared=True)
    assert err < 1e-12


def test_softmax_poly_slot_sim():
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, SLOTS)
    coeffs = rng.uniform(-2, 2, 16)
    valid = (rng.uniform(size=SLOTS) < 0.7).astype(np.float64)
    ops = mm.SlotOps(SLOTS)
    out = mm.poly15_masked(ops, mm.SV(x.astype(np.complex128), 10), coeffs, valid, 1.0)
    want = np.polynomial.polynomial.polyval(x, coeffs) * valid
    assert np.max(np.abs(out.z - want)) < 1e-12
    assert out.lv == 5


# ---------------------------------------------------------------------------
# Encrypted oracle, N = 2^13 (s = 4096 slots)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def o13():
    return ckks.Oracle(ckks.params_n13(), seed=1)


@pytest.fixture(scope="module")
def o13deep():
    # six rescale primes so that DiagATB's RotLeft and PRotUp branches both fit
    return ckks.Oracle(ckks.Params(13, 60, 6, 40, 2, 61, alpha=2, log_delta=40), seed=2)


def _enc_mat(o, M, s0, s1, lv, nonce):
    p = o.p
    blocks = mm.block_split(M, s0, s1)
    return mm.EncMat([[o.encrypt_int(ckks.encode(b, p.delta, p.N), lv, p.delta, nonce + 64 * r + j)
                       for j, b in enumerate(row)] for r, row in enumerate(blocks)],
                     M.shape[0], M.shape[1], s0, s1)


def _dec_mat(o, E, rows, cols):
    return mm.block_join([[o.decrypt_slots(x).real for x in row] for row in E.blocks], E.s0, E.s1, rows, cols)


@pytest.mark.parametrize("radix", [False, True], ids=["log", "radix"])
def test_encrypted_diag_abt_n13(o13, radix):
    """128x32 times (16x32)^T at N=2^13, scale 2^40: max |err| <= 1e-4 against FP64."""
    o = o13
    s0, s1, c = 128, 32, 16
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, (128, 32))
    W = rng.uniform(-1, 1, (16, 32))
    EX = _enc_mat(o, X, s0, s1, o.p.top, 100)
    EW = _enc_mat(o, mm.tile_vertical(W, c, s0), s0, s1, o.p.top, 200)
    ops = mm.RnsOps(o, hoist=True, lazy_relin=True, radix_sum=radix)
    out = mm.diag_abt(ops, EX, EW, c, 1.0)
    assert out.blocks[0][0].lv == 0
    got = _dec_mat(o, out, 128, s1)
    assert np.max(np.abs(got - np.tile(X @ W.T, (1, s1 // c)))) <= 1e-4
    # 8 RotUp rotations; each of the 8 SumCols sums over 32 columns twice: 2 x 5 rotations
    # as log-depth steps, 2 x (7 + 3) as radix-8 and radix-4 steps
    assert _cmr(ops) == [16, 8, 168 if radix else 88] and ops.counts["Conj"] == 1


@pytest.mark.parametrize("lvA,radix,shared", [(6, False, False), (5, False, False), (5, True, False), (6, False, True),
                                              (5, True, True)],
                         ids=["rotleft", "protup", "protup-radix", "rotleft-shared", "protup-radix-shared"])
def test_encrypted_diag_atb_n13(o13deep, lvA, radix, shared):
    o = o13deep
    s0, s1, c = 128, 32, 4
    rng = np.random.default_rng(lvA)
    A = rng.uniform(-1, 1, (128, 3))
    B = rng.uniform(-1, 1, (128, 40))
    EA = _enc_mat(o, mm.tile_horizontal(A, c, s1), s0, s1, lvA, 300)
    EB = _enc_mat(o, B, s0, s1, 6, 400)
    ops = mm.RnsOps(o, hoist=True, lazy_relin=True, radix_sum=radix, shared_rot=shared)
    t = 1.0 / 128
    out = mm.diag_atb(ops, EA, EB, c, t)
    got = _dec_mat(o, out, s0, 40)
    Ap = np.zeros((128, c))
    Ap[:, :3] = A
    want = np.tile(t * Ap.T @ B, (s0 // c, 1))
    assert np.max(np.abs(got - want)) <= 1e-4


def test_encrypted_softmax_poly_n13(o13deep):
    o = o13deep
    p = o.p
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, p.slots)
    coeffs = rng.uniform(-3, 3, 16)
    valid = (rng.uniform(size=p.slots) < 0.5).astype(np.float64)
    ct = o.encrypt_int(ckks.encode(x, p.delta, p.N), p.top, p.delta, 77)
    ops = mm.RnsOps(o)
    out = mm.poly15_masked(ops, ct, coeffs, valid, p.delta)
    assert out.lv == p.top - 5 and out.scale == p.delta
    want = np.polynomial.polynomial.polyval(x, coeffs) * valid
    assert np.max(np.abs(o.decrypt_slots(out).real - want)) <= 1e-4


# ---------------------------------------------------------------------------
# Planted mistakes: each must make a pin fail.
# ---------------------------------------------------------------------------
def test_planted_wrong_mask_sign_is_caught(monkeypatch):
    good = mm.mask_cplx
    monkeypatch.setattr(mm, "mask_cplx", lambda k, c, s0, s1: np.conj(good(k, c, s0, s1)))
    _, err = run_abt_sim(128, 128, 4, 128)
    assert err > 1e-3


def test_planted_transposed_offdiag_is_caught(monkeypatch):
    monkeypatch.setattr(mm, "mask_offdiag",
                        lambda k, c, s0, s1: ((np.arange(s1)[None, :] - np.arange(s0)[:, None] + k) % c == 0)
                        .astype(np.float64).reshape(-1))
    _, err = run_atb_sim(256, 256, 8, 256, lvA=12)
    assert err > 1e-3


def test_planted_sumrows_stride_is_caught(monkeypatch):
    def bad_sum_rows(ops, x, s0, s1):
        for u in range(mm.log2i(s0)):
            x = ops.add(x, ops.rot(x, 1 << u))
        return x
    monkeypatch.setattr(mm, "sum_rows", bad_sum_rows)
    _, err = run_atb_sim(128, 128, 4, 128, lvA=11)
    assert err > 1e-3


def test_planted_rotation_direction_is_caught(monkeypatch):
    monkeypatch.setattr(mm.SlotOps, "rot",
                        lambda self, a, r: a if r % self.s == 0 else (self._c("Rot"), mm.SV(np.roll(a.z, r), a.lv))[1])
    _, err = run_abt_sim(128, 128, 4, 128)
    assert err > 1e-3
