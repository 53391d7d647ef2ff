"""CKKS bootstrapping in the oracle (oracle/bootstrap.py): each step pinned against the
mathematics that defines it, then the whole procedure on RNS ciphertexts against the
message it refreshes."""
import math

import numpy as np
import pytest

from oracle import bootstrap as bt
from oracle import ckks, matmul as mm, softmax as sm


def test_encoding_matrix_is_the_canonical_embedding():
    N = 64
    n = N // 2
    U = bt.encoding_matrix(N)
    rng = np.random.default_rng(0)
    t = rng.integers(-1000, 1000, N).astype(float)
    # sigma(t)_j = t(zeta^(5^j)), by the oracle's decoder (pinned against the O(N^2) definition)
    z = ckks.decode_real_coeffs(t, 1.0, N)
    assert np.max(np.abs(U @ (t[:n] + 1j * t[n:]) - z)) < 1e-9
    assert np.max(np.abs(np.linalg.inv(U) - (2.0 / N) * U.conj().T)) < 1e-12


@pytest.mark.parametrize("n1", [0, 4, 32])
def test_baby_step_giant_step_is_the_matrix_product(n1):
    n = 64
    rng = np.random.default_rng(1)
    M = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    z = rng.normal(size=n) + 1j * rng.normal(size=n)
    ops = mm.SlotOps(n)
    out = bt.lintrans(ops, mm.SV(z, 5), M, "m", 1.0, bt.BootParams(n1=n1))
    assert np.max(np.abs(out.z - M @ z)) < 1e-10
    assert out.lv == 4


@pytest.mark.parametrize("N", [16, 64, 1024])
@pytest.mark.parametrize("per", [1, 2, 3, 4])
def test_factored_transforms_are_the_embedding(N, per):
    """S_L .. S_1 applied to the bit-reversed vector is U x; the inverse levels give
    (1/2) U^-1 z in bit-reversed order; every level has at most 2^(per+1) - 1 diagonals."""
    n = N // 2
    bits = n.bit_length() - 1
    perm = [int(format(i, "0%db" % bits)[::-1], 2) for i in range(n)]
    U = bt.encoding_matrix(N)
    rng = np.random.default_rng(per)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    y = x[perm]
    for M in bt.factored(N, False, per):
        assert len(M) <= 2 ** (per + 1) - 1
        y = sum(M[r] * np.roll(y, -r) for r in M)
    assert np.max(np.abs(y - U @ x)) < 1e-11
    w = U @ x
    for M in bt.factored(N, True, per):
        w = sum(M[r] * np.roll(w, -r) for r in M)
    assert np.max(np.abs(w - 0.5 * x[perm])) < 1e-12


def test_factored_procedure_on_the_slot_simulator():
    N = 1024
    q0, d_in = float(2 ** 60 - 7 * 2 ** 32 + 1), 2.0 ** 50
    rng = np.random.default_rng(6)
    m = rng.uniform(-1, 1, N // 2)
    t = ckks.encode(m, d_in, N).astype(float) + rng.normal(0, 3.2, N).round() + q0 * rng.normal(0, 4, N).round()
    prm = bt.BootParams()
    ops = mm.SlotOps(N // 2)
    out = bt.bootstrap_raised(ops, mm.SV(ckks.decode_real_coeffs(t, q0, N), 30), N, 1.0, prm)
    assert 30 - out.lv == bt.depth(prm, N)
    assert np.max(np.abs(out.z * q0 / d_in - m)) < 1e-6


def test_coeff_to_slot_and_back():
    N = 128
    n = N // 2
    rng = np.random.default_rng(2)
    t = rng.integers(-50, 50, N).astype(float)
    ops = mm.SlotOps(n)
    lo, hi = bt.coeff_to_slot(ops, mm.SV(ckks.decode_real_coeffs(t, 1.0, N), 5), N, 1.0, bt.BootParams())
    assert np.max(np.abs(lo.z - t[:n])) < 1e-9 and np.max(np.abs(hi.z - t[n:])) < 1e-9
    back = bt.slot_to_coeff(ops, lo, hi, N, 1.0, bt.BootParams())
    assert np.max(np.abs(back.z - ckks.decode_real_coeffs(t, 1.0, N))) < 1e-8


def test_eval_mod_is_the_sine_on_its_range():
    prm = bt.BootParams()
    x = np.linspace(-prm.K, prm.K, 40001)
    ops = mm.SlotOps(len(x))
    y = bt.eval_mod(ops, mm.SV(x.astype(complex), 30), prm, 1.0)
    assert np.max(np.abs(y.z.real - np.sin(2 * np.pi * x) / (2 * np.pi))) < 1e-10
    assert 30 - y.lv == bt.depth(prm) - 2
    # near an integer it removes the integer: x = I + eps -> eps (1 - (2 pi eps)^2 / 6 + ...)
    eps = 1e-4
    z = np.arange(-24, 25) + eps
    y = bt.eval_mod(mm.SlotOps(len(z)), mm.SV(z.astype(complex), 30), prm, 1.0).z.real
    assert np.max(np.abs(y - eps)) < 1e-10


def test_mod_raise_keeps_the_residues_and_adds_a_small_multiple_of_q0():
    p = ckks.Params(10, 60, 4, 60, 1, 61, 1, log_delta=50)
    o = ckks.Oracle(p, seed=2)
    z = np.random.default_rng(3).uniform(-1, 1, p.slots)
    ct = o.encrypt_int(ckks.encode(z, 2.0 ** 50, p.N), 0, 2.0 ** 50, 4)
    r = o.mod_raise(ct, p.top)
    assert r.lv == p.top and r.scale == float(p.q[0])
    assert np.array_equal(r.data[:, 0, :], ct.data[:, 0, :])
    t_low = o.decrypt_int(ct)          # centred mod q_0
    t_high = o.decrypt_int(r)          # centred mod q_0..q_top: the phase over the integers
    I = np.round((t_high - t_low) / float(p.q[0]))
    assert np.max(np.abs(t_high - t_low - I * float(p.q[0]))) < 1e-3 * float(p.q[0])
    assert 0 < np.max(np.abs(I)) <= 24


@pytest.mark.parametrize("fft", [True, False], ids=["factored", "dense"])
def test_bootstrap_refreshes_a_level_zero_ciphertext(fft):
    prm = bt.BootParams(fft=fft)
    log_n = 10
    p = ckks.Params(log_n, 60, bt.depth(prm, 1 << log_n) + 3, 60, 2, 61, 2, log_delta=40)
    o = ckks.Oracle(p, seed=4)
    m = np.random.default_rng(1).uniform(-1, 1, p.slots)
    d_in, d_w = 2.0 ** 50, 2.0 ** 50
    ct = o.encrypt_int(ckks.encode(m, d_in, p.N), 0, d_in, 9)
    ops = sm.ScaledOps(o, d_w, hoist=True)
    out = bt.bootstrap_raised(ops, o.mod_raise(ct, p.top), p.N, d_w, prm)
    assert out.lv == p.top - bt.depth(prm, p.N)
    res = ckks.Ct(out.data, out.lv, out.scale * d_in / float(p.q[0]))
    assert abs(math.log2(res.scale) - 40) < 1e-6
    got = o.decrypt_slots(res)
    assert np.max(np.abs(got - m)) < 5e-5


def _slot_pipeline(N, cts=bt.coeff_to_slot, prm=None, ops_cls=mm.SlotOps):
    """The whole procedure on the slot simulator, from t = Delta m + e + q_0 I."""
    prm = prm or bt.BootParams()
    n = N // 2
    q0, d_in = float(2 ** 60 - 7 * 2 ** 32 + 1), 2.0 ** 50
    rng = np.random.default_rng(5)
    m = rng.uniform(-1, 1, n)
    t = ckks.encode(m, d_in, N).astype(float) + rng.normal(0, 3.2, N).round() + q0 * rng.normal(0, 4, N).round()
    ops = ops_cls(n)
    lo, hi = cts(ops, mm.SV(ckks.decode_real_coeffs(t, q0, N), 20), N, 1.0, prm)
    out = bt.slot_to_coeff(ops, bt.eval_mod(ops, lo, prm, 1.0), bt.eval_mod(ops, hi, prm, 1.0), N, 1.0, prm)
    return np.max(np.abs(out.z * q0 / d_in - m))


def test_slot_level_procedure_and_planted_mistakes():
    assert _slot_pipeline(1024) < 1e-6

    def cts_wrong_sign(ops, ct, N, out_scale, prm):   # imaginary part with the wrong sign
        lo, hi = bt.coeff_to_slot(ops, ct, N, out_scale, prm)
        return lo, ops.mul_int(hi, -1)
    assert _slot_pipeline(1024, cts=cts_wrong_sign) > 1e-2
    class NoShift(mm.SlotOps):   # EvalMod without its -1/4: cos(2 pi x) instead of sin(2 pi x)
        def add_plain(self, a, vals, key):
            return a if key[0] == "em_shift" else super().add_plain(a, vals, key)
    assert _slot_pipeline(1024, ops_cls=NoShift) > 1e-2
