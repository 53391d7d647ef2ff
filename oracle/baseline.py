"""CPU baseline of the encrypted training step, from the oracle as it stands.

TEST INFRASTRUCTURE ONLY: used by the benchmark's CPU-baseline leg (and its
reference arm) and by tests.

A whole N = 2^16 step takes the single-threaded oracle hours, so the baseline
is a bounded sample: the step's algorithm is run once on the FP64 slot
simulator to count its ciphertext operations by (kind, level, group size);
each distinct kind is then timed once on the RNS oracle at that level, and the
step time is the count-weighted sum.  Additions and level drops (under 1 % of
the oracle's time) are left out.
"""
import time

import numpy as np

from . import ckks, matmul as mm


def step_operation_counts(rows, dim, c, classes, s0, s1, levels, hoist=True, lazy_relin=True):
    """Operation histogram of one training step (train_step) on the slot simulator."""
    ops = mm.SlotOps(s0 * s1, hoist=hoist, lazy_relin=lazy_relin)
    top = levels - 1
    X = mm.EncMat([[mm.SV(np.zeros(s0 * s1, complex), top) for _ in range(-(-dim // s1))]
                   for _ in range(-(-rows // s0))], rows, dim, s0, s1)
    W = mm.EncMat([[mm.SV(np.zeros(s0 * s1, complex), top) for _ in range(X.n)]], s0, dim, s0, s1)
    lvP = top - 3 - 5
    Y = mm.EncMat([[mm.SV(np.zeros(s0 * s1, complex), lvP)]], rows, s1, s0, s1)
    coeffs = np.zeros(16)
    valid = np.ones(s0 * s1)
    mm.train_step(ops, X, W, Y, coeffs, valid, c, 1.0 / rows, 1.0)
    return dict(ops.by_level)


def _fresh(o, lv, nonce, rng):
    p = o.p
    z = rng.uniform(-0.5, 0.5, p.slots)
    return o.encrypt_int(ckks.encode(z, p.delta, p.N), lv, p.delta, nonce)


def time_operation(o, kind, lv, size, rng):
    """Seconds the oracle spends on one operation of the histogram."""
    p = o.p
    a = _fresh(o, lv, 1, rng)
    ops = mm.RnsOps(o, hoist=True, lazy_relin=True)
    if kind == "rot":
        o.key(ckks.kid_rot(1))
        t = time.perf_counter()
        o.rot_raw(a, 1)
    elif kind == "conj":
        o.key(ckks.KID_CONJ)
        t = time.perf_counter()
        o.conj_raw(a)
    elif kind == "hoist":
        rs = list(range(1, size + 1))
        for r in rs:
            o.key(ckks.kid_rot(r))
        t = time.perf_counter()
        ops.rot_many(a, rs)
    elif kind == "mult":
        b = _fresh(o, lv, 2, rng)
        o.key(ckks.KID_RELIN)
        pairs = [(a, b)] * size
        t = time.perf_counter()
        ops.mult_sum(pairs)
    elif kind == "cmult":
        mask = rng.uniform(-1, 1, p.slots)
        t = time.perf_counter()
        ops.cmult(a, mask, ("t", 0))
    else:
        raise ValueError(kind)
    return time.perf_counter() - t


def estimate_step_seconds(params, rows=1024, dim=768, classes=10, c=16, s0=1024, s1=32, seed=1,
                          hoist=True, lazy_relin=True):
    """(estimated seconds per step, sample description, per-kind detail)."""
    hist = step_operation_counts(rows, dim, c, classes, s0, s1, params.L, hoist, lazy_relin)
    o = ckks.Oracle(params, seed=seed)
    rng = np.random.default_rng(seed)
    detail = []
    total = 0.0
    sampled = 0.0
    for (kind, lv, size), count in sorted(hist.items()):
        sec = time_operation(o, kind, lv, size, rng)
        sampled += sec
        total += count * sec
        detail.append((kind, lv, size, count, sec))
    desc = ("%d distinct (operation, level, group) kinds of one training step, each timed once on the "
            "single-threaded oracle (%.1f s measured) and weighted by its count in the step"
            % (len(hist), sampled))
    return total, desc, detail
