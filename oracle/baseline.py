"""CPU baseline of the encrypted training step, from the oracle as it stands.

TEST INFRASTRUCTURE ONLY: used by the benchmark's CPU-baseline leg (and its
reference arm) and by tests.

The oracle's ring arithmetic splits independent limbs over threads
(ckks.set_threads); every timing below is taken with the thread count in force.
A small DiagABT (N = 2^13) is timed whole (time_diag_abt).  A whole N = 2^16
step takes the single-threaded oracle about an hour, so that baseline is a
bounded sample, extrapolated.  The step's algorithm runs once on the FP64 slot
simulator to count its ciphertext operations by (kind, level, group size).
Five operations are then timed once each on the RNS oracle: at the top level
a rotation, a hoisted pair of rotations, a Mult-and-sum of two pairs and a
CMult, and a rotation at level 1 (about 15-30 s in all).  Each operation of
the step is charged the time of its top-level counterpart, scaled by the
ratio of their modular products at the two levels (the oracle's ring
arithmetic is plain loops); key-switch times follow a power of that count
fitted to the two rotations.  Additions and level drops are left out.
"""
import time

import numpy as np

from . import ckks, matmul as mm


def abt_operation_counts(rows, dim, c, s0, s1, levels, hoist=True, lazy_relin=True, radix_sum=False,
                         shared_rot=False):
    """Operation histogram of one DiagABT (both inputs at the top level) on the slot simulator."""
    ops = mm.SlotOps(s0 * s1, hoist=hoist, lazy_relin=lazy_relin, radix_sum=radix_sum, shared_rot=shared_rot)
    top = levels - 1
    X = mm.EncMat([[mm.SV(np.zeros(s0 * s1, complex), top) for _ in range(-(-dim // s1))]
                   for _ in range(-(-rows // s0))], rows, dim, s0, s1)
    W = mm.EncMat([[mm.SV(np.zeros(s0 * s1, complex), top) for _ in range(X.n)]], s0, dim, s0, s1)
    mm.diag_abt(ops, X, W, c, 1.0)
    return dict(ops.by_level)


def _abt_rotations(s0, s1, c, radix_sum):
    """Left-rotation amounts DiagABT uses: RotUp by k s1 (k <= c/2) and SumCols' amounts
    (+-2^u, or the radix steps' j t)."""
    s, rs = s0 * s1, set()
    for k in range(1, c // 2 + 1):
        rs.add(k * s1 % s)
    bits = mm.log2i(s1)
    for sign in (1, -1):
        if radix_sum:
            t = 1
            for b in mm.radix_plan(bits):
                rs |= {(sign * j * t) % s for j in range(1, 1 << b)}
                t <<= b
        else:
            rs |= {(sign * (1 << u)) % s for u in range(bits)}
    return sorted(rs - {0})


def time_diag_abt(params, rows, dim, c, s0, s1, seed=1, hoist=True, lazy_relin=True, radix_sum=False,
                  shared_rot=False):
    """Seconds the oracle takes for one whole DiagABT of a rows x dim matrix by (c x dim)^T at the
    top level (keys generated beforehand, not timed), and the largest error of its decryption
    against the FP64 product."""
    p = params
    o = ckks.Oracle(p, seed=seed)
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (rows, dim))
    W = rng.uniform(-1, 1, (c, dim))

    def enc(M, nonce):
        return mm.EncMat([[o.encrypt_int(ckks.encode(b, p.delta, p.N), p.top, p.delta, nonce + 64 * r + j)
                           for j, b in enumerate(row)] for r, row in enumerate(mm.block_split(M, s0, s1))],
                         M.shape[0], M.shape[1], s0, s1)

    EX, EW = enc(X, 100), enc(mm.tile_vertical(W, c, s0), 200)
    for kid in [ckks.KID_RELIN, ckks.KID_CONJ]:
        o.key(kid)
    for r in _abt_rotations(s0, s1, c, radix_sum):
        o.key(ckks.kid_rot(r))
    ops = mm.RnsOps(o, hoist=hoist, lazy_relin=lazy_relin, radix_sum=radix_sum, shared_rot=shared_rot)
    t = time.perf_counter()
    out = mm.diag_abt(ops, EX, EW, c, 1.0)
    sec = time.perf_counter() - t
    dec = np.concatenate([o.decrypt_slots(b[0]).real.reshape(s0, s1) for b in out.blocks])[:rows]
    err = float(np.max(np.abs(dec - np.tile(X @ W.T, (1, s1 // c)))))
    return sec, err


def step_operation_counts(rows, dim, c, classes, s0, s1, levels, hoist=True, lazy_relin=True, radix_sum=False,
                          shared_rot=False):
    """Operation histogram of one training step (train_step) on the slot simulator."""
    ops = mm.SlotOps(s0 * s1, hoist=hoist, lazy_relin=lazy_relin, radix_sum=radix_sum, shared_rot=shared_rot)
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
    elif kind == "rotsum":
        rs = list(range(1, size + 1))
        for r in rs:
            o.key(ckks.kid_rot(r))
        t = time.perf_counter()
        ops.rot_sum(a, rs)
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


def _ntt(p):
    return p.N // 2 * int(np.log2(p.N))


def keyswitch_work(p, lv, hoisted_step=False):
    """Modular products of one key switch at level lv: INTT, ModUp, key inner product, ModDown
    (dnum digits of alpha primes, K special primes); a further hoisted step skips INTT and ModUp."""
    l, K, a, N = lv + 1, p.K, p.alpha, p.N
    d = p.dnum(lv)
    w = 2 * d * (l + K) * N + 2 * K * _ntt(p) + 2 * (K + K * l) * N + 2 * l * _ntt(p) + 2 * l * N
    if not hoisted_step:
        w += l * _ntt(p) + d * (a * N + a * (l + K - a) * N + (l + K - a) * _ntt(p))
    return w


def rescale_work(p, lv):
    return 2 * (lv + 1) * _ntt(p) + 2 * lv * p.N


def tensor_work(p, lv):
    return 4 * (lv + 1) * p.N


def kip_work(p, lv):
    return 2 * p.dnum(lv) * (lv + 1 + p.K) * p.N


def estimate_step_seconds(params, rows=1024, dim=768, classes=10, c=16, s0=1024, s1=32, seed=1,
                          hoist=True, lazy_relin=True, radix_sum=False, shared_rot=False):
    """(estimated seconds per step, sample description, per-kind detail)."""
    hist = step_operation_counts(rows, dim, c, classes, s0, s1, params.L, hoist, lazy_relin, radix_sum, shared_rot)
    return estimate_seconds(params, hist, seed)


def estimate_seconds(params, hist, seed=1):
    """(estimated seconds of the operations in hist, sample description, per-kind detail)."""
    p = params
    o = ckks.Oracle(p, seed=seed)
    rng = np.random.default_rng(seed)
    top = p.L - 1
    t_rot = time_operation(o, "rot", top, 1, rng)
    t_hoist2 = time_operation(o, "hoist", top, 2, rng)
    t_mult2 = time_operation(o, "mult", top, 2, rng)
    t_cmult = time_operation(o, "cmult", top, 1, rng)
    t_rot1 = time_operation(o, "rot", 1, 1, rng)
    sampled = t_rot + t_hoist2 + t_mult2 + t_cmult + t_rot1
    n_timed = 5
    t_kip = None
    if any(k[0] == "rotsum" for k in hist):
        t_kip1 = max(time_operation(o, "rotsum", 1, 2, rng) - t_rot1, 1e-9)   # one more summed rotation, level 1
        sampled += t_kip1 + t_rot1
        t_kip = t_kip1 * kip_work(p, top) / kip_work(p, 1)
        n_timed += 1
    ks_full, ks_step = keyswitch_work(p, top), keyswitch_work(p, top, True)
    # key-switch time as a power of its work, through the rotations at the top level and at level 1
    e = np.log(t_rot / t_rot1) / np.log(ks_full / keyswitch_work(p, 1))

    def ks(lv, hoisted_step=False, t_top=t_rot, w_top=ks_full):
        return t_top * (keyswitch_work(p, lv, hoisted_step) / w_top) ** e

    step_t = max(t_hoist2 - t_rot, 1e-9)                    # one further hoisted rotation
    per_rescale = t_cmult / rescale_work(p, top)
    per_tensor = max(t_mult2 - t_rot - t_cmult, 1e-9) / 2 / tensor_work(p, top)
    detail = []
    total = 0.0
    for (kind, lv, size), count in sorted(hist.items()):
        if kind in ("rot", "conj"):
            sec = ks(lv)
        elif kind == "hoist":
            sec = ks(lv) + (size - 1) * ks(lv, True, step_t, ks_step)
        elif kind == "rotsum":
            sec = ks(lv) + (size - 1) * t_kip * kip_work(p, lv) / kip_work(p, top)
        elif kind == "mult":
            sec = size * per_tensor * tensor_work(p, lv) + ks(lv) + per_rescale * rescale_work(p, lv)
        elif kind == "cmult":
            sec = per_rescale * rescale_work(p, lv)
        else:
            raise ValueError(kind)
        total += count * float(sec)
        detail.append((kind, lv, size, count, float(sec)))
    desc = ("%d operations timed once on the oracle with %d thread(s) (at the top level a rotation, a hoisted "
            "pair, a Mult-and-sum of 2 pairs and a CMult; at level 1 a rotation%s: %.1f s measured); each of the "
            "%d operations is charged its counterpart's time scaled by their modular-product counts (key switches "
            "as a power of that count fitted to the two rotations)"
            % (n_timed, ckks.threads(), " and a 2-term rotation sum" if t_kip is not None else "", sampled,
               sum(hist.values())))
    return total, desc, detail
