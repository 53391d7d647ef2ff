"""Pins for the oracle's ring arithmetic, each against something other than
the oracle itself: a library routine (sympy primality, numpy's Philox), a
definition evaluated with Python big integers (schoolbook negacyclic product,
exact CRT and rounding), or an invariant of the construction."""
import numpy as np
import pytest
import sympy

from oracle import ckks

L = ckks.lib


def tiny_params():
    # N = 32, four ciphertext primes, two special primes, two primes per digit.
    return ckks.Params(5, 60, 3, 40, 2, 61, alpha=2, h=8)


def test_is_prime_matches_sympy():
    rng = np.random.default_rng(3)
    cands = [2, 3, 4, 561, 1105, 2 ** 61 - 1, 2 ** 64 - 59, 3215031751, 2152302898747]
    cands += [int(x) for x in rng.integers(2, 2 ** 62, size=300, dtype=np.int64)]
    cands += [int(x) | 1 for x in rng.integers(2 ** 40, 2 ** 41, size=300, dtype=np.int64)]
    for n in cands:
        assert bool(L().orc_is_prime(n)) == sympy.isprime(n), n


@pytest.mark.parametrize("step_log", [14, 17, 32])
@pytest.mark.parametrize("bits", [40, 50, 60, 61])
def test_gen_primes_are_the_largest(step_log, bits):
    step = 1 << step_log
    ps = ckks.gen_primes(step, bits, 4)
    assert len(ps) == 4
    assert ps == sorted(ps, reverse=True)
    for p in ps:
        assert p < 1 << bits and p % step == 1 and sympy.isprime(p)
    # every candidate = 1 mod step from 2^bits down to the last prime returned
    # is in the list exactly when it is prime (none skipped, none invented)
    x = ((1 << bits) - 1) // step * step + 1
    if x >= 1 << bits:
        x -= step
    while x >= ps[-1]:
        assert (x in ps) == sympy.isprime(x), x
        x -= step


@pytest.mark.parametrize("chain", [(13, 60, 3, 40, 1, 61), (13, 60, 6, 40, 2, 61), (16, 60, 11, 50, 2, 61),
                                   (16, 60, 14, 50, 4, 61, 21, 60), (10, 60, 14, 50, 2, 61, 19, 60)])
def test_prime_chain(chain):
    """Single chains and mixed ones (an upper group of primes above the rescale primes; here
    of q_0's size, so that it must skip q_0)."""
    log_n, q0_bits, n_rescale, rescale_bits, n_special, special_bits = chain[:6]
    n_upper, upper_bits = (chain[6], chain[7]) if len(chain) > 6 else (0, 0)
    qs, ps = ckks.prime_chain(*chain)
    assert len(qs) == 1 + n_rescale + n_upper and len(ps) == n_special
    allp = qs + ps
    assert len(set(allp)) == len(allp)
    for p in allp:
        # 1 mod 2^32 implies 1 mod 2N: the negacyclic NTT of length N exists
        assert sympy.isprime(p) and p % (1 << 32) == 1 and p % (2 << log_n) == 1
    taken = set()
    groups = [(qs[:1], q0_bits), (qs[1:1 + n_rescale], rescale_bits)]
    if n_upper:
        groups.append((qs[1 + n_rescale:], upper_bits))
    for group, bits in groups + [(ps, special_bits)]:
        assert group == sorted(group, reverse=True)
        x = (1 << bits) - (1 << 32) + 1
        while x >= group[-1]:
            if x not in taken:
                assert (x in group) == sympy.isprime(x), x
            x -= 1 << 32
        taken.update(group)


def _schoolbook_bigint(a, b, q):
    n = len(a)
    out = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += int(a[i]) * int(b[j])
            else:
                out[k - n] -= int(a[i]) * int(b[j])
    return [v % q for v in out]


@pytest.mark.parametrize("bits", [40, 50, 60, 61])
@pytest.mark.parametrize("n", [16, 64])
def test_polymul_equals_schoolbook(n, bits):
    q = ckks.gen_primes(2 * n, bits, 1)[0]
    psi = L().orc_find_psi(q, 2 * n)
    rng = np.random.default_rng(n + bits)
    a = ckks.u64(rng.integers(0, q, n, dtype=np.uint64))
    b = ckks.u64(rng.integers(0, q, n, dtype=np.uint64))
    out = np.zeros(n, dtype=np.uint64)
    L().orc_polymul(ckks.P(a), ckks.P(b), ckks.P(out), n, q, psi)
    assert [int(x) for x in out] == _schoolbook_bigint(a, b, q)
    out2 = np.zeros(n, dtype=np.uint64)
    L().orc_polymul_schoolbook(ckks.P(a), ckks.P(b), ckks.P(out2), n, q)
    assert np.array_equal(out, out2)


def test_ntt_is_evaluation_at_odd_powers_and_inverts():
    n = 16
    q = ckks.gen_primes(2 * n, 50, 1)[0]
    psi = L().orc_find_psi(q, 2 * n)
    assert pow(psi, n, q) == q - 1
    rng = np.random.default_rng(1)
    a = ckks.u64(rng.integers(0, q, n, dtype=np.uint64))
    t = a.copy()
    L().orc_ntt_fwd(ckks.P(t), n, q, psi)
    for k in range(n):
        x = pow(psi, 2 * k + 1, q)
        assert int(t[k]) == sum(int(a[i]) * pow(x, i, q) for i in range(n)) % q
    L().orc_ntt_inv(ckks.P(t), n, q, psi)
    assert np.array_equal(t, a)


def test_philox_matches_numpy():
    rng = np.random.default_rng(7)
    for _ in range(20):
        key = [int(x) for x in rng.integers(0, 2 ** 63, 2, dtype=np.int64)]
        ctr = [int(x) for x in rng.integers(0, 2 ** 40, 4, dtype=np.int64)]
        ctr[0] += 1  # numpy increments its counter before producing a block
        before = list(ctr)
        before[0] -= 1
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(before, dtype=np.uint64))
        want = [int(x) for x in bg.random_raw(4)]
        out = np.zeros(4, dtype=np.uint64)
        L().orc_philox4x64(ckks.P(ckks.u64(ctr)), ckks.P(ckks.u64(key)), ckks.P(out))
        assert [int(x) for x in out] == want


def test_samplers():
    n = 1 << 14
    q = ckks.gen_primes(2 * n, 50, 1)[0]
    u = np.zeros(n, dtype=np.uint64)
    L().orc_sample_uniform(5, 9, n, 2, q, ckks.P(u))
    assert int(u.max()) < q
    f = u.astype(np.float64) / q
    assert abs(f.mean() - 0.5) < 0.02 and abs(f.var() - 1 / 12) < 0.01
    hist = np.histogram(f, bins=16, range=(0, 1))[0]
    assert hist.min() > 0.8 * n / 16
    e = np.zeros(n, dtype=np.int64)
    L().orc_sample_cbd(5, 9, n, ckks.P(e))
    assert e.min() >= -21 and e.max() <= 21
    assert abs(e.mean()) < 0.2 and abs(e.var() - 10.5) < 0.6
    s = np.zeros(n, dtype=np.int64)
    L().orc_sample_secret(5, 9, n, 192, ckks.P(s))
    assert np.count_nonzero(s) == 192 and set(np.unique(s[s != 0])) <= {-1, 1}
    assert 60 < np.count_nonzero(s == 1) < 132


def _crt(res, mods):
    Q = 1
    for m in mods:
        Q *= m
    v = 0
    for r, m in zip(res, mods):
        Qm = Q // m
        v += int(r) * Qm * pow(Qm % m, -1, m)
    return v % Q, Q


def test_modup_invariant_bigint():
    p = tiny_params()
    n, lv = p.N, 3
    rng = np.random.default_rng(11)
    x = np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in p.q[:lv + 1]])
    x = ckks.u64(x)
    for j in range(p.dnum(lv)):
        out = np.zeros((lv + 1 + p.K, n), dtype=np.uint64)
        L().orc_modup(p.c, lv, j, ckks.P(x), ckks.P(out))
        lo, hi = j * p.alpha, min((j + 1) * p.alpha, lv + 1)
        dig = list(range(lo, hi))
        mods = p.q[:lv + 1] + p.p
        for c in range(n):
            xv, D = _crt([x[i, c] for i in dig], [p.q[i] for i in dig])
            for t, m in enumerate(mods):
                if t in dig:
                    assert out[t, c] == x[t, c]
                    continue
                diff = (int(out[t, c]) - xv) % m
                assert any(diff == (u * D) % m for u in range(len(dig))), (j, t, c)


def test_moddown_invariant_bigint():
    p = tiny_params()
    n, lv = p.N, 2
    rng = np.random.default_rng(12)
    mods = p.q[:lv + 1] + p.p
    x = ckks.u64(np.stack([rng.integers(0, m, n, dtype=np.uint64) for m in mods]))
    out = np.zeros((lv + 1, n), dtype=np.uint64)
    L().orc_moddown(p.c, lv, ckks.P(x), ckks.P(out))
    Pp = 1
    for m in p.p:
        Pp *= m
    for c in range(n):
        y, _ = _crt([x[t, c] for t in range(len(mods))], mods)
        yP, _ = _crt([x[lv + 1 + k, c] for k in range(p.K)], p.p)
        o, Q = _crt([out[i, c] for i in range(lv + 1)], p.q[:lv + 1])
        diff = (o * Pp - (y - yP)) % Q
        assert any(diff == (-u * Pp) % Q for u in range(p.K)), c


def test_rescale_is_exact_rounding_bigint():
    p = tiny_params()
    n, lv = p.N, 3
    rng = np.random.default_rng(13)
    ct = ckks.u64(np.stack([np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in p.q[:lv + 1]])
                            for _ in range(2)]))
    out = np.zeros((2, lv, n), dtype=np.uint64)
    L().orc_rescale(p.c, ckks.P(ct), lv, ckks.P(out))
    ql = p.q[lv]
    for c in range(2):
        for x in range(n):
            y, _ = _crt([ct[c, i, x] for i in range(lv + 1)], p.q[:lv + 1])
            want = (2 * y + ql) // (2 * ql)          # round(y / q_lv), q_lv odd: no ties
            o, Q = _crt([out[c, i, x] for i in range(lv)], p.q[:lv])
            assert o == want % Q


def _poly_bigint_mul(a, b):
    n = len(a)
    out = [0] * n
    for i in range(n):
        if a[i] == 0:
            continue
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += a[i] * b[j]
            else:
                out[k - n] -= a[i] * b[j]
    return out


def test_keyswitch_relation_bigint():
    """KS(d) = (k0, k1) with k0 + k1*s = d*s' + small noise (mod Q_lv), s' = s(X^g)."""
    p = tiny_params()
    o = ckks.Oracle(p, seed=21)
    n, lv = p.N, 3
    g = p.galois_rot(3)
    key = o.key(ckks.kid_rot(3))
    rng = np.random.default_rng(14)
    d = ckks.u64(np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in p.q[:lv + 1]]))
    k0 = np.zeros((lv + 1, n), dtype=np.uint64)
    k1 = np.zeros((lv + 1, n), dtype=np.uint64)
    L().orc_keyswitch(p.c, lv, ckks.P(d), ckks.P(key), ckks.P(k0), ckks.P(k1))
    mods = p.q[:lv + 1]
    Q = 1
    for m in mods:
        Q *= m
    s = [int(v) for v in o.sk]
    sp = [0] * n
    for i in range(n):
        e = (i * g) % (2 * n)
        if e < n:
            sp[e] = s[i]
        else:
            sp[e - n] = -s[i]
    D = [_crt([d[i, x] for i in range(lv + 1)], mods)[0] for x in range(n)]
    K0 = [_crt([k0[i, x] for i in range(lv + 1)], mods)[0] for x in range(n)]
    K1 = [_crt([k1[i, x] for i in range(lv + 1)], mods)[0] for x in range(n)]
    lhs = _poly_bigint_mul(K1, s)
    rhs = _poly_bigint_mul(D, sp)
    for x in range(n):
        v = (K0[x] + lhs[x] - rhs[x]) % Q
        if v > Q // 2:
            v -= Q
        assert abs(v) < 2 ** 70, v    # Q ~ 2^180; a wrong gadget or digit gives ~Q


def test_automorphism_group_law():
    n = 64
    q = ckks.gen_primes(2 * n, 40, 1)[0]
    rng = np.random.default_rng(2)
    a = ckks.u64(rng.integers(0, q, n, dtype=np.uint64))
    g1, g2 = pow(5, 3, 2 * n), pow(5, 7, 2 * n)
    t1 = np.zeros(n, dtype=np.uint64)
    t2 = np.zeros(n, dtype=np.uint64)
    t3 = np.zeros(n, dtype=np.uint64)
    L().orc_automorphism(ckks.P(a), ckks.P(t1), n, g1, q)
    L().orc_automorphism(ckks.P(t1), ckks.P(t2), n, g2, q)
    L().orc_automorphism(ckks.P(a), ckks.P(t3), n, (g1 * g2) % (2 * n), q)
    assert np.array_equal(t2, t3)
    # X -> X^g is a ring map: (a*b)(X^g) = a(X^g) * b(X^g)
    psi = L().orc_find_psi(q, 2 * n)
    b = ckks.u64(rng.integers(0, q, n, dtype=np.uint64))
    ab = np.zeros(n, dtype=np.uint64)
    L().orc_polymul(ckks.P(a), ckks.P(b), ckks.P(ab), n, q, psi)
    abg = np.zeros(n, dtype=np.uint64)
    L().orc_automorphism(ckks.P(ab), ckks.P(abg), n, g1, q)
    bg = np.zeros(n, dtype=np.uint64)
    L().orc_automorphism(ckks.P(b), ckks.P(bg), n, g1, q)
    prod = np.zeros(n, dtype=np.uint64)
    L().orc_polymul(ckks.P(t1), ckks.P(bg), ckks.P(prod), n, q, psi)
    assert np.array_equal(prod, abg)
