"""The step-level roofline's work model: its operation counts are the paper's
(Table "tab:matnum_fixed", App. D, s0 = a, s = 32768, both DiagATB branches),
and its primitive costs follow from their definitions on small parameters."""
import os

import pytest

from paper_2403_14111_gb300 import workmodel as wm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tab_matnum_fixed.txt")


def rows():
    with open(GOLDEN) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                yield [int(x) for x in ln.split()]


@pytest.mark.parametrize("row", list(rows()), ids=lambda r: "%dx%dx%d" % tuple(r[:3]))
def test_counts_are_the_papers(row):
    a, b, c = row[:3]
    s0, s1 = a, 32768 // a
    C = wm.Costs(1 << 16, 2, 2)
    ab = wm.diag_abt(C, a, b, c, s0, s1, 11).counts
    assert (ab["cmult"], ab["mult"], ab["rot"]) == tuple(row[3:6])
    rl = wm.diag_atb(C, a, b, c, s0, s1, 11, 11).counts
    assert (rl["cmult"], rl["mult"], rl["rot"]) == tuple(row[6:9])
    pr = wm.diag_atb(C, a, b, c, s0, s1, 9, 10).counts
    assert (pr["cmult"], pr["mult"], pr["rot"]) == tuple(row[9:12])
    assert ab["conj"] == 1 and rl["conj"] == -(-b // s1) and pr["conj"] == -(-b // s1)


def test_primitive_costs():
    N, K, alpha = 1 << 4, 2, 2
    C = wm.Costs(N, K, alpha)
    ntt = N // 2 * 4
    assert C.ntt == ntt
    # level 2 (3 limbs): digits {2, 1}; ModUp converts to 3 + 2 - a moduli per digit
    ks = C.keyswitch(2, "k")
    modup_bf = (3 + 2 - 2) * ntt + (3 + 2 - 1) * ntt
    modup_mac = (2 * N + 2 * 3 * N) + (1 * N + 1 * 4 * N)
    kip = 2 * 2 * (3 + 2) * N
    md_bf, md_mac = 2 * K * ntt + 2 * 3 * ntt, 2 * (K + K * 3) * N + 2 * 3 * N
    assert ks.bfly == 3 * ntt + modup_bf + md_bf
    assert ks.mac == modup_mac + kip + md_mac
    ex = C.keyswitch(2, "k", hoisted_extra=True)
    assert (ex.bfly, ex.mac) == (md_bf, kip + md_mac)
    rs = C.rescale(2)
    assert (rs.bfly, rs.mac) == (2 * 3 * ntt, 2 * 2 * N)
    mu = C.mult(2)
    assert mu.bfly == ks.bfly + rs.bfly and mu.mac == 4 * 3 * N + ks.mac + rs.mac
    cm = C.cmult(2)
    assert (cm.bfly, cm.mac) == (rs.bfly, 2 * 3 * N + rs.mac)


def test_hoisting_shares_one_modup():
    C = wm.Costs(1 << 16, 2, 2)
    a, b, c, s0, s1 = 1024, 768, 16, 1024, 32
    w = wm.diag_abt(C, a, b, c, s0, s1, 11)
    n, h = 24, 8
    plain = wm.Work()
    for _ in range(h):   # RotUp(B-bar, c/2) and c/2 - 1 RotUp(B_cplx, k), every one a full key switch
        plain.add(wm._times(C.rot(11, 0), n))
    hoisted = wm.Work()
    hoisted.add(wm._times(C.rot(11, 0), 2 * n))
    hoisted.add(wm._times(C.rot(11, 0, hoisted_extra=True), (h - 2) * n))
    diff = plain.bfly + plain.mac - hoisted.bfly - hoisted.mac
    full, extra = C.keyswitch(11, 0), C.keyswitch(11, 0, hoisted_extra=True)
    assert diff == (h - 2) * n * (full.bfly + full.mac - extra.bfly - extra.mac) > 0


def test_training_step_levels_end_at_zero():
    C = wm.Costs(1 << 16, 2, 2)
    w = wm.finish(wm.training_step(C, 1024, 768, 16, 1024, 32, 11), C)
    assert w.counts["mult"] == 8 * 24 + 7 + 8 * 24 and w.counts["conj"] == 1 + 24
    eq = w.equivalents(0.66)
    assert 1e10 < eq < 1e12 and w.nbytes > 0
    with pytest.raises(Exception):
        wm.training_step(C, 1024, 768, 16, 1024, 32, 7)   # not enough levels: a level below 0
